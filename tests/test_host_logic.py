"""Host-side logic that needs no GPU: option names of every schedule the
benchmark and the autotuner use, the autotuner's candidate set and cache
keys, and the benchmark's lookup of the committed DRAM-traffic figure."""
import hashlib
import os

import pytest

import bench
from gen import grids
from paper_1109_1146_gb300 import autotune, mf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FIELDS = {name for name, _ in mf.mf_opts._fields_ if name != "reserved"}


def test_unknown_option_names_are_rejected():
    __import__("__graft_entry__").build()
    with pytest.raises(TypeError):
        mf.default_opts(global_relabel_periods=4)
    o = mf.default_opts(boundary_relabel_period=2, global_relabel_first=1)
    assert o.boundary_relabel_period == 2 and o.global_relabel_first == 1


def test_schedule_tables_use_real_option_names():
    for name, kw in bench.RELABEL_SCHEDULES.items():
        assert set(kw) <= FIELDS, name
    for conn in (4, 8, 6):
        for tile, kw in autotune.candidates(conn):
            assert set(kw) <= FIELDS


@pytest.mark.parametrize("conn", [4, 8, 6])
def test_candidates_cover_tiles_and_schedules(conn):
    cands = autotune.candidates(conn)
    tiles = {t for t, _ in cands}
    assert tiles == {t for t, _ in autotune.CANDIDATES[conn]}
    if conn == 6:
        assert all(t[0] == 32 for t in tiles)  # the bit-parallel 3D tiles
    # every tile gets each global-relabel period and the boundary relabel
    for t in tiles:
        periods = {kw.get("global_relabel_period") for tt, kw in cands if tt == t and "boundary_relabel_period" not in kw}
        assert periods >= set(autotune.GLR_PERIODS)
        assert any(tt == t and kw.get("boundary_relabel_period") == autotune.BR_PERIOD for tt, kw in cands)
    assert len(cands) == len(set((t, tuple(sorted(kw.items()))) for t, kw in cands))


def test_cache_key_follows_size_class_and_candidate_set(monkeypatch):
    a = grids.segmentation_2d(128, 128, 1, conn=4)
    b = grids.segmentation_2d(130, 126, 2, conn=4)
    c = grids.segmentation_2d(512, 512, 3, conn=4)
    assert autotune.key_of(a) == autotune.key_of(b) != autotune.key_of(c)
    assert autotune.key_of(a, single=True).startswith("single_")
    k0 = autotune.key_of(a)
    monkeypatch.setattr(autotune, "GLR_PERIODS", (0, 4))
    assert autotune.key_of(a) != k0  # a cache written for other candidates is not reused


def test_batch_schedule_follows_the_heaviest_class():
    small = [grids.random_grid((20, 20, 1), 4, s) for s in range(3)]
    big = [grids.random_grid((90, 90, 1), 4, 7)]
    table = {autotune.key_of(small[0]): {"tile": [32, 32, 1], "opts": {"global_relabel_period": 0}, "ms": 1.0},
             autotune.key_of(big[0]): {"tile": [64, 64, 1], "opts": {"global_relabel_period": 8}, "ms": 2.0}}
    assert autotune.batch_schedule(small + big, table) == {"global_relabel_period": 8}
    assert autotune.choose(small[1], table) == ((32, 32, 1), {"global_relabel_period": 0})


def test_committed_traffic_belongs_to_the_current_kernel_source():
    p = os.path.join(ROOT, "profiles", "ard_discharge_seg2d_2048_c8.txt")
    src = os.path.join(ROOT, "paper_1109_1146_gb300", "csrc", "ard_discharge2d.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    recorded = [ln.split("=", 1)[1].strip() for ln in open(p) if ln.startswith("bench: kernel_sha256_16=")]
    kname = bench.kernel_name(8, (32, 32, 1))
    assert kname == "ard_discharge2d_kernel<8,32,32,256>"
    v = bench.committed_traffic(kname, (32, 32, 1))
    if recorded == [sha]:
        assert v is not None and 20.0 < v < 200.0
    else:
        assert v is None  # a stale figure is never reported
    assert bench.committed_traffic(kname, (64, 64, 1)) is None  # measured for 32x32 tiles only
    assert bench.committed_traffic(bench.kernel_name(6, (32, 8, 4), batch=True), (32, 8, 4)) is None or recorded


def test_batch_kinds_and_the_3d_traffic_figure():
    # the batched line's sub-workloads keep only their members, in batch order
    d3 = bench.batch_instances(0, count=2, kind="3d")
    assert [x.conn for x in d3] == [6, 6] and all(x.dims[0] == x.dims[1] == x.dims[2] for x in d3)
    d2 = bench.batch_instances(0, count=2, kind="2d")
    assert [x.conn for x in d2] == [4, 4]
    # the committed DRAM figure of the dominant kernel belongs to its source, or is not reported
    p = os.path.join(ROOT, "profiles", "ard_discharge3d_batch_3d24.txt")
    src = os.path.join(ROOT, "paper_1109_1146_gb300", "csrc", "ard_discharge3d.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    recorded = [ln.split("=", 1)[1].strip() for ln in open(p) if ln.startswith("bench: kernel_sha256_16=")]
    v = bench.committed_traffic(bench.kernel_name(6, (32, 8, 4), batch=True), (32, 8, 4))
    if recorded == [sha]:
        # rows that did not change are not written back: below the 72 B algorithmic count is possible
        assert v is not None and 20.0 < v < 200.0
    else:
        assert v is None
