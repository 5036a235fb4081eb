"""Region reduction of Sec. 8 on the GPU (mf_region_reduction and
opts.region_reduction) against the oracle.

* The class code of every vertex (strong source, strong sink, weak source,
  weak sink) equals oracle.reduction.region_reduction bit for bit, on random
  and segmentation grids, 2D 4/8-connected and 3D 6-connected, with tiles
  that leave ragged edge regions; the counts add up.
* A solve with the reduction (strong sources merged into s, strong sinks into
  t, the sweeps on the rest) gives Dinic's flow value, S_min and S_max; its
  final preflow is accepted by the independent verifier on the reduced
  network the oracle builds from its own codes; mf_certify certifies it.
"""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity
from oracle.reduction import STRONG_SINK, STRONG_SOURCE, WEAK_SINK, WEAK_SOURCE, reduce_instance, region_reduction
from paper_1109_1146_gb300 import Grid, default_opts, mf

pytestmark = pytest.mark.gpu

CASES = [
    # (instance maker, solver tile, reduction tile)
    (lambda: grids.random_grid((45, 37, 1), 4, 1, cmax=15, tmax=30, p_zero=0.3), (32, 32, 1), (8, 8, 1)),
    (lambda: grids.random_grid((40, 33, 1), 8, 2, cmax=15, tmax=30, p_zero=0.3), (32, 32, 1), (8, 6, 1)),
    (lambda: grids.segmentation_2d(70, 50, 3, conn=4), (32, 32, 1), (32, 32, 1)),
    (lambda: grids.segmentation_2d(66, 41, 4, conn=8, hard_seed_frac=0.05), (32, 32, 1), (16, 16, 1)),
    (lambda: grids.random_grid((14, 11, 9), 6, 5, cmax=15, tmax=30, p_zero=0.3), (32, 8, 4), (4, 4, 4)),
    (lambda: grids.volume_3d(36, 20, 11, 6), (32, 8, 4), (32, 8, 4)),
]


@pytest.mark.parametrize("make,tile,rtile", CASES)
def test_codes_match_the_oracle(make, tile, rtile):
    inst = make()
    want = region_reduction(inst.dims, inst.conn, rtile, inst.cs, inst.ct, inst.nlink)["codes"]
    with Grid(inst.dims, inst.conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        codes, counts = g.region_reduction(tile=rtile)
    bad = np.flatnonzero(codes != want)
    assert bad.size == 0, f"codes differ at {bad[:10]}: gpu {codes[bad[:10]]} oracle {want[bad[:10]]}"
    assert counts == [int(((want & b) != 0).sum()) for b in (STRONG_SOURCE, STRONG_SINK, WEAK_SOURCE, WEAK_SINK)]


@pytest.mark.parametrize("make,tile,rtile", CASES)
@pytest.mark.parametrize("graph", [0, 1])
def test_solve_with_reduction_is_exact(make, tile, rtile, graph):
    inst = make()
    ref = oracle.solve_instance(inst)
    with Grid(inst.dims, inst.conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st = g.solve(default_opts(region_reduction=1, graph_loop=graph))
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
        ok, cut, bad = g.certify()
        assert ok and cut == ref["flow"] and bad == 0
        codes, _ = g.region_reduction()  # the codes this solve used (the solver's tile)
    assert_parity(inst, got, ref=ref, verify=False)
    assert st.reduced_vertices == int(((codes & (STRONG_SOURCE | STRONG_SINK)) != 0).sum())
    # the final preflow is a maximum preflow of the reduced network
    cs2, ct2, nl2, K = reduce_instance(inst.dims, inst.conn, inst.cs, inst.ct, inst.nlink, codes)
    S, T = (codes & STRONG_SOURCE) != 0, (codes & STRONG_SINK) != 0
    smin_red = got["smin"].astype(bool) & ~S
    smax_red = got["smax"].astype(bool) | T
    ok, msg, info = oracle.verify(inst.dims, inst.conn, cs2, ct2, nl2, got["res"], got["tres"], got["exc"],
                                  got["flow"] - K, smin_red.astype(np.uint8), smax_red.astype(np.uint8))
    assert ok, msg


def test_reduction_in_a_batch_is_exact():
    insts = [grids.segmentation_2d(90, 70, 7, conn=4), grids.volume_3d(40, 24, 12, 8),
             grids.random_grid((50, 40, 1), 8, 9, cmax=15, tmax=30, p_zero=0.3)]
    handles = []
    for x in insts:
        g = Grid(x.dims, x.conn)
        g.set_caps(x.cs, x.ct, x.nlink)
        handles.append(g)
    stats = mf.solve_batch(handles, default_opts(region_reduction=1, graph_loop=1))
    for x, g, st in zip(insts, handles, stats):
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        assert_parity(x, got, verify=False)
        assert st.reduced_vertices > 0
        g.close()


def test_reduction_rejects_warm_start_and_oversized_tiles():
    inst = grids.seg2d_256_c4(0)
    with Grid(inst.dims, 4, tile=(64, 64, 1)) as g:
        with pytest.raises(mf.MFError) as ei:
            g.region_reduction()  # before set_caps
        assert ei.value.status == mf.MF_ESTATE
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        with pytest.raises(mf.MFError) as ei:
            g.region_reduction(tile=(128, 128, 1))  # its region network does not fit shared memory
        assert ei.value.status == mf.MF_EINVAL
        codes, counts = g.region_reduction()
        assert counts[0] + counts[1] > 0
