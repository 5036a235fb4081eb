"""Discharge = PRD (the push-relabel region discharge of Sec. 3), run by the
same parallel sweep (Algorithm 2) as ARD: kernel_variant = 2.

* Exact results: flow value, S_min and S_max equal to Dinic, the final
  preflow verified, on random and segmentation grids (2D 4/8-connected, 3D),
  with the host and the graph sweep loop, with and without the global
  relabel, in batches, and on the paper's synthetic 4-connected family
  (Sec. 7.1: excess U[-500, 500], constant strength).
* Per-sweep invariants of push-relabel: feasible preflow, labels valid for
  unit arc lengths (d(u) <= d(w) + 1 on every residual arc, d(u) <= 1 where
  u -> t), labels never decrease, d_inf = n.
"""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity, gpu_solve
from paper_1109_1146_gb300 import Grid, default_opts, mf
from test_gpu_invariants import _arc_targets

pytestmark = pytest.mark.gpu

CASES = [
    (lambda: grids.random_grid((70, 45, 1), 4, 1, cmax=20, tmax=40, p_zero=0.3), (32, 32, 1)),
    (lambda: grids.segmentation_2d(90, 70, 2, conn=8, hard_seed_frac=0.04), (32, 32, 1)),
    (lambda: grids.segmentation_2d(130, 100, 3, conn=4), (64, 64, 1)),
    (lambda: grids.paper_synthetic(120, 90, 4, strength=150), (32, 32, 1)),
    (lambda: grids.paper_synthetic(100, 100, 5, strength=40), (64, 32, 1)),
    (lambda: grids.volume_3d(40, 30, 20, 6), (32, 8, 4)),
    (lambda: grids.random_grid((20, 18, 17), 6, 7, cmax=20, tmax=40, p_zero=0.3), (8, 8, 8)),
]


@pytest.mark.parametrize("make,tile", CASES)
@pytest.mark.parametrize("graph,glr", [(0, 4), (1, 4), (0, 0)])
def test_prd_is_exact(make, tile, graph, glr):
    inst = make()
    got = gpu_solve(inst, tile=tile, opts=default_opts(kernel_variant=2, graph_loop=graph,
                                                         global_relabel_period=glr))
    assert_parity(inst, got)
    assert got["dinf"] == inst.n


@pytest.mark.parametrize("make,tile", CASES[:4] + CASES[5:6])
def test_prd_sweep_invariants(make, tile):
    inst = make()
    targets = _arc_targets(inst.dims, inst.conn)
    with Grid(inst.dims, inst.conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        # with the global relabel every 4th sweep (its region distances are valid
        # unit-length labels too); without it, excess that cannot reach t climbs
        # one label per sweep up to d_inf = n
        g.begin(default_opts(kernel_variant=2, global_relabel_period=4))
        prev = None
        for _ in range(10000):
            active = g.sweep()
            res, tres, exc = g.get_residual()
            lab, dinf = g.get_labels()
            assert dinf == inst.n
            assert (res >= 0).all() and (tres >= 0).all() and (exc >= 0).all()
            assert (lab >= 0).all() and (lab <= dinf).all()
            assert (lab[tres > 0] <= 1).all()
            for d, t in enumerate(targets):
                ok = (t >= 0) & (res[d] > 0)
                u = np.flatnonzero(ok)
                bad = lab[u] > lab[t[ok]].astype(np.int64) + 1
                assert not bad.any(), f"unit-length labeling invalid on {bad.sum()} arcs"
            if prev is not None:
                assert (lab >= prev).all(), "a label decreased"
            prev = lab
            if active == 0:
                break
        else:
            raise AssertionError("no termination")
        g.finish()
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
    assert_parity(inst, got, verify=False)


def test_prd_in_a_batch_and_against_ard():
    insts = [grids.paper_synthetic(150, 120, 8, strength=150), grids.segmentation_2d(100, 80, 9, conn=4),
             grids.volume_3d(36, 24, 16, 10)]
    refs = [oracle.solve_instance(x) for x in insts]
    for variant in (0, 2):
        handles = []
        for x in insts:
            g = Grid(x.dims, x.conn)
            g.set_caps(x.cs, x.ct, x.nlink)
            handles.append(g)
        stats = mf.solve_batch(handles, default_opts(kernel_variant=variant, graph_loop=1))
        for x, g, ref in zip(insts, handles, refs):
            got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
            assert_parity(x, got, ref=ref, verify=False)
            g.close()
        assert all(s.sweeps > 0 for s in stats)


def test_prd_rejects_warm_start_and_reduction():
    inst = grids.seg2d_256_c4(0)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        for kw in (dict(region_reduction=1), dict(kernel_variant=3)):
            with pytest.raises(mf.MFError) as ei:
                g.solve(default_opts(kernel_variant=2, **kw) if "region_reduction" in kw else default_opts(**kw))
            assert ei.value.status == mf.MF_EINVAL
