"""Per-sweep invariants of P-ARD on the GPU state (Sec. 4.4, Statement on the
properties of the parallel sweep), checked on the CPU after every sweep:

  * the preflow is feasible (capacity, antisymmetry, e >= 0);
  * the labeling is valid for the region distance (Sec. 4.1):
        d(u) <= d(w) + 1 on residual arcs with both ends in B,
        d(u) <= d(w)     on the other residual arcs,  d(u) = 0 if c_f(u,t) > 0;
  * labels never decrease (labeling monotony);
  * after a sweep no vertex outside B is active (optimality), when partial
    discharges are off;
  * the sweep count stays within 2|B|^2 + 1.
"""
import numpy as np
import pytest

import oracle
from gen import grids
from paper_1109_1146_gb300 import Grid, default_opts

pytestmark = pytest.mark.gpu

_FWD = grids.FWD


def _arc_targets(dims, conn):
    """For every arc direction d: target index of each vertex (-1 outside)."""
    X, Y, Z = dims
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    out = []
    for h, (dx, dy, dz) in enumerate(_FWD[conn]):
        for sg in (1, -1):
            x2, y2, z2 = xx + sg * dx, yy + sg * dy, zz + sg * dz
            ok = (x2 >= 0) & (x2 < X) & (y2 >= 0) & (y2 < Y) & (z2 >= 0) & (z2 < Z)
            t = np.where(ok, (z2 * Y + y2) * X + x2, -1)
            out.append(t.ravel())
    return out


def check_state(inst, res, tres, exc, lab, dinf, inB, targets):
    n = inst.n
    assert (res >= 0).all() and (tres >= 0).all() and (exc >= 0).all()
    assert (tres <= inst.ct).all()
    # antisymmetry + excess recomputed from residuals
    e = inst.cs.astype(np.int64) - (inst.ct.astype(np.int64) - tres)
    for d, t in enumerate(targets):
        ok = t >= 0
        h = d >> 1
        c = np.where(d & 1, 0, inst.nlink[h]).astype(np.int64)
        if d & 1:
            c = np.zeros(n, np.int64)
            c[ok] = inst.nlink[h][t[ok]]
        assert (res[d][~ok] == 0).all()
        back = np.zeros(n, np.int64)
        back[ok] = res[d ^ 1][t[ok]]
        assert (res[d][ok].astype(np.int64) + back[ok] == 2 * c[ok]).all()
        e -= np.where(ok, c - res[d], 0)
    assert (e == exc).all()
    # validity of the labeling
    assert (lab >= 0).all() and (lab <= dinf).all()
    assert (lab[tres > 0] == 0).all()
    for d, t in enumerate(targets):
        ok = (t >= 0) & (res[d] > 0)
        u = np.flatnonzero(ok)
        w = t[ok]
        slack = (inB[u] & inB[w]).astype(np.int64)
        bad = lab[u] > lab[w].astype(np.int64) + slack
        assert not bad.any(), f"labeling invalid on {bad.sum()} arcs (dir {d})"


@pytest.mark.parametrize("conn,dims,tile,partial", [
    (4, (192, 160, 1), (64, 64, 1), 0), (8, (150, 130, 1), (64, 64, 1), 0),
    (8, (100, 90, 1), (32, 32, 1), 0), (4, (120, 96, 1), (32, 32, 1), 1), (8, (140, 70, 1), (64, 32, 1), 0),
    (8, (90, 70, 1), (32, 16, 1), 0), (4, (100, 60, 1), (32, 16, 1), 1),
    (6, (40, 36, 30), (16, 16, 16), 0), (6, (24, 20, 18), (8, 8, 8), 1),
    (6, (70, 36, 20), (32, 16, 8), 0), (6, (40, 20, 18), (32, 8, 8), 1), (6, (50, 20, 14), (32, 8, 4), 0),
    (6, (45, 18, 14), (32, 4, 4), 0), (6, (40, 20, 9), (32, 8, 2), 1)])
@pytest.mark.parametrize("variant,glr", [(0, 0), (1, 0), (0, 1)])
def test_sweep_invariants(conn, dims, tile, partial, variant, glr):
    inst = (grids.volume_3d(*dims, seed=2) if conn == 6 else
            grids.segmentation_2d(dims[0], dims[1], 2, conn=conn, hard_seed_frac=0.04))
    inB = oracle.boundary_mask(inst.dims, conn, tile)
    targets = _arc_targets(inst.dims, conn)
    bound = oracle.sweep_bound(inst.dims, conn, tile)
    with Grid(inst.dims, conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.begin(default_opts(partial_discharge=partial, kernel_variant=variant, global_relabel_period=glr))
        prev, dinf = g.get_labels()
        sweeps = 0
        while True:
            active = g.sweep()
            sweeps += 1
            res, tres, exc = g.get_residual()
            lab, dinf = g.get_labels()
            check_state(inst, res, tres, exc, lab, dinf, inB, targets)
            assert (lab >= prev).all(), "labels decreased"
            if not partial:
                act = (exc > 0) & (lab < dinf)
                assert not (act & ~inB).any(), "active vertex outside B after a sweep"
            prev = lab
            if active == 0:
                break
            assert sweeps <= bound
        g.finish()
        ref = oracle.solve_instance(inst)
        assert g.flow_value() == ref["flow"]
        np.testing.assert_array_equal(g.get_cut(0), ref["smin"])


@pytest.mark.parametrize("make", [
    lambda: grids.segmentation_2d(300, 170, 4, conn=4, hard_seed_frac=0.02),
    lambda: grids.segmentation_2d(257, 190, 5, conn=8, hard_seed_frac=0.02),
    lambda: grids.volume_3d(40, 33, 29, 6),
])
def test_certificate_agrees_with_oracle(make):
    inst = make()
    ref = oracle.solve_instance(inst)
    with Grid(inst.dims, inst.conn) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.solve()
        ok, cut, bad = g.certify()
        smin = g.get_cut(0)
    assert ok and bad == 0
    assert cut == ref["flow"]
    assert cut == oracle.cut_cost(inst.dims, inst.conn, inst.cs, inst.ct, inst.nlink, smin)


def test_certify_needs_a_finished_solve():
    inst = grids.random_grid((20, 20, 1), 4, 1)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        with pytest.raises(Exception):
            g.certify()


@pytest.mark.parametrize("conn,dims,tile", [(4, (96, 80, 1), (32, 32, 1)), (8, (100, 70, 1), (64, 64, 1)),
                                            (8, (90, 66, 1), (64, 32, 1)), (8, (80, 70, 1), (32, 16, 1)),
                                            (6, (64, 24, 20), (32, 8, 4)),
                                            (6, (40, 30, 20), (32, 8, 8)), (6, (50, 22, 18), (32, 4, 4)),
                                            (6, (40, 20, 11), (32, 8, 2))])
def test_global_relabel_labels_are_region_distances(conn, dims, tile):
    # labels stay lower bounds of the region distance d* (non-increasing on
    # inner residual arcs, +1 at most across regions), so the relabel's
    # max(d, d*) is d* itself: after every sweep with P = 1 the labels equal
    # the oracle's 0-1 BFS distances (d_inf where t is unreachable)
    inst = (grids.volume_3d(*dims, seed=5) if conn == 6 else
            grids.segmentation_2d(dims[0], dims[1], 5, conn=conn, hard_seed_frac=0.03))
    checked = 0
    with Grid(inst.dims, conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.begin(default_opts(global_relabel_period=1))
        for _ in range(500):
            if g.sweep() == 0:
                break
            lab, dinf = g.get_labels()
            res, tres, _ = g.get_residual()
            d = oracle.region_distance(inst.dims, conn, tile, res, tres)
            np.testing.assert_array_equal(lab, np.where(d >= 0, d, dinf))
            checked += 1
        g.finish()
    assert checked >= 1
