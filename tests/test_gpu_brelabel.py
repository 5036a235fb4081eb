"""Boundary-relabel heuristic (Sec. 6.1) on the GPU against the oracle.

* After real sweeps of the solver (2D 4/8-connected, 3D 6-connected, the
  bit-parallel and the generic tiles, with and without partial discharges),
  the state is downloaded, the oracle's boundary relabel is applied to it, and
  mf_boundary_relabel must leave exactly the same labels (bit for bit), with
  no staircase merged; the labeling it starts from must be valid in the strong
  form the heuristic relies on.
* Solves with the heuristic after every sweep (alone, with the global
  relabel, in the CUDA-graph loop, in a batch) must end with the oracle's
  flow, S_min and S_max, and a batch must take each instance's single-solve
  sweeps.
"""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity
from paper_1109_1146_gb300 import Grid, default_opts, mf

pytestmark = pytest.mark.gpu

FWD = grids.FWD


def _targets(dims, conn):
    X, Y, Z = dims
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    out = []
    for dx, dy, dz in FWD[conn]:
        for sg in (1, -1):
            x2, y2, z2 = xx + sg * dx, yy + sg * dy, zz + sg * dz
            ok = (x2 >= 0) & (x2 < X) & (y2 >= 0) & (y2 < Y) & (z2 >= 0) & (z2 < Z)
            out.append(np.where(ok, (z2 * Y + y2) * X + x2, -1).ravel())
    return out


def _regions(dims, tile):
    X, Y, Z = dims
    tx, ty, tz = tile
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return ((zz // tz * -(-Y // ty) + yy // ty) * -(-X // tx) + xx // tx).ravel()


def _strong_violations(dims, conn, tile, res, tres, lab):
    reg = _regions(dims, tile)
    bad = int((lab[tres > 0] != 0).sum())
    for d, t in enumerate(_targets(dims, conn)):
        u = np.flatnonzero((t >= 0) & (res[d] > 0))
        w = t[u]
        slack = (reg[u] != reg[w]).astype(np.int64)
        bad += int((lab[u].astype(np.int64) > lab[w].astype(np.int64) + slack).sum())
    return bad


def _instance(conn, dims, seed):
    if conn == 6:
        return grids.volume_3d(*dims, seed=seed)
    return grids.segmentation_2d(dims[0], dims[1], seed, conn=conn, hard_seed_frac=0.04)


CASES = [(4, (150, 120, 1), (32, 32, 1), 0), (4, (130, 100, 1), (64, 64, 1), 1), (8, (140, 90, 1), (32, 32, 1), 0),
         (8, (150, 100, 1), (64, 32, 1), 0), (6, (70, 30, 18), (32, 8, 4), 0), (6, (40, 36, 30), (16, 16, 16), 0),
         (6, (30, 20, 17), (8, 8, 8), 1), (6, (70, 36, 20), (32, 16, 8), 0)]


@pytest.mark.parametrize("conn,dims,tile,partial", CASES)
def test_boundary_relabel_matches_oracle(conn, dims, tile, partial):
    inst = _instance(conn, dims, 3)
    checked = raised = 0
    with Grid(inst.dims, conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.begin(default_opts(partial_discharge=partial, global_relabel_period=0))
        for s in range(60):
            active = g.sweep()
            if active == 0:
                break
            if s in (0, 1, 2, 4, 8, 16, 32):
                res, tres, _ = g.get_residual()
                lab, dinf = g.get_labels()
                assert _strong_violations(inst.dims, conn, tile, res, tres, lab) == 0
                want = oracle.boundary_relabel(inst.dims, conn, tile, res, lab, dinf)
                info = g.boundary_relabel()
                got, _ = g.get_labels()
                assert info["applied"] and info["merged"] == 0
                np.testing.assert_array_equal(got, want)
                assert info["active"] == int(np.unique(_regions(inst.dims, tile)[
                    (g.get_residual()[2] > 0) & (got < dinf)]).size)
                checked += 1
                raised += int((got > lab).sum())
        g.finish()
        ref = oracle.solve_instance(inst)
        assert g.flow_value() == ref["flow"]
        np.testing.assert_array_equal(g.get_cut(0), ref["smin"])
        np.testing.assert_array_equal(g.get_cut(1), ref["smax"])
    assert checked >= 2
    assert raised > 0  # the heuristic did something on these states


def test_boundary_relabel_on_the_initial_state():
    # after Init every label is 0: every group is a target and nothing changes
    inst = _instance(4, (100, 70, 1), 1)
    with Grid(inst.dims, 4, tile=(32, 32, 1)) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.begin(default_opts())
        info = g.boundary_relabel()
        lab, _ = g.get_labels()
        assert info["applied"] and (lab == 0).all()


def test_boundary_relabel_needs_begin():
    inst = _instance(4, (40, 30, 1), 1)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        with pytest.raises(mf.MFError):
            g.boundary_relabel()


SOLVES = [(4, (257, 190, 1), (32, 32, 1)), (8, (300, 170, 1), (32, 32, 1)), (8, (200, 150, 1), (64, 64, 1)),
          (6, (64, 40, 30), (32, 8, 4)), (6, (40, 33, 29), (16, 16, 16))]


@pytest.mark.parametrize("conn,dims,tile", SOLVES)
@pytest.mark.parametrize("kw", [dict(boundary_relabel_period=1, global_relabel_period=0),
                                dict(boundary_relabel_period=1, global_relabel_period=4),
                                dict(boundary_relabel_period=2, global_relabel_period=0, partial_discharge=1),
                                dict(boundary_relabel_period=1, global_relabel_period=0, graph_loop=1),
                                dict(boundary_relabel_period=3, global_relabel_period=2, graph_loop=1)])
def test_solve_with_boundary_relabel(conn, dims, tile, kw):
    inst = _instance(conn, dims, 7)
    with Grid(inst.dims, conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st = g.solve(default_opts(**kw))
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
    assert_parity(inst, got)
    if st.sweeps > 1:
        assert st.boundary_relabels >= 1
    assert st.sweeps <= oracle.sweep_bound(inst.dims, conn, tile)


def test_graph_loop_takes_the_host_loop_sweeps():
    inst = _instance(8, (300, 200, 1), 11)
    out = []
    for gl in (0, 1):
        with Grid(inst.dims, 8, tile=(32, 32, 1)) as g:
            g.set_caps(inst.cs, inst.ct, inst.nlink)
            st = g.solve(default_opts(boundary_relabel_period=2, global_relabel_period=3, graph_loop=gl))
            out.append((st.sweeps, st.discharges, st.boundary_relabels, st.global_relabels, g.flow_value()))
    assert out[0] == out[1]


@pytest.mark.parametrize("kw", [dict(boundary_relabel_period=1, global_relabel_period=0),
                                dict(boundary_relabel_period=1, global_relabel_period=3),
                                dict(boundary_relabel_period=2, global_relabel_period=0, graph_loop=1)])
def test_batch_with_boundary_relabel(kw):
    insts = [(grids.segmentation_2d(150, 110, 1, conn=4), (32, 32, 1)),
             (grids.segmentation_2d(130, 170, 5, conn=8, hard_seed_frac=0.05), (64, 64, 1)),
             (grids.volume_3d(40, 25, 20, 10), (32, 8, 4)),
             (grids.volume_3d(30, 28, 26, 7), (16, 16, 16)),
             (grids.random_grid((5, 1, 1), 4, 9, cmax=10, tmax=20), (32, 32, 1))]
    opts = default_opts(**kw)
    handles = []
    for inst, tile in insts:
        g = Grid(inst.dims, inst.conn, tile=tile)
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        handles.append(g)
    stats = mf.solve_batch(handles, opts)
    for (inst, tile), g, st in zip(insts, handles, stats):
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
        assert_parity(inst, got)
        with Grid(inst.dims, inst.conn, tile=tile) as h:
            h.set_caps(inst.cs, inst.ct, inst.nlink)
            s1 = h.solve(opts)
            assert (s1.sweeps, s1.discharges, s1.boundary_relabels) == (st.sweeps, st.discharges,
                                                                         st.boundary_relabels)
    for g in handles:
        g.close()
