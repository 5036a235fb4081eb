"""Batched persistent solve (mf_solve_batch): many grids of uneven sizes,
mixed connectivities and tile shapes in one sweep loop.  Every instance must
match the oracle bit-exactly and agree with its own single solve (same
sweeps: the batch runs the same per-instance sequence of operations)."""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity
from paper_1109_1146_gb300 import Grid, default_opts, mf

pytestmark = pytest.mark.gpu


def _batch_instances():
    out = []
    out.append((grids.segmentation_2d(100, 90, 1, conn=4), (64, 64, 1)))
    out.append((grids.segmentation_2d(64, 64, 2, conn=4), (64, 64, 1)))
    out.append((grids.segmentation_2d(213, 150, 3, conn=4, hard_seed_frac=0.05), (64, 64, 1)))
    out.append((grids.segmentation_2d(97, 61, 4, conn=4), (32, 32, 1)))
    out.append((grids.segmentation_2d(120, 75, 13, conn=4), (32, 16, 1)))
    out.append((grids.segmentation_2d(90, 66, 14, conn=8), (32, 16, 1)))
    out.append((grids.segmentation_2d(130, 170, 5, conn=8, hard_seed_frac=0.05), (64, 64, 1)))
    out.append((grids.random_grid((77, 55, 1), 8, 6, cmax=30, tmax=60, p_zero=0.3), (32, 32, 1)))
    out.append((grids.volume_3d(30, 28, 26, 7), (16, 16, 16)))
    out.append((grids.volume_3d(20, 20, 20, 8), (8, 8, 8)))
    out.append((grids.volume_3d(50, 30, 17, 9), (32, 16, 8)))
    out.append((grids.volume_3d(40, 25, 20, 10), (32, 8, 8)))
    out.append((grids.volume_3d(45, 22, 18, 11), (32, 4, 4)))
    out.append((grids.volume_3d(36, 24, 9, 12), (32, 8, 2)))
    out.append((grids.random_grid((5, 1, 1), 4, 9, cmax=10, tmax=20), (64, 64, 1)))
    return out


@pytest.mark.parametrize("kw", [dict(global_relabel_period=0), dict(partial_discharge=1, global_relabel_period=0),
                                dict(global_relabel_period=0, graph_loop=1),
                                dict(partial_discharge=1, global_relabel_period=0, graph_loop=1),
                                dict(global_relabel_period=2), dict(global_relabel_period=3, graph_loop=1),
                                dict(global_relabel_period=8, global_relabel_first=1),
                                dict(global_relabel_period=4, global_relabel_first=1, graph_loop=1)])
def test_batch_matches_oracle_and_single_solves(kw):
    insts = _batch_instances()
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
        assert st.flow_value == got["flow"]
        # the same instance alone
        with Grid(inst.dims, inst.conn, tile=tile) as h:
            h.set_caps(inst.cs, inst.ct, inst.nlink)
            s1 = h.solve(opts)
            assert s1.sweeps == st.sweeps
            assert s1.discharges == st.discharges
            # counters and level counts reach the host through the batch's
            # own read-back launches: the same values as the single solve's
            assert (s1.stages, s1.rounds, s1.discharged_vertices) == (st.stages, st.rounds, st.discharged_vertices)
            assert (s1.global_relabels, s1.relabel_levels) == (st.global_relabels, st.relabel_levels)
            assert st.cut_passes >= 2  # each of the two closures makes at least one pass
    for g in handles:
        g.close()


@pytest.mark.parametrize("kw", [dict(global_relabel_period=2), dict(global_relabel_period=2, graph_loop=1)])
def test_batch_with_instances_done_at_init(kw):
    # grids with nothing to do (all capacities zero) or only terminal links
    # (what Init leaves cannot move) finish before the first sweep; they must
    # keep exact results while the others sweep, relabel and cut beside them
    insts = [(grids.random_grid((70, 40, 1), 4, 1, cmax=0, tmax=0), (32, 32, 1)),
             (grids.random_grid((66, 50, 1), 8, 2, cmax=0, tmax=50), (64, 64, 1)),
             (grids.segmentation_2d(150, 120, 3, conn=4), (32, 32, 1)),
             (grids.random_grid((40, 30, 20), 6, 4, cmax=0, tmax=0), (32, 8, 4)),
             (grids.volume_3d(45, 30, 21, 5), (32, 8, 4)),
             (grids.random_grid((33, 17, 9), 6, 6, cmax=0, tmax=40), (32, 4, 4))]
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
        assert st.flow_value == got["flow"]
        with Grid(inst.dims, inst.conn, tile=tile) as h:
            h.set_caps(inst.cs, inst.ct, inst.nlink)
            s1 = h.solve(opts)
            assert (s1.sweeps, s1.discharges, s1.stages) == (st.sweeps, st.discharges, st.stages)
    assert stats[0].flow_value == 0 and stats[3].flow_value == 0
    for g in handles:
        g.close()


@pytest.mark.parametrize("graph_loop", [0, 1])
def test_batch_sweep_cap_then_exact_solve(graph_loop):
    # a sweep cap below what the instances need ends the batch with
    # MF_ESWEEPLIMIT; the grids stay usable and a full batched solve is exact
    insts = [(grids.segmentation_2d(150, 120, 7, conn=4), (32, 32, 1)),
             (grids.volume_3d(45, 30, 21, 8), (32, 8, 4))]
    handles = []
    for inst, tile in insts:
        g = Grid(inst.dims, inst.conn, tile=tile)
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        handles.append(g)
    with pytest.raises(mf.MFError) as err:
        mf.solve_batch(handles, default_opts(max_sweeps=1, graph_loop=graph_loop))
    assert err.value.status == mf.MF_ESWEEPLIMIT
    with pytest.raises(mf.MFError) as err:  # no finished solve, so no cut to read
        mf.get_cuts_batch(handles, 0)
    assert err.value.status == mf.MF_ESTATE
    mf.solve_batch(handles, default_opts(graph_loop=graph_loop))
    for (inst, tile), g in zip(insts, handles):
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        assert_parity(inst, got)
        g.close()


def test_batch_of_one_and_repeat():
    inst = grids.seg2d_256_c4(3)
    ref = oracle.solve_instance(inst)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        for _ in range(2):
            mf.solve_batch([g])
            assert g.flow_value() == ref["flow"]
            np.testing.assert_array_equal(g.get_cut(0), ref["smin"])


def test_batch_rejects_bad_input():
    inst = grids.seg2d_256_c4(0)
    a = Grid(inst.dims, 4)
    with pytest.raises(mf.MFError):
        mf.solve_batch([a])  # no capacities yet
    a.set_caps(inst.cs, inst.ct, inst.nlink)
    with pytest.raises(mf.MFError):
        mf.solve_batch([a, a])  # the same grid twice
    a.close()


def test_batched_set_caps_and_cut_reads():
    # mf_set_caps_batch / mf_get_cuts_batch: the same state and results as the
    # per-grid calls, host and device buffers, errors reported for the batch
    import torch
    insts = [grids.segmentation_2d(90, 70, 21, conn=4), grids.volume_3d(40, 30, 20, 22),
             grids.random_grid((70, 50, 1), 8, 23, cmax=20, tmax=40, p_zero=0.3)]
    refs = [oracle.solve_instance(x) for x in insts]
    handles = [Grid(x.dims, x.conn) for x in insts]
    for device in (False, True):
        caps = [(x.cs, x.ct, x.nlink) for x in insts]
        if device:
            caps = [tuple(torch.from_numpy(a).cuda() for a in c) for c in caps]
        mf.set_caps_batch(handles, caps)
        mf.solve_batch(handles, default_opts(graph_loop=1))
        outs = None if not device else [torch.empty(x.n, dtype=torch.uint8, device="cuda") for x in insts]
        outs, flows = mf.get_cuts_batch(handles, 0, outs)
        smax, _ = mf.get_cuts_batch(handles, 1)
        for x, ref, o, f, sm, g in zip(insts, refs, outs, flows, smax, handles):
            o = o.cpu().numpy() if device else o
            assert f == ref["flow"] == g.flow_value()
            np.testing.assert_array_equal(o, ref["smin"])
            np.testing.assert_array_equal(sm, ref["smax"])
    # pinned host buffers (the gathered copy and the batched validation)
    pinned = [tuple(torch.from_numpy(a).pin_memory() for a in (x.cs, x.ct, x.nlink)) for x in insts]
    mf.set_caps_batch(handles, pinned)
    mf.solve_batch(handles, default_opts())
    outs, flows = mf.get_cuts_batch(handles, 0)
    for ref, o, f in zip(refs, outs, flows):
        assert f == ref["flow"]
        np.testing.assert_array_equal(o, ref["smin"])
    # a negative capacity, a link leaving the grid or an overflow in one grid:
    # the batch fails with that grid's status (pageable, pinned and device buffers)
    for kind, status in (("negative", mf.MF_EINVAL), ("leaving", mf.MF_EINVAL), ("overflow", mf.MF_EOVERFLOW)):
        cs, nl = insts[1].cs.copy(), insts[1].nlink.copy()
        if kind == "negative":
            cs[5] = -1
        elif kind == "leaving":
            X = insts[1].dims[0]
            nl[0, X - 1] = 3  # the +x link of the last column
        else:
            cs[7] = 2 ** 31 - 2
        caps = [(insts[0].cs, insts[0].ct, insts[0].nlink), (cs, insts[1].ct, nl),
                (insts[2].cs, insts[2].ct, insts[2].nlink)]
        for mode in ("pageable", "pinned", "device"):
            if mode == "pinned":
                cc = [tuple(torch.from_numpy(a).pin_memory() for a in c) for c in caps]
            elif mode == "device":
                cc = [tuple(torch.from_numpy(a).cuda() for a in c) for c in caps]
            else:
                cc = caps
            with pytest.raises(mf.MFError) as ei:
                mf.set_caps_batch(handles, cc)
            assert ei.value.status == status, (kind, mode)
    # a grid without a finished solve: MF_ESTATE
    with pytest.raises(mf.MFError) as ei:
        mf.get_cuts_batch(handles, 0)
    assert ei.value.status == mf.MF_ESTATE
    for g in handles:
        g.close()


def test_flow_value_follows_extra_sweeps():
    # the flow value read back with a finished solve is returned without a
    # device read; a later sweep invalidates it
    inst = grids.segmentation_2d(120, 90, 24, conn=4)
    ref = oracle.solve_instance(inst)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.solve(default_opts())
        assert g.flow_value() == ref["flow"]
        g.begin(default_opts())  # a new solve: the finished one's value no longer holds
        assert g.flow_value() <= ref["flow"]
        g.sweep()
        partial = g.flow_value()
        while g.sweep():
            pass
        g.finish()
        assert g.flow_value() == ref["flow"] >= partial
