"""Grids whose planes live in host (Grace) memory (MF_STATE_HOST): the
kernels stage the regions from pinned host memory over NVLink-C2C and write
them back there.  The results must be those of device placement — flow
value, S_min and S_max equal to Dinic, the final preflow verified, the same
sweeps — for single solves (host and graph loop), the step-wise form, the
warm start and batches that mix both placements."""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity
from paper_1109_1146_gb300 import Grid, default_opts, mf

pytestmark = pytest.mark.gpu

CASES = [
    (lambda: grids.segmentation_2d(200, 130, 1, conn=4), None),
    (lambda: grids.segmentation_2d(170, 140, 2, conn=8, hard_seed_frac=0.05), (64, 64, 1)),
    (lambda: grids.random_grid((97, 61, 1), 8, 3, cmax=30, tmax=60, p_zero=0.3), (32, 32, 1)),
    (lambda: grids.volume_3d(70, 30, 22, 4), None),
    (lambda: grids.volume_3d(40, 35, 20, 5), (16, 16, 16)),
]


def _solve(inst, tile, host, opts=None):
    with Grid(inst.dims, inst.conn, tile=tile, host_state=host) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st = g.solve(opts)
        out = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1), "stats": st}
        out["res"], out["tres"], out["exc"] = g.get_residual()
        out["cert"] = g.certify()
    return out


@pytest.mark.parametrize("make,tile", CASES)
@pytest.mark.parametrize("graph", [0, 1])
def test_host_state_matches_device_state_and_oracle(make, tile, graph):
    inst = make()
    ref = oracle.solve_instance(inst)
    opts = default_opts(graph_loop=graph)
    dev = _solve(inst, tile, False, opts)
    host = _solve(inst, tile, True, opts)
    assert_parity(inst, host, ref=ref)
    assert host["cert"][0] and host["cert"][1] == ref["flow"]
    assert host["stats"].sweeps == dev["stats"].sweeps
    assert host["stats"].discharges == dev["stats"].discharges
    for k in ("res", "tres", "exc"):
        np.testing.assert_array_equal(host[k], dev[k])


def test_host_state_in_a_mixed_batch_and_with_device_inputs():
    import torch
    insts = [grids.segmentation_2d(120, 90, 6, conn=4), grids.volume_3d(50, 40, 20, 7),
             grids.random_grid((80, 70, 1), 8, 8, cmax=20, tmax=40, p_zero=0.3)]
    handles = []
    for k, x in enumerate(insts):
        g = Grid(x.dims, x.conn, host_state=(k != 1))
        if k == 2:  # capacities from device buffers into host-resident planes
            g.set_caps(*(torch.from_numpy(a).cuda() for a in (x.cs, x.ct, x.nlink)))
        else:
            g.set_caps(x.cs, x.ct, x.nlink)
        handles.append(g)
    mf.solve_batch(handles, default_opts(graph_loop=1))
    for x, g in zip(insts, handles):
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
        assert_parity(x, got)
        g.close()


def test_unknown_placement_flag_is_rejected():
    import ctypes
    lib = mf.load()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 3)(16, 16, 1)
    assert lib.mf_create_grid_ex(ctypes.byref(h), 2, dims, 4, None, None, 2) == mf.MF_EINVAL
    assert not h.value
