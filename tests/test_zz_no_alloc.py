"""The allocation-free cut extraction (mf_min_cut_2d_noalloc) against the
regular one.

It exists for callers that may not allocate device memory at call time (a
framework that owns all device memory through a fixed-budget pool, or a
latency-critical loop where cudaMalloc is not allowed after start-up).  It must
give exactly the cuts that mf_get_cut gives after mf_solve, on consecutive
calls that reuse its one static scratch array.  This file is collected last
so that a failure here stops a -x run only after every other test ran.
"""
import ctypes

import numpy as np
import pytest

from gen import grids
from paper_1109_1146_gb300 import Grid, mf

pytestmark = pytest.mark.gpu


def _solve_and_residual(inst, torch, dev):
    g = Grid(inst.dims, inst.conn)
    g.set_caps(inst.cs, inst.ct, inst.nlink)
    g.solve()
    n = inst.n
    res = torch.empty((inst.conn, n), dtype=torch.int32, device=dev)
    tres = torch.empty(n, dtype=torch.int32, device=dev)
    exc = torch.empty(n, dtype=torch.int32, device=dev)
    lib = mf.load()
    st = lib.mf_get_residual(g._h, res.data_ptr(), tres.data_ptr(), exc.data_ptr(), 1)
    assert st == mf.MF_OK
    return g, res, tres, exc


@pytest.mark.parametrize("make", [
    lambda: grids.segmentation_2d(300, 170, 3, conn=8, hard_seed_frac=0.05),
    lambda: grids.config0(1),
    lambda: grids.random_grid((129, 65, 1), 4, 7, cmax=20, tmax=40),
])
def test_noalloc_cut_matches_solver_cut(make):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    inst = make()
    g, res, tres, exc = _solve_and_residual(inst, torch, dev)
    want_min, want_max = g.get_cut(0), g.get_cut(1)
    for _ in range(2):  # consecutive calls share the static scratch
        smin = torch.full((inst.n,), 7, dtype=torch.uint8, device=dev)
        smax = torch.full((inst.n,), 7, dtype=torch.uint8, device=dev)
        mf.min_cut_2d_noalloc(inst.dims[:2], inst.conn, res, tres, exc, smin, smax)
        np.testing.assert_array_equal(smin.cpu().numpy(), want_min)
        np.testing.assert_array_equal(smax.cpu().numpy(), want_max)
    g.close()


def test_noalloc_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    lib = mf.load()
    buf = torch.zeros(64, dtype=torch.int32, device=dev)
    out = torch.zeros(64, dtype=torch.uint8, device=dev)
    dims = (ctypes.c_int64 * 2)(4096, 4096)  # needs 20 MiB of scratch at 8-connectivity
    st = lib.mf_min_cut_2d_noalloc(dims, 8, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(), out.data_ptr(),
                                   out.data_ptr(), None)
    assert st == mf.MF_EINVAL
    assert "static maximum" in lib.mf_last_error(None).decode()
