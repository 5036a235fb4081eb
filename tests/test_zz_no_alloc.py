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
    lambda: grids.seg2d_256_c4(1),
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


@pytest.mark.parametrize("side,conn,ok", [(2560, 8, True), (2561, 8, False), (3328, 4, True), (3329, 4, False)])
def test_noalloc_size_limit(side, conn, ok):
    """The largest square grids that fit the 8 MiB array: 2560^2 at
    8-connectivity and 3328^2 at 4-connectivity; one more row and column is
    rejected.  An all-zero residual has S_min empty and S_max = V."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    lib = mf.load()
    n = side * side
    res = torch.zeros((conn, n) if ok else (1,), dtype=torch.int32, device=dev)
    tz = torch.zeros(n if ok else 1, dtype=torch.int32, device=dev)
    smin = torch.full((n if ok else 1,), 7, dtype=torch.uint8, device=dev)
    smax = torch.full((n if ok else 1,), 7, dtype=torch.uint8, device=dev)
    dims = (ctypes.c_int64 * 2)(side, side)
    st = lib.mf_min_cut_2d_noalloc(dims, conn, res.data_ptr(), tz.data_ptr(), tz.data_ptr(), smin.data_ptr(),
                                   smax.data_ptr(), None)
    if ok:
        assert st == mf.MF_OK, lib.mf_last_error(None).decode()
        assert int(smin.sum()) == 0 and int(smax.min()) == 1 and int(smax.max()) == 1
    else:
        assert st == mf.MF_EINVAL
        assert "static maximum" in lib.mf_last_error(None).decode()
