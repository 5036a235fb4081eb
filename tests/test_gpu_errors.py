"""Error contracts of the C ABI (include/mf.h), called through the binding.

mf_set_caps validates its input on the device: a negative capacity or a
nonzero link leaving the grid is MF_EINVAL; cs(v) plus the capacities of the
edges at v above INT32_MAX, or an edge capacity c with 2c above INT32_MAX, is
MF_EOVERFLOW (the residual arithmetic is int32, Sec. 2's capacities in N0).
mf_solve / mf_begin before a successful mf_set_caps is MF_ESTATE.  After a
rejected input the same handle must accept valid capacities and solve them
exactly (oracle parity)."""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity
from paper_1109_1146_gb300 import Grid, mf

pytestmark = pytest.mark.gpu

INT_MAX = 2 ** 31 - 1


def _base(conn):
    if conn == 6:
        return grids.volume_3d(37, 21, 11, 5)
    return grids.segmentation_2d(70, 45, 5, conn=conn)


def _fh(inst, h):
    """Flat index of forward link h leaving the grid: the last cell along the
    link's positive axis (or the first along a negative x)."""
    X, Y, Z = inst.dims
    dx, dy, dz = grids.FWD[inst.conn][h]
    x = X - 1 if dx > 0 else (0 if dx < 0 else X // 2)
    y = Y - 1 if dy > 0 else Y // 2
    z = Z - 1 if dz > 0 else Z // 2
    return (z * Y + y) * X + x


def _solve_status(g):
    return g._lib.mf_solve(g._h, None, None)


def _expect(g, status, cs, ct, nl, on_device):
    with pytest.raises(mf.MFError) as ei:
        g.set_caps(cs, ct, nl)
    assert ei.value.status == status, str(ei.value)
    # the handle has no valid capacities now
    assert _solve_status(g) == mf.MF_ESTATE


def _bufs(inst, on_device, cs=None, ct=None, nl=None):
    cs = inst.cs if cs is None else cs
    ct = inst.ct if ct is None else ct
    nl = inst.nlink if nl is None else nl
    if not on_device:
        return np.ascontiguousarray(cs), np.ascontiguousarray(ct), np.ascontiguousarray(nl)
    import torch
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (cs, ct, nl))


@pytest.mark.parametrize("conn", [4, 8, 6])
def test_solve_before_set_caps_is_state_error(conn):
    inst = _base(conn)
    with Grid(inst.dims, conn) as g:
        assert _solve_status(g) == mf.MF_ESTATE
        assert g._lib.mf_begin(g._h, None) == mf.MF_ESTATE
        assert "mf_set_caps" in g._lib.mf_last_error(g._h).decode()
        with pytest.raises(mf.MFError) as ei:
            mf.solve_batch([g])
        assert ei.value.status == mf.MF_ESTATE


@pytest.mark.parametrize("on_device", [0, 1])
@pytest.mark.parametrize("conn", [4, 8, 6])
def test_rejected_inputs_then_exact_solve(conn, on_device):
    inst = _base(conn)
    ref = oracle.solve_instance(inst)
    n, H = inst.n, inst.conn // 2
    v = n // 3
    with Grid(inst.dims, conn) as g:
        # negative terminal capacities
        cs = inst.cs.copy(); cs[v] = -1
        _expect(g, mf.MF_EINVAL, *_bufs(inst, on_device, cs=cs), on_device)
        ct = inst.ct.copy(); ct[v] = -5
        _expect(g, mf.MF_EINVAL, *_bufs(inst, on_device, ct=ct), on_device)
        # negative edge capacity
        nl = inst.nlink.copy(); nl[H - 1, v] = -2
        _expect(g, mf.MF_EINVAL, *_bufs(inst, on_device, nl=nl), on_device)
        # a nonzero link leaving the grid, for every forward direction
        for h in range(H):
            nl = inst.nlink.copy(); nl[h, _fh(inst, h)] = 3
            _expect(g, mf.MF_EINVAL, *_bufs(inst, on_device, nl=nl), on_device)
        # cs(v) + sum of the capacities at v above INT32_MAX
        cs = inst.cs.copy(); nl = inst.nlink.copy()
        nl[0, v] = 7
        cs[v] = INT_MAX - 6
        _expect(g, mf.MF_EOVERFLOW, *_bufs(inst, on_device, cs=cs, nl=nl), on_device)
        # one edge with 2c > INT32_MAX (its residual pair could not be stored)
        nl = inst.nlink.copy(); nl[0, v] = INT_MAX // 2 + 1
        _expect(g, mf.MF_EOVERFLOW, *_bufs(inst, on_device, nl=nl), on_device)
        # the same handle then solves valid input exactly
        g.set_caps(*_bufs(inst, on_device))
        g.solve()
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
    assert_parity(inst, got, ref=ref)


def test_capacity_at_the_int32_limit_is_accepted():
    """cs(v) + sum of its edge capacities = INT32_MAX exactly is allowed and
    solved exactly (flow = min(cs, ct) per vertex with no links)."""
    inst = grids.random_grid((9, 7, 1), 4, 3, cmax=0, tmax=0, p_zero=0.0)
    cs = np.zeros(inst.n, np.int32); ct = np.zeros(inst.n, np.int32)
    cs[10] = INT_MAX; ct[10] = INT_MAX
    cs[11] = INT_MAX; ct[11] = 5
    inst = grids.GridInstance(inst.dims, 4, cs, ct, np.zeros_like(inst.nlink), "int32_limit")
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.solve()
        assert g.flow_value() == INT_MAX + 5
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
    assert_parity(inst, got)
