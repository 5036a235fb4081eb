"""Shared test helpers: run the CUDA solver through the C ABI and compare it
with the oracle."""
import numpy as np

import oracle
from paper_1109_1146_gb300 import Grid, default_opts


def gpu_solve(inst, tile=None, opts=None, residual=True):
    with Grid(inst.dims, inst.conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st = g.solve(opts)
        out = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1), "stats": st}
        if residual:
            out["res"], out["tres"], out["exc"] = g.get_residual()
            out["lab"], out["dinf"] = g.get_labels()
    return out


def assert_parity(inst, got, ref=None, verify=True):
    """Bit-exact flow value, S_min and S_max against Dinic; the final preflow
    independently verified (feasible, maximal, cut cost = flow)."""
    ref = ref if ref is not None else oracle.solve_instance(inst)
    assert got["flow"] == ref["flow"], (got["flow"], ref["flow"])
    bad = np.flatnonzero(got["smin"] != ref["smin"])
    assert bad.size == 0, f"S_min differs at {bad[:10]} ({bad.size} vertices)"
    bad = np.flatnonzero(got["smax"] != ref["smax"])
    assert bad.size == 0, f"S_max differs at {bad[:10]} ({bad.size} vertices)"
    if verify and "res" in got:
        ok, msg, info = oracle.verify(inst.dims, inst.conn, inst.cs, inst.ct, inst.nlink, got["res"],
                                      got["tres"], got["exc"], got["flow"], got["smin"], got["smax"])
        assert ok, msg
    return ref


def opts(**kw):
    return default_opts(**kw)
