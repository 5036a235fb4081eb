"""Full-size workloads, in the launch configurations the benchmark times.

* 2048x2048 8-connected segmentation (the benchmark's instance, seed 0): the
  autotuned configuration (32x32 tiles, global relabel every 8 sweeps) with
  the host-driven and the graph sweep loop, and 64x64 tiles with the default
  options: bit-exact flow, S_min and S_max against Dinic, final preflow
  verified.
* 512x512x384 6-connected volume (1.0e8 vertices): Dinic would take hours
  here, so the oracle certifies the GPU's final preflow instead (feasible
  against the original capacities, no excess vertex reaches t, cut cost =
  claimed flow) and recomputes S_min and S_max from it with its own closure
  code, which must equal the GPU's.
"""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity, gpu_solve, opts

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_bench_workload_full_size():
    inst = grids.seg2d_2048_c8_hard(0)
    ref = oracle.solve_instance(inst)
    got = gpu_solve(inst, tile=(32, 32, 1), opts=opts(global_relabel_period=8))
    assert_parity(inst, got, ref=ref)
    got = gpu_solve(inst, tile=(64, 64, 1), opts=opts())
    assert_parity(inst, got, ref=ref)
    got = gpu_solve(inst, tile=(32, 32, 1), opts=opts(global_relabel_period=8, graph_loop=1), residual=False)
    assert got["flow"] == ref["flow"]
    np.testing.assert_array_equal(got["smin"], ref["smin"])
    np.testing.assert_array_equal(got["smax"], ref["smax"])


def test_volume_full_size_certified():
    inst = grids.vol3d_512x512x384(0)
    got = gpu_solve(inst)  # default 3D tile (32x8x8, bit-parallel discharge)
    ok, msg, info = oracle.verify(inst.dims, 6, inst.cs, inst.ct, inst.nlink, got["res"], got["tres"], got["exc"],
                                  got["flow"], got["smin"], got["smax"])
    assert ok, msg
    assert info["cut_cost"] == got["flow"] and info["n_smin"] == int(got["smin"].sum())
    print("volume 512x512x384: flow", got["flow"], "sweeps", got["stats"].sweeps, "ms", got["stats"].ms_total)
