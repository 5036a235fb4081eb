"""The sweep loop as one CUDA graph (conditional while node, opts.graph_loop):
the same computation as the host-driven loop, so identical flow, cuts,
residual network, sweep count and relabel count, and oracle parity."""
import numpy as np
import pytest

from gen import grids
from helpers import assert_parity, gpu_solve, opts
from paper_1109_1146_gb300 import Grid, MFError

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,tile", [
    (lambda: grids.segmentation_2d(230, 190, 3, conn=8, hard_seed_frac=0.05), (32, 32, 1)),
    (lambda: grids.segmentation_2d(300, 170, 4, conn=4, hard_seed_frac=0.02), (64, 64, 1)),
    (lambda: grids.volume_3d(41, 37, 30, 2), (8, 8, 8)),
    (lambda: grids.volume_3d(70, 37, 30, 2), (32, 16, 8)),
])
@pytest.mark.parametrize("kw", [dict(), dict(partial_discharge=1), dict(global_relabel_period=2),
                                dict(global_relabel_period=3, partial_discharge=1, global_gap=0),
                                dict(global_relabel_period=8, global_relabel_first=1),
                                dict(global_relabel_period=0, global_relabel_first=2)])
def test_graph_loop_equals_host_loop(make, tile, kw):
    inst = make()
    host = gpu_solve(inst, tile=tile, opts=opts(**kw))
    dev = gpu_solve(inst, tile=tile, opts=opts(graph_loop=1, **kw))
    assert_parity(inst, dev)
    assert dev["flow"] == host["flow"]
    for k in ("smin", "smax", "res", "tres", "exc", "lab"):
        np.testing.assert_array_equal(dev[k], host[k])
    assert dev["stats"].sweeps == host["stats"].sweeps
    assert dev["stats"].global_relabels == host["stats"].global_relabels
    assert dev["stats"].gaps == host["stats"].gaps


def test_graph_loop_sweep_cap_and_reuse():
    inst = grids.seg2d_256_c4(3)
    with Grid(inst.dims, inst.conn, tile=(64, 64, 1)) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        with pytest.raises(MFError, match="SWEEPLIMIT"):
            g.solve(opts(graph_loop=1, max_sweeps=1, global_relabel_period=0))
        # the handle stays usable; the graph is rebuilt only when baked options change
        a = g.solve(opts(graph_loop=1))
        fa = g.flow_value()
        b = g.solve(opts(graph_loop=1, partial_discharge=1))
        assert g.flow_value() == fa and a.sweeps >= 1 and b.sweeps >= 1
