"""Oracle parity at the sizes of the batched and warm-start workloads.

* A 20-instance share of the uneven batch (the benchmark's generator and
  instance seeds): its largest 2D grid and its largest 3D volume, plus 18
  instances spread over the batch order, solved in ONE batched persistent
  solve with the CUDA-graph sweep loop and the relabel period the benchmark
  uses, once cold and once with the learned warm start on the 2D members.
  The tiles rotate over every kernel type the autotuner can pick.  Every
  instance: flow value, S_min and S_max bit-identical to Dinic, final preflow
  accepted by the independent verifier.
* A held-out 1024x1024 grid of the warm-start set, solved warm, against
  Dinic (not against the GPU's own cold solve).
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from gen import grids
from helpers import assert_parity
from paper_1109_1146_gb300 import Grid, default_opts, mf, warmstart

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_1109_1146_gb300", "weights", "warm_seg2d_1024_c4.npy")
TILES2 = [(32, 32, 1), (64, 32, 1), (64, 64, 1)]
TILES3 = [(32, 8, 4), (32, 8, 8), (32, 16, 8), (32, 4, 4), (32, 8, 2)]


def _batch_share():
    shapes = grids.uneven_batch_shapes(0)
    n2 = [i for i, s in enumerate(shapes) if s[2] == 1]
    n3 = [i for i, s in enumerate(shapes) if s[2] > 1]
    big2 = max(n2, key=lambda i: shapes[i][0])
    big3 = max(n3, key=lambda i: shapes[i][0])
    spread = [i for i in range(0, len(shapes), 29) if i not in (big2, big3)][:18]
    idx = sorted({big2, big3, *spread})

    def make(i):
        X, Y, Z = shapes[i]
        return grids.segmentation_2d(X, Y, 5000 + i, conn=4) if Z == 1 else grids.volume_3d(X, Y, Z, 5000 + i)
    with ThreadPoolExecutor(8) as ex:
        insts = list(ex.map(make, idx))
    return idx, insts, shapes[big2], shapes[big3]


def _check_all(insts, handles, refs):
    for inst, g, ref in zip(insts, handles, refs):
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
        assert_parity(inst, got, ref=ref)


def test_uneven_batch_share_cold_and_warm_vs_oracle():
    idx, insts, big2, big3 = _batch_share()
    assert len(insts) >= 16 and big2[0] >= 1000 and big3[0] >= 125  # the batch's largest members are in
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        refs = list(ex.map(oracle.solve_instance, insts))
    handles = []
    for k, inst in enumerate(insts):
        tiles = TILES2 if inst.conn == 4 else TILES3
        tile = tiles[k % len(tiles)]
        g = Grid(inst.dims, inst.conn, tile=tile)
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        handles.append(g)
    # cold, the benchmark's launch configuration (graph loop, relabel every 8 sweeps)
    mf.solve_batch(handles, default_opts(graph_loop=1, global_relabel_period=8))
    _check_all(insts, handles, refs)
    # warm start on the 2D members from the committed network
    net = warmstart.load_network(WEIGHTS)
    dev = torch.device("cuda", torch.cuda.current_device())
    used = 0
    for inst, g in zip(insts, handles):
        if inst.conn != 4:
            continue
        X, Y = inst.dims[0], inst.dims[1]
        x = torch.empty((1, 6, Y, X), dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        g.warm_features(x)
        net.infer(x, y)
        st, _ = g.warm_start(y, check=False)
        used += st == mf.MF_OK
    assert used > 0
    mf.solve_batch(handles, default_opts(graph_loop=1, global_relabel_period=8, warm_start=1))
    _check_all(insts, handles, refs)
    for g in handles:
        g.close()


def test_warm_start_1024_vs_dinic():
    inst = grids.seg2d_1024_c4_mu(warmstart.EVAL_SEED0 + 5)
    ref = oracle.solve_instance(inst)
    net = warmstart.load_network(WEIGHTS)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st, _, rounds, used = warmstart.warm_solve(g, net)
        assert used and rounds > 0
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
    assert_parity(inst, got, ref=ref)
    np.testing.assert_array_equal(got["smin"], ref["smin"])
