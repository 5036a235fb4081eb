"""Learned warm start: training examples from exact solves, the training loop
and warm solves.  All arithmetic runs in the library's kernels (feature and
target extraction, the network's forward / backward / Adam, the projection
to a preflow); this module only moves device buffers around.

A warm solve = features -> network -> projection to a valid preflow -> the
usual sweeps from that preflow.  If the projection runs out of rounds the
solve starts cold.  The exact answer does not depend on the start.
"""
from __future__ import annotations

import time

import torch

from .mf import CNN, MF_OK, Grid, default_opts


def channels(conn: int) -> int:
    return conn + 2


def example(inst, dev, stream=None, opts=None):
    """Solve `inst` exactly and return device tensors (x, t) of shape
    [C, Y, X]: the network input and the flows of the solution."""
    C = channels(inst.conn)
    X, Y = inst.dims[0], inst.dims[1]
    x = torch.empty((C, Y, X), dtype=torch.float32, device=dev)
    t = torch.empty((C, Y, X), dtype=torch.float32, device=dev)
    with Grid(inst.dims, inst.conn, stream=stream) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.solve(opts)
        g.warm_features(x)
        g.warm_targets(t)
        flow = g.flow_value()
    return x, t, flow


def train(cnn: CNN, xs, ts, steps: int, batch: int = 8, lr: float = 2e-3, seed: int = 0, log=None):
    """Adam on the mean squared error between prediction and solution flows;
    xs / ts: lists of equal-shape device tensors [C, H, W]."""
    gen = torch.Generator().manual_seed(seed)
    dev = xs[0].device
    C, H, W = xs[0].shape
    xb = torch.empty((batch, C, H, W), dtype=torch.float32, device=dev)
    tb = torch.empty_like(xb)
    yb = torch.empty_like(xb)
    dy = torch.empty_like(xb)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, len(xs), (batch,), generator=gen).tolist()
        for j, i in enumerate(idx):
            xb[j].copy_(xs[i])
            tb[j].copy_(ts[i])
        cnn.forward(xb, yb)
        loss = cnn.mse(yb, tb, dy)
        cnn.zero_grad()
        cnn.backward(xb, dy)
        cnn.adam_step(lr=lr)
        losses.append(loss)
        if log and (s % max(1, steps // 10) == 0 or s == steps - 1):
            log(f"step {s} loss {loss:.5f}")
    return losses


def warm_solve(g: Grid, cnn: CNN, opts=None, max_rounds: int = 0):
    """Warm solve of a grid whose capacities are set.  Returns (stats,
    wall-clock ms of inference + projection + solve, projection rounds, used
    warm start)."""
    C = channels(g.conn)
    X, Y = g.dims[0], g.dims[1]
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.empty((1, C, Y, X), dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.warm_features(x)
    cnn.forward(x, y)
    st, rounds = g.warm_start(y, max_rounds=max_rounds, check=False)
    used = st == MF_OK
    o = opts if opts is not None else default_opts()
    o.warm_start = 1 if used else 0
    stats = g.solve(o)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    return stats, ms, rounds, used
