"""Learned warm start: training examples from exact solves, the training loop,
warm solves, and the train / evaluate driver.

All arithmetic of the path runs in the library's kernels (feature and target
extraction, the network's forward / backward / Adam and tensor-core
inference, the projection to a preflow, the solve, the certificate); this
module moves device buffers around and keeps the books.

A warm solve = features -> network -> projection to a valid preflow -> one
exact region-distance relabel -> the usual sweeps.  If the projection runs
out of rounds the solve starts cold.  The exact answer does not depend on the
start; every warm result is compared with the cold one.

  python -m paper_1109_1146_gb300.warmstart train --out W.npy [--train 2000]
  python -m paper_1109_1146_gb300.warmstart eval --weights W.npy [--seeds 200]
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import sys
import time
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import torch

from .mf import CNN, MF_OK, Grid, default_opts

# seeds 0 .. n-1 train; held-out evaluation seeds start here
EVAL_SEED0 = 1_000_000


def channels(conn: int) -> int:
    return conn + 2


def example(inst, dev, stream=None, opts=None, dtype=torch.float32):
    """Solve `inst` exactly, check the optimality certificate, and return
    device tensors (x, t) of shape [C, Y, X] (network input, solution flows)
    and the flow value."""
    C = channels(inst.conn)
    X, Y = inst.dims[0], inst.dims[1]
    x = torch.empty((C, Y, X), dtype=torch.float32, device=dev)
    t = torch.empty((C, Y, X), dtype=torch.float32, device=dev)
    with Grid(inst.dims, inst.conn, stream=stream) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.solve(opts)
        ok, _, bad = g.certify()
        if not ok:
            raise RuntimeError(f"solve of {inst.name} failed its certificate ({bad} violations)")
        g.warm_features(x)
        g.warm_targets(t)
        flow = g.flow_value()
    if dtype != torch.float32:
        x, t = x.to(dtype), t.to(dtype)
    return x, t, flow


def train(cnn: CNN, xs, ts, steps: int, batch: int = 8, lr: float = 2e-3, seed: int = 0, crop: int | None = None,
          log=None):
    """Adam with a cosine learning-rate schedule on the mean squared error
    between prediction and solution flows.  xs / ts: lists of equal-shape
    device tensors [C, H, W]; with `crop`, each batch element is a random
    crop x crop window of a random example."""
    gen = torch.Generator().manual_seed(seed)
    dev = xs[0].device
    C, H, W = xs[0].shape
    ch, cw = (crop, crop) if crop else (H, W)
    xb = torch.empty((batch, C, ch, cw), dtype=torch.float32, device=dev)
    tb = torch.empty_like(xb)
    yb = torch.empty_like(xb)
    dy = torch.empty_like(xb)
    losses = []
    for s in range(steps):
        idx = torch.randint(0, len(xs), (batch,), generator=gen).tolist()
        oy = torch.randint(0, H - ch + 1, (batch,), generator=gen).tolist()
        ox = torch.randint(0, W - cw + 1, (batch,), generator=gen).tolist()
        for j, i in enumerate(idx):
            xb[j].copy_(xs[i][:, oy[j]:oy[j] + ch, ox[j]:ox[j] + cw])
            tb[j].copy_(ts[i][:, oy[j]:oy[j] + ch, ox[j]:ox[j] + cw])
        cnn.forward(xb, yb)
        loss = cnn.mse(yb, tb, dy)
        cnn.zero_grad()
        cnn.backward(xb, dy)
        cnn.adam_step(lr=lr * 0.5 * (1.0 + math.cos(math.pi * s / steps)))
        losses.append(loss)
        if log and (s % max(1, steps // 10) == 0 or s == steps - 1):
            log(f"step {s} loss {loss:.5f}")
    return losses


def warm_solve(g: Grid, cnn: CNN, opts=None, max_rounds: int = 0):
    """Warm solve of a grid whose capacities are set.  Returns (stats, device
    ms of features + inference + projection + solve, projection rounds, used
    warm start)."""
    C = channels(g.conn)
    X, Y = g.dims[0], g.dims[1]
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.empty((1, C, Y, X), dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.warm_features(x)
    cnn.infer(x, y)
    st, rounds = g.warm_start(y, max_rounds=max_rounds, check=False)
    used = st == MF_OK
    o = opts if opts is not None else default_opts()
    o.warm_start = 1 if used else 0
    stats = g.solve(o)
    e1.record()
    e1.synchronize()
    return stats, e0.elapsed_time(e1), rounds, used


def save_weights(cnn: CNN, path: str, meta: dict):
    np.save(path, cnn.get_params())
    with open(path.rsplit(".", 1)[0] + ".json", "w") as f:
        json.dump(meta, f, indent=1, sort_keys=True)


def load_network(path: str, conn: int = 4) -> CNN:
    net = CNN(channels=channels(conn), seed=0)
    net.load(path)
    return net


def _make(seed_side):
    from gen import grids
    seed, side = seed_side
    return grids.seg2d_1024_c4_mu(seed, side=side)


def _instances(pool, seeds, side):
    return pool.map(_make, [(s, side) for s in seeds], chunksize=4)


def cmd_train(a):
    ctx = mp.get_context("spawn")
    with ProcessPoolExecutor(max_workers=a.workers, mp_context=ctx) as pool:  # before any CUDA call
        dev = torch.device("cuda:0")
        xs, ts = [], []
        t0 = time.perf_counter()
        for inst in _instances(pool, range(a.train), a.side):
            x, t, _ = example(inst, dev, dtype=torch.bfloat16)
            xs.append(x)
            ts.append(t)
        t_data = time.perf_counter() - t0
    print(f"{len(xs)} certified examples of {a.side}x{a.side} in {t_data:.1f} s", flush=True)
    net = CNN(channels=channels(4), seed=a.seed)
    t0 = time.perf_counter()
    losses = train(net, xs, ts, a.steps, batch=a.batch, lr=a.lr, seed=a.seed, crop=a.crop,
                   log=lambda m: print(m, flush=True))
    t_train = time.perf_counter() - t0
    meta = {"instances": a.train, "side": a.side, "steps": a.steps, "batch": a.batch, "crop": a.crop, "lr": a.lr,
            "seed": a.seed, "final_loss_mean_last100": float(np.mean(losses[-100:])), "train_s": t_train,
            "data_s": t_data, "recipe": "seg2d 4-connected, mu_fg and mu_bg ~ U[60,200] per seed"}
    save_weights(net, a.out, meta)
    print(json.dumps(meta), flush=True)


def cmd_eval(a):
    ctx = mp.get_context("spawn")
    rows = []
    with ProcessPoolExecutor(max_workers=a.workers, mp_context=ctx) as pool:
        net = load_network(a.weights)
        for i, inst in enumerate(_instances(pool, range(EVAL_SEED0, EVAL_SEED0 + a.seeds), a.side)):
            with Grid(inst.dims, 4) as g:
                g.set_caps(inst.cs, inst.ct, inst.nlink)
                if i == 0:
                    g.solve()
                    warm_solve(g, net)
                cold = g.solve()
                flow, smin, smax = g.flow_value(), g.get_cut(0), g.get_cut(1)
                ws, ms, rounds, used = warm_solve(g, net)
                same = g.flow_value() == flow and np.array_equal(g.get_cut(0), smin) and np.array_equal(
                    g.get_cut(1), smax)
                if not same:
                    raise RuntimeError(f"warm and cold results differ on {inst.name}")
                rows.append({"seed": EVAL_SEED0 + i, "cold_ms": cold.ms_total, "cold_sweeps": cold.sweeps,
                             "warm_ms": ms, "warm_solve_ms": ws.ms_total, "warm_sweeps": ws.sweeps,
                             "projection_rounds": rounds, "warm_used": used})

    def stats(k):
        v = np.array([r[k] for r in rows], dtype=np.float64)
        return {"mean": float(v.mean()), "median": float(np.median(v)), "p90": float(np.percentile(v, 90))}

    summary = {"instances": len(rows), "side": a.side, "identical_results": True,
               **{k: stats(k) for k in ("cold_ms", "warm_ms", "warm_solve_ms", "cold_sweeps", "warm_sweeps",
                                        "projection_rounds")},
               "warm_fewer_sweeps": int(sum(r["warm_sweeps"] < r["cold_sweeps"] for r in rows)),
               "warm_more_sweeps": int(sum(r["warm_sweeps"] > r["cold_sweeps"] for r in rows))}
    print(json.dumps(summary, indent=1), flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump({"summary": summary, "rows": rows}, f, indent=1)


def main(argv=None):
    p = argparse.ArgumentParser(prog="python -m paper_1109_1146_gb300.warmstart")
    sub = p.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", required=True)
    t.add_argument("--train", type=int, default=2000)
    t.add_argument("--side", type=int, default=1024)
    t.add_argument("--steps", type=int, default=4000)
    t.add_argument("--batch", type=int, default=8)
    t.add_argument("--crop", type=int, default=256)
    t.add_argument("--lr", type=float, default=5e-3)
    t.add_argument("--seed", type=int, default=3)
    t.add_argument("--workers", type=int, default=12)
    e = sub.add_parser("eval")
    e.add_argument("--weights", required=True)
    e.add_argument("--seeds", type=int, default=200)
    e.add_argument("--side", type=int, default=1024)
    e.add_argument("--workers", type=int, default=12)
    e.add_argument("--json", default=None)
    a = p.parse_args(argv)
    {"train": cmd_train, "eval": cmd_eval}[a.cmd](a)


if __name__ == "__main__":
    sys.exit(main())
