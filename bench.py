#!/usr/bin/env python
"""Benchmark of the CUDA P-ARD solver on the batched-solve workload: 512
uneven synthetic instances (384 2D 4-connected segmentation grids with side
uniform in [64, 1024] and 128 3D 6-connected Perlin volumes with side uniform
in [48, 128]; about 2.6e8 vertices), solved exactly through the C ABI.

One step = one mf_solve_batch of all 512 instances from capacities already
resident on the device: Init, every sweep of Algorithm 2 (discharge, fusion,
global gap, relabels) for every instance, the cut extraction (S_min, S_max)
and the flow values, all on the GPU.  ``value`` is ms per instance of that
batched solve.  Beside it, in the same run and on the same instances: the
batched solve with the learned warm start on the 2D members (features,
network inference and projection inside the timed region), the plain
cold-start solve of every instance one by one with the default settings,
sweeps per instance of all three, the end-to-end time through the C ABI from
pinned host buffers, the roofline of the dominant discharge kernel, and the
CPU oracle (Dinic) on a sample of the instances.  The single 2048^2
8-connected grid and the 512x512x384 volume are carried as extra keys.

Prints one JSON line (rank 0).  Multi-GPU: one process per GPU (torchrun),
each rank solves its own batch (batch seed = rank): replicas, weak scaling,
no data-path collective.  ``--impl reference`` times the CPU oracle on the
same 512 instances (each timed step a disjoint share of them, all host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact-maxflow solve ms + sweeps per instance, learned/batched vs plain; HBM GB/s"
UNIT = "ms/instance"
SIDE = 2048
CONN = 8
# algorithmic bytes per discharged vertex: read + write of cap[2H], tcap, exc, lab (int32)
BYTES_PER_VERTEX = {4: (4 + 3) * 4 * 2, 8: (8 + 3) * 4 * 2, 6: (6 + 3) * 4 * 2}
L2_FLUSH_BYTES = 256 << 20
WEIGHTS = os.path.join(ROOT, "paper_1109_1146_gb300", "weights", "warm_seg2d_1024_c4.npy")
BATCH_WORKLOAD = ("uneven batch of 512: 384 seg2d 4-connected grids side U{64..1024} (value-noise intensity, "
                  "cs=|I-80| ct=|I-170|, n-links round(100exp(-dI^2/800))) + 128 vol3d 6-connected Perlin volumes "
                  "side U{48..128} (t-links -log N(I;mu,30^2) x10, n-links round(50exp(-dI^2/450))), PCG64 batch seed")


def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def batch_instance(i, shape, batch_seed=0):
    """Instance i of the uneven batch (instance seed 5000 + i, offset per batch seed)."""
    from gen import grids
    X, Y, Z = shape
    seed = 5000 + i + 100000 * batch_seed
    if Z == 1:
        return grids.segmentation_2d(X, Y, seed, conn=4)
    return grids.volume_3d(X, Y, Z, seed)


def batch_instances(batch_seed=0, count=0, threads=None, only=None, kind="all"):
    """The uneven batch, generated on host threads (numpy releases the GIL);
    kind "2d" / "3d" keeps only those members."""
    from gen import grids
    shapes = grids.uneven_batch_shapes(batch_seed)
    idx = list(range(len(shapes))) if only is None else list(only)
    if kind != "all":
        idx = [i for i in idx if (shapes[i][2] == 1) == (kind == "2d")]
    if count:
        idx = idx[:count]
    with ThreadPoolExecutor(threads or host_threads()) as ex:
        return list(ex.map(lambda i: batch_instance(i, shapes[i], batch_seed), idx))


def oracle_solve_many(insts, threads):
    """Dinic + S_min/S_max of every instance on `threads` host threads (the C
    oracle releases the GIL); returns (results, wall seconds)."""
    import oracle
    oracle._load()
    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(oracle.solve_instance, insts))
    return res, time.perf_counter() - t0


def workload_name(side=SIDE):
    return (f"seg2d {side}x{side} 8-connected, value-noise intensity, cs=|I-80| ct=|I-170|, "
            f"n-links round(100exp(-dI^2/800)) (diagonals /sqrt2), 5% hard seeds at 1e6")


def kernel_name(conn, tile, batch=False):
    tx, ty, tz = tile
    if conn == 6:
        nt = 512 if ty * tz >= 128 else 128 if ty * tz == 16 else 256
        return f"ard_discharge3d{'_batch' if batch else ''}_kernel<{ty},{tz},{nt}>"
    return f"ard_discharge2d{'_batch' if batch else ''}_kernel<{conn},{tx},{ty},{256 if tx * ty <= 2048 else 512}>"


def make_instance(seed, side=SIDE):
    from gen import grids
    return grids.seg2d_2048_c8_hard(seed=seed, side=side)


def directed_arcs(dims, conn):
    from gen.grids import FWD
    X, Y, Z = dims
    return 2 * sum((X - abs(dx)) * (Y - abs(dy)) * (Z - abs(dz)) for dx, dy, dz in FWD[conn])


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def job_time_ms(local_ms, ws, device=None):
    """Timed total of the whole job: the maximum over ranks of each rank's
    timed total (every rank solves its own instance; the slowest bounds it)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(total_ms, ws, steps):
    """ms per instance over the whole job: ws ranks each solved `steps` instances."""
    return total_ms / (ws * steps)


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.dev_id = dev_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev_id), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        rows = []
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                rows.append((float(p[0]), float(p[1]), p[4:8]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, fl in rows for i, f in enumerate(fl) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def committed_traffic(kernel, tile):
    """DRAM bytes per discharged vertex of a discharge kernel from the
    committed ncu summaries (profiles/*.txt lines "bench: key = value"), or
    None if no summary covers this kernel and tile, or if the kernel's source
    changed since it was taken."""
    import glob
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.txt"))):
        kv = {}
        try:
            for ln in open(p):
                if ln.startswith("bench:"):
                    k, v = ln[len("bench:"):].split("=", 1)
                    kv[k.strip()] = v.strip()
        except Exception:
            continue
        if kv.get("kernel") != kernel or kv.get("tile") != "x".join(str(t) for t in tile):
            continue
        src = os.path.join(ROOT, "paper_1109_1146_gb300", "csrc", kv.get("source", ""))
        try:
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        except Exception:
            continue
        if kv.get("kernel_sha256_16") == sha:
            return float(kv["dram_bytes_per_discharged_vertex"])
    return None


def kernel_source(conn):
    return "ard_discharge3d.cu" if conn == 6 else "ard_discharge2d.cu"


def roofline_of(stats, insts, tiles, batch):
    """Roofline line of the dominant discharge kernel type: algorithmic bytes
    (discharged vertices x bytes per vertex) over that kernel's event-timed
    duration, per launch."""
    by_type = {}
    for st, x, t in zip(stats, insts, tiles):
        k = (x.conn, tuple(t))
        e = by_type.setdefault(k, {"ms": 0.0, "launches": 0, "vertices": 0})
        if batch:  # every instance of a type reports the type's total
            e["ms"] = st.ms_discharge
            e["launches"] = st.discharge_launches
        else:
            e["ms"] += st.ms_discharge
            e["launches"] += st.discharge_launches
        e["vertices"] += st.discharged_vertices
    (conn, tile), e = max(by_type.items(), key=lambda kv: kv[1]["ms"])
    peak, peak_kind = measured_peak_hbm()
    alg = e["vertices"] * BYTES_PER_VERTEX[conn]
    achieved = alg / (e["ms"] * 1e-3) / 1e9 if e["ms"] > 0 else 0.0
    kname = kernel_name(conn, tile, batch)
    tb = committed_traffic(kname, tile)
    launches = max(1, e["launches"])
    share = {f"{kernel_name(c, t, batch)}": round(v["ms"], 3) for (c, t), v in by_type.items()}
    return {"kernel": kname, "bound": "hbm", "achieved": round(achieved, 2), "peak": peak,
            "peak_kind": f"{peak_kind} hbm_gbs", "unit": "GB/s", "frac": round(achieved / peak, 5),
            "traffic": None if tb is None else round(tb * e["vertices"] / launches),
            "alg_bytes_per_launch": round(alg / launches), "launch_ms_avg": round(e["ms"] / launches, 4),
            "launches": e["launches"], "discharged_vertices": e["vertices"],
            "bytes_per_discharged_vertex": BYTES_PER_VERTEX[conn],
            "discharge_ms_by_kernel": share}


def run_uneven_batch(args):
    """The batched-solve workload: batched (value), batched with the learned
    warm start, and plain one-by-one solves of the same 512 instances."""
    import numpy as np
    import torch

    from paper_1109_1146_gb300 import Grid, autotune, default_opts, mf, warmstart

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    t_gen = time.perf_counter()
    insts = batch_instances(batch_seed=rank, count=args.batch_count, kind=args.batch_kind)
    t_gen = time.perf_counter() - t_gen
    count = len(insts)
    nv = sum(x.n for x in insts)
    stream = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # tile and schedule per size class from the autotuner (measured solves, untimed)
    t_tune = time.perf_counter()
    table = autotune.tune(insts, cache_path=os.path.join(tempfile.gettempdir(), f"mf_autotune_c4_{rank}.json"))
    sched = autotune.batch_schedule(insts, table)
    t_tune = time.perf_counter() - t_tune
    tiles = [autotune.choose(x, table)[0] for x in insts]
    # capacities resident on the device; one handle per instance for the
    # batched solves (autotuned tiles), one per instance for the plain solves
    # (the library's default tile)
    dcs = [torch.from_numpy(x.cs).to(dev) for x in insts]
    dct = [torch.from_numpy(x.ct).to(dev) for x in insts]
    dnl = [torch.from_numpy(x.nlink).to(dev) for x in insts]
    hb, hp = [], []
    for x, t, a, b, c in zip(insts, tiles, dcs, dct, dnl):
        g = Grid(x.dims, x.conn, tile=t, stream=stream)
        g.set_caps(a, b, c)
        hb.append(g)
        g = Grid(x.dims, x.conn, stream=stream)
        g.set_caps(a, b, c)
        hp.append(g)
    idx2 = [i for i, x in enumerate(insts) if x.conn == 4]
    net = warmstart.load_network(WEIGHTS)
    wx = {}
    for i in idx2:
        X, Y = insts[i].dims[0], insts[i].dims[1]
        wx[i] = (torch.empty((1, 6, Y, X), dtype=torch.float32, device=dev),
                 torch.empty((1, 6, Y, X), dtype=torch.float32, device=dev))

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        out = None
        for k in range(steps):
            ev[k][0].record(stream)
            out = fn()
            ev[k][1].record(stream)
        barrier()
        return [a.elapsed_time(b) for a, b in ev], out

    bopts = default_opts(graph_loop=1, **sched)
    wopts = default_opts(graph_loop=1, warm_start=1, **sched)

    def batched():
        return mf.solve_batch(hb, bopts)

    preds = [None] * count
    for i in idx2:
        preds[i] = wx[i][1]

    def batched_warm():
        for i in idx2:
            x, y = wx[i]
            hb[i].warm_features(x)
            net.infer(x, y)
        mf.warm_start_batch(hb, preds)  # a grid whose projection fails stays cold
        return mf.solve_batch(hb, wopts)

    def plain():
        return [g.solve() for g in hp]

    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    with ClockSampler(f"GPU-{uuid}" if uuid else local) as clk:
        b_ms, b_stats = timed(batched, args.steps, args.warmup)
    smin_b = [g.get_cut(0) for g in hb]
    flow_b = [g.flow_value() for g in hb]
    kw = max(1, min(args.steps, args.aux_steps))
    w_ms, w_stats = timed(batched_warm, kw, min(args.warmup, 2))
    assert [g.flow_value() for g in hb] == flow_b, "warm and cold batched solves disagree on a flow value"
    assert all(np.array_equal(g.get_cut(0), s) for g, s in zip(hb, smin_b)), "warm and cold S_min differ"
    p_ms, p_stats = timed(plain, kw, 1)
    assert [g.flow_value() for g in hp] == flow_b, "batched and plain solves disagree on a flow value"
    assert all(np.array_equal(g.get_cut(0), s) for g, s in zip(hp, smin_b)), "batched and plain S_min differ"
    # host-driven batch loop: the same solve with per-kernel-type event timing
    # (roofline); an NVTX range names it for profilers (ncu --nvtx-include)
    torch.cuda.nvtx.range_push("batched_host_loop")
    _, h_stats = timed(lambda: mf.solve_batch(hb, default_opts(**sched)), 1, 1)
    torch.cuda.nvtx.range_pop()
    # end to end through the C ABI from pinned host buffers: H2D of every
    # instance's capacities (mf_set_caps_batch), the batched solve, D2H of
    # every S_min and flow value (mf_get_cuts_batch)
    pin = [(torch.from_numpy(x.cs).pin_memory(), torch.from_numpy(x.ct).pin_memory(),
            torch.from_numpy(x.nlink).pin_memory(), torch.empty(x.n, dtype=torch.uint8).pin_memory())
           for x in insts]
    e2e_ms = []
    ke = max(1, min(args.steps, args.aux_steps))
    for k in range(ke + 1):
        barrier()
        t0 = time.perf_counter()
        mf.set_caps_batch(hb, [(a, b, c) for a, b, c, _ in pin])
        mf.solve_batch(hb, bopts)
        _, fl = mf.get_cuts_batch(hb, 0, [p[3] for p in pin])
        t1 = time.perf_counter()
        if k > 0:
            e2e_ms.append((t1 - t0) * 1e3)
        assert fl == flow_b
    assert all(np.array_equal(p[3].numpy(), s) for p, s in zip(pin, smin_b))

    total_b = job_time_ms(sum(b_ms), ws, dev)
    total_w = job_time_ms(sum(w_ms), ws, dev)
    total_p = job_time_ms(sum(p_ms), ws, dev)
    total_e = job_time_ms(sum(e2e_ms), ws, dev)
    roof = roofline_of(h_stats, insts, tiles, batch=True)
    h0 = h_stats[0]
    dis_total = sum(roof["discharge_ms_by_kernel"].values())
    breakdown = {"note": "one host-driven batched solve (events): ms of the whole batch by phase",
                 "total": round(h0.ms_total, 2), "init": round(h0.ms_init, 2), "cut": round(h0.ms_cut, 2),
                 "discharge": round(dis_total, 2), "relabel": round(h0.ms_relabel, 2),
                 "fusion_gap_activity_and_loop": round(h0.ms_sweeps - dis_total - h0.ms_relabel, 2)}
    for g in hb + hp:
        g.close()
    del dcs, dct, dnl

    extras = {}
    extra_keys = args.extras.split(",")
    if rank == 0 and "seg2048" in extra_keys:
        extras["seg2d_2048_c8"] = run_single_extra(args, make_instance(0), stream, dev)
    if rank == 0 and "seg2048_host" in extra_keys:
        extras["seg2d_2048_c8_grace_state"] = run_single_extra(args, make_instance(0), stream, dev, host_state=True)
    if rank == 0 and "vol512" in extra_keys:
        from gen import grids
        extras["vol3d_512x512x384"] = run_single_extra(args, grids.vol3d_512x512x384(0), stream, dev)

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    def per(total, steps):
        return round(total / (ws * steps * count), 4)

    def sweeps(st):
        return round(sum(s.sweeps for s in st) / count, 3)

    value = per(total_b, args.steps)
    h2d = int(sum(x.cs.nbytes + x.ct.nbytes + x.nlink.nbytes for x in insts))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_b / args.steps, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD + (f" ({args.batch_kind} members only)" if args.batch_kind != "all" else "")
                   + (f" (first {count})" if args.batch_count else ""),
                   "instances": count, "vertices": nv, "batch_seed": "rank",
                   "parallelism": f"replicas x{ws}", "mode": "batched persistent solve, CUDA-graph sweep loop",
                   "schedule": sched, "tiles": sorted({"x".join(map(str, t)) for t in tiles}),
                   "l2": "not flushed: the batch's device state (about 8 GB) is far larger than L2",
                   "generation_s": round(t_gen, 1), "autotune_s": round(t_tune, 1)},
        "sweeps_per_instance": sweeps(b_stats),
        "vertices_per_s": nv * ws / (total_b / args.steps * 1e-3),
        "batched_cold": {"ms_per_instance": value, "sweeps_per_instance": sweeps(b_stats)},
        "batched_warm": {"ms_per_instance": per(total_w, kw), "sweeps_per_instance": sweeps(w_stats),
                         "note": "learned warm start on the 384 2D members (features, tensor-core inference, "
                                 "projection to a preflow, all timed); 3D members cold",
                         "projection_phases_mean_2d": round(statistics.mean([w_stats[i].projection_rounds
                                                                              for i in idx2] or [0]), 2),
                         "steps": kw},
        "plain": {"ms_per_instance": per(total_p, kw), "sweeps_per_instance": sweeps(p_stats),
                  "note": "cold-start mf_solve of each instance one by one, default tile and options", "steps": kw},
        "speedup_batched_vs_plain": round(total_p / kw / (total_b / args.steps), 3),
        "speedup_batched_warm_vs_plain": round(total_p / kw / (total_w / kw), 3),
        "roofline": roof,
        "breakdown_ms": breakdown,
        "e2e": {"value": per(total_e, ke), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(sum(x.n + 8 for x in insts)), "steps": ke},
        "gpu_launches": int(sum(s.launches for s in b_stats)) * args.steps,
        "clocks": clk.summary(),
    }
    line.update(extras)
    if ws == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample: every 16th instance (24 2D + 8 3D),
        # all host threads; every sampled result compared with the GPU's
        sample = list(range(0, count, 16))
        thr = host_threads()
        refs, wall = oracle_solve_many([insts[i] for i in sample], thr)
        for i, r in zip(sample, refs):
            assert r["flow"] == flow_b[i], (i, r["flow"], flow_b[i])
            assert np.array_equal(r["smin"], smin_b[i]), f"S_min of instance {i} differs from the oracle"
        line["cpu_baseline"] = {"value": round(wall * 1e3 / len(sample), 2), "unit": UNIT, "cores": thr,
                                "kind": "oracle",
                                "sample": f"every 16th instance of the batch ({len(sample)} instances, "
                                          f"{sum(insts[i].n for i in sample)} vertices): Dinic + S_min/S_max BFS, "
                                          f"one instance per host thread; flow and S_min equal to the GPU's"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_single_extra(args, inst, stream, dev, host_state=False):
    """Plain single solve of one large instance with the default tile and
    options (extra key of the batched line): ms, sweeps, discharge roofline;
    host_state keeps the grid's planes in Grace memory (MF_STATE_HOST)."""
    import torch

    from paper_1109_1146_gb300 import Grid, default_opts
    with Grid(inst.dims, inst.conn, stream=stream, host_state=host_state) as g:
        g.set_caps(torch.from_numpy(inst.cs).to(dev), torch.from_numpy(inst.ct).to(dev),
                   torch.from_numpy(inst.nlink).to(dev))
        opts = default_opts()
        for _ in range(2):
            g.solve(opts)
        torch.cuda.synchronize()
        sts = [g.solve(opts) for _ in range(max(1, min(args.steps, 3)))]
        tile = (32, 32, 1) if inst.conn != 6 else (32, 8, 4)
        roof = roofline_of(sts, [inst] * len(sts), [tile] * len(sts), batch=False)
        ok, cut, bad = g.certify()
        ms = statistics.median(s.ms_total for s in sts)
        plane_bytes = sum(s_.discharged_vertices for s_ in sts) / len(sts) * BYTES_PER_VERTEX[inst.conn]
        return {"workload": inst.name, "vertices": inst.n, "tile": list(tile), "ms": round(ms, 3),
                "state": "pinned host (Grace) memory over NVLink-C2C" if host_state else "device (HBM)",
                "discharge_plane_bytes_per_solve": int(plane_bytes),
                "sweeps": sts[-1].sweeps, "vertices_per_s": inst.n / (ms * 1e-3), "flow_value": g.flow_value(),
                "certified": ok, "roofline": {k: roof[k] for k in ("kernel", "achieved", "frac", "launch_ms_avg")}}


def run_ours(args):
    """The single 2048x2048 8-connected grid (--workload seg2048): one step =
    one mf_solve from device-resident capacities."""
    import numpy as np
    import torch

    from paper_1109_1146_gb300 import Grid, autotune, default_opts

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    inst = make_instance(seed=rank)
    stream = torch.cuda.current_stream()
    cs = torch.from_numpy(inst.cs).to(dev)
    ct = torch.from_numpy(inst.ct).to(dev)
    nl = torch.from_numpy(inst.nlink).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    # tile and schedule from the autotuner (measured solves of this instance, untimed)
    table = autotune.tune([inst], single=True,
                          cache_path=os.path.join(tempfile.gettempdir(), f"mf_autotune_single_{rank}.json"))
    tile, sched = autotune.choose(inst, table, single=True)
    g = Grid(inst.dims, CONN, tile=tile, stream=stream)
    g.set_caps(cs, ct, nl)
    opts = default_opts(**sched)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        g.solve(opts)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    with ClockSampler(f"GPU-{uuid}" if uuid else local) as clk:
        barrier()
        for k in range(args.steps):
            flush.zero_()  # L2 flush between timed iterations (not timed)
            ev[k][0].record(stream)
            stats.append(g.solve(opts))
            ev[k][1].record(stream)
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # the same steps with the sweep loop as one CUDA graph (no per-kernel events
    # exist inside a graph, so the roofline above comes from the host-driven loop)
    gopts = default_opts(graph_loop=1, **sched)
    for _ in range(args.warmup):
        g.solve(gopts)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        gev[k][0].record(stream)
        g.solve(gopts)
        gev[k][1].record(stream)
    barrier()
    graph_ms = sum(a.elapsed_time(b) for a, b in gev)
    total_ms = job_time_ms(sum(step_ms), ws, dev)
    flow = g.flow_value()

    # end to end through the public API with host buffers (pinned)
    pc = torch.from_numpy(inst.cs).pin_memory()
    pt = torch.from_numpy(inst.ct).pin_memory()
    pn = torch.from_numpy(inst.nlink).pin_memory()
    cut_host = torch.empty(inst.n, dtype=torch.uint8).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.set_caps(pc, pt, pn)
        g.solve(opts)
        g.get_cut(0, out=cut_host)
        f_host = g.flow_value()
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_ms.append((t1 - t0) * 1e3)
        assert f_host == flow
    e2e_total = job_time_ms(sum(e2e_ms), ws, dev)
    graph_total = job_time_ms(graph_ms, ws, dev)
    g.close()

    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return

    units = ws * args.steps
    value = job_value(total_ms, ws, args.steps)
    sweeps = statistics.mean(s.sweeps for s in stats)
    dis_ms = sum(s.ms_discharge for s in stats)
    dis_launches = sum(s.sweeps for s in stats)
    dis_vertices = sum(s.discharged_vertices for s in stats)
    alg_bytes = dis_vertices * BYTES_PER_VERTEX[CONN]
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (dis_ms * 1e-3) / 1e9 if dis_ms > 0 else 0.0
    tb = committed_traffic(kernel_name(CONN, tile), tile)
    traffic = None if tb is None else tb * dis_vertices / dis_launches
    solve_bytes = alg_bytes / args.steps
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(), "vertices": inst.n, "directed_arcs": directed_arcs(inst.dims, CONN),
                   "tile": list(tile), "schedule": sched, "autotuned": True,
                   "regions": (SIDE // tile[0]) * (SIDE // tile[1]), "seed": "rank",
                   "parallelism": f"replicas x{ws}", "l2": "flushed between steps (256 MiB write)",
                   "flow_value": flow},
        "sweeps_per_instance": sweeps,
        "vertices_per_s": inst.n / (value * 1e-3),
        "hbm_gbs_solve": solve_bytes / (value * 1e-3) / 1e9,
        "phase_ms": {"discharge": dis_ms / args.steps, "fuse_gap": sum(s.ms_fuse for s in stats) / args.steps,
                     "cut": sum(s.ms_cut for s in stats) / args.steps,
                     "init": sum(s.ms_init for s in stats) / args.steps},
        "roofline": {"kernel": kernel_name(CONN, tile), "bound": "hbm",
                     "achieved": round(achieved, 2), "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs",
                     "unit": "GB/s", "frac": round(achieved / peak, 5),
                     "traffic": None if traffic is None else round(traffic),
                     "alg_bytes_per_launch": round(alg_bytes / dis_launches),
                     "launch_ms_avg": round(dis_ms / dis_launches, 4)},
        "e2e": {"value": round(job_value(e2e_total, ws, args.steps), 4), "unit": UNIT,
                "h2d_bytes_per_step": int(inst.cs.nbytes + inst.ct.nbytes + inst.nlink.nbytes),
                "d2h_bytes_per_step": int(inst.n + 8)},
        "gpu_launches": int(sum(s.launches for s in stats)),
        "graph_loop": {"value": round(job_value(graph_total, ws, args.steps), 4), "unit": UNIT,
                       "note": "same steps, sweep loop as one CUDA graph with a device-side while node"},
        "clocks": clk.summary(),
    }
    if ws == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.solve_instance(inst)
        t1 = time.perf_counter()
        assert ref["flow"] == flow, (ref["flow"], flow)
        line["cpu_baseline"] = {"value": round((t1 - t0) * 1e3, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "the full instance (seed 0): Dinic on the explicit s-t network + "
                                          "S_min/S_max BFS, single thread"}
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def run_batch_warm(args):
    """Learned warm start with the batched solve: held-out 1024x1024 4-connected
    segmentation grids (mu_fg, mu_bg per seed) solved one by one cold, batched
    cold, and batched warm (features, network inference and projection of every
    instance inside the timed region)."""
    import torch

    from gen import grids
    from paper_1109_1146_gb300 import Grid, default_opts, mf, warmstart

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    count = args.batch_count or 64
    insts = [grids.seg2d_1024_c4_mu(warmstart.EVAL_SEED0 + i) for i in range(count)]
    stream = torch.cuda.current_stream()
    weights = os.path.join(ROOT, "paper_1109_1146_gb300", "weights", "warm_seg2d_1024_c4.npy")
    net = warmstart.load_network(weights)
    plain_ms, plain_sweeps, flows = 0.0, 0, []
    for x in insts:
        with Grid(x.dims, x.conn, stream=stream) as g:
            g.set_caps(x.cs, x.ct, x.nlink)
            g.solve()
            st = g.solve()
            plain_ms += st.ms_total
            plain_sweeps += st.sweeps
            flows.append(g.flow_value())
    handles = []
    for x in insts:
        g = Grid(x.dims, x.conn, stream=stream)
        g.set_caps(x.cs, x.ct, x.nlink)
        handles.append(g)
    C, X, Y = 6, insts[0].dims[0], insts[0].dims[1]
    xf = torch.empty((1, C, Y, X), dtype=torch.float32, device=dev)
    yp = torch.empty_like(xf)

    def one_step(warm):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        if warm:
            for g in handles:
                g.warm_features(xf)
                net.infer(xf, yp)
                g.warm_start(yp, check=False)
        stats = mf.solve_batch(handles, default_opts(warm_start=1 if warm else 0, graph_loop=1))
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b), stats

    res = {}
    for warm in (False, True):
        for _ in range(args.warmup):
            one_step(warm)
        runs = [one_step(warm) for _ in range(args.steps)]
        assert [h.flow_value() for h in handles] == flows, "batched and single solves disagree"
        res[warm] = (statistics.median(r[0] for r in runs), sum(s.sweeps for s in runs[-1][1]) / count)
    line = {"metric": METRIC, "workload": "batch_warm", "value": round(res[True][0] / count, 4), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "%d held-out seg2d 1024x1024 4-connected grids, mu_fg and mu_bg ~ U[60,200] per "
                                   "seed; committed warm-start network" % count, "instances": count},
            "plain_cold_ms_per_instance": round(plain_ms / count, 4),
            "batch_cold_ms_per_instance": round(res[False][0] / count, 4),
            "batch_warm_ms_per_instance": round(res[True][0] / count, 4),
            "sweeps_per_instance_plain_cold": plain_sweeps / count,
            "sweeps_per_instance_batch_cold": res[False][1],
            "sweeps_per_instance_batch_warm": res[True][1],
            "speedup_batch_warm_vs_plain": round(plain_ms / res[True][0], 3)}
    for h in handles:
        h.close()
    print(json.dumps(line), flush=True)


def run_prd(args):
    """P-ARD against P-PRD (Discharge = PRD, kernel_variant 2) on the paper's
    synthetic family (Sec. 7.1: displacements from the paper's list, excess
    U[-500, 500], constant strength): sweeps and device ms of both on the same
    instances and schedule (global relabel every 4 sweeps), over strength,
    size and connectivity (at connectivity c the strength is 150 * 8 / c, as
    in the paper's connectivity series), and over the region size (the
    number of regions) at connectivity 8 and 4; every pair must reach the
    same flow value."""
    from gen import grids
    from paper_1109_1146_gb300 import Grid, default_opts

    t32 = (32, 32, 1)
    cases = [(1000, s, 8, t32) for s in (20, 50, 150, 400, 1000)]        # strength, connectivity 8
    cases += [(n, 150, 8, t32) for n in (250, 500, 2000)]                 # size
    cases += [(1000, 1200 // c, c, t32) for c in (4, 12, 16, 20, 24, 28)]  # connectivity
    cases += [(1000, s, 4, t32) for s in (20, 150, 400, 1000)]
    cases += [(1000, 150, 8, t) for t in ((64, 32, 1), (64, 64, 1))]      # number of regions, connectivity 8
    cases += [(1000, 150, 4, t) for t in ((64, 64, 1), (64, 32, 1))]      # and 4
    for side, strength, conn, tile in cases:
        rows = {}
        for seed in range(args.prd_seeds):
            inst = grids.paper_synthetic(side, side, seed, strength=strength, connectivity=conn)
            flows = set()
            with Grid(inst.dims, inst.conn, tile=tile) as g:
                g.set_caps(inst.cs, inst.ct, inst.nlink)
                for name, variant in (("ard", 0), ("prd", 2)):
                    opts = default_opts(kernel_variant=variant)
                    g.solve(opts)
                    st = g.solve(opts)
                    flows.add(g.flow_value())
                    r = rows.setdefault(name, {"sweeps": [], "ms": [], "rounds": []})
                    r["sweeps"].append(st.sweeps)
                    r["ms"].append(st.ms_total)
                    r["rounds"].append(st.rounds / max(1, st.discharges))
            assert len(flows) == 1, (side, strength, conn, seed, flows)
        print(json.dumps({"workload": "prd", "instance": f"paper synthetic {side}x{side} connectivity {conn}",
                          "connectivity": conn, "strength": strength, "tile": list(tile), "seeds": args.prd_seeds,
                          **{f"{k}_{m}_mean": round(statistics.mean(v[m]), 3) for k, v in rows.items() for m in v}}),
              flush=True)


RELABEL_SCHEDULES = {
    "none": dict(global_relabel_period=0),
    "glr2": dict(global_relabel_period=2),
    "glr4": dict(global_relabel_period=4),
    "glr8": dict(global_relabel_period=8),
    "br1": dict(global_relabel_period=0, boundary_relabel_period=1),
    "br2": dict(global_relabel_period=0, boundary_relabel_period=2),
    "pd": dict(global_relabel_period=0, partial_discharge=1),
    "pd+br1": dict(global_relabel_period=0, partial_discharge=1, boundary_relabel_period=1),
    "br1+glr8": dict(global_relabel_period=8, boundary_relabel_period=1),
    "glr8f1": dict(global_relabel_period=8, global_relabel_first=1),
    "glr8f2": dict(global_relabel_period=8, global_relabel_first=2),
    "glr4f1": dict(global_relabel_period=4, global_relabel_first=1),
}


def run_relabel(args):
    """Relabel schedules compared on the named workloads: no relabel, the exact
    global relabel every P sweeps (glrP), the boundary-relabel heuristic of
    Sec. 6.1 every P sweeps (brP), partial discharges (pd) and combinations.
    One JSON line per (workload, schedule): median device ms of a solve,
    sweeps, discharges and the relabels run; every schedule must reach the
    same flow value."""
    from gen import grids
    from paper_1109_1146_gb300 import Grid, default_opts, warmstart

    glr = ["none", "glr2", "glr4", "glr8", "br1", "br2", "pd", "pd+br1", "br1+glr8"]
    no_glr = ["none", "br1", "br2", "pd", "pd+br1"]
    cases = [("seg2d 2048x2048 8-connected, 5% hard seeds", lambda: grids.seg2d_2048_c8_hard(0), (32, 32, 1), glr),
             ("seg2d 1024x1024 4-connected, held-out seed of the warm-start set",
              lambda: grids.seg2d_1024_c4_mu(warmstart.EVAL_SEED0), (32, 32, 1), glr),
             ("seg2d 256x256 4-connected", lambda: grids.seg2d_256_c4(0), (32, 32, 1), glr),
             ("volume 256x256x128 6-connected", lambda: grids.vol3d_512x512x384(0, dims=(256, 256, 128)), (32, 8, 4), glr),
             ("volume 256x256x128 6-connected, 16^3 tiles (no global relabel)",
              lambda: grids.vol3d_512x512x384(0, dims=(256, 256, 128)), (16, 16, 16), no_glr),
             ("volume 512x512x384 6-connected", lambda: grids.vol3d_512x512x384(0), (32, 8, 4),
              ["glr4", "br1", "br2", "br1+glr8"])]
    if args.relabel_case >= 0:
        cases = [cases[args.relabel_case]]
    for name, make, tile, scheds in cases:
        if args.relabel_schedule:
            scheds = [args.relabel_schedule]
        inst = make()
        flows = set()
        with Grid(inst.dims, inst.conn, tile=tile) as g:
            g.set_caps(inst.cs, inst.ct, inst.nlink)
            for sn in scheds:
                opts = default_opts(**RELABEL_SCHEDULES[sn])
                runs = [g.solve(opts) for _ in range(args.warmup + args.steps)][args.warmup:]
                st = runs[-1]
                flows.add(g.flow_value())
                print(json.dumps({"workload": "relabel", "instance": name, "tile": list(tile), "schedule": sn,
                                  "opts": RELABEL_SCHEDULES[sn], "ms": round(statistics.median(r.ms_total for r in runs), 3),
                                  "sweeps": st.sweeps, "discharges": st.discharges,
                                  "global_relabels": st.global_relabels, "boundary_relabels": st.boundary_relabels,
                                  "boundary_relabel_levels": st.boundary_relabel_levels,
                                  "ms_discharge": round(st.ms_discharge, 3), "ms_fuse": round(st.ms_fuse, 3)}),
                      flush=True)
        assert len(flows) == 1, f"schedules disagree on {name}: {flows}"


def reference_shares(count, steps):
    """Instances of each timed step of the reference arm: step k solves the
    instances i with i mod steps = k (disjoint; together every instance once)."""
    return [[i for i in range(count) if i % steps == k] for k in range(steps)]


def run_reference(args):
    """The oracle (Dinic + S_min/S_max BFS, plain C) on the same workload as
    the default line: the 512 instances of the uneven batch, solved on all
    host threads (one instance per thread).  Each timed step solves a
    disjoint, interleaved share of the batch (instance i in step i mod K), so
    the K timed steps together solve every instance exactly once; generation
    is not timed.  Warm-up steps solve the smallest instances."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from gen import grids
    shapes = grids.uneven_batch_shapes(0)
    count = args.batch_count or len(shapes)
    thr = host_threads()
    steps = max(1, args.steps)
    by_size = sorted(range(count), key=lambda i: shapes[i][0] * shapes[i][1] * shapes[i][2])
    for w in range(args.warmup):
        oracle_solve_many(batch_instances(0, only=[by_size[w % count]]), thr)
    times, nv, solved = [], 0, 0
    for share in reference_shares(count, steps):
        if not share:
            continue
        insts = batch_instances(0, only=share)
        res, wall = oracle_solve_many(insts, thr)
        times.append(wall * 1e3)
        nv += sum(x.n for x in insts)
        solved += len(insts)
    total = sum(times)
    value = total / solved
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
            "steps": steps, "warmup": args.warmup, "ms_per_step": round(total / len(times), 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "instances": solved, "vertices": nv, "batch_seed": 0,
                       "parallelism": f"{thr} host threads, one instance each"},
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": thr, "kind": "oracle",
                             "sample": f"all {solved} instances of the batch over the {steps} timed steps "
                                       f"(step k: instances i with i mod {steps} = k), untimed generation"},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="batch512", choices=["batch512", "seg2048", "batch_warm", "relabel", "prd"])
    ap.add_argument("--prd-seeds", type=int, default=3, help="prd workload: instances per point")
    ap.add_argument("--batch-count", type=int, default=0, help="first N instances of the batch (0 = all 512)")
    ap.add_argument("--batch-kind", default="all", choices=["all", "2d", "3d"],
                    help="batched line: all members, or only the 2D / 3D ones")
    ap.add_argument("--aux-steps", type=int, default=3,
                    help="timed steps of the warm, plain and end-to-end modes of the batched line (<= --steps)")
    ap.add_argument("--extras", default="seg2048,seg2048_host,vol512",
                    help="extra keys of the batched line: seg2048 = 2048^2 8-connected grid, seg2048_host = the same "
                         "with its state in Grace memory, vol512 = 512x512x384 volume; none = no extra")
    ap.add_argument("--relabel-case", type=int, default=-1, help="relabel workload: only this instance (index)")
    ap.add_argument("--relabel-schedule", default="", help="relabel workload: only this schedule")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_uneven_batch(args)
    elif args.workload == "batch_warm":
        run_batch_warm(args)
    elif args.workload == "relabel":
        run_relabel(args)
    elif args.workload == "prd":
        run_prd(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
