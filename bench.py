#!/usr/bin/env python
"""Benchmark: exact max-flow / min-cut solve of the 2048x2048 8-connected
segmentation grid (4.19M vertices, 33.5M arcs, 5% hard seeds at 10^6; tile
and schedule from the autotuner) by the CUDA P-ARD solver, through the C ABI.

One step = one mf_solve from capacities already resident on the device:
Init, all sweeps of Algorithm 2 (discharge, fusion, global gap), the cut
extraction (S_min, S_max) and the flow value, all on the GPU.

Prints one JSON line (rank 0).  Multi-GPU: one process per GPU
(torchrun), each rank solves its own instance (seed = rank): replicas, weak
scaling, no data-path collective.  ``--impl reference`` times the CPU
oracle (Dinic) on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact-maxflow solve ms + sweeps per instance, learned/batched vs plain; HBM GB/s"
UNIT = "ms/instance"
SIDE = 2048
CONN = 8
BYTES_PER_VERTEX = (CONN + 3) * 4 * 2  # read + write of cap[8], tcap, exc, lab (int32)
L2_FLUSH_BYTES = 256 << 20
REF_SAMPLE_SIDE = 1024


def workload_name(side=SIDE):
    return (f"seg2d {side}x{side} 8-connected, value-noise intensity, cs=|I-80| ct=|I-170|, "
            f"n-links round(100exp(-dI^2/800)) (diagonals /sqrt2), 5% hard seeds at 1e6")


def kernel_name(tile):
    return f"ard_discharge2d_kernel<{CONN},{tile[0]},{tile[1]},{256 if tile[0] == 32 else 512}>"


def make_instance(seed, side=SIDE):
    from gen import grids
    return grids.config1(seed=seed, side=side)


def directed_arcs(dims):
    from gen.grids import FWD
    X, Y, _ = dims
    return 2 * sum((X - abs(dx)) * (Y - abs(dy)) for dx, dy, _ in FWD[CONN])


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


def committed_traffic(tile):
    """DRAM bytes per discharged vertex of the discharge kernel from the
    committed ncu summary, or None if the kernel source or the tile differs
    from the ones measured there."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ard_discharge_seg2d_2048_c8.txt")
    src = os.path.join(ROOT, "paper_1109_1146_gb300", "csrc", "ard_discharge2d.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        kv = {}
        for ln in open(p):
            if ln.startswith("bench:"):
                k, v = ln[len("bench:"):].split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("kernel_sha256_16") != sha or kv.get("tile") != "x".join(str(t) for t in tile):
            return None
        return float(kv["dram_bytes_per_discharged_vertex"])
    except Exception:
        return None


def run_ours(args):
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
    alg_bytes = dis_vertices * BYTES_PER_VERTEX
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (dis_ms * 1e-3) / 1e9 if dis_ms > 0 else 0.0
    tb = committed_traffic(tile)
    traffic = None if tb is None else tb * dis_vertices / dis_launches
    solve_bytes = alg_bytes / args.steps
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(), "vertices": inst.n, "directed_arcs": directed_arcs(inst.dims),
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
        "roofline": {"kernel": kernel_name(tile), "bound": "hbm",
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


def run_batch(args):
    """Batched persistent solve of the uneven batch (384 2D 4-connected grids,
    side U{64..1024}, and 128 3D 6-connected grids, side U{48..128}) against
    the same instances solved one by one with the default settings."""
    import tempfile

    import torch

    from gen import grids
    from paper_1109_1146_gb300 import Grid, autotune, default_opts, mf

    torch.cuda.set_device(0)
    shapes = grids.config4_shapes(0)[: args.batch_count] if args.batch_count else grids.config4_shapes(0)
    insts = []
    for i, (X, Y, Z) in enumerate(shapes):
        if Z == 1:
            insts.append(grids.segmentation_2d(X, Y, 5000 + i, conn=4))
        else:
            insts.append(grids.volume_3d(X, Y, Z, 5000 + i))
    nv = sum(x.n for x in insts)
    stream = torch.cuda.current_stream()
    # plain: one solve per instance, default tile and options
    plain_ms, plain_sweeps, flows = 0.0, 0, []
    for x in insts:
        with Grid(x.dims, x.conn, stream=stream) as g:
            g.set_caps(x.cs, x.ct, x.nlink)
            g.solve()
            st = g.solve()
            plain_ms += st.ms_total
            plain_sweeps += st.sweeps
            flows.append(g.flow_value())
    table = autotune.tune(insts, cache_path=os.path.join(tempfile.gettempdir(), "mf_autotune.json"))
    sched = autotune.batch_schedule(insts, table)
    handles = []
    for x in insts:
        tile, _ = autotune.choose(x, table)
        g = Grid(x.dims, x.conn, tile=tile, stream=stream)
        g.set_caps(x.cs, x.ct, x.nlink)
        handles.append(g)
    def timed(opts):
        for _ in range(args.warmup):
            mf.solve_batch(handles, opts)
        times, stats = [], None
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            stats = mf.solve_batch(handles, opts)
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        return times, stats

    # the sweep loop of the batch as one CUDA graph (device-side while node); the
    # host-driven loop is timed beside it
    host_times, _ = timed(default_opts(**sched))
    times, stats = timed(default_opts(graph_loop=1, **sched))
    bflows = [h.flow_value() for h in handles]
    assert bflows == flows, "batched and single solves disagree"
    bms = statistics.median(times)
    line = {"metric": METRIC, "workload": "batch", "value": round(bms / len(insts), 4), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": "uneven batch: 384 2D 4-conn grids side U{64..1024} + 128 3D 6-conn side "
                                   "U{48..128} (first %d), segmentation / volume generators" % len(insts),
                       "instances": len(insts), "vertices": nv, "autotune": table, "schedule": sched},
            "batch_ms": round(bms, 3), "batch_ms_host_loop": round(statistics.median(host_times), 3),
            "plain_sequential_ms": round(plain_ms, 3),
            "plain_ms_per_instance": round(plain_ms / len(insts), 4),
            "speedup_vs_plain": round(plain_ms / bms, 3),
            "sweeps_per_instance_batch": sum(s.sweeps for s in stats) / len(insts),
            "sweeps_per_instance_plain": plain_sweeps / len(insts),
            "vertices_per_s_batch": nv / (bms * 1e-3)}
    for h in handles:
        h.close()
    print(json.dumps(line), flush=True)


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
    insts = [grids.config3(warmstart.EVAL_SEED0 + i) for i in range(count)]
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
    cases = [("seg2d 2048x2048 8-connected (config of the headline)", lambda: grids.config1(0), (32, 32, 1), glr),
             ("seg2d 1024x1024 4-connected, held-out seed of the warm-start set",
              lambda: grids.config3(warmstart.EVAL_SEED0), (32, 32, 1), glr),
             ("seg2d 256x256 4-connected", lambda: grids.config0(0), (32, 32, 1), glr),
             ("volume 256x256x128 6-connected", lambda: grids.config2(0, dims=(256, 256, 128)), (32, 8, 4), glr),
             ("volume 256x256x128 6-connected, 16^3 tiles (no global relabel)",
              lambda: grids.config2(0, dims=(256, 256, 128)), (16, 16, 16), no_glr),
             ("volume 512x512x384 6-connected", lambda: grids.config2(0), (32, 8, 4),
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


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    inst = make_instance(seed=0, side=REF_SAMPLE_SIDE)
    scale = (SIDE * SIDE) / inst.n
    for _ in range(args.warmup):
        oracle.solve_instance(inst)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve_instance(inst)
    t1 = time.perf_counter()
    value = (t1 - t0) * 1e3 / args.steps * scale
    sample = (f"{REF_SAMPLE_SIDE}x{REF_SAMPLE_SIDE} instance of the same recipe per step (1/{scale:g} of the "
              f"vertices), time scaled x{scale:g} to one {SIDE}x{SIDE} instance")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value, 2),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": workload_name(), "vertices": SIDE * SIDE,
                                            "parallelism": "1 host thread"},
            "cpu_baseline": {"value": round(value, 2), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 2), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="seg2048", choices=["seg2048", "batch", "batch_warm", "relabel"])
    ap.add_argument("--batch-count", type=int, default=0, help="first N instances of the batch (0 = all 512)")
    ap.add_argument("--relabel-case", type=int, default=-1, help="relabel workload: only this instance (index)")
    ap.add_argument("--relabel-schedule", default="", help="relabel workload: only this schedule")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "batch_warm":
        run_batch_warm(args)
    elif args.workload == "relabel":
        run_relabel(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
