"""Autotuner: region tile shape and sweep schedule per (connectivity, size
class), for batched solves and for single solves.

For every class present in a list of instances it solves one representative
instance (real data from the list) with each candidate configuration through
the C ABI, keeps the fastest by the library's own device timing, and caches
the choice in a JSON file so later runs reuse it.  Candidates vary the tile,
partial discharges, the global-relabel period and the boundary-relabel
heuristic (Sec. 6.1).
"""
from __future__ import annotations

import hashlib
import json
import math
import os

from .mf import Grid, default_opts

# (tile, schedule) candidates per connectivity
CANDIDATES = {
    4: [((64, 64, 1), {}), ((32, 32, 1), {}), ((64, 32, 1), {}), ((64, 64, 1), {"partial_discharge": 1}),
        ((32, 32, 1), {"partial_discharge": 1})],
    8: [((64, 64, 1), {}), ((32, 32, 1), {}), ((64, 32, 1), {}), ((64, 64, 1), {"partial_discharge": 1}),
        ((32, 32, 1), {"partial_discharge": 1})],
    6: [((32, 8, 4), {}), ((32, 4, 4), {}), ((32, 8, 8), {}), ((32, 16, 8), {}), ((32, 8, 4), {"partial_discharge": 1})],
}


# global-relabel periods tried (0 = never); the relabel exists for 2D tiles and
# for 3D tiles 32 voxels wide
GLR_PERIODS = (0, 2, 4, 8)
# boundary-relabel period tried without the global relabel (any tile)
BR_PERIOD = 2


def _relabel_supported(conn: int, tile) -> bool:
    return conn != 6 or tile[0] == 32


def candidates(conn: int, single: bool = False):
    """(tile, opts kwargs) candidates of one connectivity (the same for single
    and batched solves; `single` only separates the cache entries)."""
    out = []
    for t, kw in CANDIDATES[conn]:
        periods = GLR_PERIODS if _relabel_supported(conn, t) else (0,)
        out += [(t, dict(kw, global_relabel_period=p)) for p in periods]
        out.append((t, dict(kw, global_relabel_period=0, boundary_relabel_period=BR_PERIOD)))
    return out


def size_class(dims) -> int:
    """Half-octave bucket of the number of vertices."""
    n = 1
    for d in dims:
        n *= max(1, int(d))
    return int(round(2 * math.log2(n)))


def key_of(inst, single: bool = False) -> str:
    """Cache key: connectivity, size class and a digest of the candidate set
    (a cache written for other candidates is not reused)."""
    fp = hashlib.sha1(repr(candidates(inst.conn)).encode()).hexdigest()[:8]
    return f"{'single_' if single else ''}c{inst.conn}_s{size_class(inst.dims)}_{fp}"


def _time_config(inst, tile, kw, reps):
    best = float("inf")
    with Grid(inst.dims, inst.conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        opts = default_opts(**kw)
        for _ in range(reps + 1):
            st = g.solve(opts)
            best = min(best, st.ms_total)
    return best


def tune(instances, cache_path: str | None = None, reps: int = 2, single: bool = False):
    """Return {class key: {"tile": [...], "opts": {...}, "ms": t}} for the
    classes of `instances` (objects with dims, conn, cs, ct, nlink); with
    `single`, for single solves (keys prefixed "single_")."""
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    reps_by_key = {}
    for inst in instances:
        reps_by_key.setdefault(key_of(inst, single), inst)
    changed = False
    for k, inst in reps_by_key.items():
        if k in cache:
            continue
        trials = []
        for tile, kw in candidates(inst.conn, single):
            trials.append((_time_config(inst, tile, kw, reps), tile, kw))
        t, tile, kw = min(trials, key=lambda x: x[0])
        cache[k] = {"tile": list(tile), "opts": kw, "ms": t}
        changed = True
    if cache_path and changed:
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return cache


def choose(inst, table, single: bool = False):
    """(tile, opts kwargs) chosen for one instance."""
    e = table[key_of(inst, single)]
    return tuple(e["tile"]), dict(e["opts"])


def batch_schedule(instances, table):
    """One schedule for a whole batch (a batch runs one set of options): the
    choice of the class that holds the most vertices."""
    weight = {}
    for inst in instances:
        weight[key_of(inst)] = weight.get(key_of(inst), 0) + inst.n
    k = max(weight, key=weight.get)
    return dict(table[k]["opts"])
