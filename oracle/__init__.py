"""CPU oracle for the grid s-t min-cut / max-flow problem — TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The solver library never calls it and
shares no code with it: the C sources here (``dinic.c``, ``verify.c``) and the
Python below implement the plain definitions of Sec. 2 of the paper
(Shekhovtsov & Hlavac, "A Distributed Mincut/Maxflow Algorithm Combining Path
Augmentation and Push-Relabel"):

  * ``maxflow``     — Dinic on the explicit s-t network (Sec. 2, Eq. 1);
  * ``verify``      — preflow feasibility, maximality and the cut-cost
                      certificate of a claimed solution (Sec. 2);
  * ``brute_force`` — exhaustive enumeration of all 2^n source sets of Eq. 1
                      (n <= 20): the minimum cost, S_min = intersection of all
                      minimisers, S_max = union of all minimisers;
  * ``chain_min_cut`` — the exact minimum of Eq. 1 on a 1 x n chain by dynamic
                      programming over the two sides (a closed form that shares
                      nothing with max-flow);
  * ``boundary_size`` — |B| of Sec. 4.1 (the union of the region boundaries
                      B^R of Eq. 2) by its definition, and the sweep bound
                      2|B|^2 + 1 of the P-ARD termination theorem (Sec. 4.4);
  * ``region_distance`` — the region distance d* of Sec. 4.1 (eq. 3) by a
                      0-1 BFS over the residual graph;
  * ``boundary_relabel`` — the boundary-relabel heuristic of Sec. 6.1 on an
                      explicit auxiliary graph of (region, label) groups.
  The stencils are the 4/8-connected 2D and 6-connected 3D grids and the
  synthetic networks of Sec. 7.1 (connectivity code 100 + c).
  ``oracle.cnn`` and ``oracle.warm`` hold the float64 warm-start network and
  the projection of a prediction to a preflow; ``oracle.reduction`` the
  region reduction of Sec. 8 on explicit per-region networks.

Every function here is pinned by the ``-m "not gpu"`` tests against values
fixed by mathematics (brute force on tiny inputs, closed forms, special
cases), not against itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "_lib")
_LIBPATH = os.path.join(_LIBDIR, "liboracle.so")
_SOURCES = [os.path.join(_HERE, f) for f in ("dinic.c", "verify.c")]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_lib/liboracle.so (gcc, -O2)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES)
    if not force and os.path.exists(_LIBPATH) and os.path.getmtime(_LIBPATH) >= newest:
        return _LIBPATH
    tmp = _LIBPATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp] + _SOURCES)
    os.replace(tmp, _LIBPATH)
    return _LIBPATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIBPATH)
            P = ctypes.c_void_p
            lib.orc_maxflow.restype = ctypes.c_int64
            lib.orc_maxflow.argtypes = [P, ctypes.c_int, P, P, P, P, P, P]
            lib.orc_maxflow_state.restype = ctypes.c_int64
            lib.orc_maxflow_state.argtypes = [P, ctypes.c_int, P, P, P, P, P, P]
            lib.orc_cut_cost.restype = ctypes.c_int64
            lib.orc_cut_cost.argtypes = [P, ctypes.c_int, P, P, P, P]
            lib.orc_closure.restype = None
            lib.orc_closure.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
            lib.orc_verify.restype = ctypes.c_int
            lib.orc_verify.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, ctypes.c_int64, P, P,
                                       ctypes.c_char_p, ctypes.c_int, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dims(dims):
    X, Y, Z = (tuple(dims) + (1, 1))[:3]
    return np.array([X, Y, Z], dtype=np.int64)


def maxflow(dims, conn, cs, ct, nlink):
    """Dinic on the explicit network -> dict(flow, smin, smax, phases)."""
    lib = _load()
    d = _dims(dims)
    n = int(np.prod(d))
    cs, ct, nl = _i32(cs), _i32(ct), _i32(nlink)
    smin = np.zeros(n, dtype=np.uint8)
    smax = np.zeros(n, dtype=np.uint8)
    ph = np.zeros(1, dtype=np.int64)
    f = lib.orc_maxflow(_p(d), conn, _p(cs), _p(ct), _p(nl), _p(smin), _p(smax), _p(ph))
    if f < 0:
        raise RuntimeError(f"orc_maxflow failed ({f})")
    return {"flow": int(f), "smin": smin, "smax": smax, "phases": int(ph[0])}


def maxflow_state(dims, conn, cs, ct, nlink):
    """Dinic's maximum flow exported as a maximum preflow in the solver's
    residual layout -> dict(flow, res [2H, n], tres, exc)."""
    lib = _load()
    d = _dims(dims)
    n = int(np.prod(d))
    H = len(_FWD[conn])
    res = np.zeros((2 * H, n), dtype=np.int32)
    tres = np.zeros(n, dtype=np.int32)
    exc = np.zeros(n, dtype=np.int32)
    f = lib.orc_maxflow_state(_p(d), conn, _p(_i32(cs)), _p(_i32(ct)), _p(_i32(nlink)),
                              _p(res), _p(tres), _p(exc))
    if f < 0:
        raise RuntimeError(f"orc_maxflow_state failed ({f})")
    return {"flow": int(f), "res": res, "tres": tres, "exc": exc}


def solve_instance(inst):
    return maxflow(inst.dims, inst.conn, inst.cs, inst.ct, inst.nlink)


def cut_cost(dims, conn, cs, ct, nlink, S):
    """Cost of Eq. 1 for the source set S (uint8/bool per vertex)."""
    lib = _load()
    d = _dims(dims)
    S = np.ascontiguousarray(S, dtype=np.uint8)
    return int(lib.orc_cut_cost(_p(d), conn, _p(_i32(cs)), _p(_i32(ct)), _p(_i32(nlink)), _p(S)))


def closure(dims, conn, res, seeds, backward=False):
    """Residual closure of a seed set (forward: reachable from the seeds;
    backward: vertices that reach the seeds)."""
    lib = _load()
    d = _dims(dims)
    S = np.ascontiguousarray(seeds, dtype=np.uint8).copy()
    lib.orc_closure(_p(d), conn, _p(_i32(res)), 1 if backward else 0, _p(S))
    return S


def verify(dims, conn, cs, ct, nlink, res, tres, exc, flow, smin=None, smax=None):
    """Check a claimed maximum preflow.  Returns (ok, message, info)."""
    lib = _load()
    d = _dims(dims)
    msg = ctypes.create_string_buffer(512)
    out = np.zeros(4, dtype=np.int64)
    smin = None if smin is None else np.ascontiguousarray(smin, dtype=np.uint8)
    smax = None if smax is None else np.ascontiguousarray(smax, dtype=np.uint8)
    rc = lib.orc_verify(_p(d), conn, _p(_i32(cs)), _p(_i32(ct)), _p(_i32(nlink)), _p(_i32(res)),
                        _p(_i32(tres)), _p(_i32(exc)), int(flow), _p(smin), _p(smax), msg, 512, _p(out))
    info = {"flow": int(out[0]), "n_smin": int(out[1]), "n_smax": int(out[2]), "cut_cost": int(out[3])}
    return rc == 0, msg.value.decode(), info


# --- pure-Python pieces --------------------------------------------------------

_FWD = {4: ((1, 0, 0), (0, 1, 0)),
        8: ((1, 0, 0), (0, 1, 0), (1, 1, 0), (-1, 1, 0)),
        6: ((1, 0, 0), (0, 1, 0), (0, 0, 1))}
# The synthetic networks of Sec. 7.1: edges at the listed relative
# displacements, read as (dx, dy); connectivity c takes the first c/2 of them
# (code 100 + c).  The list's first pair, (0,1), (1,0), is kept here as
# (1,0), (0,1) so that its planes are those of the 4-connected grid.
_PAPER_LIST = ((1, 0), (0, 1), (1, 2), (2, 1), (1, 3), (3, 1), (2, 3), (3, 2), (0, 2), (2, 0), (2, 2), (3, 3),
               (3, 4), (4, 2))
for _c in range(8, 29, 4):
    _FWD[100 + _c] = tuple((dx, dy, 0) for dx, dy in _PAPER_LIST[:_c // 2])


def edge_list(dims, conn, nlink):
    """Undirected edges (u, w, c) of the grid, by the forward half-stencil."""
    X, Y, Z = _dims(dims).tolist()
    n = X * Y * Z
    nl = np.asarray(nlink).reshape(len(_FWD[conn]), n)
    edges = []
    for h, (dx, dy, dz) in enumerate(_FWD[conn]):
        for z in range(Z):
            for y in range(Y):
                for x in range(X):
                    xx, yy, zz = x + dx, y + dy, z + dz
                    if 0 <= xx < X and 0 <= yy < Y and 0 <= zz < Z:
                        v = (z * Y + y) * X + x
                        edges.append((v, (zz * Y + yy) * X + xx, int(nl[h, v])))
    return edges


def brute_force(dims, conn, cs, ct, nlink):
    """Enumerate all 2^n source sets of Eq. 1 (n <= 20).

    Returns dict(min_cost, smin, smax, n_min): smin / smax are the
    intersection / union of all minimising source sets."""
    X, Y, Z = _dims(dims).tolist()
    n = X * Y * Z
    if n > 20:
        raise ValueError("brute force is limited to n <= 20")
    masks = np.arange(1 << n, dtype=np.int64)
    bits = ((masks[:, None] >> np.arange(n)[None, :]) & 1).astype(bool)  # [2^n, n]
    cs = np.asarray(cs, dtype=np.int64)
    ct = np.asarray(ct, dtype=np.int64)
    cost = np.where(bits, ct[None, :], cs[None, :]).sum(axis=1)
    for (u, w, c) in edge_list(dims, conn, nlink):
        cost += c * (bits[:, u] != bits[:, w])
    best = cost.min()
    arg = bits[cost == best]
    return {"min_cost": int(best), "smin": arg.all(axis=0).astype(np.uint8),
            "smax": arg.any(axis=0).astype(np.uint8), "n_min": int(len(arg))}


def chain_min_cut(cs, ct, w):
    """Exact minimum of Eq. 1 on a chain v_0 - v_1 - ... - v_{n-1} with edge
    capacities w[i] between v_i and v_{i+1}: Viterbi over the two sides
    (side 1 = source set, paying ct; side 0 pays cs; a side change pays w)."""
    INF = float("inf")
    best = [cs[0], ct[0]]  # [sink side, source side]
    for i in range(1, len(cs)):
        b0 = min(best[0], best[1] + w[i - 1]) + cs[i]
        b1 = min(best[1], best[0] + w[i - 1]) + ct[i]
        best = [b0, b1]
    return int(min(best)) if best[0] < INF else 0


def boundary_mask(dims, conn, tile):
    """B of Sec. 4.1 by its definition: the union over regions R of
    B^R = {w not in R : (u, w) in E for some u in R} (Eq. 2), where E is the
    full grid stencil (zero-capacity arcs included, E being symmetric) and the
    regions are the tiles of the given shape.  A vertex is in B iff it has a
    stencil neighbour in a different tile."""
    X, Y, Z = _dims(dims).tolist()
    tx, ty, tz = (tuple(tile) + (1, 1))[:3]
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    reg = (zz // tz * ((Y + ty - 1) // ty) + yy // ty) * ((X + tx - 1) // tx) + xx // tx
    inB = np.zeros((Z, Y, X), dtype=bool)
    for (dx, dy, dz) in _FWD[conn]:
        for sg in (1, -1):
            ox, oy, oz = sg * dx, sg * dy, sg * dz
            x2, y2, z2 = xx + ox, yy + oy, zz + oz
            ok = (x2 >= 0) & (x2 < X) & (y2 >= 0) & (y2 < Y) & (z2 >= 0) & (z2 < Z)
            r2 = np.zeros_like(reg)
            r2[ok] = reg[z2[ok], y2[ok], x2[ok]]
            inB |= ok & (r2 != reg)
    return inB.ravel()


def boundary_size(dims, conn, tile):
    return int(boundary_mask(dims, conn, tile).sum())


def sweep_bound(dims, conn, tile):
    """2|B|^2 + 1: the P-ARD sweep bound (Sec. 4.4)."""
    b = boundary_size(dims, conn, tile)
    return 2 * b * b + 1


def region_distance(dims, conn, tile, res, tres):
    """Exact region distance d*(u) (Sec. 4.1, eq. 3): the least number of
    inter-region arcs on a residual path from u to t, the arcs inside a region
    counting 0; -1 where t is unreachable.  A 0-1 BFS from {u : c_f(u,t) > 0}
    over reversed residual arcs (pure Python: small grids only)."""
    from collections import deque
    X, Y, Z = _dims(dims).tolist()
    tx, ty, tz = (tuple(tile) + (1, 1))[:3]
    n = X * Y * Z
    H = len(_FWD[conn])
    res = np.asarray(res, dtype=np.int64).reshape(2 * H, n)
    RX, RY = (X + tx - 1) // tx, (Y + ty - 1) // ty

    def coords(v):
        return v % X, (v // X) % Y, v // (X * Y)

    def region(x, y, z):
        return (z // tz * RY + y // ty) * RX + x // tx

    # in-arcs of w: (u, d) with u + D(d) = w and c_f(u -> w) > 0
    arcs = []
    for h, (dx, dy, dz) in enumerate(_FWD[conn]):
        arcs.append((2 * h, dx, dy, dz))
        arcs.append((2 * h + 1, -dx, -dy, -dz))
    dist = np.full(n, -1, dtype=np.int64)
    q = deque()
    for v in np.flatnonzero(np.asarray(tres) > 0):
        dist[v] = 0
        q.append(int(v))
    done = np.zeros(n, dtype=bool)
    while q:
        w = q.popleft()
        if done[w]:
            continue
        done[w] = True
        wx, wy, wz = coords(w)
        rw = region(wx, wy, wz)
        for d, dx, dy, dz in arcs:
            ux, uy, uz = wx - dx, wy - dy, wz - dz
            if not (0 <= ux < X and 0 <= uy < Y and 0 <= uz < Z):
                continue
            u = (uz * Y + uy) * X + ux
            if res[d, u] <= 0:
                continue
            c = 0 if region(ux, uy, uz) == rw else 1
            nd = dist[w] + c
            if dist[u] < 0 or nd < dist[u]:
                dist[u] = nd
                if c == 0:
                    q.appendleft(u)
                else:
                    q.append(u)
    return dist


def boundary_relabel(dims, conn, tile, res, lab, dinf):
    """Boundary-relabel heuristic (Sec. 6.1, the auxiliary graph of its
    figure, the update d := max(d, d')).

    Only boundary vertices (B of Sec. 4.1) with d < d_inf take part.  They are
    grouped by (region, label).  Within a region, consecutive group labels
    l_i < l_{i+1} get a length-0 arc (l_i) -> (l_{i+1}): validity lets a
    vertex reach higher labels of its region but not lower ones.  Every
    residual arc (u, w) between two regions, both ends with d < d_inf, gives a
    length-1 arc group(u) -> group(w).  d' of a group is its distance to the
    groups of label 0 (a 0-1 BFS on reversed arcs), d_inf if none is reached.

    The section defines d' on B only; inner vertices are read here as
    follows (the reading keeps the labeling valid, because d' never
    decreases along a region's label order): a vertex v of region R with
    0 < d(v) < d_inf gets d'(v) = the least d' of R's groups with label >=
    d(v), d_inf if there is none; d(v) = 0 keeps 0.  For a boundary vertex
    this is its own group's d'.  Returns max(d, d') clipped to d_inf
    (int64[n]).  Requires a labeling valid in the strong form the region
    relabel yields (non-increasing along residual arcs inside a region)."""
    from collections import deque
    X, Y, Z = _dims(dims).tolist()
    tx, ty, tz = (tuple(tile) + (1, 1))[:3]
    n = X * Y * Z
    H = len(_FWD[conn])
    res = np.asarray(res, dtype=np.int64).reshape(2 * H, n)
    lab = np.asarray(lab, dtype=np.int64).ravel()
    RX, RY = (X + tx - 1) // tx, (Y + ty - 1) // ty
    inB = boundary_mask(dims, conn, tile)

    def region(v):
        x, y, z = v % X, (v // X) % Y, v // (X * Y)
        return (z // tz * RY + y // ty) * RX + x // tx

    # groups (R, l) of boundary vertices with finite labels
    node = {}
    labels_of = {}
    for u in np.flatnonzero(inB & (lab < dinf)):
        key = (region(int(u)), int(lab[u]))
        if key not in node:
            node[key] = len(node)
            labels_of.setdefault(key[0], []).append(key[1])
    rev = [[] for _ in node]  # rev[b] = [(a, length)] for the arcs a -> b
    for R, ls in labels_of.items():
        ls.sort()
        for a, b in zip(ls, ls[1:]):
            rev[node[(R, b)]].append((node[(R, a)], 0))
    arcs = []
    for h, (dx, dy, dz) in enumerate(_FWD[conn]):
        arcs.append((2 * h, dx, dy, dz))
        arcs.append((2 * h + 1, -dx, -dy, -dz))
    for d, dx, dy, dz in arcs:
        for u in np.flatnonzero(res[d] > 0):
            u = int(u)
            if lab[u] >= dinf:
                continue
            x, y, z = u % X + dx, (u // X) % Y + dy, u // (X * Y) + dz
            if not (0 <= x < X and 0 <= y < Y and 0 <= z < Z):
                continue
            w = (z * Y + y) * X + x
            if lab[w] >= dinf or region(u) == region(w):
                continue
            rev[node[(region(w), int(lab[w]))]].append((node[(region(u), int(lab[u]))], 1))
    # 0-1 BFS from the label-0 groups over reversed arcs
    INF = np.iinfo(np.int64).max
    dist = [INF] * len(node)
    q = deque()
    for (R, l), i in node.items():
        if l == 0:
            dist[i] = 0
            q.append(i)
    while q:
        b = q.popleft()
        for a, ln in rev[b]:
            if dist[b] + ln < dist[a]:
                dist[a] = dist[b] + ln
                (q.appendleft if ln == 0 else q.append)(a)
    out = lab.copy()
    for v in range(n):
        l = int(lab[v])
        if l == 0 or l >= dinf:
            continue
        R = region(v)
        best = INF
        for m in labels_of.get(R, []):
            if m >= l:
                best = min(best, dist[node[(R, m)]])
        out[v] = dinf if best == INF else min(dinf, max(l, best))
    return out
