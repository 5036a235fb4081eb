"""Region reduction (Sec. 8, Algorithm "Region Reduction (G^R, B^R)") —
TEST INFRASTRUCTURE: only the tests may import this module.

For every region R of a tiling the region network G^R holds the vertices of
R with their terminal links, the neighbour arcs inside R, and the neighbour
arcs between R and its boundary B^R (the vertices outside R adjacent to R)
in both directions; boundary vertices have no terminal links and no arcs
among themselves.  Starting from the zero flow the algorithm
  1. augments s -> t to a maximum flow;
  2. splits the boundary into B^S = {v in B^R : s -> v} and
     B^T = {v in B^R : v -> t} (disjoint after step 1);
  3. augments s -> B^S (B^S as sinks);
  4. augments B^T -> t (B^T as sources);
  5. classifies each vertex v of R in the final residual network:
     s -> v: strong source; v -> t: strong sink; otherwise v is a weak source
     if v cannot reach B^R and a weak sink if B^R cannot reach v.
The section's argument (a path of G leaving R passes through B^R) makes
these classes hold for the whole network G: a strong source is on the source
side of every minimum cut, a strong sink on the sink side of every one, a
weak source / sink on that side of some minimum cut.

Plain augmenting paths by breadth-first search on the explicit network
(pure Python: small grids only).
"""
from __future__ import annotations

from collections import deque

import numpy as np

STRONG_SOURCE, STRONG_SINK, WEAK_SOURCE, WEAK_SINK = 1, 2, 4, 8
_INF = 1 << 60

_FWD = {4: ((1, 0, 0), (0, 1, 0)),
        8: ((1, 0, 0), (0, 1, 0), (1, 1, 0), (-1, 1, 0)),
        6: ((1, 0, 0), (0, 1, 0), (0, 0, 1))}


class _Net:
    """Residual network with paired arcs (arc e and its reverse e ^ 1)."""

    def __init__(self, n):
        self.adj = [[] for _ in range(n)]
        self.to, self.cap = [], []

    def add(self, u, v, c):
        self.adj[u].append(len(self.to))
        self.to.append(v)
        self.cap.append(c)
        self.adj[v].append(len(self.to))
        self.to.append(u)
        self.cap.append(0)
        return len(self.to) - 2

    def augment(self, src, dst):
        """Augment along shortest residual paths from node src to node dst
        until none is left; returns the flow sent."""
        total = 0
        while True:
            prev = {src: -1}
            q = deque([src])
            while q and dst not in prev:
                u = q.popleft()
                for e in self.adj[u]:
                    w = self.to[e]
                    if self.cap[e] > 0 and w not in prev:
                        prev[w] = e
                        q.append(w)
            if dst not in prev:
                return total
            path, w = [], dst
            while w != src:
                e = prev[w]
                path.append(e)
                w = self.to[e ^ 1]
            d = min(self.cap[e] for e in path)
            for e in path:
                self.cap[e] -= d
                self.cap[e ^ 1] += d
            total += d

    def reach(self, seeds, skip=(), backward=False):
        """Nodes reachable from the seeds over residual arcs (backward: nodes
        that reach a seed), never entering the nodes in skip."""
        seen = set(seeds)
        q = deque(seeds)
        while q:
            u = q.popleft()
            for e in self.adj[u]:
                w = self.to[e]
                ok = self.cap[e ^ 1] > 0 if backward else self.cap[e] > 0
                if ok and w not in seen and w not in skip:
                    seen.add(w)
                    q.append(w)
        return seen


def region_reduction(dims, conn, tile, cs, ct, nlink):
    """Classes of every vertex (uint8 bit set of STRONG_SOURCE, STRONG_SINK,
    WEAK_SOURCE, WEAK_SINK) and, per region, the checks the section states:
    dict(codes, regions=[dict(BS, BT, s_to_boundary_or_t, boundary_or_s_to_t)])."""
    X, Y, Z = (tuple(int(d) for d in dims) + (1, 1))[:3]
    tx, ty, tz = (tuple(tile) + (1, 1))[:3]
    n = X * Y * Z
    H = len(_FWD[conn])
    cs = np.asarray(cs, dtype=np.int64).ravel()
    ct = np.asarray(ct, dtype=np.int64).ravel()
    nl = np.asarray(nlink, dtype=np.int64).reshape(H, n)
    RX, RY, RZ = -(-X // tx), -(-Y // ty), -(-Z // tz)

    def idx(x, y, z):
        return (z * Y + y) * X + x

    codes = np.zeros(n, dtype=np.uint8)
    info = []
    for rz in range(RZ):
        for ry in range(RY):
            for rx in range(RX):
                R = [idx(x, y, z) for z in range(rz * tz, min(Z, rz * tz + tz))
                     for y in range(ry * ty, min(Y, ry * ty + ty)) for x in range(rx * tx, min(X, rx * tx + tx))]
                inR = set(R)
                local = {v: i for i, v in enumerate(R)}
                edges = []  # (u, w, c) with u in R
                for v in R:
                    x, y, z = v % X, (v // X) % Y, v // (X * Y)
                    for h, (dx, dy, dz) in enumerate(_FWD[conn]):
                        for sg in (1, -1):
                            x2, y2, z2 = x + sg * dx, y + sg * dy, z + sg * dz
                            if not (0 <= x2 < X and 0 <= y2 < Y and 0 <= z2 < Z):
                                continue
                            w = idx(x2, y2, z2)
                            c = int(nl[h, v] if sg > 0 else nl[h, w])
                            if w in inR and w < v:
                                continue  # each inner edge once
                            if w not in inR and w not in local:
                                local[w] = len(local)
                            edges.append((v, w, c))
                B = [w for w in local if w not in inR]
                s, t = len(local), len(local) + 1
                net = _Net(len(local) + 4)
                for (u, w, c) in edges:
                    net.add(local[u], local[w], c)
                    net.add(local[w], local[u], c)
                for v in R:
                    net.add(s, local[v], int(cs[v]))
                    net.add(local[v], t, int(ct[v]))
                Bl = [local[w] for w in B]
                # 1. s -> t
                net.augment(s, t)
                # 2. boundary split
                from_s = net.reach([s])
                to_t = net.reach([t], backward=True)
                BS = [b for b in Bl if b in from_s]
                BT = [b for b in Bl if b in to_t]
                # 3. s -> B^S through a super sink; 4. B^T -> t from a super source
                # (each super terminal leaves the network before the next step:
                # it is not part of G^R)
                ss, tt = len(local) + 2, len(local) + 3
                sink_arcs = [net.add(b, tt, _INF) for b in BS]
                net.augment(s, tt)
                for e in sink_arcs:
                    net.cap[e] = net.cap[e ^ 1] = 0
                source_arcs = [net.add(ss, b, _INF) for b in BT]
                net.augment(ss, t)
                for e in source_arcs:
                    net.cap[e] = net.cap[e ^ 1] = 0
                skip = (ss, tt)
                from_s = net.reach([s], skip)
                to_t = net.reach([t], skip, backward=True)
                to_B = net.reach(Bl, skip, backward=True)
                from_B = net.reach(Bl, skip)
                for v in R:
                    i = local[v]
                    c = 0
                    if i in from_s:
                        c |= STRONG_SOURCE
                    if i in to_t:
                        c |= STRONG_SINK
                    if not c:
                        if i not in to_B:
                            c |= WEAK_SOURCE
                        if i not in from_B:
                            c |= WEAK_SINK
                    codes[v] = c
                info.append({"BS": sorted(B[Bl.index(b)] for b in BS), "BT": sorted(B[Bl.index(b)] for b in BT),
                             "s_to_boundary_or_t": bool((set(Bl) | {t}) & from_s),
                             "boundary_or_s_to_t": bool((set(Bl) | {s}) & to_t)})
    return {"codes": codes, "regions": info}


def reduce_instance(dims, conn, cs, ct, nlink, codes):
    """The network with the strong source vertices merged into s and the
    strong sink vertices into t (every minimum cut already puts them there):
    for a vertex w left open, cs'(w) = cs(w) + c(edges of w to strong
    sources), ct'(w) = ct(w) + c(edges of w to strong sinks); edges with a
    merged endpoint and the terminal links of merged vertices are removed.
    Every cut that keeps S* on the source side and T* on the sink side costs
    the reduced network's cut plus the constant
        K = sum_{S*} ct + sum_{T*} cs + c(S*, T*).
    Returns (cs', ct', nlink', K)."""
    X, Y, Z = (tuple(int(d) for d in dims) + (1, 1))[:3]
    n = X * Y * Z
    H = len(_FWD[conn])
    cs = np.asarray(cs, dtype=np.int64).ravel()
    ct = np.asarray(ct, dtype=np.int64).ravel()
    nl = np.asarray(nlink, dtype=np.int64).reshape(H, n).copy()
    codes = np.asarray(codes).ravel()
    S = (codes & STRONG_SOURCE) != 0
    T = (codes & STRONG_SINK) != 0
    cs2, ct2 = cs.copy(), ct.copy()
    K = int(ct[S].sum() + cs[T].sum())
    for h, (dx, dy, dz) in enumerate(_FWD[conn]):
        for v in range(n):
            c = int(nl[h, v])
            if c == 0:
                continue
            x, y, z = v % X, (v // X) % Y, v // (X * Y)
            w = ((z + dz) * Y + (y + dy)) * X + (x + dx)
            if (S[v] and T[w]) or (T[v] and S[w]):
                K += c
            if not (S[v] or T[v]):
                cs2[v] += c if S[w] else 0
                ct2[v] += c if T[w] else 0
            if not (S[w] or T[w]):
                cs2[w] += c if S[v] else 0
                ct2[w] += c if T[v] else 0
            if S[v] or T[v] or S[w] or T[w]:
                nl[h, v] = 0
    cs2[S | T] = 0
    ct2[S | T] = 0
    return cs2.astype(np.int32), ct2.astype(np.int32), nl.astype(np.int32), K
