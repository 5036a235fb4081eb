"""CPU oracle of the warm start's projection to a preflow — TEST
INFRASTRUCTURE ONLY (the solver library never calls it).

The paper starts from the zero flow (Init, Sec. 2) and says nothing of a
predicted start; this is the plain statement of the projection rule the
library uses, written with numpy over whole arrays:

  * edge flow of the edge (v, v + h-th forward offset) = the prediction of
    its lower endpoint v in channel 2h, times S = 100 in float32, rounded to
    the nearest integer (ties to even), clamped to [-c, c] (0 if c = 0);
  * sink flow = channel N+1 times S, rounded, clamped to [0, ct - min(cs,ct)];
  * every s-link saturated, min(cs, ct) sent straight from s to t;
  * synchronous rounds: every vertex with negative excess lowers its own
    outflows — sink flow first, then arcs 0..N-1 in order — by its deficit,
    until no excess is negative (or the round cap).

Pinned in tests/test_oracle_warm.py (hand case, preflow properties, and the
projection of a valid preflow returning it unchanged in zero rounds).
"""
from __future__ import annotations

import numpy as np

from . import _FWD, _dims

SCALE = np.float32(100.0)


def project(dims, conn, cs, ct, nlink, pred, max_rounds=4096):
    """Returns (F [H, n] int64 edge flows, ft [n] sink flows, E [n] excess,
    rounds), or None if max_rounds trim rounds left a negative excess."""
    X, Y, Z = _dims(dims).tolist()
    n = X * Y * Z
    fwd = _FWD[conn]
    H = len(fwd)
    cs = np.asarray(cs, dtype=np.int64)
    ct = np.asarray(ct, dtype=np.int64)
    nl = np.asarray(nlink, dtype=np.int64).reshape(H, n)
    p = np.asarray(pred, dtype=np.float32).reshape(2 * H + 2, n)
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    xx, yy, zz = xx.ravel(), yy.ravel(), zz.ravel()
    head_in = []   # does v + fwd_h lie in the grid
    tail = []      # index of v - fwd_h, -1 outside
    for dx, dy, dz in fwd:
        ok = (xx + dx < X) & (xx + dx >= 0) & (yy + dy < Y) & (yy + dy >= 0) & (zz + dz < Z) & (zz + dz >= 0)
        head_in.append(ok)
        tx, ty, tz = xx - dx, yy - dy, zz - dz
        okt = (tx >= 0) & (tx < X) & (ty >= 0) & (ty < Y) & (tz >= 0) & (tz < Z)
        tail.append(np.where(okt, (tz * Y + ty) * X + tx, -1))
    F = np.zeros((H, n), dtype=np.int64)
    for h in range(H):
        c = np.where(head_in[h], nl[h], 0)
        f = np.rint(p[2 * h] * SCALE).astype(np.int64)
        F[h] = np.where(c > 0, np.clip(f, -c, c), 0)
    m = np.minimum(cs, ct)
    ft = np.clip(np.rint(p[2 * H + 1] * SCALE).astype(np.int64), 0, ct - m)
    base = cs - m

    def excess():
        e = base - ft - F.sum(axis=0)
        for h in range(H):
            t = tail[h]
            e = e + np.where(t >= 0, F[h][np.maximum(t, 0)], 0)
        return e

    for r in range(max_rounds + 1):
        E = excess()
        if (E >= 0).all():
            return F, ft, E, r
        if r == max_rounds:
            return None
        deficit = np.maximum(-E, 0)
        take = np.minimum(ft, deficit)
        ft = ft - take
        deficit = deficit - take
        for d in range(2 * H):
            h = d >> 1
            if d % 2 == 0:   # own forward edge: positive flow is an outflow
                take = np.where(F[h] > 0, np.minimum(F[h], deficit), 0)
                F[h] = F[h] - take
            else:            # edge from v - fwd_h: negative flow is an outflow of v
                t = tail[h]
                ok = t >= 0
                fl = np.where(ok, F[h][np.maximum(t, 0)], 0)
                take = np.where(ok & (fl < 0), np.minimum(-fl, deficit), 0)
                np.add.at(F[h], t[take > 0], take[take > 0])
            deficit = deficit - take
    return None


def residual(dims, conn, cs, ct, nlink, F, ft):
    """Residual network (res [2H, n], tres, exc) of the preflow (F, ft) with
    every s-link saturated, in the solver's layout."""
    X, Y, Z = _dims(dims).tolist()
    n = X * Y * Z
    fwd = _FWD[conn]
    H = len(fwd)
    nl = np.asarray(nlink, dtype=np.int64).reshape(H, n)
    cs = np.asarray(cs, dtype=np.int64)
    ct = np.asarray(ct, dtype=np.int64)
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    xx, yy, zz = xx.ravel(), yy.ravel(), zz.ravel()
    res = np.zeros((2 * H, n), dtype=np.int64)
    exc = cs - np.minimum(cs, ct) - ft
    for h, (dx, dy, dz) in enumerate(fwd):
        ok = (xx + dx < X) & (xx + dx >= 0) & (yy + dy < Y) & (yy + dy >= 0) & (zz + dz < Z) & (zz + dz >= 0)
        c = np.where(ok, nl[h], 0)
        res[2 * h] = c - F[h]
        w = np.where(ok, ((zz + dz) * Y + (yy + dy)) * X + (xx + dx), 0)
        rev = np.zeros(n, dtype=np.int64)
        np.add.at(rev, w[ok], c[ok] + F[h][ok])   # arc w -> v of the same edge: c + f(v, w)
        res[2 * h + 1] = rev
        exc -= F[h]
        np.add.at(exc, w[ok], F[h][ok])
    tres = ct - np.minimum(cs, ct) - ft
    return res, tres, exc
