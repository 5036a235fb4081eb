"""Pins of the projection oracle (oracle/warm.py) and the region-distance
oracle (oracle.region_distance), on the CPU."""
import numpy as np
import pytest

import oracle
from gen import grids
from oracle import warm


def _flows_of(inst, st):
    """Edge flows and sink flows of a residual state (solver layout)."""
    H = inst.nlink.shape[0]
    X, Y, Z = inst.dims
    n = X * Y * Z
    F = np.zeros((H, n), dtype=np.int64)
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    xx, yy, zz = xx.ravel(), yy.ravel(), zz.ravel()
    for h, (dx, dy, dz) in enumerate(grids.FWD[inst.conn]):
        ok = (xx + dx >= 0) & (xx + dx < X) & (yy + dy < Y) & (yy + dy >= 0) & (zz + dz < Z)
        F[h] = np.where(ok, inst.nlink[h].astype(np.int64) - st["res"][2 * h], 0)
    m = np.minimum(inst.cs, inst.ct).astype(np.int64)
    ft = inst.ct.astype(np.int64) - m - st["tres"]
    return F, ft


def test_hand_chain():
    # 1x3 chain, cs = [5,0,0], ct = [0,0,5], links 4 and 4.  Predicted flows 7
    # and 6 clamp to 4 and 4; the predicted sink flow 9 clamps to 5; v2 then
    # receives 4 and sends 5: one trim round lowers its sink flow to 4.
    cs = np.array([5, 0, 0]); ct = np.array([0, 0, 5]); nl = np.array([[4, 4, 0], [0, 0, 0]])
    pred = np.zeros((6, 3), dtype=np.float32)
    pred[0, 0], pred[0, 1], pred[5, 2] = 0.07, 0.06, 0.09
    F, ft, E, rounds = warm.project((3, 1, 1), 4, cs, ct, nl, pred)
    assert rounds == 1
    assert F[0].tolist() == [4, 4, 0] and F[1].tolist() == [0, 0, 0]
    assert ft.tolist() == [0, 0, 4] and E.tolist() == [1, 0, 0]


@pytest.mark.parametrize("conn,dims", [(4, (23, 17, 1)), (8, (19, 15, 1)), (6, (9, 8, 7))])
def test_a_valid_preflow_projects_to_itself(conn, dims):
    inst = (grids.volume_3d(*dims, seed=3) if conn == 6 else
            grids.segmentation_2d(dims[0], dims[1], 3, conn=conn, hard_seed_frac=0.05))
    st = oracle.maxflow_state(inst.dims, conn, inst.cs, inst.ct, inst.nlink)
    F0, ft0 = _flows_of(inst, st)
    H = len(grids.FWD[conn])
    pred = np.zeros((2 * H + 2, inst.n), dtype=np.float32)
    for h in range(H):
        pred[2 * h] = F0[h].astype(np.float32) / np.float32(100)
    pred[2 * H + 1] = ft0.astype(np.float32) / np.float32(100)
    F, ft, E, rounds = warm.project(inst.dims, conn, inst.cs, inst.ct, inst.nlink, pred)
    assert rounds == 0
    np.testing.assert_array_equal(F, F0)
    np.testing.assert_array_equal(ft, ft0)
    res, tres, exc = warm.residual(inst.dims, conn, inst.cs, inst.ct, inst.nlink, F, ft)
    np.testing.assert_array_equal(res, st["res"])
    np.testing.assert_array_equal(tres, st["tres"])
    np.testing.assert_array_equal(exc, st["exc"])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_projection_gives_a_preflow_and_only_lowers_flows(seed):
    inst = grids.segmentation_2d(31, 22, seed, conn=8)
    rng = np.random.Generator(np.random.PCG64(seed))
    pred = (rng.standard_normal((10, inst.n)) * 0.6).astype(np.float32)
    F, ft, E, rounds = warm.project(inst.dims, 8, inst.cs, inst.ct, inst.nlink, pred)
    assert (E >= 0).all() and rounds > 0
    res, tres, exc = warm.residual(inst.dims, 8, inst.cs, inst.ct, inst.nlink, F, ft)
    assert (res >= 0).all() and (tres >= 0).all()
    np.testing.assert_array_equal(exc, E)
    # the clamped prediction itself is not a preflow here, so the round cap 0 fails
    assert warm.project(inst.dims, 8, inst.cs, inst.ct, inst.nlink, pred, max_rounds=0) is None
    # trimming only moves flows toward zero
    for h in range(4):
        c = inst.nlink[h].astype(np.int64)
        raw = np.clip(np.rint(pred[2 * h] * np.float32(100)).astype(np.int64), -c, c)
        assert (np.abs(F[h]) <= np.abs(raw)).all() and (F[h] * raw >= 0).all()


def test_region_distance_matches_dijkstra():
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    for conn, dims, tile, seed in [(4, (13, 11, 1), (4, 4, 1), 0), (8, (12, 9, 1), (4, 4, 1), 1),
                                   (6, (7, 6, 5), (4, 4, 2), 2)]:
        rng = np.random.Generator(np.random.PCG64(seed))
        X, Y, Z = dims
        n = X * Y * Z
        H = len(grids.FWD[conn])
        res = (rng.random((2 * H, n)) < 0.55).astype(np.int32)
        tres = (rng.random(n) < 0.08).astype(np.int32)
        got = oracle.region_distance(dims, conn, tile, res, tres)
        # Dijkstra from t on the reversed residual graph: weight 1 across
        # regions, 1e-6 inside (scipy drops explicit zero weights)
        rows, cols, wts = [], [], []
        zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
        xx, yy, zz = xx.ravel(), yy.ravel(), zz.ravel()
        tx, ty, tz = tile
        reg = (zz // tz * ((Y + ty - 1) // ty) + yy // ty) * ((X + tx - 1) // tx) + xx // tx
        for h, (dx, dy, dz) in enumerate(grids.FWD[conn]):
            for d, sg in ((2 * h, 1), (2 * h + 1, -1)):
                wx, wy, wz = xx + sg * dx, yy + sg * dy, zz + sg * dz
                ok = (wx >= 0) & (wx < X) & (wy >= 0) & (wy < Y) & (wz >= 0) & (wz < Z) & (res[d] > 0)
                u = np.flatnonzero(ok)
                w = ((wz * Y + wy) * X + wx)[ok]
                rows += list(w + 1)      # reversed arc w -> u; node 0 is t
                cols += list(u + 1)
                wts += list(np.where(reg[u] == reg[w], 1e-6, 1.0))
        tv = np.flatnonzero(tres > 0)
        rows += [0] * len(tv); cols += list(tv + 1); wts += [1e-6] * len(tv)
        G = sp.csr_matrix((wts, (rows, cols)), shape=(n + 1, n + 1))
        dist = csgraph.dijkstra(G, directed=True, indices=0)[1:]
        ref = np.where(np.isfinite(dist), np.floor(dist + 0.5), -1).astype(np.int64)
        np.testing.assert_array_equal(got, ref)


def _project_one_at_a_time(dims, conn, cs, ct, nlink, pred, order_seed):
    """The projection's trims applied one vertex at a time in a random order
    (each vertex trims its current deficit from the current flows), instead
    of in synchronous rounds: a plain loop written from the rule, sharing
    nothing with oracle.warm beyond its initial rounding and clamping."""
    X, Y, Z = (tuple(dims) + (1, 1))[:3]
    n = X * Y * Z
    fwd = grids.FWD[conn]
    H = len(fwd)
    res = warm.project(dims, conn, cs, ct, nlink, pred, max_rounds=0)
    assert res is None or res[3] == 0
    # the initial flows: zero rounds of trimming
    p = np.asarray(pred, dtype=np.float32).reshape(2 * H + 2, n)
    nl = np.asarray(nlink, dtype=np.int64).reshape(H, n)
    F = np.zeros((H, n), dtype=np.int64)
    for v in range(n):
        x, y, z = v % X, (v // X) % Y, v // (X * Y)
        for h, (dx, dy, dz) in enumerate(fwd):
            if 0 <= x + dx < X and 0 <= y + dy < Y and 0 <= z + dz < Z and nl[h, v] > 0:
                F[h, v] = int(np.clip(np.rint(p[2 * h, v] * np.float32(100.0)), -nl[h, v], nl[h, v]))
    cs = np.asarray(cs, dtype=np.int64); ct = np.asarray(ct, dtype=np.int64)
    m = np.minimum(cs, ct)
    ft = np.clip(np.rint(p[2 * H + 1] * np.float32(100.0)).astype(np.int64), 0, ct - m)

    def tail_of(v, h):
        x, y, z = v % X, (v // X) % Y, v // (X * Y)
        dx, dy, dz = fwd[h]
        if 0 <= x - dx < X and 0 <= y - dy < Y and 0 <= z - dz < Z:
            return ((z - dz) * Y + (y - dy)) * X + (x - dx)
        return -1

    def excess(v):
        e = cs[v] - m[v] - ft[v] - F[:, v].sum()
        for h in range(H):
            w = tail_of(v, h)
            if w >= 0:
                e += F[h, w]
        return e

    rng = np.random.default_rng(order_seed)
    while True:
        changed = False
        for v in rng.permutation(n):
            d = -excess(v)
            if d <= 0:
                continue
            changed = True
            t = min(ft[v], d); ft[v] -= t; d -= t
            for a in range(2 * H):
                h = a >> 1
                if a % 2 == 0 and F[h, v] > 0:
                    t = min(F[h, v], d); F[h, v] -= t; d -= t
                elif a % 2 == 1:
                    w = tail_of(v, h)
                    if w >= 0 and F[h, w] < 0:
                        t = min(-F[h, w], d); F[h, w] += t; d -= t
            if d > 0:
                return None
        if not changed:
            return F, ft


@pytest.mark.parametrize("conn,dims", [(4, (13, 11, 1)), (8, (12, 9, 1))])
@pytest.mark.parametrize("seed", range(3))
def test_trim_order_does_not_matter(conn, dims, seed):
    """The synchronous rounds reach the least fixed point of a monotone map
    (trim totals only grow, and a vertex's deficit only grows when its
    neighbours trim), so trimming the vertices in any order reaches the same
    flows: the basis for computing the projection tile by tile."""
    inst = grids.random_grid(dims, conn, 40 + seed, cmax=20, tmax=40, p_zero=0.2)
    H = len(grids.FWD[conn])
    rng = np.random.default_rng(seed)
    pred = rng.normal(0.1, 0.15, size=(2 * H + 2, inst.n)).astype(np.float32)
    want = warm.project(inst.dims, conn, inst.cs, inst.ct, inst.nlink, pred)
    assert want is not None and want[3] > 1  # several rounds: the order matters for the path, not the end
    for order in range(3):
        got = _project_one_at_a_time(inst.dims, conn, inst.cs, inst.ct, inst.nlink, pred, order)
        assert got is not None
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
