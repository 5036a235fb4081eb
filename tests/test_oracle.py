"""Pins of the CPU oracle against values fixed by mathematics, not by itself.

* hand-derived minimum cuts (tests/golden/hand_examples.json, Eq. 1 of Sec. 2);
* brute-force enumeration of all 2^n source sets on tiny grids;
* the exact chain minimum by dynamic programming (shares nothing with max-flow);
* closed-form special cases (no neighbour links; neighbour links too strong to cut);
* the preflow verifier accepting Dinic's optimum and rejecting planted mistakes;
* |B| of Sec. 4.1 against a closed-form count of the tile geometry.
"""
import json
import os

import numpy as np
import pytest

import oracle
from gen import grids

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")


def _load_golden():
    with open(GOLDEN) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _load_golden(), ids=lambda e: e["name"])
def test_hand_examples(ex):
    dims, conn = tuple(ex["dims"]), ex["conn"]
    cs, ct = np.array(ex["cs"]), np.array(ex["ct"])
    nl = np.array(ex["nlink"]).reshape(2, -1)
    r = oracle.maxflow(dims, conn, cs, ct, nl)
    assert r["flow"] == ex["flow"]
    assert r["smin"].tolist() == ex["smin"]
    assert r["smax"].tolist() == ex["smax"]
    b = oracle.brute_force(dims, conn, cs, ct, nl)
    assert b["min_cost"] == ex["flow"]
    assert b["smin"].tolist() == ex["smin"] and b["smax"].tolist() == ex["smax"]
    assert oracle.chain_min_cut(cs.tolist(), ct.tolist(), nl[0].tolist()) == ex["flow"]


TINY = [((4, 4, 1), 4), ((5, 3, 1), 4), ((1, 16, 1), 4), ((2, 9, 1), 4), ((4, 4, 1), 8),
        ((3, 5, 1), 8), ((2, 2, 4), 6), ((3, 2, 3), 6), ((1, 1, 1), 4), ((2, 1, 1), 8)]


@pytest.mark.parametrize("dims,conn", TINY)
@pytest.mark.parametrize("seed", range(6))
def test_dinic_vs_brute_force(dims, conn, seed):
    # small capacity ranges make ties (several minimisers) common
    g = grids.random_grid(dims, conn, seed, cmax=4 + seed, tmax=6, p_zero=0.25)
    r = oracle.solve_instance(g)
    b = oracle.brute_force(g.dims, conn, g.cs, g.ct, g.nlink)
    assert r["flow"] == b["min_cost"]
    np.testing.assert_array_equal(r["smin"], b["smin"])
    np.testing.assert_array_equal(r["smax"], b["smax"])


def test_brute_force_sees_ties():
    # the pins above must exercise S_min != S_max somewhere
    seen = 0
    for dims, conn in TINY:
        for seed in range(6):
            g = grids.random_grid(dims, conn, seed, cmax=4 + seed, tmax=6, p_zero=0.25)
            b = oracle.brute_force(g.dims, conn, g.cs, g.ct, g.nlink)
            seen += int((b["smin"] != b["smax"]).any())
    assert seen >= 5


@pytest.mark.parametrize("n,seed", [(2, 0), (17, 1), (64, 2), (200, 3), (333, 4)])
def test_chain_dp_closed_form(n, seed):
    g = grids.random_grid((n, 1, 1), 4, seed, cmax=30, tmax=50, p_zero=0.1)
    r = oracle.solve_instance(g)
    w = g.nlink[0][:-1].tolist()
    assert r["flow"] == oracle.chain_min_cut(g.cs.tolist(), g.ct.tolist(), w)


@pytest.mark.parametrize("dims,conn", [((23, 17, 1), 4), ((19, 11, 1), 8), ((7, 6, 5), 6)])
def test_no_neighbour_links(dims, conn):
    g = grids.random_grid(dims, conn, 5, cmax=0, tmax=60)
    r = oracle.solve_instance(g)
    assert r["flow"] == int(np.minimum(g.cs, g.ct).astype(np.int64).sum())
    np.testing.assert_array_equal(r["smin"], (g.cs > g.ct).astype(np.uint8))
    np.testing.assert_array_equal(r["smax"], (g.cs >= g.ct).astype(np.uint8))


@pytest.mark.parametrize("dims,conn,seed", [((20, 9, 1), 4, 0), ((12, 12, 1), 8, 1), ((5, 6, 7), 6, 2),
                                            ((20, 9, 1), 4, 3)])
def test_uncuttable_neighbour_links(dims, conn, seed):
    g = grids.random_grid(dims, conn, seed, cmax=0, tmax=50)
    X, Y, Z = g.dims
    big = int(g.cs.sum() + g.ct.sum() + 1)
    nl = np.zeros_like(g.nlink)
    for h, (dx, dy, dz) in enumerate(grids.FWD[conn]):
        m = np.ones((Z, Y, X), dtype=bool)
        if dx > 0: m[:, :, X - dx:] = False
        if dx < 0: m[:, :, :-dx] = False
        if dy > 0: m[:, Y - dy:, :] = False
        if dz > 0: m[Z - dz:, :, :] = False
        nl[h] = np.where(m.ravel(), big, 0)
    if seed == 3:  # force the tie sum(cs) == sum(ct)
        ct = g.ct.copy()
        ct[0] += int(g.cs.sum() - g.ct.sum())
        if ct[0] < 0:
            pytest.skip("cannot balance")
        g.ct = ct
    r = oracle.maxflow(g.dims, conn, g.cs, g.ct, nl)
    scs, sct = int(g.cs.sum()), int(g.ct.sum())
    assert r["flow"] == min(scs, sct)
    # every vertex is on one side: S_min is everything iff flow cannot use all source capacity
    assert int(r["smin"].sum()) == (g.n if scs > sct else 0)
    assert int(r["smax"].sum()) == (g.n if scs >= sct else 0)


@pytest.mark.parametrize("dims,conn,seed", [((31, 17, 1), 4, 0), ((23, 19, 1), 8, 1), ((9, 8, 7), 6, 2),
                                            ((40, 40, 1), 4, 3)])
def test_verifier_accepts_optimum(dims, conn, seed):
    g = grids.random_grid(dims, conn, seed)
    st = oracle.maxflow_state(g.dims, conn, g.cs, g.ct, g.nlink)
    r = oracle.solve_instance(g)
    assert st["flow"] == r["flow"]
    ok, msg, info = oracle.verify(g.dims, conn, g.cs, g.ct, g.nlink, st["res"], st["tres"], st["exc"],
                                  st["flow"], r["smin"], r["smax"])
    assert ok, msg
    assert info["cut_cost"] == r["flow"]
    # closure of the excess set equals s-reachability in Dinic's explicit network
    S = oracle.closure(g.dims, conn, st["res"], st["exc"] > 0)
    np.testing.assert_array_equal(S, r["smin"])
    T = oracle.closure(g.dims, conn, st["res"], st["tres"] > 0, backward=True)
    np.testing.assert_array_equal(1 - T, r["smax"])


def _state(conn=8, dims=(21, 13, 1), seed=4):
    g = grids.random_grid(dims, conn, seed)
    st = oracle.maxflow_state(g.dims, conn, g.cs, g.ct, g.nlink)
    r = oracle.solve_instance(g)
    return g, st, r


def _check(g, st, flow, smin=None, smax=None):
    return oracle.verify(g.dims, g.conn, g.cs, g.ct, g.nlink, st["res"], st["tres"], st["exc"], flow,
                         smin, smax)


def test_verifier_rejects_broken_antisymmetry():
    g, st, r = _state()
    d, v = np.argwhere(st["res"] > 0)[0]
    st["res"][d, v] -= 1
    ok, msg, _ = _check(g, st, r["flow"])
    assert not ok and "antisymmetry" in msg


def test_verifier_rejects_wrong_excess():
    g, st, r = _state()
    st["exc"][5] += 1
    ok, msg, _ = _check(g, st, r["flow"])
    assert not ok and "excess" in msg


def test_verifier_rejects_wrong_flow_value():
    g, st, r = _state()
    ok, msg, _ = _check(g, st, r["flow"] + 1)
    assert not ok and "flow value" in msg


def test_verifier_rejects_wrong_cut():
    g, st, r = _state()
    smin = r["smin"].copy()
    smin[np.argmin(smin)] ^= 1
    ok, msg, _ = _check(g, st, r["flow"], smin=smin)
    assert not ok and "S_min" in msg


def test_verifier_rejects_non_maximal_preflow():
    # the preflow right after Init plus the terminal reduction (no flow on
    # neighbour links) is feasible but not maximal on a coupled grid
    g = grids.random_grid((16, 16, 1), 4, 9)
    r = oracle.solve_instance(g)
    m = np.minimum(g.cs, g.ct)
    assert r["flow"] > int(m.sum())
    H = 2
    n = g.n
    res = np.zeros((2 * H, n), dtype=np.int32)
    for h in range(H):
        res[2 * h] = g.nlink[h]
        # backward arc at w = v + FWD[h] carries the same edge capacity
        dx, dy, _ = grids.FWD[4][h]
        c = g.nlink[h].reshape(16, 16)
        back = np.zeros_like(c)
        back[dy:, dx:] = c[:16 - dy, :16 - dx]
        res[2 * h + 1] = back.ravel()
    st = {"res": res, "tres": (g.ct - m).astype(np.int32), "exc": (g.cs - m).astype(np.int32)}
    ok, msg, _ = _check(g, st, int(m.sum()))
    assert not ok and "not maximal" in msg


def test_verifier_rejects_negative_excess():
    g, st, r = _state(conn=4, dims=(12, 12, 1), seed=2)
    # move one unit of flow out of a vertex with zero excess along a residual arc
    d, v = next((d, v) for d, v in np.argwhere(st["res"] > 0) if st["exc"][v] == 0 and d == 0)
    w = v + 1
    st["res"][d, v] -= 1
    st["res"][d ^ 1, w] += 1
    st["exc"][v] -= 1
    st["exc"][w] += 1
    ok, msg, _ = _check(g, st, r["flow"])
    assert not ok and "negative excess" in msg


def _closed_form_B(dims, tile):
    # a coordinate c of an axis of length D cut into tiles of length T is on a
    # region border if c is the first of a tile (c > 0) or the last (c < D-1)
    inner = 1
    n = 1
    for D, T in zip(dims, tile):
        border = sum(1 for c in range(D) if (c % T == 0 and c > 0) or (c % T == T - 1 and c < D - 1))
        inner *= D - border
        n *= D
    return n - inner


@pytest.mark.parametrize("dims,conn,tile", [((256, 256, 1), 4, (64, 64, 1)), ((256, 256, 1), 8, (64, 64, 1)),
                                            ((200, 150, 1), 4, (64, 64, 1)), ((130, 70, 1), 8, (64, 64, 1)),
                                            ((40, 35, 20), 6, (16, 16, 16)), ((64, 64, 1), 4, (64, 64, 1))])
def test_boundary_size_closed_form(dims, conn, tile):
    assert oracle.boundary_size(dims, conn, tile) == _closed_form_B(dims, tile)


def test_boundary_size_of_named_workloads():
    # the two 2D workloads: 4 and 32 tiles per axis
    assert _closed_form_B((256, 256, 1), (64, 64, 1)) == 65536 - 250 ** 2 == 3036
    assert _closed_form_B((2048, 2048, 1), (64, 64, 1)) == 2048 ** 2 - 1986 ** 2 == 250108
    assert oracle.boundary_size((256, 256, 1), 4, (64, 64, 1)) == 3036
    assert oracle.sweep_bound((256, 256, 1), 4, (64, 64, 1)) == 2 * 3036 ** 2 + 1
    assert _closed_form_B((512, 512, 384), (16, 16, 16)) == 512 * 512 * 384 - 450 * 450 * 338


# ---- the synthetic stencils of Sec. 7.1 (connectivity code 100 + c) --------
# the displacement list as printed in Sec. 7.1 (each pair adds 4 to the connectivity)
PRINTED_DISPLACEMENTS = [(0, 1), (1, 0), (1, 2), (2, 1), (1, 3), (3, 1), (2, 3), (3, 2), (0, 2), (2, 0), (2, 2),
                         (3, 3), (3, 4), (4, 2)]


def _paper_fwd(c):
    # the list read as (dx, dy), its first pair as (1,0), (0,1) (the 4-connected planes)
    return [(1, 0), (0, 1)] + PRINTED_DISPLACEMENTS[2:c // 2]


def _paper_random(dims, c, seed, cmax=5, tmax=7):
    X, Y, _ = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    cs = rng.integers(0, tmax + 1, X * Y).astype(np.int32)
    ct = rng.integers(0, tmax + 1, X * Y).astype(np.int32)
    nl = rng.integers(0, cmax + 1, (c // 2, Y, X)).astype(np.int32)
    for h, (dx, dy) in enumerate(_paper_fwd(c)):  # no edge whose partner leaves the grid
        nl[h, max(0, Y - dy):, :] = 0
        nl[h, :, max(0, X - dx):] = 0
    return cs, ct, nl.reshape(c // 2, -1)


def test_paper_stencil_tables_are_the_printed_list():
    for c in range(8, 29, 4):
        assert [(dx, dy) for dx, dy, dz in oracle._FWD[100 + c]] == _paper_fwd(c)
        assert all(dz == 0 for _, _, dz in oracle._FWD[100 + c])


@pytest.mark.parametrize("c", [8, 12, 20, 28])
@pytest.mark.parametrize("seed", range(4))
def test_paper_stencil_cut_cost_by_hand(c, seed):
    # Eq. 1 from an edge list written here from the printed displacements:
    # pins the C oracle's stencil table (cut_cost) independently of the Python one
    dims = (9, 7, 1)
    X, Y, _ = dims
    cs, ct, nl = _paper_random(dims, c, seed)
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    for _ in range(5):
        S = rng.integers(0, 2, X * Y).astype(np.uint8)
        cost = int(np.where(S == 1, ct, cs).astype(np.int64).sum())
        for h, (dx, dy) in enumerate(_paper_fwd(c)):
            for y in range(Y - dy):
                for x in range(X - dx):
                    u, w = y * X + x, (y + dy) * X + x + dx
                    if S[u] != S[w]:
                        cost += int(nl[h, u])
        assert oracle.cut_cost(dims, 100 + c, cs, ct, nl, S) == cost


@pytest.mark.parametrize("c", [8, 12, 20, 28])
@pytest.mark.parametrize("seed", range(4))
def test_paper_stencil_dinic_vs_brute_force(c, seed):
    dims = (5, 4, 1)
    cs, ct, nl = _paper_random(dims, c, seed)
    r = oracle.maxflow(dims, 100 + c, cs, ct, nl)
    b = oracle.brute_force(dims, 100 + c, cs, ct, nl)
    assert r["flow"] == b["min_cost"]
    np.testing.assert_array_equal(r["smin"], b["smin"])
    np.testing.assert_array_equal(r["smax"], b["smax"])


@pytest.mark.parametrize("c", [8, 28])
def test_paper_stencil_verifier_accepts_optimum(c):
    dims = (23, 19, 1)
    cs, ct, nl = _paper_random(dims, c, 7, cmax=40, tmax=60)
    st = oracle.maxflow_state(dims, 100 + c, cs, ct, nl)
    r = oracle.maxflow(dims, 100 + c, cs, ct, nl)
    assert st["flow"] == r["flow"]
    ok, msg, info = oracle.verify(dims, 100 + c, cs, ct, nl, st["res"], st["tres"], st["exc"], st["flow"],
                                  r["smin"], r["smax"])
    assert ok, msg
    assert info["cut_cost"] == r["flow"]


def test_paper_stencil_boundary_size_by_definition():
    # |B|: vertices with a stencil neighbour (either direction) in another tile
    for c in (8, 16, 28):
        for dims, tile in (((70, 45, 1), (32, 32, 1)), ((100, 96, 1), (32, 32, 1))):
            X, Y, _ = dims
            inB = 0
            for y in range(Y):
                for x in range(X):
                    hit = False
                    for dx, dy in _paper_fwd(c):
                        for s in (1, -1):
                            x2, y2 = x + s * dx, y + s * dy
                            if 0 <= x2 < X and 0 <= y2 < Y and (x2 // 32, y2 // 32) != (x // 32, y // 32):
                                hit = True
                    inB += hit
            assert oracle.boundary_size(dims, 100 + c, tile) == inB
