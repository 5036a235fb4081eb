"""Pins of the oracle's boundary-relabel heuristic (Sec. 6.1) against values
fixed by hand and by mathematics, not by itself:

* two hand-worked chains (tests/golden/boundary_relabel_examples.json): the
  length-0 arcs between a region's consecutive labels, and their direction;
* regions of one vertex: every arc crosses regions and every group is one
  vertex, so from the labeling min(d*, 1) the heuristic must reach the
  region distance d* of Sec. 4.1 exactly (a plain BFS distance here);
* regions whose inner arcs are all residual both ways: a group is a whole
  region, and again the result must be d*;
* on random valid labelings (d* clipped or halved): the result is valid, not
  below the input, not above d*, and d* itself is a fixed point;
* a single region has no boundary: nothing changes.
"""
import json
import os

import numpy as np
import pytest

import oracle
from gen import grids

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "boundary_relabel_examples.json")
FWD = grids.FWD


def _examples():
    with open(GOLDEN) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _examples(), ids=lambda e: e["name"])
def test_hand_worked_chains(ex):
    n = ex["dims"][0]
    res = np.zeros((4, n), np.int64)
    res[0], res[1] = ex["right"], ex["left"]
    tile = tuple(ex["tile"])
    assert oracle.boundary_size(ex["dims"], 4, tile) == ex["dinf"]
    lab = np.array(ex["lab"])
    assert _strongly_valid(ex["dims"], 4, tile, res, np.array(ex["tres"]), lab)
    out = oracle.boundary_relabel(ex["dims"], 4, tile, res, lab, ex["dinf"])
    assert out.tolist() == ex["expected"]


def _targets(dims, conn):
    X, Y, Z = dims
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    out = []
    for dx, dy, dz in FWD[conn]:
        for sg in (1, -1):
            x2, y2, z2 = xx + sg * dx, yy + sg * dy, zz + sg * dz
            ok = (x2 >= 0) & (x2 < X) & (y2 >= 0) & (y2 < Y) & (z2 >= 0) & (z2 < Z)
            out.append(np.where(ok, (z2 * Y + y2) * X + x2, -1).ravel())
    return out


def _regions(dims, tile):
    X, Y, Z = dims
    tx, ty, tz = tile
    zz, yy, xx = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    return ((zz // tz * -(-Y // ty) + yy // ty) * -(-X // tx) + xx // tx).ravel()


def _strongly_valid(dims, conn, tile, res, tres, lab):
    """d(u) <= d(w) on residual arcs inside a region, d(u) <= d(w) + 1 across
    regions, d = 0 where c_f(u, t) > 0."""
    reg = _regions(dims, tile)
    if (lab[np.asarray(tres) > 0] != 0).any():
        return False
    for d, t in enumerate(_targets(dims, conn)):
        u = np.flatnonzero((t >= 0) & (res[d] > 0))
        w = t[u]
        slack = (reg[u] != reg[w]).astype(np.int64)
        if (lab[u] > lab[w] + slack).any():
            return False
    return True


def _random_state(dims, conn, seed, p_zero=0.45):
    rng = np.random.default_rng(seed)
    n = int(np.prod(dims))
    tg = _targets(dims, conn)
    res = np.zeros((len(tg), n), np.int64)
    for d, t in enumerate(tg):
        res[d] = np.where((t >= 0) & (rng.random(n) > p_zero), rng.integers(1, 9, n), 0)
    tres = np.where(rng.random(n) < 0.06, rng.integers(1, 5, n), 0)
    return res, tres


def _dstar(dims, conn, tile, res, tres):
    dinf = max(oracle.boundary_size(dims, conn, tile), 1)
    d = oracle.region_distance(dims, conn, tile, res, tres)
    return np.where(d >= 0, d, dinf), dinf


CASES = [((9, 7, 1), 4, (1, 1, 1)), ((8, 6, 1), 8, (1, 1, 1)), ((4, 3, 3), 6, (1, 1, 1))]


@pytest.mark.parametrize("dims,conn,tile", CASES)
@pytest.mark.parametrize("seed", range(4))
def test_one_vertex_regions_reach_the_region_distance(dims, conn, tile, seed):
    res, tres = _random_state(dims, conn, seed)
    dstar, dinf = _dstar(dims, conn, tile, res, tres)
    lab = np.minimum(dstar, 1)
    assert _strongly_valid(dims, conn, tile, res, tres, lab)
    out = oracle.boundary_relabel(dims, conn, tile, res, lab, dinf)
    np.testing.assert_array_equal(out, dstar)


@pytest.mark.parametrize("dims,conn,tile", [((12, 9, 1), 4, (3, 3, 1)), ((12, 8, 1), 8, (4, 2, 1)),
                                            ((6, 6, 4), 6, (2, 3, 2))])
@pytest.mark.parametrize("seed", range(4))
def test_inner_arcs_both_ways_reach_the_region_distance(dims, conn, tile, seed):
    res, tres = _random_state(dims, conn, seed, p_zero=0.7)
    reg = _regions(dims, tile)
    for d, t in enumerate(_targets(dims, conn)):
        inner = (t >= 0) & (reg == reg[np.maximum(t, 0)])
        res[d][inner] = 5
    dstar, dinf = _dstar(dims, conn, tile, res, tres)
    lab = np.minimum(dstar, 1)
    assert _strongly_valid(dims, conn, tile, res, tres, lab)
    out = oracle.boundary_relabel(dims, conn, tile, res, lab, dinf)
    np.testing.assert_array_equal(out, dstar)


@pytest.mark.parametrize("dims,conn,tile", [((16, 12, 1), 4, (4, 4, 1)), ((14, 10, 1), 8, (4, 4, 1)),
                                            ((8, 6, 6), 6, (4, 2, 2)), ((20, 9, 1), 4, (8, 4, 1))])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("lower", ["clip1", "clip2", "half"])
def test_valid_monotone_and_below_the_region_distance(dims, conn, tile, seed, lower):
    res, tres = _random_state(dims, conn, seed, p_zero=0.3)
    dstar, dinf = _dstar(dims, conn, tile, res, tres)
    lab = {"clip1": np.minimum(dstar, 1), "clip2": np.minimum(dstar, 2), "half": dstar // 2}[lower]
    assert _strongly_valid(dims, conn, tile, res, tres, lab)
    out = oracle.boundary_relabel(dims, conn, tile, res, lab, dinf)
    assert (out >= lab).all()
    assert (out <= dstar).all()
    assert _strongly_valid(dims, conn, tile, res, tres, out)
    np.testing.assert_array_equal(oracle.boundary_relabel(dims, conn, tile, res, dstar, dinf), dstar)


def test_single_region_changes_nothing():
    dims, conn = (7, 5, 1), 4
    res, tres = _random_state(dims, conn, 3)
    lab = np.where(tres > 0, 0, 1)
    out = oracle.boundary_relabel(dims, conn, (8, 8, 1), res, lab, 1)
    np.testing.assert_array_equal(out, lab)
