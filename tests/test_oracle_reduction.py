"""Pins of the oracle's region reduction (Sec. 8) against values fixed by
hand and by the whole network's minimum cuts, not by itself:

* a hand-worked two-region chain (tests/golden/region_reduction_examples.json);
* one region covering the grid (no boundary): the strong sources are exactly
  S_min and the strong sinks exactly the complement of S_max (Dinic);
* on random grids cut into small regions, the classes the section states:
  strong source => in every minimum cut's source set (S_min), strong sink =>
  in none (outside S_max), weak source => in some (S_max), weak sink => not
  in all (outside S_min) — against Dinic, and against brute force on tiny
  grids;
* the section's statements about the algorithm: B^S and B^T are disjoint, and
  at the end s reaches neither B^R nor t and neither B^R nor s reaches t.
"""
import json
import os

import numpy as np
import pytest

import oracle
from gen import grids
from oracle.reduction import STRONG_SINK, STRONG_SOURCE, WEAK_SINK, WEAK_SOURCE, region_reduction

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "region_reduction_examples.json")


@pytest.mark.parametrize("ex", json.load(open(GOLDEN))["examples"], ids=lambda e: e["name"])
def test_hand_worked_chain(ex):
    r = region_reduction(ex["dims"], ex["conn"], ex["tile"], ex["cs"], ex["ct"], np.array(ex["nlink"]))
    assert r["codes"].tolist() == ex["codes"]
    assert [g["BS"] for g in r["regions"]] == ex["BS"]
    assert [g["BT"] for g in r["regions"]] == ex["BT"]


def _check_classes(codes, smin, smax):
    smin, smax = smin.astype(bool), smax.astype(bool)
    assert not ((codes & STRONG_SOURCE).astype(bool) & ~smin).any(), "strong source outside S_min"
    assert not ((codes & STRONG_SINK).astype(bool) & smax).any(), "strong sink inside S_max"
    assert not ((codes & WEAK_SOURCE).astype(bool) & ~smax).any(), "weak source outside S_max"
    assert not ((codes & WEAK_SINK).astype(bool) & smin).any(), "weak sink inside S_min"


@pytest.mark.parametrize("dims,conn", [((9, 7, 1), 4), ((8, 6, 1), 8), ((5, 4, 3), 6)])
@pytest.mark.parametrize("seed", range(3))
def test_single_region_gives_the_global_cuts(dims, conn, seed):
    inst = grids.random_grid(dims, conn, seed, cmax=12, tmax=20, p_zero=0.3)
    ref = oracle.maxflow(inst.dims, conn, inst.cs, inst.ct, inst.nlink)
    r = region_reduction(inst.dims, conn, inst.dims, inst.cs, inst.ct, inst.nlink)
    codes = r["codes"]
    np.testing.assert_array_equal((codes & STRONG_SOURCE) != 0, ref["smin"].astype(bool))
    np.testing.assert_array_equal((codes & STRONG_SINK) != 0, ~ref["smax"].astype(bool))
    rest = (codes & (STRONG_SOURCE | STRONG_SINK)) == 0
    assert (codes[rest] == (WEAK_SOURCE | WEAK_SINK)).all()


@pytest.mark.parametrize("dims,conn,tile", [((12, 10, 1), 4, (4, 4, 1)), ((12, 9, 1), 8, (4, 3, 1)),
                                            ((6, 6, 4), 6, (3, 3, 2)), ((16, 8, 1), 4, (8, 4, 1))])
@pytest.mark.parametrize("seed", range(4))
def test_classes_agree_with_the_global_cuts(dims, conn, tile, seed):
    inst = grids.random_grid(dims, conn, seed, cmax=15, tmax=30, p_zero=0.3)
    ref = oracle.maxflow(inst.dims, conn, inst.cs, inst.ct, inst.nlink)
    r = region_reduction(inst.dims, conn, tile, inst.cs, inst.ct, inst.nlink)
    _check_classes(r["codes"], ref["smin"], ref["smax"])
    for g in r["regions"]:
        assert not set(g["BS"]) & set(g["BT"])
        assert not g["s_to_boundary_or_t"] and not g["boundary_or_s_to_t"]


@pytest.mark.parametrize("dims,conn,tile", [((4, 4, 1), 4, (2, 2, 1)), ((4, 3, 1), 8, (2, 2, 1)),
                                            ((2, 2, 3), 6, (1, 2, 2))])
@pytest.mark.parametrize("seed", range(5))
def test_classes_agree_with_brute_force(dims, conn, tile, seed):
    inst = grids.random_grid(dims, conn, 100 + seed, cmax=8, tmax=12, p_zero=0.25)
    bf = oracle.brute_force(inst.dims, conn, inst.cs, inst.ct, inst.nlink)
    r = region_reduction(inst.dims, conn, tile, inst.cs, inst.ct, inst.nlink)
    _check_classes(r["codes"], bf["smin"], bf["smax"])


def test_classes_decide_vertices():
    # not vacuous: on a segmentation grid many vertices are decided (strong
    # sink or weak source, the paper's measure) and some are left open
    inst = grids.segmentation_2d(24, 20, 3, conn=4)
    r = region_reduction(inst.dims, 4, (8, 8, 1), inst.cs, inst.ct, inst.nlink)
    decided = ((r["codes"] & (STRONG_SINK | WEAK_SOURCE)) != 0).mean()
    assert 0.05 < decided < 1.0


@pytest.mark.parametrize("dims,conn,tile", [((12, 10, 1), 4, (4, 4, 1)), ((12, 9, 1), 8, (4, 3, 1)),
                                            ((6, 6, 4), 6, (3, 3, 2))])
@pytest.mark.parametrize("seed", range(3))
def test_reduced_instance_keeps_the_minimum_cuts(dims, conn, tile, seed):
    """Merging the strong sources into s and the strong sinks into t keeps
    the minimum cut value (plus the constant of the merged edges) and both
    canonical cuts: S_min = S* + S_min(reduced), S_max = S_max(reduced) - T*
    (Dinic on both networks)."""
    from oracle.reduction import reduce_instance
    inst = grids.random_grid(dims, conn, 30 + seed, cmax=15, tmax=30, p_zero=0.3)
    ref = oracle.maxflow(inst.dims, conn, inst.cs, inst.ct, inst.nlink)
    codes = region_reduction(inst.dims, conn, tile, inst.cs, inst.ct, inst.nlink)["codes"]
    S, T = (codes & STRONG_SOURCE) != 0, (codes & STRONG_SINK) != 0
    cs2, ct2, nl2, K = reduce_instance(inst.dims, conn, inst.cs, inst.ct, inst.nlink, codes)
    red = oracle.maxflow(inst.dims, conn, cs2, ct2, nl2)
    assert red["flow"] + K == ref["flow"]
    np.testing.assert_array_equal(red["smin"].astype(bool) | S, ref["smin"].astype(bool))
    np.testing.assert_array_equal(red["smax"].astype(bool) & ~T, ref["smax"].astype(bool))
    assert (S | T).any()  # not vacuous


def test_classes_do_not_depend_on_the_augmenting_paths(monkeypatch):
    """The classes are functions of the network alone: augmenting along other
    paths (depth-first, adjacency shuffled before every step) gives the same
    codes, so a parallel implementation can be compared with them exactly."""
    import random
    import oracle.reduction as R
    inst = grids.random_grid((12, 10, 1), 4, 5, cmax=6, tmax=10, p_zero=0.3)
    want = region_reduction(inst.dims, 4, (4, 4, 1), inst.cs, inst.ct, inst.nlink)["codes"]
    rng = random.Random(1)

    def dfs_augment(self, src, dst):
        for a in self.adj:
            rng.shuffle(a)
        total = 0
        while True:
            prev, stack = {src: -1}, [src]
            while stack and dst not in prev:
                u = stack.pop()
                for e in self.adj[u]:
                    w = self.to[e]
                    if self.cap[e] > 0 and w not in prev:
                        prev[w] = e
                        stack.append(w)
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
    monkeypatch.setattr(R._Net, "augment", dfs_augment)
    for tile in ((4, 4, 1), (6, 5, 1), (12, 10, 1)):
        w = region_reduction(inst.dims, 4, tile, inst.cs, inst.ct, inst.nlink)["codes"]
        monkeypatch.undo()
        base = region_reduction(inst.dims, 4, tile, inst.cs, inst.ct, inst.nlink)["codes"]
        monkeypatch.setattr(R._Net, "augment", dfs_augment)
        np.testing.assert_array_equal(w, base)
    monkeypatch.undo()
    np.testing.assert_array_equal(region_reduction(inst.dims, 4, (4, 4, 1), inst.cs, inst.ct, inst.nlink)["codes"], want)
