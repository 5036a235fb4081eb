"""The synthetic networks of Sec. 7.1 on the GPU: 2D grids whose edges join
the nodes at the paper's listed displacements (connectivity 8 .. 28,
displacements up to 4; connectivity code 100 + c), solved by P-ARD and P-PRD
with the generic region discharge on 32x32 tiles.

* Flow value, S_min and S_max equal to Dinic, the final preflow verified, on
  the paper's family (constant strength, excess in [-500, 500]) and on random
  capacities, ragged and degenerate shapes, host and graph sweep loops.
* |B| of the solve (the boundary of Sec. 4.1 under the longer displacements)
  equals the oracle's count by definition; the global relabel gives the
  oracle's region distances after every sweep.
* The calls these stencils do not support fail with MF_EINVAL.
"""
import numpy as np
import pytest

import oracle
from gen import grids
from gen.grids import GridInstance
from helpers import assert_parity, gpu_solve
from paper_1109_1146_gb300 import Grid, default_opts, mf

pytestmark = pytest.mark.gpu

CONNS = [8, 12, 16, 20, 24, 28]


def _random(dims, c, seed, cmax=30, tmax=60):
    """Random capacities on the stencil of connectivity c (no edge leaves the grid)."""
    X, Y = dims
    rng = np.random.Generator(np.random.PCG64(seed))
    cs = rng.integers(0, tmax + 1, X * Y).astype(np.int32)
    ct = rng.integers(0, tmax + 1, X * Y).astype(np.int32)
    nl = rng.integers(0, cmax + 1, (c // 2, Y, X)).astype(np.int32)
    nl[rng.random(nl.shape) < 0.3] = 0
    disp = ((1, 0), (0, 1)) + grids.PAPER_DISPLACEMENTS[2:c // 2]
    for h, (dx, dy) in enumerate(disp):
        nl[h, max(0, Y - dy):, :] = 0
        nl[h, :, max(0, X - dx):] = 0
    return GridInstance((X, Y, 1), 100 + c, cs, ct, nl.reshape(c // 2, -1), f"paper_rand_{X}x{Y}_c{c}_s{seed}")


@pytest.mark.parametrize("c", CONNS)
@pytest.mark.parametrize("variant", [0, 2])
def test_paper_family_is_exact(c, variant):
    inst = grids.paper_synthetic(100, 75, 3, strength=1200 // c, connectivity=c)
    got = gpu_solve(inst, tile=(32, 32, 1), opts=default_opts(kernel_variant=variant))
    assert_parity(inst, got)
    assert got["stats"].boundary_size == oracle.boundary_size(inst.dims, inst.conn, (32, 32, 1))


@pytest.mark.parametrize("c", [8, 20, 28])
@pytest.mark.parametrize("dims,seed", [((70, 45), 1), ((33, 97), 2), ((129, 40), 3)])
@pytest.mark.parametrize("graph", [0, 1])
def test_random_capacities_are_exact(c, dims, seed, graph):
    inst = _random(dims, c, seed)
    got = gpu_solve(inst, tile=(32, 32, 1), opts=default_opts(graph_loop=graph))
    assert_parity(inst, got)


@pytest.mark.parametrize("c", [8, 28])
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("kw", [dict(), dict(partial_discharge=1), dict(global_gap=0)])
def test_options_keep_exact_results(c, variant, kw):
    inst = _random((90, 64), c, 4)
    got = gpu_solve(inst, tile=(32, 32, 1), opts=default_opts(kernel_variant=variant, **kw))
    assert_parity(inst, got)


@pytest.mark.parametrize("c", [8, 28])
@pytest.mark.parametrize("dims", [(1, 1), (5, 4), (3, 50), (32, 32), (36, 5)])
def test_degenerate_shapes(c, dims):
    inst = _random(dims, c, 5, cmax=10, tmax=20)
    got = gpu_solve(inst, tile=(32, 32, 1))
    assert_parity(inst, got)


def test_strength_sweep_matches_the_oracle():
    # the paper's dependence-on-strength series at connectivity 8 (small size)
    for strength in (20, 150, 400, 1000):
        inst = grids.paper_synthetic(120, 90, 11, strength=strength, connectivity=8)
        for variant in (0, 2):
            got = gpu_solve(inst, tile=(32, 32, 1), opts=default_opts(kernel_variant=variant), residual=False)
            assert_parity(inst, got, verify=False)


@pytest.mark.parametrize("tile", [(64, 32, 1), (64, 64, 1)])
@pytest.mark.parametrize("variant", [0, 2])
def test_larger_tiles_at_connectivity_8(tile, variant):
    # the paper's dependence on the number of regions at its default connectivity
    inst = grids.paper_synthetic(150, 140, 9, strength=150, connectivity=8)
    got = gpu_solve(inst, tile=tile, opts=default_opts(kernel_variant=variant))
    assert_parity(inst, got)
    assert got["stats"].boundary_size == oracle.boundary_size(inst.dims, inst.conn, tile)
    assert got["stats"].global_relabels > 0
    inst = _random((130, 70), 8, 10)
    got = gpu_solve(inst, tile=tile, opts=default_opts(kernel_variant=variant, graph_loop=1))
    assert_parity(inst, got)


def test_unsupported_uses_are_rejected():
    inst = grids.paper_synthetic(64, 64, 1, connectivity=8)
    big = grids.paper_synthetic(64, 64, 1, connectivity=12)
    with pytest.raises(mf.MFError) as ei:
        Grid(big.dims, big.conn, tile=(64, 64, 1))  # 15 planes of 64x64 do not fit in shared memory
    assert ei.value.status == mf.MF_EINVAL
    with pytest.raises(mf.MFError) as ei:
        Grid(inst.dims, inst.conn, host_state=True)
    assert ei.value.status == mf.MF_EINVAL
    with Grid(inst.dims, inst.conn) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        for kw in (dict(region_reduction=1), dict(boundary_relabel_period=2)):
            with pytest.raises(mf.MFError) as ei:
                g.solve(default_opts(**kw))
            assert ei.value.status == mf.MF_EINVAL
        with pytest.raises(mf.MFError) as ei:
            g.region_reduction()
        assert ei.value.status == mf.MF_EINVAL
        with pytest.raises(mf.MFError) as ei:
            mf.solve_batch([g], default_opts())
        assert ei.value.status == mf.MF_EINVAL
        st = g.solve(default_opts())  # and the handle still solves
        assert st.sweeps > 0
        assert g.flow_value() == oracle.solve_instance(inst)["flow"]


@pytest.mark.parametrize("c,tile", [(8, (32, 32, 1)), (16, (32, 32, 1)), (28, (32, 32, 1)), (8, (64, 32, 1)),
                                    (8, (64, 64, 1))])
def test_global_relabel_gives_region_distances(c, tile):
    # with the relabel after every sweep the labels equal the oracle's 0-1 BFS
    # region distances (d_inf where t is unreachable), as for the unit stencils
    inst = _random((140, 70), c, 6)
    checked = 0
    with Grid(inst.dims, inst.conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        g.begin(default_opts(global_relabel_period=1))
        for _ in range(500):
            if g.sweep() == 0:
                break
            lab, dinf = g.get_labels()
            res, tres, _ = g.get_residual()
            d = oracle.region_distance(inst.dims, inst.conn, tile, res, tres)
            np.testing.assert_array_equal(lab, np.where(d >= 0, d, dinf))
            checked += 1
        g.finish()
    assert checked >= 1


@pytest.mark.parametrize("c", [8, 28])
@pytest.mark.parametrize("variant,glr", [(0, 1), (0, 4), (2, 2), (2, 4)])
def test_exact_with_the_global_relabel(c, variant, glr):
    inst = grids.paper_synthetic(130, 100, 8, strength=1200 // c, connectivity=c)
    for graph in (0, 1):
        got = gpu_solve(inst, tile=(32, 32, 1), opts=default_opts(kernel_variant=variant, global_relabel_period=glr,
                                                                 graph_loop=graph))
        assert_parity(inst, got)
        assert got["stats"].global_relabels > 0
