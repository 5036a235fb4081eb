"""Parity of the CUDA P-ARD solver with the CPU oracle (called through the C ABI).

Bar: flow value, S_min and S_max bit-identical to Dinic; the final preflow
accepted by the independent verifier; sweeps within the P-ARD bound 2|B|^2+1
(Sec. 4.4).  Sizes span several regions and ragged edge tiles."""
import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity, gpu_solve, opts

pytestmark = pytest.mark.gpu


def _bound_ok(inst, got, tile):
    b = oracle.boundary_size(inst.dims, inst.conn, tile)
    assert got["stats"].boundary_size == b
    assert got["stats"].sweeps <= 2 * b * b + 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_seg2d_256_workload(seed):
    inst = grids.seg2d_256_c4(seed)
    got = gpu_solve(inst, tile=(64, 64, 1))
    assert_parity(inst, got)
    _bound_ok(inst, got, (64, 64, 1))


CASES = [
    # (dims, conn, tile)
    ((200, 150, 1), 4, (64, 64, 1)),
    ((130, 70, 1), 8, (64, 64, 1)),
    ((97, 61, 1), 4, (32, 32, 1)),
    ((75, 90, 1), 8, (32, 32, 1)),
    ((150, 77, 1), 8, (64, 32, 1)),
    ((131, 100, 1), 4, (64, 32, 1)),
    ((97, 61, 1), 4, (32, 16, 1)),
    ((75, 90, 1), 8, (32, 16, 1)),
    ((40, 35, 20), 6, (16, 16, 16)),
    ((21, 19, 13), 6, (8, 8, 8)),
    ((70, 37, 21), 6, (32, 16, 8)),
    ((45, 30, 19), 6, (32, 8, 8)),
    ((96, 48, 24), 6, (32, 16, 8)),
    ((70, 30, 22), 6, (32, 8, 4)),
    ((75, 27, 22), 6, (32, 4, 4)),
    ((66, 33, 13), 6, (32, 8, 2)),
]


@pytest.mark.parametrize("dims,conn,tile", CASES)
@pytest.mark.parametrize("kind", ["seg", "rand"])
def test_ragged_multi_region(dims, conn, tile, kind):
    if kind == "seg":
        inst = (grids.volume_3d(*dims, seed=3) if conn == 6 else
                grids.segmentation_2d(dims[0], dims[1], 3, conn=conn, hard_seed_frac=0.03))
    else:
        inst = grids.random_grid(dims, conn, 11, cmax=30, tmax=60, p_zero=0.3)
    got = gpu_solve(inst, tile=tile)
    assert_parity(inst, got)
    _bound_ok(inst, got, tile)


@pytest.mark.parametrize("dims,conn,tile", [((1, 1, 1), 4, (64, 64, 1)), ((5, 1, 1), 4, (64, 64, 1)),
                                            ((64, 64, 1), 8, (64, 64, 1)), ((16, 16, 16), 6, (16, 16, 16)),
                                            ((1, 300, 1), 4, (32, 32, 1)), ((3, 3, 40), 6, (8, 8, 8)),
                                            ((1, 1, 1), 6, (32, 16, 8)), ((33, 1, 9), 6, (32, 8, 8)),
                                            ((32, 16, 8), 6, (32, 16, 8)), ((1, 1, 1), 6, (32, 4, 4)),
                                            ((33, 5, 3), 6, (32, 8, 2)), ((32, 4, 4), 6, (32, 4, 4)),
                                            ((1, 40, 1), 8, (32, 16, 1)), ((32, 16, 1), 4, (32, 16, 1))])
def test_degenerate_shapes(dims, conn, tile):
    inst = grids.random_grid(dims, conn, 5, cmax=25, tmax=40)
    got = gpu_solve(inst, tile=tile)
    assert_parity(inst, got)


def test_single_region_is_one_sweep():
    # one region: stage 0 of ARD is a complete augmenting-path max-flow (d_inf = 1)
    inst = grids.segmentation_2d(64, 64, 2, conn=4)
    got = gpu_solve(inst, tile=(64, 64, 1))
    assert_parity(inst, got)
    assert got["stats"].sweeps == 1


@pytest.mark.parametrize("conn", [4, 8, 6])
def test_zero_neighbour_links(conn):
    dims = (50, 40, 1) if conn != 6 else (20, 20, 20)
    inst = grids.random_grid(dims, conn, 1, cmax=0, tmax=50)
    got = gpu_solve(inst, tile=(32, 32, 1) if conn != 6 else (8, 8, 8))
    assert_parity(inst, got)
    assert got["flow"] == int(np.minimum(inst.cs, inst.ct).astype(np.int64).sum())


def test_all_zero_capacities():
    inst = grids.random_grid((70, 70, 1), 4, 1, cmax=0, tmax=0)
    got = gpu_solve(inst)
    assert got["flow"] == 0 and got["smin"].sum() == 0 and got["smax"].sum() == inst.n


def test_strong_links_carry_everything():
    inst = grids.random_grid((100, 90, 1), 4, 3, cmax=0, tmax=50)
    inst.nlink[:] = 10 ** 6
    inst.nlink[0].reshape(90, 100)[:, -1] = 0
    inst.nlink[1].reshape(90, 100)[-1, :] = 0
    got = gpu_solve(inst)
    assert_parity(inst, got)
    assert got["flow"] == min(int(inst.cs.sum()), int(inst.ct.sum()))


@pytest.mark.parametrize("conn,dims,t1,t2", [(4, (150, 130, 1), (64, 64, 1), (32, 32, 1)),
                                             (8, (150, 130, 1), (64, 64, 1), (32, 32, 1)),
                                             (6, (40, 40, 24), (16, 16, 16), (8, 8, 8)),
                                             (6, (70, 40, 24), (32, 16, 8), (16, 16, 16)),
                                             (6, (64, 40, 24), (32, 8, 8), (8, 8, 8))])
def test_result_invariant_under_tile_shape(conn, dims, t1, t2):
    inst = (grids.volume_3d(*dims, seed=4) if conn == 6 else
            grids.segmentation_2d(dims[0], dims[1], 4, conn=conn))
    a = gpu_solve(inst, tile=t1, residual=False)
    b = gpu_solve(inst, tile=t2, residual=False)
    assert a["flow"] == b["flow"]
    np.testing.assert_array_equal(a["smin"], b["smin"])
    np.testing.assert_array_equal(a["smax"], b["smax"])


@pytest.mark.parametrize("kw", [dict(partial_discharge=1), dict(global_gap=0),
                                dict(partial_discharge=1, global_gap=0), dict(global_relabel_period=1),
                                dict(global_relabel_period=2, partial_discharge=1),
                                dict(global_relabel_period=1, global_gap=0)])
@pytest.mark.parametrize("conn,tile", [(8, (64, 64, 1)), (4, (32, 32, 1))])
def test_options_keep_exact_results(kw, conn, tile):
    inst = grids.segmentation_2d(190, 170, 6, conn=conn, hard_seed_frac=0.05)
    got = gpu_solve(inst, tile=tile, opts=opts(**kw))
    assert_parity(inst, got)
    if kw.get("global_relabel_period"):
        assert got["stats"].global_relabels >= 1


def test_repeat_solve_same_handle():
    from paper_1109_1146_gb300 import Grid
    inst = grids.seg2d_256_c4(5)
    ref = oracle.solve_instance(inst)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        for _ in range(3):
            g.solve()
            assert g.flow_value() == ref["flow"]
            np.testing.assert_array_equal(g.get_cut(0), ref["smin"])


def test_device_resident_inputs():
    torch = pytest.importorskip("torch")
    from paper_1109_1146_gb300 import Grid
    inst = grids.segmentation_2d(150, 100, 8, conn=8)
    ref = oracle.solve_instance(inst)
    dev = torch.device("cuda:0")
    cs = torch.from_numpy(inst.cs).to(dev)
    ct = torch.from_numpy(inst.ct).to(dev)
    nl = torch.from_numpy(inst.nlink).to(dev)
    with Grid(inst.dims, 8, stream=torch.cuda.current_stream()) as g:
        g.set_caps(cs, ct, nl)
        g.solve()
        out = torch.empty(inst.n, dtype=torch.uint8, device=dev)
        g.get_cut(0, out=out)
        torch.cuda.synchronize()
        assert g.flow_value() == ref["flow"]
        np.testing.assert_array_equal(out.cpu().numpy(), ref["smin"])


@pytest.mark.parametrize("conn,dims,tile", [(4, (200, 150, 1), (64, 64, 1)), (8, (130, 170, 1), (64, 64, 1)),
                                            (4, (97, 61, 1), (32, 32, 1)), (8, (75, 90, 1), (32, 32, 1))])
@pytest.mark.parametrize("kind", ["seg", "rand"])
def test_generic_kernel_variant(conn, dims, tile, kind):
    # the generic per-vertex discharge kernel (variant 1) must give the same exact answer
    inst = (grids.segmentation_2d(dims[0], dims[1], 9, conn=conn, hard_seed_frac=0.05) if kind == "seg"
            else grids.random_grid(dims, conn, 13, cmax=30, tmax=60, p_zero=0.3))
    got = gpu_solve(inst, tile=tile, opts=opts(kernel_variant=1))
    assert_parity(inst, got)


@pytest.mark.parametrize("tile", [(32, 8, 8, ), (32, 16, 8)])
@pytest.mark.parametrize("kw", [dict(global_relabel_period=1), dict(global_relabel_period=2, partial_discharge=1),
                                dict(global_relabel_period=3, global_gap=0)])
def test_3d_global_relabel_keeps_exact_results(tile, kw):
    inst = grids.volume_3d(75, 43, 37, 12)
    got = gpu_solve(inst, tile=tile, opts=opts(**kw))
    assert_parity(inst, got)
    assert got["stats"].global_relabels >= 1


def test_resume_after_sweep_cap_and_get_flow():
    # a sweep cap leaves a consistent state: the caller can keep sweeping and
    # finish, with exact results; mf_get_flow is the residual of mf_get_residual
    from paper_1109_1146_gb300 import Grid, MFError
    inst = grids.segmentation_2d(230, 170, 8, conn=8, hard_seed_frac=0.03)
    with Grid(inst.dims, 8) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        with pytest.raises(MFError, match="SWEEPLIMIT"):
            g.solve(opts(max_sweeps=1))
        for _ in range(10000):
            if g.sweep() == 0:
                break
        g.finish()
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
        np.testing.assert_array_equal(g.get_flow(), got["res"])
    assert_parity(inst, got)


@pytest.mark.parametrize("conn,tile", [(8, (32, 32, 1)), (4, (64, 64, 1)), (6, (32, 8, 4))])
def test_round_cap_reports_and_leaves_a_valid_state(conn, tile):
    # one Augment round per stage cannot finish a discharge here: the device
    # loop stops at the cap, sets the error word, and the host reports
    # MF_EROUNDLIMIT; the preflow stays feasible and a normal solve afterwards
    # on the same handle is exact
    from paper_1109_1146_gb300 import Grid, MFError
    inst = (grids.volume_3d(40, 24, 16, 4) if conn == 6 else
            grids.segmentation_2d(120, 90, 4, conn=conn, hard_seed_frac=0.03))
    with Grid(inst.dims, conn, tile=tile) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        with pytest.raises(MFError, match="ROUNDLIMIT"):
            g.solve(opts(max_rounds=1))
        res, tres, exc = g.get_residual()
        assert (res >= 0).all() and (tres >= 0).all() and (exc >= 0).all()
        got = gpu_solve(inst, tile=tile)
    assert_parity(inst, got)
