"""Learned warm start on the GPU: the network's kernels against the float64
oracle, the projection to a preflow, exactness of warm solves, and the gain
of a trained network over the cold start."""
import os

import numpy as np
import pytest

import oracle
from gen import grids
from helpers import assert_parity
from oracle import cnn as ocnn
from paper_1109_1146_gb300 import Grid, default_opts, mf, warmstart

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("c,shape", [(6, (2, 6, 20, 17)), (10, (1, 10, 33, 16)), (6, (1, 6, 48, 64))])
def test_forward_and_gradients_match_oracle(c, shape):
    net = mf.CNN(channels=c, seed=11)
    p = net.get_params()
    rng = np.random.Generator(np.random.PCG64(5))
    x = rng.standard_normal(shape).astype(np.float32)
    dy = rng.standard_normal(shape).astype(np.float32)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.empty_like(xt)
    net.forward(xt, yt)
    ref, _, _ = ocnn.forward(p, x.astype(np.float64), c)
    np.testing.assert_allclose(yt.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)
    net.zero_grad()
    net.backward(xt, torch.from_numpy(dy).to(DEV))
    g = net.get_grads()
    gref = ocnn.backward(p, x.astype(np.float64), c, dy.astype(np.float64))
    scale = np.abs(gref).max()
    np.testing.assert_allclose(g, gref, rtol=2e-3, atol=2e-4 * scale)


@pytest.mark.parametrize("c,shape", [(6, (2, 6, 20, 17)), (10, (1, 10, 33, 40)), (6, (1, 6, 64, 48))])
def test_tensor_core_inference_matches_oracle(c, shape):
    net = mf.CNN(channels=c, seed=12)
    p = net.get_params()
    rng = np.random.Generator(np.random.PCG64(7))
    x = rng.standard_normal(shape).astype(np.float32)
    xt = torch.from_numpy(x).to(DEV)
    yt = torch.empty_like(xt)
    net.infer(xt, yt)
    got = yt.cpu().numpy()
    ref, _, _ = ocnn.forward(p, x.astype(np.float64), c, bf16_activations=True)
    # FP32 against float64 sums: a hidden value next to a BF16 rounding
    # boundary may round to the neighbouring BF16 value (2^-8 relative)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=1e-2, atol=1e-2 * scale)
    assert np.abs(got - ref).mean() < 1e-3 * scale
    # and close to the FP32-activation forward
    yf = torch.empty_like(xt)
    net.forward(xt, yf)
    np.testing.assert_allclose(got, yf.cpu().numpy(), rtol=5e-2, atol=3e-2 * scale)


def test_adam_reduces_loss_on_fixed_batch():
    net = mf.CNN(channels=6, seed=2)
    rng = np.random.Generator(np.random.PCG64(6))
    x = torch.from_numpy(rng.standard_normal((4, 6, 16, 16)).astype(np.float32)).to(DEV)
    t = torch.from_numpy(rng.standard_normal((4, 6, 16, 16)).astype(np.float32) * 0.1).to(DEV)
    y, dy = torch.empty_like(x), torch.empty_like(x)
    losses = []
    for _ in range(60):
        net.forward(x, y)
        losses.append(net.mse(y, t, dy))
        net.zero_grad()
        net.backward(x, dy)
        net.adam_step(lr=3e-3)
    assert losses[-1] < 0.5 * losses[0]


def _solved_targets(inst):
    C = inst.conn + 2
    X, Y = inst.dims[0], inst.dims[1]
    t = torch.empty((C, Y, X), dtype=torch.float32, device=DEV)
    with Grid(inst.dims, inst.conn) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st = g.solve(default_opts(global_relabel_period=0))
        g.warm_targets(t)
    return t, st


@pytest.mark.parametrize("conn", [4, 8])
def test_projection_of_the_exact_flows_is_immediate(conn):
    inst = grids.segmentation_2d(150, 110, 3, conn=conn, hard_seed_frac=0.03)
    t, cold = _solved_targets(inst)
    with Grid(inst.dims, conn) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st, rounds = g.warm_start(t)
        assert rounds == 0  # the solution's flows already form a preflow
        ws = g.solve(default_opts(warm_start=1, global_relabel_period=0))
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
    assert_parity(inst, got)
    # the relabel before the first sweep already sees a maximum preflow
    assert ws.sweeps == 0 and ws.global_relabels == 1 and cold.sweeps > 0


@pytest.mark.parametrize("noise", [0.0, 0.3, 3.0])
def test_noisy_predictions_project_and_solve_exactly(noise):
    inst = grids.seg2d_1024_c4_mu(7, side=128)
    t, _ = _solved_targets(inst)
    gen = torch.Generator(device=DEV).manual_seed(1)
    pred = t + noise * torch.randn(t.shape, generator=gen, device=DEV)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st, rounds = g.warm_start(pred)
        ws = g.solve(default_opts(warm_start=1))
        assert ws.projection_rounds == rounds
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
    assert_parity(inst, got)


def test_projection_trims_a_chain_by_hand():
    # 1x3 chain, cs = [5,0,0], ct = [0,0,5], links 4 and 4.  Predicted flows 7
    # and 6 exceed what s supplies: v0 has excess 5-4 (after clamping 7 -> 4);
    # v1 receives 4 and sends 4 (6 clamped to 4): fine; so clamping alone gives
    # a preflow.  Predict 4 on the first link and 4 on the second but a sink
    # flow the capacity allows: v2 gets 4 and may send 4 -> flow 4 = max flow.
    cs = np.array([5, 0, 0], np.int32)
    ct = np.array([0, 0, 5], np.int32)
    nl = np.array([[4, 4, 0], [0, 0, 0]], np.int32)
    g = Grid((3, 1, 1), 4)
    g.set_caps(cs, ct, nl)
    pred = torch.zeros((6, 1, 3), dtype=torch.float32, device=DEV)
    pred[0, 0, 0] = 0.07   # v0 -> v1: 7, clamped to 4
    pred[0, 0, 1] = 0.06   # v1 -> v2: 6, clamped to 4
    pred[5, 0, 2] = 0.09   # v2 -> t: 9, clamped to 5
    st, rounds = g.warm_start(pred)
    # v2: in 4, out 5 -> deficit 1 -> sink flow trimmed to 4 in one round
    assert rounds == 1
    g.solve(default_opts(warm_start=1))
    assert g.flow_value() == 4
    res, tres, exc = g.get_residual()
    assert exc.tolist() == [1, 0, 0] and tres.tolist() == [0, 0, 1]
    g.close()


WEIGHTS = os.path.join(os.path.dirname(warmstart.__file__), "weights", "warm_seg2d_1024_c4.npy")


def test_trained_network_saves_sweeps():
    # the committed network (trained by `python -m paper_1109_1146_gb300.warmstart
    # train` on 2,000 certified 1024x1024 solves) against the cold start on the
    # first 32 held-out seeds: identical exact results, fewer sweeps in total
    net = warmstart.load_network(WEIGHTS)
    cold_sw, warm_sw = [], []
    for seed in range(warmstart.EVAL_SEED0, warmstart.EVAL_SEED0 + 32):
        inst = grids.seg2d_1024_c4_mu(seed)
        with Grid(inst.dims, 4) as g:
            g.set_caps(inst.cs, inst.ct, inst.nlink)
            cold = g.solve()
            flow, smin = g.flow_value(), g.get_cut(0)
            ws, _, _, used = warmstart.warm_solve(g, net)
            assert used
            assert g.flow_value() == flow
            np.testing.assert_array_equal(g.get_cut(0), smin)
            assert g.certify()[0]
        cold_sw.append(cold.sweeps)
        warm_sw.append(ws.sweeps)
    print("cold sweeps", sum(cold_sw), "warm sweeps", sum(warm_sw))
    assert sum(warm_sw) < sum(cold_sw)


def test_untrained_network_gives_exact_results():
    inst = grids.seg2d_1024_c4_mu(warmstart.EVAL_SEED0 + 77, side=512)
    ref = oracle.solve_instance(inst)
    net = mf.CNN(channels=6, seed=99)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        warmstart.warm_solve(g, net)
        assert g.flow_value() == ref["flow"]
        np.testing.assert_array_equal(g.get_cut(0), ref["smin"])


def test_batched_warm_start_is_exact():
    # a batch of 2D 4-connected grids, half of them warm-started from noisy
    # solution flows, plus one 3D grid that stays cold: exact results for all
    from paper_1109_1146_gb300 import mf as mfmod
    insts = [grids.seg2d_1024_c4_mu(30 + i, side=96 + 32 * i) for i in range(4)] + [grids.volume_3d(40, 30, 20, 3)]
    handles = []
    for k, inst in enumerate(insts):
        g = Grid(inst.dims, inst.conn)
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        if k % 2 == 0 and inst.conn == 4:
            t, _ = _solved_targets(inst)
            gen = torch.Generator(device=DEV).manual_seed(k)
            g.warm_start(t + 0.2 * torch.randn(t.shape, generator=gen, device=DEV))
        handles.append(g)
    for graph in (0, 1):
        mfmod.solve_batch(handles, default_opts(warm_start=1, global_relabel_period=0, graph_loop=graph))
        for inst, g in zip(insts, handles):
            got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
            got["res"], got["tres"], got["exc"] = g.get_residual()
            assert_parity(inst, got)
    for g in handles:
        g.close()


def test_load_model_reads_the_trainers_file(tmp_path):
    net = mf.CNN(channels=6, seed=5)
    net.load(WEIGHTS)
    np.testing.assert_array_equal(net.get_params(), np.load(WEIGHTS))
    bad = tmp_path / "short.npy"
    np.save(bad, np.zeros(10, dtype=np.float32))
    with pytest.raises(mf.MFError, match="shape"):
        net.load(str(bad))
    f64 = tmp_path / "f64.npy"
    np.save(f64, np.zeros(net.num_params, dtype=np.float64))
    with pytest.raises(mf.MFError, match="float32"):
        net.load(str(f64))
    with pytest.raises(mf.MFError, match="cannot open"):
        net.load(str(tmp_path / "missing.npy"))


@pytest.mark.parametrize("conn", [4, 8])
@pytest.mark.parametrize("noise", [0.05, 0.5])
def test_projection_matches_oracle(conn, noise):
    # the projected preflow of the library equals the oracle's, bit for bit
    from oracle import warm as owarm
    inst = grids.segmentation_2d(97, 83, 5, conn=conn, hard_seed_frac=0.02)
    t, _ = _solved_targets(inst)
    gen = torch.Generator(device=DEV).manual_seed(7)
    pred = (t + noise * torch.randn(t.shape, generator=gen, device=DEV)).contiguous()
    with Grid(inst.dims, conn) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        _, rounds = g.warm_start(pred)
        g.begin(default_opts(warm_start=1))
        res, tres, exc = g.get_residual()
        g.finish()
    ref = owarm.project(inst.dims, conn, inst.cs, inst.ct, inst.nlink, pred.cpu().numpy().reshape(conn + 2, -1))
    assert ref is not None
    F, ft, E, r = ref
    assert (r == 0) == (rounds == 0)  # the library counts tile phases, the oracle synchronous rounds
    rres, rtres, rexc = owarm.residual(inst.dims, conn, inst.cs, inst.ct, inst.nlink, F, ft)
    np.testing.assert_array_equal(res, rres)
    np.testing.assert_array_equal(tres, rtres)
    np.testing.assert_array_equal(exc, rexc)


def test_projection_round_cap_falls_back_to_cold():
    # a prediction whose trims need many rounds, with a cap of one round:
    # mf_warm_start reports MF_EROUNDLIMIT, the warm solve starts cold, and the
    # result is exact
    inst = grids.seg2d_1024_c4_mu(11, side=128)
    t, _ = _solved_targets(inst)
    pred = t * 3.0  # large over-predictions cascade through many trim rounds
    net = mf.CNN(channels=6, seed=1)
    with Grid(inst.dims, 4) as g:
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        st, rounds = g.warm_start(pred, max_rounds=1, check=False)
        assert st == mf.MF_EROUNDLIMIT
        ws = g.solve(default_opts(warm_start=0))
        assert ws.projection_rounds == 0
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        got["res"], got["tres"], got["exc"] = g.get_residual()
        _, _, _, used = warmstart.warm_solve(g, net, default_opts(), max_rounds=1)
        assert g.flow_value() == got["flow"]  # warm if the projection fit in one round, else cold
    assert_parity(inst, got)


def test_batched_projection_matches_single_projections():
    # mf_warm_start_batch enqueues every projection and waits once: the same
    # preflows (hence the same warm solves) as mf_warm_start one grid at a time,
    # a grid with no prediction stays cold, results exact against the oracle
    insts = [grids.seg2d_1024_c4_mu(60 + i, side=80 + 24 * i) for i in range(3)]
    preds = []
    for k, inst in enumerate(insts):
        t, _ = _solved_targets(inst)
        gen = torch.Generator(device=DEV).manual_seed(k)
        preds.append((t + 0.3 * torch.randn(t.shape, generator=gen, device=DEV)).contiguous())
    single = []
    for inst, p in zip(insts, preds):
        with Grid(inst.dims, 4) as g:
            g.set_caps(inst.cs, inst.ct, inst.nlink)
            _, r = g.warm_start(p)
            g.begin(default_opts(warm_start=1))
            single.append((r, g.get_residual()))
            g.finish()
    handles = []
    for inst in insts:
        g = Grid(inst.dims, 4)
        g.set_caps(inst.cs, inst.ct, inst.nlink)
        handles.append(g)
    rounds = mf.warm_start_batch(handles, [preds[0], None, preds[2]])
    assert rounds[0] == single[0][0] and rounds[1] == -1 and rounds[2] == single[2][0]
    stats = mf.solve_batch(handles, default_opts(warm_start=1, graph_loop=1))
    assert stats[1].projection_rounds == 0 and stats[0].projection_rounds == rounds[0]
    for inst, g in zip(insts, handles):
        got = {"flow": g.flow_value(), "smin": g.get_cut(0), "smax": g.get_cut(1)}
        assert_parity(inst, got, verify=False)
    for k in (0, 2):
        h = handles[k]
        h.begin(default_opts(warm_start=1))  # the projected preflow is kept for the next warm solve
        res = h.get_residual()
        for a, b in zip(res, single[k][1]):
            np.testing.assert_array_equal(a, b)
        h.finish()
    for g in handles:
        g.close()
