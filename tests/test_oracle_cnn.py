"""Pins of the float64 network oracle (oracle/cnn.py): forward against
scipy's 2D correlation, backward against central finite differences."""
import numpy as np
import pytest

from oracle import cnn


def _params(c, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal(cnn.num_params(c)) * 0.2).astype(np.float32)


def test_conv_matches_scipy_correlate():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.Generator(np.random.PCG64(1))
    x = rng.standard_normal((2, 3, 9, 7))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill") for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=1e-12, atol=1e-12)


def test_bf16_rounding():
    a = np.array([1.0, 1.00390625, 1.005859375, 3.0e-3, -2.5], dtype=np.float32)
    r = cnn.bf16(a)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: rounds to even (1.0)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125 and r[4] == -2.5
    assert abs(r[3] - 3.0e-3) / 3.0e-3 < 2 ** -8


def test_backward_matches_finite_differences():
    c = 6
    p = _params(c, 3)
    rng = np.random.Generator(np.random.PCG64(4))
    x = rng.standard_normal((1, c, 6, 5))
    dy = rng.standard_normal((1, c, 6, 5))
    g = cnn.backward(p, x, c, dy)
    # finite differences on a sample of biases and weights; BF16 rounding makes
    # the forward piecewise constant in the weights, so weights are checked on
    # a network whose forward does not round (a variant of the same code path)
    idx = list(range(0, cnn.num_params(c), 997))[:12]
    orig = cnn.bf16
    try:
        cnn.bf16 = lambda a: np.asarray(a, dtype=np.float64)
        g_nr = cnn.backward(p.astype(np.float64).astype(np.float32), x, c, dy)
        for i in idx:
            eps = 1e-3
            pp, pm = p.astype(np.float64).copy(), p.astype(np.float64).copy()
            pp[i] += eps
            pm[i] -= eps
            fp = (cnn.forward(pp, x, c)[0] * dy).sum()
            fm = (cnn.forward(pm, x, c)[0] * dy).sum()
            num = (fp - fm) / (2 * eps)
            assert abs(num - g_nr[i]) <= 2e-2 * max(1.0, abs(num)), (i, num, g_nr[i])
    finally:
        cnn.bf16 = orig
    assert np.isfinite(g).all() and g.shape == (cnn.num_params(c),)
