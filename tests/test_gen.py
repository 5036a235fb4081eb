"""The seeded input generators: determinism, value ranges, the stated recipes."""
import math

import numpy as np
import pytest

from gen import grids


def test_splitmix64_reference_values():
    # SplitMix64 output sequence for state 0 (Steele, Lea & Flood 2014;
    # the generator as published by Vigna): first outputs of next() from seed 0
    x = np.array([0], dtype=np.uint64)
    assert int(grids.splitmix64(x)[0]) == 0xE220A8397B1DCDAF
    x2 = np.array([0x9E3779B97F4A7C15], dtype=np.uint64)
    assert int(grids.splitmix64(x2)[0]) == 0x6E789E6AA1B965F4


def test_deterministic():
    a, b = grids.seg2d_256_c4(3), grids.seg2d_256_c4(3)
    assert grids.instance_digest(a) == grids.instance_digest(b)
    assert grids.instance_digest(a) != grids.instance_digest(grids.seg2d_256_c4(4))


def test_seg2d_256_recipe():
    g = grids.seg2d_256_c4(0)
    assert g.dims == (256, 256, 1) and g.conn == 4 and g.nlink.shape == (2, 65536)
    I = grids.value_noise_2d(256, 256, 0).ravel()
    assert I.min() == 0 and I.max() == 255
    np.testing.assert_array_equal(g.cs, np.abs(I - 80))
    np.testing.assert_array_equal(g.ct, np.abs(I - 170))
    # n-link = round(100 exp(-dI^2 / 800)) between right neighbours
    Im = I.reshape(256, 256)
    d = np.abs(Im[:, 1:] - Im[:, :-1])
    want = np.floor(100 * np.exp(-d.astype(float) ** 2 / 800.0) + 0.5).astype(np.int32)
    np.testing.assert_array_equal(g.nlink[0].reshape(256, 256)[:, :-1], want)
    assert (g.nlink[0].reshape(256, 256)[:, -1] == 0).all()
    assert (g.nlink[1].reshape(256, 256)[-1, :] == 0).all()


def test_hard_seeds_small():
    g = grids.segmentation_2d(256, 256, 1, conn=8, hard_seed_frac=0.05)
    hard = (g.cs == 10 ** 6) | (g.ct == 10 ** 6)
    assert 0.04 < hard.mean() < 0.06
    assert ((g.cs == 10 ** 6) <= (g.ct == 0)).all()
    diag = grids.nlink_lut(100, 20, diag=True)
    assert diag[0] == 71 and round(100 / math.sqrt(2)) == 71
    # edges to (-1,+1) vanish on the first column and last row
    nl3 = g.nlink[3].reshape(256, 256)
    assert (nl3[:, 0] == 0).all() and (nl3[-1, :] == 0).all()


def test_volume_luts():
    bg = grids.neglog_gauss_lut(80.0, 30.0)
    c = 10 * math.log(30 * math.sqrt(2 * math.pi))
    assert bg[80] == round(c)
    assert bg[0] == math.floor(c + 10 * 80 ** 2 / 1800 + 0.5)
    assert (grids.nlink_lut(50, 15) <= 50).all() and grids.nlink_lut(50, 15)[0] == 50


def test_volume_small():
    g = grids.volume_3d(20, 18, 9, 0)
    assert g.nlink.shape == (3, 20 * 18 * 9)
    assert g.cs.min() >= 0 and g.ct.min() >= 0
    nl = g.nlink.reshape(3, 9, 18, 20)
    assert (nl[0, :, :, -1] == 0).all() and (nl[1, :, -1, :] == 0).all() and (nl[2, -1] == 0).all()


def test_seg2d_1024_mu_range():
    for s in range(5):
        g = grids.seg2d_1024_c4_mu(s, side=64)
        assert g.cs.max() <= 200 and g.ct.max() <= 200


def test_uneven_batch_shapes():
    sh = grids.uneven_batch_shapes(0)
    assert len(sh) == 512
    assert all(64 <= s[0] <= 1024 and s[2] == 1 for s in sh[:384])
    assert all(48 <= s[0] <= 128 and s[0] == s[2] for s in sh[384:])


def test_paper_synthetic_family():
    # Sec. 7.1: excess/deficit uniform in [-500, 500] as one terminal link per
    # node, every edge the constant strength, 4-connected (displacements
    # (0,1), (1,0)); edges leaving the grid have no capacity
    inst = grids.paper_synthetic(60, 40, 3, strength=150)
    assert inst.conn == 4 and inst.dims == (60, 40, 1)
    assert ((inst.cs == 0) | (inst.ct == 0)).all()
    e = inst.cs.astype(int) - inst.ct.astype(int)
    assert e.min() >= -500 and e.max() <= 500 and e.min() < -400 and e.max() > 400
    assert abs(e.mean()) < 40
    nl = inst.nlink.reshape(2, 40, 60)
    assert (nl[0, :, :59] == 150).all() and (nl[0, :, 59] == 0).all()
    assert (nl[1, :39, :] == 150).all() and (nl[1, 39, :] == 0).all()
    again = grids.paper_synthetic(60, 40, 3, strength=150)
    assert (again.cs == inst.cs).all() and (again.ct == inst.ct).all()
    for bad in (6, 10, 32):
        with pytest.raises(ValueError):
            grids.paper_synthetic(10, 10, 0, connectivity=bad)


# Sec. 7.1, the displacement list as printed (each pair adds 4 to the connectivity)
PRINTED_DISPLACEMENTS = [(0, 1), (1, 0), (1, 2), (2, 1), (1, 3), (3, 1), (2, 3), (3, 2), (0, 2), (2, 0), (2, 2),
                         (3, 3), (3, 4), (4, 2)]


def test_paper_synthetic_higher_connectivity():
    assert list(grids.PAPER_DISPLACEMENTS) == PRINTED_DISPLACEMENTS
    X, Y = 37, 29
    for c in (8, 12, 16, 20, 24, 28):
        inst = grids.paper_synthetic(X, Y, 5, strength=1200 // c, connectivity=c)
        assert inst.conn == 100 + c and inst.nlink.shape == (c // 2, X * Y)
        # the same terminal links as connectivity 4 with the same seed
        base = grids.paper_synthetic(X, Y, 5, connectivity=4)
        assert (inst.cs == base.cs).all() and (inst.ct == base.ct).all()
        nl = inst.nlink.reshape(c // 2, Y, X)
        disp = [(1, 0), (0, 1)] + PRINTED_DISPLACEMENTS[2:c // 2]
        for h, (dx, dy) in enumerate(disp):
            # an edge per node whose displaced partner lies in the grid, none otherwise
            yy, xx = np.mgrid[0:Y, 0:X]
            inside = (xx + dx < X) & (yy + dy < Y)
            assert (nl[h][inside] == 1200 // c).all() and (nl[h][~inside] == 0).all()
        # connectivity = the number of edges at a node far from the boundary
        deg = np.zeros((Y, X), dtype=int)
        for h, (dx, dy) in enumerate(disp):
            deg += nl[h] > 0
            deg[dy:, dx:] += nl[h][: Y - dy, : X - dx] > 0
        assert deg[10, 10] == c
