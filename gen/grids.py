"""Seeded synthetic grid instances for the s-t min-cut problem (Sec. 2, Eq. 1).

This module only produces INPUTS: per-vertex terminal capacities cs (source
link), ct (sink link) and the symmetric neighbour-link capacities of a 2D or 3D
grid graph.  It contains none of the max-flow arithmetic; both the CPU oracle
and the CUDA solver read the very same int32 arrays produced here.

Array conventions (shared by every consumer):
  * vertex index v = (z * Y + y) * X + x, x fastest;
  * cs, ct : int32[n];
  * nlink  : int32[H, n] with H = connectivity // 2; nlink[h, v] is the
    capacity c(v, w) = c(w, v) of the edge between v and w = v + FWD[conn][h]
    (0 where w is outside the grid).  The forward half-stencil FWD lists, for
    every undirected edge, the endpoint that comes later in raster order.

The vision-style workloads follow the shapes of the paper's experiments
(Sec. 7: 2D 4-connected stereo/segmentation grids, 3D 6-connected volumes);
their exact recipes are stated in the docstrings below.

Floating point is used only where it is deterministic across machines: the
noise fields use +, *, / (IEEE-exact rounding, no libm), and every value that
goes through exp/log is tabulated over the 256 integer intensities into a
lookup table, rounded half away from zero, and checked to sit away from a
rounding tie (so a one-ulp libm difference cannot change an integer).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# forward half-stencils (dx, dy, dz)
FWD = {
    4: ((1, 0, 0), (0, 1, 0)),
    8: ((1, 0, 0), (0, 1, 0), (1, 1, 0), (-1, 1, 0)),
    6: ((1, 0, 0), (0, 1, 0), (0, 0, 1)),
}

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def _hash(*keys) -> np.ndarray:
    h = np.uint64(0x243F6A8885A308D3)
    out = None
    for k in keys:
        k = np.asarray(k).astype(np.int64).astype(np.uint64)
        out = splitmix64((h if out is None else out) ^ k)
    return out


def _u01(h: np.ndarray) -> np.ndarray:
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _fade(t: np.ndarray) -> np.ndarray:
    # quintic fade 6t^5 - 15t^4 + 10t^3 (Perlin 2002); +,* only
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def _normalise_u8(v: np.ndarray) -> np.ndarray:
    lo, hi = float(v.min()), float(v.max())
    if hi <= lo:
        return np.zeros(v.shape, dtype=np.int32)
    return np.rint((v - lo) * (255.0 / (hi - lo))).astype(np.int32)


def value_noise_2d(X: int, Y: int, seed: int, lattices=(32, 16, 8, 4)) -> np.ndarray:
    """Smooth random intensity field I[y, x] in [0, 255] (int32).

    Value noise: random lattice values u in [0,1) from SplitMix64 of
    (seed, octave, i, j), quintic-fade bilinear interpolation, octaves with
    lattice pitch 32/16/8/4 pixels and amplitude halving, normalised to
    integers 0..255 (round half to even)."""
    xs = np.arange(X, dtype=np.int64)
    ys = np.arange(Y, dtype=np.int64)
    acc = np.zeros((Y, X), dtype=np.float64)
    amp = 1.0
    for o, L in enumerate(lattices):
        gx, fx = xs // L, (xs % L).astype(np.float64) / L
        gy, fy = ys // L, (ys % L).astype(np.float64) / L
        nx, ny = int(gx[-1]) + 2, int(gy[-1]) + 2
        jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        lat = _u01(_hash(seed, o, ii, jj))  # [ny, nx]
        wx, wy = _fade(fx)[None, :], _fade(fy)[:, None]
        v00 = lat[gy][:, gx]
        v10 = lat[gy][:, gx + 1]
        v01 = lat[gy + 1][:, gx]
        v11 = lat[gy + 1][:, gx + 1]
        top = v00 + (v10 - v00) * wx
        bot = v01 + (v11 - v01) * wx
        acc += amp * (top + (bot - top) * wy)
        amp *= 0.5
    return _normalise_u8(acc)


_GRAD3 = np.array(
    [[1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0],
     [1, 0, 1], [-1, 0, 1], [1, 0, -1], [-1, 0, -1],
     [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1]], dtype=np.float64)


def perlin_3d(X: int, Y: int, Z: int, seed: int, base: int = 32, octaves: int = 3,
              zchunk: int = 8) -> np.ndarray:
    """Seeded 3D gradient ("Perlin") noise volume I[z, y, x] in [0, 255] (int32).

    Classic gradient noise: each lattice corner picks one of the 12 cube-edge
    gradients by SplitMix64(seed, octave, i, j, k) mod 12; the value is the
    quintic-fade trilinear blend of the corner dot products.  Octaves have
    lattice pitch base, base/2, ... and amplitude halving."""
    acc = np.zeros((Z, Y, X), dtype=np.float64)
    xs = np.arange(X, dtype=np.int64)
    ys = np.arange(Y, dtype=np.int64)
    amp = 1.0
    for o in range(octaves):
        L = base >> o
        gx, fx = xs // L, (xs % L).astype(np.float64) / L
        gy, fy = ys // L, (ys % L).astype(np.float64) / L
        nx, ny, nz = int(gx[-1]) + 2, int(gy[-1]) + 2, (Z - 1) // L + 2
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        gidx = (_hash(seed, 1000 + o, ii, jj, kk) % np.uint64(12)).astype(np.int64)
        G = _GRAD3[gidx]  # [nz, ny, nx, 3]
        wx = _fade(fx)[None, None, :]
        wy = _fade(fy)[None, :, None]
        for z0 in range(0, Z, zchunk):
            zs = np.arange(z0, min(Z, z0 + zchunk), dtype=np.int64)
            gz, fz = zs // L, (zs % L).astype(np.float64) / L
            wz = _fade(fz)[:, None, None]
            res = None
            for cz in (0, 1):
                for cy in (0, 1):
                    for cx in (0, 1):
                        g = G[gz + cz][:, gy + cy][:, :, gx + cx]  # [zc, Y, X, 3]
                        dot = (g[..., 0] * (fx[None, None, :] - cx)
                               + g[..., 1] * (fy[None, :, None] - cy)
                               + g[..., 2] * (fz[:, None, None] - cz))
                        w = ((wx if cx else 1.0 - wx) * (wy if cy else 1.0 - wy)
                             * (wz if cz else 1.0 - wz))
                        res = dot * w if res is None else res + dot * w
            acc[z0:z0 + len(zs)] += amp * res
        amp *= 0.5
    return _normalise_u8(acc)


def _lround_table(values, what: str) -> np.ndarray:
    """Round half away from zero, refusing values within 1e-7 of a tie."""
    out = np.empty(len(values), dtype=np.int64)
    for i, x in enumerate(values):
        frac = abs(x) - math.floor(abs(x))
        if abs(frac - 0.5) < 1e-7:
            raise ValueError(f"{what}[{i}] = {x!r} is too close to a rounding tie")
        out[i] = int(math.floor(abs(x) + 0.5)) * (1 if x >= 0 else -1)
    return out


def nlink_lut(scale: float, sigma: float, diag: bool = False) -> np.ndarray:
    """LUT[d] = round(scale * exp(-d^2 / (2 sigma^2)) [/ sqrt 2]) for d = 0..255."""
    vals = []
    for d in range(256):
        w = scale * math.exp(-(d * d) / (2.0 * sigma * sigma))
        if diag:
            w /= math.sqrt(2.0)
        vals.append(w)
    return _lround_table(vals, "nlink_lut")


def neglog_gauss_lut(mu: float, sigma: float, scale: float = 10.0) -> np.ndarray:
    """LUT[I] = round(scale * -log N(I; mu, sigma^2)) for I = 0..255."""
    c = math.log(sigma * math.sqrt(2.0 * math.pi))
    vals = [scale * (c + (i - mu) ** 2 / (2.0 * sigma * sigma)) for i in range(256)]
    return _lround_table(vals, "neglog_gauss_lut")


@dataclass
class GridInstance:
    dims: tuple  # (X, Y, Z)
    conn: int
    cs: np.ndarray
    ct: np.ndarray
    nlink: np.ndarray
    name: str = ""

    @property
    def ndim(self) -> int:
        return 3 if self.conn == 6 else 2

    @property
    def n(self) -> int:
        X, Y, Z = self.dims
        return X * Y * Z


def _edge_caps_from_intensity(I: np.ndarray, conn: int, luts) -> np.ndarray:
    """nlink[h] = LUT_h[|I(v) - I(v + FWD[h])|], 0 outside the grid."""
    if I.ndim == 2:
        I3 = I[None]
    else:
        I3 = I
    Z, Y, X = I3.shape
    H = len(FWD[conn])
    out = np.zeros((H, Z, Y, X), dtype=np.int32)
    for h, (dx, dy, dz) in enumerate(FWD[conn]):
        lut = luts[h]
        xs0, xs1 = max(0, -dx), X - max(0, dx)
        ys0, ys1 = max(0, -dy), Y - max(0, dy)
        zs0, zs1 = max(0, -dz), Z - max(0, dz)
        a = I3[zs0:zs1, ys0:ys1, xs0:xs1]
        b = I3[zs0 + dz:zs1 + dz, ys0 + dy:ys1 + dy, xs0 + dx:xs1 + dx]
        out[h, zs0:zs1, ys0:ys1, xs0:xs1] = lut[np.abs(a - b)]
    return out.reshape(H, -1)


def segmentation_2d(X: int, Y: int, seed: int, conn: int = 4, mu_fg: float = 170.0,
                    mu_bg: float = 80.0, hard_seed_frac: float = 0.0,
                    hard_cap: int = 10 ** 6, sigma: float = 20.0, scale: float = 100.0,
                    name: str = "") -> GridInstance:
    """Segmentation-style 2D instance.

    I = value_noise_2d; cs = round(|I - mu_bg|), ct = round(|I - mu_fg|)
    (a bright pixel near mu_fg is expensive to put on the sink side);
    n-links round(scale * exp(-dI^2 / (2 sigma^2))), diagonals divided by
    sqrt 2 before rounding.  With hard_seed_frac > 0 a seeded Bernoulli picks
    that fraction of pixels as hard seeds: cs = hard_cap, ct = 0 where
    I >= (mu_fg + mu_bg) / 2, else cs = 0, ct = hard_cap."""
    assert conn in (4, 8)
    I = value_noise_2d(X, Y, seed)
    Ii = np.arange(256, dtype=np.float64)
    cs_lut = _lround_table(np.abs(Ii - mu_bg), "cs")
    ct_lut = _lround_table(np.abs(Ii - mu_fg), "ct")
    cs = cs_lut[I].astype(np.int64)
    ct = ct_lut[I].astype(np.int64)
    if hard_seed_frac > 0:
        yy, xx = np.meshgrid(np.arange(Y), np.arange(X), indexing="ij")
        pick = _u01(_hash(seed, 77, xx, yy)) < hard_seed_frac
        fg = I >= (mu_fg + mu_bg) / 2.0
        cs = np.where(pick, np.where(fg, hard_cap, 0), cs)
        ct = np.where(pick, np.where(fg, 0, hard_cap), ct)
    straight = nlink_lut(scale, sigma)
    luts = [straight, straight]
    if conn == 8:
        d = nlink_lut(scale, sigma, diag=True)
        luts += [d, d]
    nl = _edge_caps_from_intensity(I, conn, luts)
    return GridInstance((X, Y, 1), conn, cs.astype(np.int32).ravel(),
                        ct.astype(np.int32).ravel(), nl, name or f"seg2d_{X}x{Y}_c{conn}_s{seed}")


def volume_3d(X: int, Y: int, Z: int, seed: int, mu_fg: float = 170.0, mu_bg: float = 80.0,
              sigma_cls: float = 30.0, sigma: float = 15.0, scale: float = 50.0,
              name: str = "") -> GridInstance:
    """3D 6-connected volume instance.

    I = perlin_3d; cs = round(10 * -log N(I; mu_bg, 30^2)),
    ct = round(10 * -log N(I; mu_fg, 30^2)) (Gaussian class likelihoods);
    n-links round(scale * exp(-dI^2 / (2 sigma^2)))."""
    I = perlin_3d(X, Y, Z, seed)
    cs = neglog_gauss_lut(mu_bg, sigma_cls)[I]
    ct = neglog_gauss_lut(mu_fg, sigma_cls)[I]
    lut = nlink_lut(scale, sigma)
    nl = _edge_caps_from_intensity(I, 6, [lut, lut, lut])
    return GridInstance((X, Y, Z), 6, cs.astype(np.int32).ravel(), ct.astype(np.int32).ravel(),
                        nl, name or f"vol3d_{X}x{Y}x{Z}_s{seed}")


def random_grid(dims, conn: int, seed: int, cmax: int = 20, tmax: int = 40,
                p_zero: float = 0.2, name: str = "") -> GridInstance:
    """Unstructured random instance: caps uniform in [0, max], a fraction
    p_zero of n-links forced to 0 (to create bottlenecks and cut-offs)."""
    X, Y, Z = (tuple(dims) + (1, 1))[:3]
    n = X * Y * Z
    rng = np.random.Generator(np.random.PCG64(seed))
    cs = rng.integers(0, tmax + 1, n)
    ct = rng.integers(0, tmax + 1, n)
    H = len(FWD[conn])
    nl = rng.integers(0, cmax + 1, (H, n))
    nl[rng.random((H, n)) < p_zero] = 0
    nl = nl.reshape(H, Z, Y, X)
    for h, (dx, dy, dz) in enumerate(FWD[conn]):
        if dx > 0:
            nl[h, :, :, X - dx:] = 0
        if dx < 0:
            nl[h, :, :, :(-dx)] = 0
        if dy > 0:
            nl[h, :, Y - dy:, :] = 0
        if dz > 0:
            nl[h, Z - dz:, :, :] = 0
    return GridInstance((X, Y, Z), conn, cs.astype(np.int32), ct.astype(np.int32),
                        nl.reshape(H, n).astype(np.int32), name or f"rand_{X}x{Y}x{Z}_c{conn}_s{seed}")


# displacements of the paper's synthetic networks (Sec. 7.1), in the order in
# which they are listed (each pair adds 4 to the connectivity), read as (dx, dy)
PAPER_DISPLACEMENTS = ((0, 1), (1, 0), (1, 2), (2, 1), (1, 3), (3, 1), (2, 3), (3, 2), (0, 2), (2, 0), (2, 2),
                       (3, 3), (3, 4), (4, 2))


def paper_connectivity_code(connectivity: int) -> int:
    """Connectivity code of the synthetic stencil of the given connectivity:
    4 is the 4-connected grid, c = 8, 12, ..., 28 the code 100 + c."""
    if connectivity not in (4, 8, 12, 16, 20, 24, 28):
        raise ValueError("the synthetic family has connectivity 4, 8, ..., 28")
    return 4 if connectivity == 4 else 100 + connectivity


def paper_synthetic(X: int, Y: int, seed: int, strength: int = 150, connectivity: int = 4,
                    name: str = "") -> GridInstance:
    """The synthetic family of Sec. 7.1: a 2D grid whose edges join the nodes
    at the first connectivity/2 listed displacements (connectivity 4, 8, ...,
    28), every edge with the same capacity (the strength), and every node
    given an integer excess or deficit drawn uniformly from [-500, 500] (PCG64
    of the seed): a positive value is a source link, a negative one a sink
    link.  Plane h holds the edges of the h-th forward displacement; the
    list's first pair, (0,1), (1,0), goes to planes 1, 0, so connectivity 4
    is this package's 4-connected grid, and higher connectivities carry the
    code 100 + connectivity."""
    code = paper_connectivity_code(connectivity)
    disp = ((1, 0), (0, 1)) + PAPER_DISPLACEMENTS[2:connectivity // 2]
    rng = np.random.Generator(np.random.PCG64(seed))
    e = rng.integers(-500, 501, X * Y)
    cs = np.where(e > 0, e, 0).astype(np.int32)
    ct = np.where(e < 0, -e, 0).astype(np.int32)
    nl = np.zeros((len(disp), Y, X), dtype=np.int32)
    for h, (dx, dy) in enumerate(disp):  # the edge exists where its head lies in the grid
        nl[h, : max(0, Y - dy), : max(0, X - dx)] = strength
    return GridInstance((X, Y, 1), code, cs, ct, nl.reshape(len(disp), -1),
                        name or f"paper_synth_{X}x{Y}_c{connectivity}_str{strength}_s{seed}")


# --- the five named workloads ------------------------------------------------

def seg2d_256_c4(seed: int = 0) -> GridInstance:
    """256x256 4-connected segmentation grid (65,536 vertices; 64x64 regions)."""
    return segmentation_2d(256, 256, seed, conn=4, name=f"seg2d_256x256_c4_s{seed}")


def seg2d_2048_c8_hard(seed: int = 0, side: int = 2048) -> GridInstance:
    """2048x2048 8-connected segmentation grid, 5% hard seeds at 10^6."""
    return segmentation_2d(side, side, seed, conn=8, hard_seed_frac=0.05,
                           name=f"seg2d_{side}x{side}_c8_hard_s{seed}")


def vol3d_512x512x384(seed: int = 0, dims=(512, 512, 384)) -> GridInstance:
    """512x512x384 6-connected Perlin volume (1.0e8 vertices; 16^3 regions)."""
    X, Y, Z = dims
    return volume_3d(X, Y, Z, seed, name=f"vol3d_{X}x{Y}x{Z}_s{seed}")


def seg2d_1024_c4_mu(seed: int, side: int = 1024) -> GridInstance:
    """1024x1024 4-connected segmentation grid, mu_fg and mu_bg ~ U[60, 200]
    per instance (drawn from SplitMix64(seed)); t-links round(|I - mu|)."""
    h = _hash(seed, 4242, np.arange(2))
    mu_fg, mu_bg = (60.0 + 140.0 * _u01(h)).tolist()
    return segmentation_2d(side, side, seed, conn=4, mu_fg=mu_fg, mu_bg=mu_bg,
                           name=f"seg2d_{side}x{side}_c4_mu_s{seed}")


def uneven_batch_shapes(seed: int = 0, n2d: int = 384, n3d: int = 128):
    """Shapes of the uneven batch: 2D sides ~ U{64..1024}, 3D sides ~ U{48..128}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    s2 = rng.integers(64, 1025, n2d)
    s3 = rng.integers(48, 129, n3d)
    return [(int(s), int(s), 1) for s in s2] + [(int(s), int(s), int(s)) for s in s3]


def instance_digest(inst: GridInstance) -> str:
    import hashlib
    h = hashlib.sha256()
    h.update(np.asarray(inst.dims, dtype=np.int64).tobytes())
    h.update(np.int64(inst.conn).tobytes())
    for a in (inst.cs, inst.ct, inst.nlink):
        h.update(np.ascontiguousarray(a, dtype=np.int32).tobytes())
    return h.hexdigest()
