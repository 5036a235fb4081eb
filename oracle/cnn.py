"""CPU oracle of the warm-start network — TEST INFRASTRUCTURE ONLY.

The warm start is not part of the paper (its hook is the zero flow of Init,
Sec. 2); this module is the plain float64 definition of the network the
solver library trains, used to check the library's forward and backward
kernels:

  four 3x3 convolutions with zero padding, C -> 32 -> 32 -> 32 -> C, ReLU
  after the first three; weights rounded to BF16 (round to nearest even) as
  the library does in every product; parameter vector = for each layer the
  weights [C_out][C_in][3][3] then the biases [C_out].

Pinned in tests/test_oracle_cnn.py against scipy's 2D correlation (forward)
and against central finite differences of this forward (backward).
"""
from __future__ import annotations

import numpy as np

HIDDEN = 32


def layer_shapes(c):
    return [(HIDDEN, c), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (c, HIDDEN)]


def num_params(c):
    return sum(co * ci * 9 + co for co, ci in layer_shapes(c))


def unpack(p, c):
    out, o = [], 0
    for co, ci in layer_shapes(c):
        w = p[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = p[o:o + co]
        o += co
        out.append((w, b))
    return out


def bf16(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b):
    """y[n,co] = b[co] + sum_ci sum_ky,kx w[co,ci,ky,kx] x[n,ci,y+ky-1,x+kx-1] (zero padding)."""
    N, C, H, W = x.shape
    xp = np.zeros((N, C, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((N, w.shape[0], H, W)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, :, ky:ky + H, kx:kx + W]                     # [N, C, H, W]
            y += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], patch)
    return y


def forward(p, x, c, bf16_activations=False):
    """Returns (output, list of layer inputs, list of layer outputs).  With
    bf16_activations the input and each hidden layer's ReLU output are rounded
    to BF16 (the inference variant of the network)."""
    layers = unpack(np.asarray(p, dtype=np.float32), c)
    ins, outs = [], []
    h = np.asarray(x, dtype=np.float64)
    if bf16_activations:
        h = bf16(h)
    for i, (w, b) in enumerate(layers):
        ins.append(h)
        h = conv3x3(h, bf16(w), b.astype(np.float64))
        if i < 3:
            h = np.maximum(h, 0.0)
            if bf16_activations:
                h = bf16(h)
        outs.append(h)
    return h, ins, outs


def backward(p, x, c, dy):
    """Gradient of sum(dy * forward(p, x)) with respect to the parameters (the
    BF16 rounding is treated as identity in the derivative, as in training)."""
    layers = unpack(np.asarray(p, dtype=np.float32), c)
    _, ins, outs = forward(p, x, c)
    g = []
    cur = np.asarray(dy, dtype=np.float64)
    for i in range(3, -1, -1):
        w, _ = layers[i]
        if i < 3:
            cur = cur * (outs[i] > 0)
        xin = ins[i]
        N, C, H, W = xin.shape
        xp = np.zeros((N, C, H + 2, W + 2))
        xp[:, :, 1:-1, 1:-1] = xin
        dw = np.zeros(w.shape)
        for ky in range(3):
            for kx in range(3):
                dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", cur, xp[:, :, ky:ky + H, kx:kx + W])
        db = cur.sum(axis=(0, 2, 3))
        g.append((dw, db))
        # input gradient: correlation with the flipped, transposed kernel
        cp = np.zeros((N, cur.shape[1], H + 2, W + 2))
        cp[:, :, 1:-1, 1:-1] = cur
        wb = bf16(w)
        dx = np.zeros(xin.shape)
        for ky in range(3):
            for kx in range(3):
                dx += np.einsum("oc,nohw->nchw", wb[:, :, 2 - ky, 2 - kx], cp[:, :, ky:ky + H, kx:kx + W])
        cur = dx
    flat = []
    for dw, db in reversed(g):
        flat.append(dw.ravel())
        flat.append(db)
    return np.concatenate(flat)
