"""FP64 reference of the learned preconditioner's building blocks: 3x3x3 convolution
forward and backward, ReLU backward, mean squared error, Adam and BF16 rounding.

TEST INFRASTRUCTURE: only tests/ import it; the CUDA library never does.

Written from the definitions, one slice per tap:
  - the convolution is the cross-correlation used by convolutional networks,
    y[co][p] = b[co] + sum_ci sum_k w[co][ci][k] x[ci][p + k - 1] over the 27 taps
    k = (kz, ky, kx) in {0, 1, 2}^3, with x read as zero outside the grid;
  - its backward passes are the derivatives of sum(dy * y): with respect to x, the
    same sum with dy read at p - k + 1 (the transposed operator); with respect to
    w[co][ci][k], sum_p dy[co][p] x[ci][p + k - 1]; with respect to b[co], sum_p dy[co][p];
  - the loss is sum (y - t)^2 / (2 n), with gradient (y - t) / n;
  - Adam is Algorithm 1 of Kingma & Ba (2015) with bias-corrected moments;
  - BF16 keeps the upper 16 bits of an IEEE binary32 value, rounded to nearest with
    ties to even;
  - the U-Net's 2x average pooling and nearest-neighbour upsampling: coarse cell q of
    a fine grid covers the fine voxels 2q, 2q + 1 along each axis, clipped to the grid;
    pooling is the mean over the cell, upsampling copies the cell's value to its voxels,
    and their backward passes are the transposed maps.
Arrays are [C][D][H][W] with W fastest; weights [C_out][C_in][27] with kx fastest.
"""
from __future__ import annotations

import numpy as np

TAPS = [(kz, ky, kx) for kz in range(3) for ky in range(3) for kx in range(3)]


def bf16_bits(a):
    """The BF16 bit patterns (uint16) nearest to the FP32 values of a (ties to even)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    return ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)


def bf16_value(bits):
    """FP64 values of BF16 bit patterns."""
    b = np.ascontiguousarray(bits, dtype=np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


def bf16_round(a):
    return bf16_value(bf16_bits(a))


def _pad(a):
    return np.pad(a, ((0, 0), (1, 1), (1, 1), (1, 1)))


def conv3d(x, w, b=None):
    """y[co][p] = b[co] + sum_ci sum_k w[co][ci][k] x[ci][p + k - 1], zero outside."""
    ci, D, H, W = x.shape
    w = np.asarray(w, dtype=np.float64).reshape(-1, ci, 27)
    xp = _pad(np.asarray(x, dtype=np.float64))
    y = np.zeros((w.shape[0], D, H, W))
    for t, (kz, ky, kx) in enumerate(TAPS):
        y += np.tensordot(w[:, :, t], xp[:, kz:kz + D, ky:ky + H, kx:kx + W], axes=(1, 0))
    if b is not None:
        y += np.asarray(b, dtype=np.float64)[:, None, None, None]
    return y


def conv3d_backward_data(dy, w, cin):
    """dx[ci][p] = sum_co sum_k w[co][ci][k] dy[co][p - k + 1], zero outside."""
    co, D, H, W = dy.shape
    w = np.asarray(w, dtype=np.float64).reshape(co, cin, 27)
    dyp = _pad(np.asarray(dy, dtype=np.float64))
    dx = np.zeros((cin, D, H, W))
    for t, (kz, ky, kx) in enumerate(TAPS):
        # dy at p - k + 1 sits at p - k + 2 of the padded array
        dx += np.tensordot(w[:, :, t], dyp[:, 2 - kz:2 - kz + D, 2 - ky:2 - ky + H, 2 - kx:2 - kx + W], axes=(0, 0))
    return dx


def conv3d_backward_weight(dy, x):
    """(dw[co][ci][k] = sum_p dy[co][p] x[ci][p + k - 1], db[co] = sum_p dy[co][p])."""
    co, D, H, W = dy.shape
    ci = x.shape[0]
    xp = _pad(np.asarray(x, dtype=np.float64))
    dy = np.asarray(dy, dtype=np.float64)
    dw = np.zeros((co, ci, 27))
    for t, (kz, ky, kx) in enumerate(TAPS):
        dw[:, :, t] = np.tensordot(dy, xp[:, kz:kz + D, ky:ky + H, kx:kx + W], axes=([1, 2, 3], [1, 2, 3]))
    return dw, dy.sum(axis=(1, 2, 3))


def relu_backward(dy, y):
    return np.where(np.asarray(y) > 0, dy, 0.0)


def mse(y, t):
    """(sum (y - t)^2 / (2 n), (y - t) / n)."""
    e = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float(np.sum(e * e) / (2 * e.size)), e / e.size


def adam(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step t >= 1; returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def _cell_index(n):
    """coarse cell of each fine index along an axis of n points, and the cell count"""
    return np.arange(n) // 2, (n + 1) // 2


def pool2(x):
    """y[c][q] = mean of x[c][p] over the fine voxels p of coarse cell q (clipped)."""
    x = np.asarray(x, dtype=np.float64)
    C, D, H, W = x.shape
    (iz, nz), (iy, ny), (ix, nx) = _cell_index(D), _cell_index(H), _cell_index(W)
    s = np.zeros((C, nz, ny, nx))
    cnt = np.zeros((nz, ny, nx))
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                s[:, iz[z], iy[y], ix[xx]] += x[:, z, y, xx]
                cnt[iz[z], iy[y], ix[xx]] += 1
    return s / cnt


def pool2_backward(dy, fine_shape):
    """dx[c][p] = dy[c][q(p)] / (voxels of cell q(p))."""
    dy = np.asarray(dy, dtype=np.float64)
    D, H, W = fine_shape
    (iz, nz), (iy, ny), (ix, nx) = _cell_index(D), _cell_index(H), _cell_index(W)
    cnt = np.zeros((nz, ny, nx))
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                cnt[iz[z], iy[y], ix[xx]] += 1
    g = dy / cnt
    return g[:, iz][:, :, iy][:, :, :, ix]


def upsample2(x, fine_shape):
    """y[c][p] = x[c][q(p)]."""
    x = np.asarray(x, dtype=np.float64)
    D, H, W = fine_shape
    iz, iy, ix = (np.arange(n) // 2 for n in (D, H, W))
    return x[:, iz][:, :, iy][:, :, :, ix]


def upsample2_backward(dy):
    """dx[c][q] = sum of dy[c][p] over the fine voxels p of cell q."""
    dy = np.asarray(dy, dtype=np.float64)
    C, D, H, W = dy.shape
    (iz, nz), (iy, ny), (ix, nx) = _cell_index(D), _cell_index(H), _cell_index(W)
    out = np.zeros((C, nz, ny, nx))
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                out[:, iz[z], iy[y], ix[xx]] += dy[:, z, y, xx]
    return out
