"""Element-wise error bounds for the network's GPU forward and backward
against the FP64 reference (``oracle.mlp``), from first-order propagation of
the rounding the GPU path performs (test helper).

The reference runs in FP64 on the same BF16-rounded weights and inputs; the
GPU path differs by:
  - FP32 accumulation of every tensor-core product (bounded by K 2^-22 of the
    sum of |terms|, four times the round-to-nearest unit roundoff, since the
    accumulation order and alignment are the hardware's);
  - FP32 bias adds and GELU evaluation (as z / (1 + e^{-2u}), the exact
    identity for the tanh form, with the hardware exponential and a fast
    divide: a few FP32 ulps, inside the 4 unit roundoffs allowed below);
  - BF16 rounding (unit roundoff 2^-8) of the hidden activations H1, H2, of
    the output gradient dY and of the pre-activation gradients dZ2, dZ1.
Each error is propagated through the next product with absolute values
(|W| @ e), the GELU by its derivative plus half its curvature bound
(|GELU''| <= 0.8) times the error squared.  The returned bounds are per
entry, so a wrong entry (a transposed bias, a dropped GELU' on a few
columns) stands out against them.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U_BF16 = 2.0 ** -8
U_F32 = 2.0 ** -24


def _gamma(k):
    return k * 2.0 ** -22


def _gelu_err(z, a, ez):
    """Error of a = GELU(z) evaluated in FP32 at z + dz, |dz| <= ez."""
    return (np.abs(mlp.gelu_grad(z)) + 0.5 * ez) * ez + 4 * U_F32 * (np.abs(z) + np.abs(a))


def forward_bounds(p, x, n_in, h1, h2):
    """Reference intermediates and per-entry bounds of the forward pass.

    Returns (y, e_y, ctx) with ctx holding z1, a1, z2, a2 and their bounds."""
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, n_in, h1, h2)
    y, (x, z1, a1, z2, a2) = mlp.forward(p, x, n_in, h1, h2)
    ax = np.abs(x)
    e_z1 = _gamma(n_in) * (ax @ np.abs(W1).T) + 2 * U_F32 * np.abs(z1)
    e_a1 = U_BF16 * np.abs(a1) + _gelu_err(z1, a1, e_z1)
    e_z2 = e_a1 @ np.abs(W2).T + _gamma(h1) * (np.abs(a1) @ np.abs(W2).T) + 2 * U_F32 * np.abs(z2)
    e_a2 = U_BF16 * np.abs(a2) + _gelu_err(z2, a2, e_z2)
    e_y = e_a2 @ np.abs(W3).T + _gamma(h2) * (np.abs(a2) @ np.abs(W3).T) + 2 * U_F32 * np.abs(y)
    ctx = dict(x=x, z1=z1, a1=a1, z2=z2, a2=a2, e_z1=e_z1, e_a1=e_a1, e_z2=e_z2, e_a2=e_a2,
               W1=W1, W2=W2, W3=W3)
    return y, e_y, ctx


def threshold_margin(y, e_y, t, vstep):
    """Distance of each sample's max(|ex|, |ey|) from vstep, in units of its
    velocity error bound (the confidence label flips inside a margin < 1)."""
    m = np.maximum(np.abs(y[:, 0] - t[:, 0]), np.abs(y[:, 1] - t[:, 1]))
    return np.abs(m - vstep) / np.maximum(np.max(e_y[:, :2], axis=1), 1e-30)


def grad_bounds(p, x, t, vstep, n_in, h1, h2):
    """Reference gradients and per-entry bounds (flat, in the parameter
    layout W1, b1, W2, b2, W3, b3), for targets away from the label flip."""
    y, e_y, c = forward_bounds(p, x, n_in, h1, h2)
    _, g, tc = mlp.loss_and_grads(p, x, t, vstep, n_in, h1, h2)
    n = x.shape[0]
    W2, W3 = c["W2"], c["W3"]
    ex, ey = y[:, 0] - t[:, 0], y[:, 1] - t[:, 1]
    sg = 1.0 / (1.0 + np.exp(-y[:, 2]))
    dy = np.stack([2 * ex, 2 * ey, sg - tc], axis=1) / n
    e_dy = U_BF16 * np.abs(dy) + np.stack([2 * e_y[:, 0], 2 * e_y[:, 1], 0.25 * e_y[:, 2] + 1e-6], 1) / n
    a1, a2, ax = np.abs(c["a1"]), np.abs(c["a2"]), np.abs(c["x"])
    gz1, gz2 = mlp.gelu_grad(c["z1"]), mlp.gelu_grad(c["z2"])
    dH2 = dy @ W3
    dz2 = dH2 * gz2
    dH1 = dz2 @ W2
    dz1 = dH1 * gz1
    e_gW3 = e_dy.T @ a2 + np.abs(dy).T @ c["e_a2"] + _gamma(n) * (np.abs(dy).T @ a2)
    e_gb3 = e_dy.sum(0) + _gamma(n) * np.abs(dy).sum(0)
    e_dH2 = e_dy @ np.abs(W3) + _gamma(3) * (np.abs(dy) @ np.abs(W3))
    e_dz2 = U_BF16 * np.abs(dz2) + np.abs(gz2) * e_dH2 + 0.8 * np.abs(dH2) * c["e_z2"] + 4 * U_F32 * np.abs(dz2)
    e_gW2 = e_dz2.T @ a1 + np.abs(dz2).T @ c["e_a1"] + _gamma(n) * (np.abs(dz2).T @ a1)
    e_gb2 = e_dz2.sum(0) + _gamma(n) * np.abs(dz2).sum(0)
    e_dH1 = e_dz2 @ np.abs(W2) + _gamma(h2) * (np.abs(dz2) @ np.abs(W2))
    e_dz1 = U_BF16 * np.abs(dz1) + np.abs(gz1) * e_dH1 + 0.8 * np.abs(dH1) * c["e_z1"] + 4 * U_F32 * np.abs(dz1)
    e_gW1 = e_dz1.T @ ax + _gamma(n) * (np.abs(dz1).T @ ax)
    e_gb1 = e_dz1.sum(0) + _gamma(n) * np.abs(dz1).sum(0)
    e = mlp.pack([e_gW1, e_gb1, e_gW2, e_gb2, e_gW3, e_gb3])
    inter = dict(dy=dy, dH2=dH2, dz2=dz2, dH1=dH1, dz1=dz1, gz1=gz1, gz2=gz2, **c)
    return g, e, tc, inter


PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def param_slices(n_in, h1, h2, n_out=3):
    sizes = [h1 * n_in, h1, h2 * h1, h2, n_out * h2, n_out]
    out, o = {}, 0
    for name, s in zip(PARAM_NAMES, sizes):
        out[name] = slice(o, o + s)
        o += s
    return out
