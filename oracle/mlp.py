"""FP64 reference of the learned velocity estimator's network (test
infrastructure only, like the rest of this package).

MLP n_in -> h1 -> h2 -> 3 with the tanh form of GELU,
  GELU(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))),
outputs (vx, vy, c).  Per-sample loss
  (vx - tx)^2 + (vy - ty)^2 + BCE(sigmoid(c), tc),
  tc = 1 if max(|vx - tx|, |vy - ty|) <= vstep else 0 (held constant),
averaged over the batch.  Gradients by the chain rule, written out layer by
layer.  Parameter layout as the library's: W1 [h1][n_in], b1, W2 [h2][h1], b2,
W3 [3][h2], b3, flattened in that order.
"""
from __future__ import annotations

import numpy as np

K0 = np.sqrt(2.0 / np.pi)
K1 = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def unpack(p, n_in, h1, h2, n_out=3):
    shapes = [(h1, n_in), (h1,), (h2, h1), (h2,), (n_out, h2), (n_out,)]
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(np.asarray(p[o:o + n], np.float64).reshape(s))
        o += n
    assert o == len(p)
    return out


def pack(parts):
    return np.concatenate([np.asarray(a, np.float64).ravel() for a in parts])


def forward(p, x, n_in, h1, h2):
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h1, h2)
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    a1 = gelu(z1)
    z2 = a1 @ W2.T + b2
    a2 = gelu(z2)
    y = a2 @ W3.T + b3
    return y, (x, z1, a1, z2, a2)


def loss_and_grads(p, x, t, vstep, n_in, h1, h2):
    """Mean loss and the gradient of the mean loss w.r.t. the flat parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, h1, h2)
    y, (x, z1, a1, z2, a2) = forward(p, x, n_in, h1, h2)
    n = x.shape[0]
    ex, ey = y[:, 0] - t[:, 0], y[:, 1] - t[:, 1]
    c = y[:, 2]
    tc = (np.maximum(np.abs(ex), np.abs(ey)) <= vstep).astype(np.float64)
    bce = np.maximum(c, 0) - c * tc + np.log1p(np.exp(-np.abs(c)))
    loss = np.mean(ex ** 2 + ey ** 2 + bce)
    dy = np.stack([2 * ex, 2 * ey, 1.0 / (1.0 + np.exp(-c)) - tc], axis=1) / n
    gW3 = dy.T @ a2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * gelu_grad(z2)
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * gelu_grad(z1)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3]), tc


def loss_only(p, x, t, tc, n_in, h1, h2):
    """Mean loss with the confidence targets tc held fixed (for finite differences)."""
    y, _ = forward(p, x, n_in, h1, h2)
    ex, ey, c = y[:, 0] - t[:, 0], y[:, 1] - t[:, 1], y[:, 2]
    bce = np.maximum(c, 0) - c * tc + np.log1p(np.exp(-np.abs(c)))
    return np.mean(ex ** 2 + ey ** 2 + bce)


def features_from_power(P):
    """(log2(P(k)/sum_k P(k) + 1e-6) + 10)/10 over a pixel's bins (last three
    axes flattened): the network's input, a normalised log-power spectrum."""
    P = np.asarray(P, np.float64)
    flat = P.reshape(P.shape[:-3] + (-1,))
    tot = flat.sum(-1, keepdims=True)
    return 0.1 * (np.log2(flat / np.where(tot > 0, tot, 1.0) + 1e-6) + 10.0)
