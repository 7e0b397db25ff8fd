"""Pins of the FP64 network reference: gradients against central finite
differences of the loss, GELU's tanh form against x*Phi(x) (the exact GELU,
within the approximation's known error), and the loss gradient at the output
against its closed form."""
import numpy as np
from scipy.special import ndtr

from oracle import mlp


def test_gelu_tanh_form_close_to_exact_gelu():
    x = np.linspace(-6, 6, 2001)
    assert np.max(np.abs(mlp.gelu(x) - x * ndtr(x))) < 1e-3
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-7


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, h1, h2, n = 12, 16, 8, 10
    npar = h1 * n_in + h1 + h2 * h1 + h2 + 3 * h2 + 3
    p = rng.normal(0, 0.4, npar)
    x = rng.normal(0, 1, (n, n_in))
    t = rng.normal(0, 0.5, (n, 2))
    loss, g, tc = mlp.loss_and_grads(p, x, t, 0.25, n_in, h1, h2)
    assert abs(loss - mlp.loss_only(p, x, t, tc, n_in, h1, h2)) < 1e-12
    eps = 1e-6
    for i in rng.choice(npar, 60, replace=False):
        d = np.zeros(npar)
        d[i] = eps
        fd = (mlp.loss_only(p + d, x, t, tc, n_in, h1, h2) - mlp.loss_only(p - d, x, t, tc, n_in, h1, h2)) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_output_gradient_closed_form():
    # with zero hidden weights the output is the bias: dL/db3 is the closed form
    n_in, h1, h2 = 4, 8, 8
    npar = h1 * n_in + h1 + h2 * h1 + h2 + 3 * h2 + 3
    p = np.zeros(npar)
    p[-3:] = [0.3, -0.2, 0.5]
    x = np.ones((6, n_in))
    t = np.tile([[0.1, 0.4]], (6, 1))
    _, g, tc = mlp.loss_and_grads(p, x, t, 0.25, n_in, h1, h2)
    assert np.allclose(tc, 0.0)   # |vy - ty| = 0.6 > 0.25
    s = 1 / (1 + np.exp(-0.5))
    assert np.allclose(g[-3:], [2 * 0.2, 2 * -0.6, s - 0.0])
