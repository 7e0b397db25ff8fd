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


# ---- the network's input: features_from_power ------------------------------------------
def _feature_pins(fn):
    """Properties of the normalised log-power input that fix it without
    restating it: returns the list of failed pins (empty when all hold)."""
    failed = []
    rng = np.random.default_rng(3)
    M, Mz = 5, 4
    P = rng.exponential(1.0, (3, 2, Mz, M, M))
    f = np.asarray(fn(P))
    # 1. invariance under a common scale of the power (P -> cP)
    if not np.allclose(np.asarray(fn(7.5 * P)), f, rtol=0, atol=1e-12):
        failed.append("scale")
    # 2. a flat spectrum: every bin holds 1/N of the power
    N = Mz * M * M
    flat = np.asarray(fn(np.full((1, 1, Mz, M, M), 2.0))).ravel()
    if not np.allclose(flat, 0.1 * (np.log(1.0 / N + 1e-6) / np.log(2.0) + 10.0), rtol=0, atol=1e-12):
        failed.append("flat")
    # 3. one bin holds all the power: 0.1 (log2(1 + 1e-6) + 10) there, 0.1 (log2(1e-6) + 10) elsewhere
    one = np.zeros((1, 1, Mz, M, M))
    one[0, 0, 1, 2, 3] = 4.0
    g = np.asarray(fn(one)).reshape(Mz, M, M)
    want = np.full((Mz, M, M), 0.1 * (np.log(1e-6) / np.log(2.0) + 10.0))
    want[1, 2, 3] = 0.1 * (np.log(1.0 + 1e-6) / np.log(2.0) + 10.0)
    if not np.allclose(g, want, rtol=0, atol=1e-12):
        failed.append("single bin")
    # 4. output shape: the three bin axes flattened in [kz][ky][kx] order
    if f.shape != (3, 2, N) or not np.allclose(f[1, 0].reshape(Mz, M, M)[2, 4, 0],
                                               np.asarray(fn(P[1:2, 0:1]))[0, 0].reshape(Mz, M, M)[2, 4, 0]):
        failed.append("layout")
    return failed


def test_features_from_power_pins():
    assert _feature_pins(mlp.features_from_power) == []


def test_features_from_power_mirror_symmetry_on_oracle_power():
    """P(-k) = P(k) for a real input (pin P8 of the spectrum), so the features of
    mirrored bins are equal: feature[kz][ky][kx] = feature[-kz][-ky][-kx]."""
    import oracle
    from paper_1408_3526_b300 import scenes
    M, Mz = 5, 4
    sc = scenes.small_scene(T=6, H=9, W=11, seed=4, tex_size=64)
    o = oracle.Oracle(M, Mz, 1.0, 0.25)
    P = o.run(sc.frames, spec_frames=[5], power=True)["power"][0]
    f = mlp.features_from_power(P).reshape(9, 11, Mz, M, M)
    # bins kz = -((Mz-1)//2) .. Mz//2: index iz -> kz = iz - 1; the mirror of kz is -kz mod Mz
    kz = np.arange(Mz) - (Mz - 1) // 2
    iz_m = [int(np.nonzero(((-k - kz) % Mz) == 0)[0][0]) for k in kz]
    mirror = f[:, :, iz_m][:, :, :, ::-1, ::-1]
    assert np.allclose(f, mirror, rtol=0, atol=1e-9)


def test_feature_pins_catch_planted_mistakes():
    """Mutants of the input definition fail the pins: natural log instead of
    log2, no normalisation by the total power, and a dropped offset."""
    def ln_mutant(P):
        P = np.asarray(P, np.float64)
        flat = P.reshape(P.shape[:-3] + (-1,))
        tot = flat.sum(-1, keepdims=True)
        return 0.1 * (np.log(flat / tot + 1e-6) + 10.0)

    def unnormalised(P):
        P = np.asarray(P, np.float64)
        flat = P.reshape(P.shape[:-3] + (-1,))
        return 0.1 * (np.log2(flat + 1e-6) + 10.0)

    def no_offset(P):
        P = np.asarray(P, np.float64)
        flat = P.reshape(P.shape[:-3] + (-1,))
        return 0.1 * np.log2(flat / flat.sum(-1, keepdims=True) + 1e-6)

    for fn in (ln_mutant, unnormalised, no_offset):
        assert _feature_pins(fn) != [], fn.__name__


# ---- the element-wise bounds the GPU network tests use ------------------------------------
def test_elementwise_bounds_catch_planted_mistakes():
    """The per-entry gradient bounds of the GPU comparison are tight enough to
    flag plausible mistakes planted in an otherwise exact FP64 backward: a
    dropped GELU' on four hidden columns of layer 1, a reversed b1 gradient,
    and W2's gradient transposed within one 8x8 block."""
    from tests import _mlp_bounds as B
    rng = np.random.default_rng(2)
    n_in, h1, h2, n = 96, 32, 16, 128
    npar = h1 * n_in + h1 + h2 * h1 + h2 + 3 * h2 + 3
    p = rng.normal(0, 1, npar)
    sl = B.param_slices(n_in, h1, h2)
    for name, (r, c) in zip(("W1", "W2", "W3"), ((h1, n_in), (h2, h1), (3, h2))):
        p[sl[name]] /= np.sqrt(c)
    for name in ("b1", "b2", "b3"):
        p[sl[name]] *= 0.1
    x = rng.normal(0, 1, (n, n_in))
    y, e_y, _ = B.forward_bounds(p, x, n_in, h1, h2)
    t = y[:, :2] + rng.uniform(-0.6, 0.6, (n, 2))
    for _ in range(20):                 # keep every label away from its flip
        bad = B.threshold_margin(y, e_y, t, 0.25) < 8
        if not bad.any():
            break
        t[bad] += 0.05
    g, e, tc, it = B.grad_bounds(p, x, t, 0.25, n_in, h1, h2)
    assert np.all(e > 0) and np.all(np.isfinite(e))
    # 1. dropped GELU' on hidden columns 0..3 of layer 1
    dz1 = it["dz1"].copy()
    dz1[:, :4] = it["dH1"][:, :4]
    g1 = g.copy()
    g1[sl["W1"]] = (dz1.T @ it["x"]).ravel()
    # 2. reversed b1 gradient
    g2 = g.copy()
    g2[sl["b1"]] = g[sl["b1"]][::-1]
    # 3. an 8 x 8 block of W2's gradient transposed
    g3 = g.copy()
    gw2 = g[sl["W2"]].reshape(h2, h1).copy()
    gw2[:8, :8] = gw2[:8, :8].T.copy()
    g3[sl["W2"]] = gw2.ravel()
    for gm in (g1, g2, g3):
        assert np.any(np.abs(gm - g) > 2 * e)


def test_folded_first_layer_equals_network_on_all_bins():
    """One input per mirror pair: with P(-k) = P(k) (the oracle's power of a real
    input, pin P8), a first layer whose columns of k and -k are summed gives
    the same pre-activations on the folded features as the original layer on
    all bins; the folded width is (M^2 Mz + 2 - Mz % 2) / 2."""
    import oracle
    from paper_1408_3526_b300 import learned, scenes
    for M, Mz in ((5, 4), (5, 3)):
        sc = scenes.small_scene(T=6, H=7, W=9, seed=11, tex_size=64)
        P = oracle.Oracle(M, Mz, 1.0, 0.25).run(sc.frames, spec_frames=[5], power=True)["power"][0]
        f_all = mlp.features_from_power(P).reshape(7 * 9, -1)
        rng = np.random.default_rng(M * 10 + Mz)
        W1 = rng.normal(0, 1, (16, M * M * Mz))
        Wf = learned.fold_first_layer(W1, M, Mz)
        assert Wf.shape[1] == learned.n_features(M, Mz) == (M * M * Mz + 2 - Mz % 2) // 2
        K, J = (M - 1) // 2, (Mz - 1) // 2
        keep = []
        for iz in range(Mz):
            kzm = -(iz - J)
            kzm += Mz if kzm < -J else 0
            for iy in range(M):
                for ix in range(M):
                    b = (iz * M + iy) * M + ix
                    if b <= ((kzm + J) * M + (2 * K - iy)) * M + (2 * K - ix):
                        keep.append(b)
        z_all = f_all @ W1.T
        z_fold = f_all[:, keep] @ Wf.T
        assert np.allclose(z_all, z_fold, rtol=1e-12, atol=1e-9)
