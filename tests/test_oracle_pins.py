"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself:
brute force on tiny inputs, a closed form, an identity, or a special case that
reduces to a textbook result.  They are chosen so that a plausible mistake in
the oracle (a dropped factor, a wrong sign or index, a transposed axis, a
wrong Hann phase, a wrong delay) fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1408_3526_b300 import scenes


def _clamp(v, n):
    return min(max(v, 0), n - 1)


def _window_block(frames, t, py, px, M, Mz):
    """x(n - m) for m in [0,M)^2 x [0,Mz): window origin n = (px+K, py+K, t),
    clamped at the frame edge, zero before frame 0.  Indexed [mz][my][mx]."""
    K = (M - 1) // 2
    T, H, W = frames.shape
    blk = np.zeros((Mz, M, M))
    for mz in range(Mz):
        tt = t - mz
        if tt < 0:
            continue
        for my in range(M):
            for mx in range(M):
                blk[mz, my, mx] = frames[tt, _clamp(py + K - my, H), _clamp(px + K - mx, W)]
    return blk


def _np_dirichlet(W, w):
    w = np.asarray(w, np.float64)
    j = np.rint(w)
    d = w - j
    sgn = np.where(((j * (W - 1)) % 2) == 0, 1.0, -1.0)
    safe = np.where(np.abs(d) < 1e-12, 1.0, d)
    val = np.sin(np.pi * W * safe) / (W * np.sin(np.pi * safe))
    return sgn * np.where(np.abs(d) < 1e-12, 1.0, val)


# --- P1: recursive spectrum == direct windowed 3-D DFT, Eq. (6)-(7) ----------
@pytest.mark.parametrize("M,Mz", [(5, 3), (5, 4), (3, 6)])
def test_recursive_spectrum_equals_direct_dft(M, Mz):
    rng = np.random.default_rng(10 + Mz)
    T, H, W = 8, 11, 13
    fr = rng.standard_normal((T, H, W)).astype(np.float32) + 3.0
    o = oracle.Oracle(M, Mz, vmax=1.0, vstep=0.5)
    ts = [1, Mz - 1, T - 1]
    S = o.run(fr, spec_frames=ts, spectrum=True)["spectrum"]
    K, kzlo = o.K, o.kzlo
    kx = np.arange(M) - K
    kz = np.arange(Mz) + kzlo
    m = np.arange(M)
    mz = np.arange(Mz)
    Fz = np.exp(2j * np.pi * np.outer(kz, mz) / Mz)      # [kz][mz]
    Fs = np.exp(2j * np.pi * np.outer(kx, m) / M)        # [k][m]
    err = 0.0
    for si, t in enumerate(ts):
        for py in range(H):
            for px in range(W):
                blk = _window_block(fr, t, py, px, M, Mz)
                # literal triple sum, Eq. (6)
                d = np.zeros((Mz, M, M), complex)
                for a in range(Mz):
                    for b in range(M):
                        for c in range(M):
                            ph = Fz[a][:, None, None] * Fs[b][None, :, None] * Fs[c][None, None, :]
                            d[a, b, c] = np.sum(ph * blk)
                d /= math.sqrt(M * M * Mz)
                err = max(err, np.max(np.abs(d - S[si, py, px])))
    assert err < 1e-11, err


def test_crop_equals_full_frame():
    rng = np.random.default_rng(3)
    fr = rng.standard_normal((6, 12, 14)).astype(np.float32)
    o = oracle.Oracle(5, 4, vmax=1.0, vstep=0.25)
    ts = list(range(6))
    full = o.run(fr, spec_frames=ts, spectrum=True, autocorr=True)
    part = o.run(fr, crop=(3, 9, 4, 5), spec_frames=ts, spectrum=True, autocorr=True)
    np.testing.assert_allclose(part["spectrum"], full["spectrum"][:, 3:7, 9:14], atol=1e-12)
    np.testing.assert_allclose(part["autocorr"], full["autocorr"][:, 3:7, 9:14], atol=1e-12)
    np.testing.assert_allclose(part["whitened"][1:], full["whitened"][1:, 3:7, 9:14], atol=1e-12)
    # the argmax is unique wherever the top two R' values are not a rounding tie
    # (at frame 0 the lz = 1 slice of R is exactly zero: a tie everywhere)
    r = np.sort(full["autocorr"][:, 3:7, 9:14].reshape(6, 4, 5, -1), axis=-1)
    clear = (r[..., -1] - r[..., -2]) > 1e-9 * np.abs(r[..., -1]).max()
    assert clear[1:].mean() > 0.9
    np.testing.assert_array_equal(part["vel_index"][clear], full["vel_index"][:, 3:7, 9:14][clear])


# --- P2: deadbeat observer ---------------------------------------------------
@pytest.mark.parametrize("Mz", [3, 4, 5, 6])
def test_deadbeat_converges_in_Mz_steps_from_any_state(Mz):
    rng = np.random.default_rng(Mz)
    n = 3 * Mz
    u = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    s0 = 100 * (rng.standard_normal(Mz) + 1j * rng.standard_normal(Mz))
    a = oracle.observer_run(u, Mz, s0)
    kz = np.arange(Mz) - (Mz - 1) // 2
    for t in range(Mz - 1, n):
        last = np.array([u[t - m] for m in range(Mz)])
        dft = np.array([np.sum(last * np.exp(2j * np.pi * k * np.arange(Mz) / Mz)) for k in kz]) / Mz
        assert np.max(np.abs(a[t] - dft)) < 1e-11
    # before Mz steps the initial state has not been forgotten
    assert np.max(np.abs(a[Mz - 2] - np.array([
        np.sum(np.array([u[Mz - 2 - m] if Mz - 2 - m >= 0 else 0 for m in range(Mz)]) *
               np.exp(2j * np.pi * k * np.arange(Mz) / Mz)) / Mz for k in kz]))) > 1e-3


def test_deadbeat_tracks_bin_sinusoid_closed_form():
    Mz = 5
    kz0 = 2
    n = 40
    t = np.arange(n)
    u = np.exp(-2j * np.pi * kz0 * t / Mz)       # delay-m sample = u(t) e^{+j2pi kz0 m/Mz}
    a = oracle.observer_run(u, Mz)
    kz = np.arange(Mz) - (Mz - 1) // 2
    for tt in range(Mz - 1, n):
        expect = np.where(kz == -kz0, u[tt], 0.0)  # sum_m e^{j2pi (kz+kz0) m/Mz}/Mz
        assert np.max(np.abs(a[tt] - expect)) < 1e-12


def test_deadbeat_no_drift_over_10k_frames():
    Mz = 6
    rng = np.random.default_rng(7)
    n = 10000
    u = 10.0 + rng.standard_normal(n)
    a = oracle.observer_run(u.astype(complex), Mz)
    kz = np.arange(Mz) - (Mz - 1) // 2
    last = u[n - Mz:][::-1]
    dft = np.array([np.sum(last * np.exp(2j * np.pi * k * np.arange(Mz) / Mz)) for k in kz]) / Mz
    assert np.max(np.abs(a[-1] - dft)) < 1e-12


# --- P3: Dirichlet kernel, Eq. (3) -------------------------------------------
@pytest.mark.parametrize("W", [4, 5, 6, 7, 9, 15])
def test_dirichlet_matches_definition_and_limit(W):
    rng = np.random.default_rng(W)
    w = rng.uniform(-3, 3, 200)
    ref = np.sin(np.pi * W * w) / (W * np.sin(np.pi * w))
    np.testing.assert_allclose(oracle.dirichlet(W, w), ref, rtol=1e-10, atol=1e-12)
    ints = np.arange(-4, 5)
    np.testing.assert_allclose(oracle.dirichlet(W, ints), (-1.0) ** (ints * (W - 1)), atol=1e-15)
    # continuity through the removable singularity
    np.testing.assert_allclose(oracle.dirichlet(W, 1 + 1e-7), oracle.dirichlet(W, 1.0), atol=1e-10)


@pytest.mark.parametrize("Mz", [4, 5, 6])
def test_dirichlet_partition_of_unity(Mz):
    """sum_kz D_Mz(kz/Mz + u)^2 = 1 for every u (Parseval on the Mz-point DFT)."""
    kz = np.arange(Mz) - (Mz - 1) // 2
    for u in np.linspace(-1.3, 1.3, 37):
        s = np.sum(oracle.dirichlet(Mz, kz / Mz + u) ** 2)
        assert abs(s - 1.0) < 1e-12


# --- P4: frequency-domain PEF (Eq. 4 + 8) == sample-domain FIR (Eq. 1 + 2) ----
@pytest.mark.parametrize("M,Mz,B,v", [(5, 4, 1, (0.37, -1.21)), (7, 5, 2, (1.625, 0.625)),
                                      (9, 6, 3, (-0.8, 0.45))])
def test_pef_frequency_domain_equals_sample_domain(M, Mz, B, v):
    rng = np.random.default_rng(M * Mz)
    T, H, W = Mz + 3, M + 4, M + 5
    fr = (5.0 + rng.standard_normal((T, H, W))).astype(np.float32)
    o = oracle.Oracle(M, Mz, vmax=1.0, vstep=0.5, B=B)
    out = o.run(fr, fixed_v=v)
    K, mpz = o.K, o.mpz
    Wb = 2 * B + 1
    mx = np.arange(M)
    mz = np.arange(Mz)
    # Eq. (2) coefficients, m' = (K, K, m'z)
    ux = (mx[None, None, :] - K - v[0] * (mz[:, None, None] - mpz)) / M
    uy = (mx[None, :, None] - K - v[1] * (mz[:, None, None] - mpz)) / M
    Hs = (Wb * Wb / (M * M * Mz)) * _np_dirichlet(Wb, ux) * _np_dirichlet(Wb, uy)
    err = 0.0
    for t in range(mpz, T):
        for py in range(H):
            for px in range(W):
                blk = _window_block(fr, t, py, px, M, Mz)
                Ihat = np.sum(Hs * blk)                     # Eq. (1)
                Ihat_oracle = fr[t - mpz, py, px] - out["whitened"][t, py, px]
                err = max(err, abs(Ihat - Ihat_oracle))
    assert err < 1e-11, err


# --- P5: PEF nulls a band-limited texture translating at the tuned velocity --
@pytest.mark.parametrize("M,Mz,B,v", [(9, 4, 3, (0.37, -1.21)), (9, 5, 3, (1.625, 0.625)),
                                      (15, 6, 5, (-2.3, 0.7))])
def test_pef_nulls_translating_bandlimited_texture(M, Mz, B, v):
    rng = np.random.default_rng(21)
    comps = []
    for _ in range(8):
        kx, ky = rng.integers(-B, B + 1, 2)
        comps.append((kx / M, ky / M, rng.uniform(0.2, 1.0), rng.uniform(0, 2 * np.pi)))
    T, H, W = Mz + 4, M + 6, M + 8
    fr = scenes.sinusoid_scene(H, W, T, comps, v[0], v[1], dc=10.0).astype(np.float32)
    # float32 frames: compare against the same frames in double
    o = oracle.Oracle(M, Mz, vmax=3.0, vstep=0.25, B=B)
    E = o.run(fr, fixed_v=v)["whitened"]
    K = o.K
    interior = E[Mz - 1:, K:H - K, K:W - K]
    # exact null of the band-limited model; only float32 input rounding remains
    assert np.max(np.abs(interior)) < 2e-5
    # and the filter is not trivially zero: a wrong velocity leaves residue
    E2 = o.run(fr, fixed_v=(v[0] + 0.5, v[1]))["whitened"]
    assert np.max(np.abs(E2[Mz - 1:, K:H - K, K:W - K])) > 1e-2


def test_pef_null_exact_in_double():
    """Same as above with frames exactly representable (integer-valued)."""
    M, Mz, B, v = 9, 4, 3, (1.0, -1.0)
    T, H, W = 8, 15, 17
    # integer translation keeps bin-centred sinusoids sampled on the same grid;
    # scale so every sample is an exact float32
    comps = [(1 / 9, 2 / 9, 1.0, 0.3), (-3 / 9, 1 / 9, 0.5, 1.1), (0.0, 3 / 9, 0.7, 2.0)]
    fr64 = scenes.sinusoid_scene(H, W, T, comps, v[0], v[1], dc=10.0)
    fr = fr64.astype(np.float32)
    o = oracle.Oracle(M, Mz, vmax=2.0, vstep=0.25, B=B)
    E = o.run(fr, fixed_v=v)["whitened"]
    K = o.K
    assert np.max(np.abs(E[Mz - 1:, K:H - K, K:W - K])) < 1e-5


# --- P6: R(l) at integer l == circular autocorrelation of the windowed block --
@pytest.mark.parametrize("M,Mz", [(5, 4), (7, 5), (5, 6)])
def test_autocorr_equals_sample_domain_circular_autocorrelation(M, Mz):
    rng = np.random.default_rng(M + 10 * Mz)
    T, H, W = Mz + 2, 9, 10
    fr = (4.0 + rng.standard_normal((T, H, W))).astype(np.float32)
    o = oracle.Oracle(M, Mz, vmax=2.0, vstep=1.0, alpha=0.0)   # alpha = 0: R' = R
    t = T - 1
    R = o.run(fr, spec_frames=[t], autocorr=True)["autocorr"][0]
    D = (M - 1) / 2.0
    Dz = (Mz - 1) / 2.0
    w = 0.5 + 0.5 * np.cos(2 * np.pi * (np.arange(M) - D) / M)
    wz = 0.5 + 0.5 * np.cos(2 * np.pi * (np.arange(Mz) - Dz) / Mz)
    win = wz[:, None, None] * w[None, :, None] * w[None, None, :]
    grid = o.grid_values().astype(int)
    err = 0.0
    for py in range(H):
        for px in range(W):
            blk = _window_block(fr, t, py, px, M, Mz)
            y = win * (blk - blk.mean(axis=(1, 2), keepdims=True))   # high-pass, then Hann
            for gy, ly in enumerate(grid):
                for gx, lx in enumerate(grid):
                    # y(m + l) with l = (lx, ly, lz = 1), indices modulo the window
                    sh = np.roll(y, shift=(-1, -ly, -lx), axis=(0, 1, 2))
                    ref = np.sum(sh * y)
                    err = max(err, abs(ref - R[py, px, gy, gx]))
    assert err < 1e-10, err


def test_hann_convolution_matches_lines_mode():
    """hp_lines flag zeroes every kx=0 or ky=0 bin; with a constant-per-row
    block both readings agree that the result is zero power."""
    fr = np.tile(np.arange(12, dtype=np.float32)[None, :, None], (6, 1, 11))   # varies in y only
    o = oracle.Oracle(5, 4, vmax=1.0, vstep=0.5, hp_lines=True)
    P = o.run(fr, spec_frames=[5], power=True)["power"][0]
    assert np.max(P) < 1e-20


# --- P7: known shift -> argmax at the true velocity ---------------------------
@pytest.mark.parametrize("v,exact_frac", [((1.0, -1.0), 0.8), ((0.5, 0.25), 0.9),
                                          ((-1.25, 0.75), 0.0), ((0.0, 0.0), 1.0)])
def test_autocorr_peak_at_known_shift(v, exact_frac):
    """A noiseless texture translating at a grid velocity peaks at +v.

    Not exact: the cyclic boundary of Eq. (10) (the paper recommends
    l << M - 1) and the Hann window's own autocorrelation envelope pull the
    peak toward zero lag, by up to one grid step at |v| >= 1.25 with M = 9.
    Pinned as: every interior pixel within one grid step of +v, never beyond
    it in magnitude, and mostly exact at small speeds.  A sign or axis error
    puts the peak far from +v.
    """
    M, Mz = 9, 4
    T, H, W = 24, 24, 24
    sc = scenes.translating_texture(H, W, T, v[0], v[1], seed=4, dc=10.0, noise_rel=0.0,
                                    tex_size=128)
    o = oracle.Oracle(M, Mz, vmax=2.0, vstep=0.25)
    vi = o.run(sc.frames, whitened=False)["vel_index"]
    g = o.grid_values()
    K = o.K
    sel = vi[T - 1, K:H - K, K:W - K]
    vx, vy = g[sel % o.L], g[sel // o.L]
    steps = np.maximum(np.abs(vx - v[0]), np.abs(vy - v[1])) / o.vstep
    assert steps.max() <= 1.0 + 1e-9
    assert np.all(np.abs(vx) <= abs(v[0]) + 1e-9) and np.all(np.abs(vy) <= abs(v[1]) + 1e-9)
    assert np.all(np.sign(vx) * np.sign(v[0]) >= 0) and np.all(np.sign(vy) * np.sign(v[1]) >= 0)
    assert np.mean(steps < 1e-9) >= exact_frac


# --- P8: conjugate symmetries ---------------------------------------------------
def test_power_symmetric_and_pef_hermitian():
    rng = np.random.default_rng(8)
    M, Mz = 7, 6
    fr = (3 + rng.standard_normal((8, 10, 10))).astype(np.float32)
    o = oracle.Oracle(M, Mz, vmax=1.0, vstep=0.5)
    out = o.run(fr, spec_frames=[7], power=True, spectrum=True)
    P = out["power"][0]                       # [h][w][Mz][M][M]
    K, kzlo = o.K, o.kzlo
    for iz in range(Mz):
        jz = ((-(iz + kzlo)) - kzlo) % Mz     # -kz mod Mz, mapped into the bin set
        for iy in range(M):
            for ix in range(M):
                np.testing.assert_allclose(P[..., iz, iy, ix], P[..., jz, 2 * K - iy, 2 * K - ix],
                                           rtol=1e-10, atol=1e-12)
    B = 2
    Hk = oracle.pef_design(M, Mz, B, o.mpz, 0.61, -1.37)
    for iz in range(Mz):
        kz = iz + kzlo
        jz = ((-kz) - kzlo) % Mz
        for jy in range(2 * B + 1):
            for jx in range(2 * B + 1):
                np.testing.assert_allclose(Hk[jz, 2 * B - jy, 2 * B - jx], np.conj(Hk[iz, jy, jx]),
                                           atol=1e-13)
    # Im(Ihat) = 0: sum_k H(k) S(k) over the band is real
    S = out["spectrum"][0]
    for (py, px) in [(2, 3), (5, 5), (9, 0)]:
        Ih = 0
        for iz in range(Mz):
            for jy in range(2 * B + 1):
                for jx in range(2 * B + 1):
                    Ih += Hk[iz, jy, jx] * S[py, px, iz, jy - B + K, jx - B + K]
        assert abs(Ih.imag) < 1e-10 * max(1.0, abs(Ih.real))


# --- smoothing and argmax conventions -------------------------------------------
def test_smoother_is_first_order_recursion_of_raw_R():
    rng = np.random.default_rng(9)
    fr = (2 + rng.standard_normal((7, 8, 9))).astype(np.float32)
    ts = list(range(7))
    raw = oracle.Oracle(5, 4, vmax=1.0, vstep=0.5, alpha=0.0).run(
        fr, spec_frames=ts, autocorr=True)["autocorr"]
    a = math.exp(-0.1)
    sm = oracle.Oracle(5, 4, vmax=1.0, vstep=0.5).run(fr, spec_frames=ts, autocorr=True)["autocorr"]
    ref = np.zeros_like(raw[0])
    for t in ts:
        ref = (1 - a) * raw[t] + a * ref
        np.testing.assert_allclose(sm[t], ref, rtol=1e-12, atol=1e-12)


def test_argmax_ties_go_to_lowest_index_and_flat_convention():
    fr = np.zeros((5, 8, 8), np.float32)           # every R' value is exactly 0: a full tie
    o = oracle.Oracle(5, 4, vmax=1.0, vstep=0.5)
    vi = o.run(fr)["vel_index"]
    assert np.all(vi == 0)


def test_whitened_delay_and_warmup():
    rng = np.random.default_rng(12)
    fr = (1 + rng.standard_normal((6, 7, 7))).astype(np.float32)
    o = oracle.Oracle(5, 6, vmax=1.0, vstep=0.5)
    assert o.mpz == 2
    E = o.run(fr)["whitened"]
    assert np.all(np.isnan(E[:2])) and np.all(np.isfinite(E[2:]))
