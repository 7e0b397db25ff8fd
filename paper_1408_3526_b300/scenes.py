"""Seeded synthetic infrared scenes: cloud-like clutter, point targets, noise.

Input creation only.  Nothing here implements any step of the whitening
method; both the FP64 oracle and the CUDA path consume the frames produced
here.  The paper's real infrared sequences (Sec. 4, Fig. 2) are not
available, so these scenes stand in for them.

Background
    A periodic texture with a 1/f^2 power spectrum (cloud-like): complex
    Gaussian noise shaped by |f|^-1 in the FFT domain, f = 0 removed, real
    part taken, scaled to unit RMS.  A DC offset of ``dc`` x RMS is added
    (the paper's own simulation, Sec. 3, uses DC 10 against component
    magnitude 0.1).
Motion
    Frame t samples the texture bilinearly at the back-mapped position of
    each pixel: uniform translation p - v t, or the exact solution of the
    linear flow dp/dt = G (p - c) (shear plus rotation), I(p,t) =
    g(c + expm(-G t)(p - c)).
Targets
    Additive Gaussian point-spread functions on straight tracks (wrapping at
    the frame edge), peak amplitude a multiple of the noise sigma.
Noise
    Additive white Gaussian.

Axes: x = column index (fast axis), y = row index; a positive velocity
moves content toward +x / +y each frame.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Scene", "make_texture", "uniform_flow", "shear_rotation_flow",
    "config1_scene", "config2_scene", "small_scene", "paper_sim_scene",
    "sinusoid_scene", "translating_texture",
]


@dataclasses.dataclass
class Scene:
    frames: np.ndarray            # float32 [T][H][W]
    true_vx: np.ndarray           # float32 [H][W] background velocity at t=0 (x)
    true_vy: np.ndarray           # float32 [H][W]
    targets: list                 # list of dicts: x0, y0, vx, vy, sigma, amp
    noise_sigma: float
    background_rms: float

    def target_positions(self, t: int):
        """Target centres (x, y) at frame t (wrapped into the frame)."""
        T, H, W = self.frames.shape
        out = []
        for tg in self.targets:
            out.append(((tg["x0"] + tg["vx"] * t) % W, (tg["y0"] + tg["vy"] * t) % H))
        return out


def make_texture(size: int, seed: int) -> np.ndarray:
    """Periodic 1/f^2-power texture of unit RMS and zero mean (float64)."""
    rng = np.random.default_rng(seed)
    fy = np.fft.fftfreq(size)[:, None]
    fx = np.fft.fftfreq(size)[None, :]
    f = np.sqrt(fx * fx + fy * fy)
    amp = np.zeros_like(f)
    amp[f > 0] = 1.0 / f[f > 0]
    noise = rng.standard_normal((size, size)) + 1j * rng.standard_normal((size, size))
    tex = np.fft.ifft2(noise * amp).real
    tex -= tex.mean()
    tex /= np.sqrt(np.mean(tex * tex))
    return tex


def _bilinear_periodic(tex: np.ndarray, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    n0, n1 = tex.shape
    x0 = np.floor(xs)
    y0 = np.floor(ys)
    fx = xs - x0
    fy = ys - y0
    ix0 = x0.astype(np.int64) % n1
    iy0 = y0.astype(np.int64) % n0
    ix1 = (ix0 + 1) % n1
    iy1 = (iy0 + 1) % n0
    return ((1 - fy) * ((1 - fx) * tex[iy0, ix0] + fx * tex[iy0, ix1])
            + fy * ((1 - fx) * tex[iy1, ix0] + fx * tex[iy1, ix1]))


def uniform_flow(vx: float, vy: float):
    """Back-map for a uniform translation: source position of pixel p at t."""
    def back(px, py, t):
        return px - vx * t, py - vy * t

    def vel(px, py):
        return np.full_like(px, vx), np.full_like(py, vy)
    return back, vel


def shear_rotation_flow(cx: float, cy: float, omega: float, shear: float):
    """Linear flow dp/dt = G (p - c), G = [[0, -w(1+s)], [w(1-s), 0]].

    Exact back-map p0 = c + expm(-G t)(p - c); since G^2 = -w^2 (1 - s^2) I,
    expm(G t) = cos(mu t) I + sin(mu t)/mu G with mu = w sqrt(1 - s^2).
    """
    a = omega * (1.0 + shear)
    b = omega * (1.0 - shear)
    mu = math.sqrt(a * b)

    def back(px, py, t):
        c, s = math.cos(mu * t), math.sin(mu * t) / mu
        dx, dy = px - cx, py - cy
        # expm(-G t) = cos(mu t) I - sin(mu t)/mu G
        return cx + c * dx + s * a * dy, cy - s * b * dx + c * dy

    def vel(px, py):
        return -a * (py - cy), b * (px - cx)
    return back, vel


def _render(tex, H, W, T, back, targets, noise_sigma, dc, seed, t0=0):
    rng = np.random.default_rng(seed + 7919)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    frames = np.empty((T, H, W), np.float32)
    for t in range(T):
        sx, sy = back(px, py, t0 + t)
        img = _bilinear_periodic(tex, sx, sy) + dc
        for tg in targets:
            cx = (tg["x0"] + tg["vx"] * (t0 + t)) % W
            cy = (tg["y0"] + tg["vy"] * (t0 + t)) % H
            ddx = (px - cx + W / 2) % W - W / 2
            ddy = (py - cy + H / 2) % H - H / 2
            img += tg["amp"] * np.exp(-(ddx * ddx + ddy * ddy) / (2 * tg["sigma"] ** 2))
        if noise_sigma > 0:
            img += noise_sigma * rng.standard_normal((H, W))
        frames[t] = img
    return frames


def translating_texture(H, W, T, vx, vy, seed, dc=10.0, noise_rel=0.0, tex_size=512,
                        targets=()):
    """A 1/f^2 texture translating uniformly (noise sigma = noise_rel x RMS)."""
    tex = make_texture(tex_size, seed)
    back, vel = uniform_flow(vx, vy)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    tvx, tvy = vel(px, py)
    frames = _render(tex, H, W, T, back, list(targets), noise_rel, dc, seed)
    return Scene(frames, tvx.astype(np.float32), tvy.astype(np.float32), list(targets),
                 noise_rel, 1.0)


def config1_scene(T=32, H=64, W=64, seed=1, tex_size=2048):
    """Plain-method scene: uniform v = (0.7, -0.4), two targets at (-1.2, 0.9).

    Noise sigma = 2% of background RMS; target peak 4 x noise sigma, PSF
    sigma 0.7 px; starts drawn in the interior.
    """
    rng = np.random.default_rng(seed)
    sig_n = 0.02
    targets = []
    for _ in range(2):
        targets.append(dict(x0=float(rng.uniform(0.25 * W, 0.75 * W)),
                            y0=float(rng.uniform(0.25 * H, 0.75 * H)),
                            vx=-1.2, vy=0.9, sigma=0.7, amp=4.0 * sig_n))
    tex = make_texture(tex_size, seed)
    back, vel = uniform_flow(0.7, -0.4)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    tvx, tvy = vel(px, py)
    frames = _render(tex, H, W, T, back, targets, sig_n, 10.0, seed)
    return Scene(frames, tvx.astype(np.float32), tvy.astype(np.float32), targets, sig_n, 1.0)


def config2_scene(T=64, H=512, W=640, seed=2, tex_size=2048, t0=0, max_speed=2.0,
                  shear=0.3, n_targets=5):
    """Non-uniform flow scene (shear plus slow rotation, speeds 0..max_speed).

    The flow centre sits inside the frame, so speeds run from 0 at the centre
    to ``max_speed`` px/frame at the farthest corner.  Five targets with PSF
    sigma U[0.6, 1.0] px, peak U[2, 6] x noise sigma, straight tracks at
    random velocities of magnitude <= 3 px/frame.  Noise sigma = 2% RMS.
    """
    rng = np.random.default_rng(seed)
    sig_n = 0.02
    cx = float(rng.uniform(0.35, 0.65) * W)
    cy = float(rng.uniform(0.35, 0.65) * H)
    rmax = max(math.hypot(x - cx, y - cy) for x in (0, W - 1) for y in (0, H - 1))
    omega = max_speed / (rmax * (1.0 + abs(shear)))
    back, vel = shear_rotation_flow(cx, cy, omega, shear)
    targets = []
    for _ in range(n_targets):
        sp = rng.uniform(0.0, 3.0)
        ang = rng.uniform(0, 2 * math.pi)
        targets.append(dict(x0=float(rng.uniform(0, W)), y0=float(rng.uniform(0, H)),
                            vx=sp * math.cos(ang), vy=sp * math.sin(ang),
                            sigma=float(rng.uniform(0.6, 1.0)),
                            amp=float(rng.uniform(2.0, 6.0)) * sig_n))
    tex = make_texture(tex_size, seed)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    tvx, tvy = vel(px, py)
    frames = _render(tex, H, W, T, back, targets, sig_n, 10.0, seed, t0=t0)
    return Scene(frames, tvx.astype(np.float32), tvy.astype(np.float32), targets, sig_n, 1.0)


def small_scene(T, H, W, seed, vx=0.7, vy=-0.4, noise=0.02, tex_size=256, n_targets=1):
    """Small cluttered scene for fast parity cases (config-1 generator, smaller)."""
    rng = np.random.default_rng(seed)
    targets = [dict(x0=float(rng.uniform(0, W)), y0=float(rng.uniform(0, H)),
                    vx=-1.2, vy=0.9, sigma=0.7, amp=4.0 * max(noise, 0.02))
               for _ in range(n_targets)]
    tex = make_texture(tex_size, seed)
    back, vel = uniform_flow(vx, vy)
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    tvx, tvy = vel(px, py)
    frames = _render(tex, H, W, T, back, targets, noise, 10.0, seed)
    return Scene(frames, tvx.astype(np.float32), tvy.astype(np.float32), targets, noise, 1.0)


def sinusoid_scene(H, W, T, comps, vx, vy, dc=0.0):
    """Sum of real sinusoids translating at (vx, vy): comps = [(fx, fy, amp, phase)]."""
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    frames = np.empty((T, H, W), np.float64)
    for t in range(T):
        img = np.full((H, W), dc, np.float64)
        for fx, fy, a, ph in comps:
            img += a * np.cos(2 * np.pi * (fx * (px - vx * t) + fy * (py - vy * t)) + ph)
        frames[t] = img
    return frames


def training_scene_set(n_scenes, T, H, W, seed0=100, vlim=1.75, tex_size=2048, noise_rel=0.02):
    """Yield (frames [T][H][W], (vx, vy)) for n_scenes config-1-style scenes:
    one 1/f^2 texture (seed seed0), each scene a random window origin and a
    uniform velocity drawn U[-vlim, vlim]^2 (scene seed = seed0 + i), additive
    white noise of noise_rel x RMS."""
    tex = make_texture(tex_size, seed0)
    for i in range(n_scenes):
        rng = np.random.default_rng(seed0 + i)
        vx, vy = rng.uniform(-vlim, vlim, 2)
        ox, oy = rng.uniform(0, tex_size, 2)
        back0, _ = uniform_flow(vx, vy)

        def back(px, py, t, ox=ox, oy=oy, back0=back0):
            sx, sy = back0(px, py, t)
            return sx + ox, sy + oy
        frames = _render(tex, H, W, T, back, [], noise_rel, 10.0, seed0 + i)
        yield frames, (float(vx), float(vy))


def paper_sim_scene(T=32, H=64, W=64, seed=5, components=25, fmax=2 / 9, magnitude=0.1, dc=10.0,
                    v_clt=(1.625, 0.625), v_tgt=(-0.625, -0.375), tgt_peak=1.0, psf_sigma=1.0,
                    truncation=0.1, noise_sigma=0.1):
    """The paper's own simulation recipe (Sec. 3), re-generated from its text
    (the defaults are the values it prints).

    `components` sinusoids with spatial frequencies U[-fmax, fmax] cycles/px,
    random phase, the given magnitude, plus the DC offset, translating at
    v_clt px/frame.  One occluding target: Gaussian PSF of psf_sigma px and
    peak tgt_peak, truncated below `truncation`, velocity v_tgt, centred in
    the last frame.  Zero-mean Gaussian noise of noise_sigma.
    """
    rng = np.random.default_rng(seed)
    comps = [(rng.uniform(-fmax, fmax), rng.uniform(-fmax, fmax), magnitude,
              rng.uniform(0, 2 * np.pi)) for _ in range(components)]
    vx, vy = v_clt
    bg = sinusoid_scene(H, W, T, comps, vx, vy, dc=dc)
    tvx, tvy = v_tgt
    cx_end, cy_end = (W - 1) / 2.0, (H - 1) / 2.0
    py, px = np.mgrid[0:H, 0:W].astype(np.float64)
    frames = np.empty((T, H, W), np.float32)
    for t in range(T):
        cx = cx_end + tvx * (t - (T - 1))
        cy = cy_end + tvy * (t - (T - 1))
        psf = tgt_peak * np.exp(-((px - cx) ** 2 + (py - cy) ** 2) / (2.0 * psf_sigma ** 2))
        img = np.where(psf >= truncation, psf, bg[t])       # the target occludes
        img = img + noise_sigma * rng.standard_normal((H, W))
        frames[t] = img
    targets = [dict(x0=cx_end + tvx * (-(T - 1)), y0=cy_end + tvy * (-(T - 1)), vx=tvx,
                    vy=tvy, sigma=psf_sigma, amp=tgt_peak)]
    return Scene(frames, np.full((H, W), vx, np.float32), np.full((H, W), vy, np.float32),
                 targets, noise_sigma, magnitude)
