"""The oracle on the paper's own simulated scene, with the filter parameters
the paper prints (Sec. 3; values in tests/golden/paper_simulation.json).

The paper prints no output numbers for this scene, so these are pins by
property:
- the parameter readings reproduce the printed filter: B = 3 at M = 9,
  m'_z = K_z, alpha = e^{-1/10}, a 17 x 17 grid from -2 to 2 in steps of 1/4;
- the whitened background falls well below the input clutter: the PEF of
  Eqs. (4) and (8) at the estimated velocity predicts the translating
  background, so E keeps little more than the sensor noise;
- the target, which moves at another velocity, stands out of the whitened
  background;
- the estimated background velocity lies near the true (1.625, 0.625), which
  sits midway between grid points.
A planted mistake (the PEF applied at the mirrored velocity) must break the
whitening pin, so the pin can tell a wrong filter from a right one.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1408_3526_b300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def printed():
    with open(os.path.join(HERE, "golden", "paper_simulation.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def run(printed):
    f, s = printed["filter"], printed["scene"]
    M, Mz = 2 * f["K_x"] + 1, 2 * f["K_z"] + 1
    sc = scenes.paper_sim_scene(
        T=32, H=f["N_y"], W=f["N_x"], seed=5, components=s["components"],
        fmax=s["frequency_range_cycles_per_px"][1], magnitude=s["component_magnitude"],
        dc=s["dc_offset"], v_clt=tuple(s["background_velocity"]),
        v_tgt=tuple(s["target_velocity"]), tgt_peak=s["target_peak"],
        psf_sigma=s["target_psf_sigma_px"], truncation=s["target_truncation"],
        noise_sigma=s["noise_sigma"])
    o = oracle.Oracle(M, Mz, f["grid_max"], f["grid_step"])
    return o, sc, o.run(sc.frames)


def test_parameter_readings_reproduce_the_printed_filter(printed, run):
    f = printed["filter"]
    o, _, _ = run
    assert o.B == f["B_x"] == f["B_y"]
    assert o.mpz == f["K_z"]
    assert o.alpha == pytest.approx(math.exp(-0.1), rel=0, abs=1e-15)
    assert o.L == int(round((f["grid_max"] - f["grid_min"]) / f["grid_step"])) + 1 == 17


def _masks(o, sc, t_in):
    H, W = sc.frames.shape[1:]
    K = (o.M - 1) // 2
    py, px = np.mgrid[0:H, 0:W]
    tg = sc.targets[0]
    d = np.hypot(px - (tg["x0"] + tg["vx"] * t_in), py - (tg["y0"] + tg["vy"] * t_in))
    interior = (px >= K) & (px < W - K) & (py >= K) & (py < H - K)
    return d, (d > 6) & interior


def _whitening_ratios(o, sc, E, t0=12):
    out = []
    for t in range(t0, sc.frames.shape[0]):
        te = t - o.mpz                    # E(t) is the whitened frame t - m'_z
        _, bg = _masks(o, sc, te)
        out.append(float(E[t][bg].std() / sc.frames[te][bg].std()))
    return np.array(out)


def test_whitened_background_is_well_below_the_clutter(run):
    o, sc, r = run
    ratios = _whitening_ratios(o, sc, r["whitened"])
    assert ratios.max() <= 0.5, ratios


def test_target_stands_out_of_the_whitened_background(run):
    o, sc, r = run
    E = r["whitened"]
    for t in range(12, sc.frames.shape[0]):
        d, bg = _masks(o, sc, t - o.mpz)
        assert np.abs(E[t][d <= 3]).max() >= 10 * E[t][bg].std(), t


def test_estimated_background_velocity_near_the_true_one(printed, run):
    o, sc, r = run
    vtx, vty = printed["scene"]["background_velocity"]
    g = -o.vmax + o.vstep * np.arange(o.L)
    fr = []
    for t in range(12, sc.frames.shape[0]):
        _, bg = _masks(o, sc, t)
        vi = r["vel_index"][t]
        ok = (np.abs(g[vi % o.L] - vtx) <= 2 * o.vstep) & (np.abs(g[vi // o.L] - vty) <= 2 * o.vstep)
        fr.append(ok[bg].mean())
    assert np.mean(fr) >= 0.75, fr


def test_planted_mistake_mirrored_velocity_breaks_the_whitening_pin(run):
    o, sc, r = run
    vi = r["vel_index"]
    mirrored = (o.L - 1 - vi % o.L) + (o.L - 1 - vi // o.L) * o.L
    bad = o.run(sc.frames, vel_override=mirrored, velocity=False)
    assert _whitening_ratios(o, sc, bad["whitened"]).min() > 0.6
