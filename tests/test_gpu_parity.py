"""GPU path vs the FP64 oracle on the same seeded inputs (needs a B300).

Cases span several tiles and a ragged tail, frames smaller than the window,
odd and even temporal orders, and the full 512 x 640 configuration in the
launch configuration the benchmark times (sampled pixels).
"""
import numpy as np
import pytest

import oracle
from paper_1408_3526_b300 import scenes
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _compare(frames, M, Mz, vmax, step, spec_frames, debug=True, check_vel_frac=True,
             win_tol=P.SPEC_TOL, **kw):
    T, H, W = frames.shape
    g = P.run_gpu(frames, M, Mz, vmax, step, spec_frames=spec_frames, debug=debug, **kw)
    kw = dict(kw)
    o = oracle.Oracle(M, Mz, vmax, step, B=kw.get("band"), mpz=kw.get("delay_z"),
                      alpha=kw.get("alpha"))
    kw.pop("precision", None)
    ref = o.run(frames, spec_frames=list(spec_frames), spectrum=True, power=debug,
                autocorr=True, windowed=debug)
    m = {"spec": 0.0, "win": 0.0, "win_raw": 0.0, "pow": 0.0, "rs": 0.0}
    for i, t in enumerate(spec_frames):
        m["spec"] = max(m["spec"], P.spectrum_rel_err(g["spectrum"][t], ref["spectrum"][i]))
        if debug:
            m["win"] = max(m["win"], P.spectrum_rel_err(g["windowed"][t], ref["windowed"][i]))
            m["win_raw"] = max(m["win_raw"], P.spectrum_rel_err(g["windowed"][t], ref["windowed"][i],
                                                                 scale_ref=ref["spectrum"][i]))
            m["pow"] = max(m["pow"], P.spectrum_rel_err(g["power"][t], ref["power"][i]))
        ar = ref["autocorr"][i]
        scale = np.abs(ar).reshape(H, W, -1).max(-1)[..., None, None]
        m["rs"] = max(m["rs"], float(np.max(np.abs(g["autocorr"][t] - ar) / np.maximum(scale, 1e-30))))
    rs = {t: ref["autocorr"][i] for i, t in enumerate(spec_frames)}
    frac, steps, tie, bad = P.velocity_report(g["vel_index"], ref["vel_index"], rs, o.L)
    wr = P.whitened_report(g["whitened"], g["vel_index"], ref["whitened"], ref["vel_index"], frames,
                           o.mpz)
    ref2 = o.run(frames, vel_override=g["vel_index"], velocity=False)
    err = P.whitened_err(g["whitened"], ref2["whitened"], frames, o.mpz)
    print(f"\n[parity M={M} Mz={Mz} {T}x{H}x{W}] spec {m['spec']:.2e} windowed {m['win']:.2e} "
          f"(vs raw RMS {m['win_raw']:.2e}) "
          f"power {m['pow']:.2e} R' {m['rs']:.2e} vel_same {frac:.5f} max_steps {steps} "
          f"tie {tie:.2e} whitened vs oracle {wr['matched']:.2e} xRMS ({wr['matched_clutter']:.2e} "
          f"x clutter RMS), at {wr['mismatched_frac']:.1e} near-tie pixels {wr['mismatched']:.2e} xRMS; "
          f"same field {err:.2e} xRMS mismatches {bad[:6]}", flush=True)
    assert m["spec"] <= P.SPEC_TOL
    assert m["win"] <= win_tol
    assert m["pow"] <= 2 * P.SPEC_TOL
    assert m["rs"] <= P.SPEC_TOL
    if check_vel_frac:
        assert frac >= P.VEL_EXACT_FRAC, (frac, bad)
    assert steps <= 1, (steps, bad)
    assert tie <= P.TIE_TOL, (tie, bad)
    assert wr["matched"] <= P.WHITE_TOL_REL, wr
    assert wr["matched_clutter"] <= P.WHITE_TOL_CLUTTER, wr
    assert err <= P.WHITE_TOL_REL, err
    return g, ref


def test_parity_paper_simulation():
    """The paper's own simulation recipe (Sec. 3) as a second regression
    workload: 25 sinusoids translating between grid points, an occluding
    truncated target, 64 x 64 x 32 frames, 9 x 9 window, order 4, grid +-2/4."""
    sc = scenes.paper_sim_scene(T=32)
    _compare(sc.frames, 9, 4, 2.0, 0.25, spec_frames=(3, 31))


def test_parity_paper_simulation_precision_form():
    """The same with the spatial sums in double (WH_PREC_SPEC_F64)."""
    sc = scenes.paper_sim_scene(T=32)
    _compare(sc.frames, 9, 4, 2.0, 0.25, spec_frames=(3, 31), precision=64)


@pytest.mark.parametrize("precision", [16, 0, 128, 32, 64 | 32],
                         ids=["tc_shortlist_rerank", "cuda_cores", "tc_dense", "tc_separable",
                              "f64_sums_tc_separable"])
def test_parity_config1_full(precision):
    """64 x 64 x 32 frames, 9 x 9 window, order 4, grid +-2 step 1/4 (in full),
    with both FP32-exact engines of the autocorrelation search."""
    sc = scenes.config1_scene(T=32)
    _compare(sc.frames, 9, 4, 2.0, 0.25, spec_frames=(3, 31), precision=precision)


@pytest.mark.parametrize("precision", [16, 0, 128, 32],
                         ids=["tc_shortlist_rerank", "cuda_cores", "tc_dense", "tc_separable"])
def test_parity_config2_shape_crop(precision):
    """15 x 15 window, order 6, grid +-3 step 1/4 on a 40 x 56 crop of the
    non-uniform-flow scene (several tiles, ragged tail)."""
    sc = scenes.config2_scene(T=14, H=512, W=640)
    fr = np.ascontiguousarray(sc.frames[:, 200:240, 300:356])
    _compare(fr, 15, 6, 3.0, 0.25, spec_frames=(13,), precision=precision)


@pytest.mark.parametrize("M,Mz,H,W", [(7, 5, 37, 53), (5, 3, 33, 70), (9, 6, 19, 41)])
def test_parity_ragged_odd_even_orders(M, Mz, H, W):
    sc = scenes.small_scene(T=12, H=H, W=W, seed=M * 10 + Mz, vx=0.6, vy=-0.3, tex_size=128)
    _compare(sc.frames, M, Mz, 1.5, 0.5, spec_frames=(Mz - 1, 11))


@pytest.mark.parametrize("M,Mz,vmax,step", [(9, 4, 3.75, 0.25), (5, 6, 1.5, 0.1)])
def test_parity_widest_grid(M, Mz, vmax, step):
    """L = 31, the widest grid the search takes: every lane of a pixel's group
    owns two grid values, and the T rows use the wider stride."""
    sc = scenes.small_scene(T=10, H=21, W=38, seed=M + 100 * Mz, vx=1.2, vy=-0.9, tex_size=128)
    _compare(sc.frames, M, Mz, vmax, step, spec_frames=(9,))


def test_parity_frame_smaller_than_window():
    sc = scenes.small_scene(T=8, H=5, W=7, seed=3, tex_size=64)
    _compare(sc.frames, 9, 4, 2.0, 0.25, spec_frames=(7,), check_vel_frac=False)


@pytest.mark.parametrize("cfg", ["config2", "config3"])
def test_parity_crop_128x160x64(cfg):
    """A 128 x 160 crop over 64 frames, compared element by element with the
    FP64 oracle: the non-uniform-flow scene at 15 x 15 / order 6 / grid +-3
    (its largest speeds, lower right of the 512 x 640 frame), and the
    uniform-flow scene at 1024 x 1280 with 15 x 15 / order 6 / grid +-2."""
    T = 64
    if cfg == "config2":
        sc = scenes.config2_scene(T=T)
        fr = np.ascontiguousarray(sc.frames[:, 360:488, 440:600])
        vmax = 3.0
    else:
        sc = scenes.config1_scene(T=T, H=1024, W=1280, seed=3)
        fr = np.ascontiguousarray(sc.frames[:, 448:576, 560:720])
        vmax = 2.0
    _compare(fr, 15, 6, vmax, 0.25, spec_frames=(T - 1,))


def test_parity_full_size_config2_sampled():
    """512 x 640, 15 x 15, order 6, grid +-3/0.25: full frames on the GPU in the
    benchmark's launch configuration, the oracle on 64 sampled pixels (edges,
    corners, interior) over every frame."""
    T = 20
    sc = scenes.config2_scene(T=T)
    H, W = 512, 640
    g = P.run_gpu(sc.frames, 15, 6, 3.0, 0.25, spec_frames=(T - 1,), debug=False)
    o = oracle.Oracle(15, 6, 3.0, 0.25)
    rng = np.random.default_rng(0)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (7, 300), (255, 319), (511, 17)]
    pts += [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(57)]
    same = 0
    wmax = 0.0
    for (y, x) in pts:
        ref = o.run(sc.frames, crop=(y, x, 1, 1), spec_frames=[T - 1], spectrum=True, autocorr=True)
        assert P.spectrum_rel_err(g["spectrum"][T - 1][y:y + 1, x:x + 1],
                                  ref["spectrum"][0]) <= P.SPEC_TOL
        ar = ref["autocorr"][0]
        assert np.max(np.abs(g["autocorr"][T - 1][y, x] - ar[0, 0])) <= P.SPEC_TOL * np.abs(ar).max()
        gi = g["vel_index"][:, y:y + 1, x:x + 1]
        ri = ref["vel_index"]
        same += int(np.sum(gi[1:] == ri[1:]))          # frame 0: exact tie, see _parity
        d = np.maximum(np.abs(gi % o.L - ri % o.L), np.abs(gi // o.L - ri // o.L))
        assert np.all(d[1:] <= 1), (y, x, d.ravel())
        wr = P.whitened_report(g["whitened"][:, y:y + 1, x:x + 1], gi, ref["whitened"], ri, sc.frames,
                               o.mpz)
        assert wr["matched"] <= P.WHITE_TOL_REL, wr
        wmax = max(wmax, wr["matched"])
        ref2 = o.run(sc.frames, crop=(y, x, 1, 1), vel_override=np.ascontiguousarray(gi),
                     velocity=False)
        err = P.whitened_err(g["whitened"][:, y:y + 1, x:x + 1], ref2["whitened"], sc.frames, o.mpz)
        assert err <= P.WHITE_TOL_REL
    n = (T - 1) * len(pts)
    print(f"\n[parity 512x640 sampled] velocity identical {same}/{n}, whitened vs oracle {wmax:.2e} xRMS",
          flush=True)
    assert same >= P.VEL_EXACT_FRAC * n


def test_parity_full_frames_config2_first12():
    """512 x 640, 15 x 15, order 6, grid +-3/0.25: every pixel of the first 12
    frames against the oracle run on the whole frame (its own velocities, no
    conditioning): smoothed R' of the last frame, velocity
    indices identical except at the oracle's near-ties (one grid step at most
    there), whitened output at every pixel-frame whose velocity agrees."""
    T = 12
    sc = scenes.config2_scene(T=T)
    g = P.run_gpu(sc.frames, 15, 6, 3.0, 0.25, spec_frames=(T - 1,), debug=False)
    o = oracle.Oracle(15, 6, 3.0, 0.25)
    ref = o.run(sc.frames, spec_frames=[T - 1], autocorr=True)
    ar = ref["autocorr"][0]
    scale = np.abs(ar).reshape(512, 640, -1).max(-1)[..., None, None]
    rs_err = float(np.max(np.abs(g["autocorr"][T - 1] - ar) / np.maximum(scale, 1e-30)))
    frac, steps, tie, bad = P.velocity_report(g["vel_index"], ref["vel_index"], {T - 1: ar}, o.L)
    wr = P.whitened_report(g["whitened"], g["vel_index"], ref["whitened"], ref["vel_index"], sc.frames,
                           o.mpz)
    print(f"\n[parity 512x640 full, 12 frames] R' {rs_err:.2e} vel_same {frac:.5f} max_steps {steps} "
          f"tie {tie:.2e} whitened vs oracle {wr['matched']:.2e} xRMS ({wr['matched_clutter']:.2e} x clutter "
          f"RMS), near-tie pixel-frames {wr['mismatched_frac']:.1e}: {wr['mismatched']:.2e} xRMS; "
          f"mismatches {bad[:6]}", flush=True)
    assert rs_err <= P.SPEC_TOL
    assert frac >= P.VEL_EXACT_FRAC, (frac, bad)
    assert steps <= 1, (steps, bad)
    assert tie <= P.TIE_TOL, (tie, bad)
    assert wr["matched"] <= P.WHITE_TOL_REL, wr
    assert wr["matched_clutter"] <= P.WHITE_TOL_CLUTTER, wr


@pytest.mark.parametrize("H,W", [(4096, 4096), (8, 65536), (65536, 8)],
                         ids=["4096x4096", "8x65536", "65536x8"])
def test_parity_large_and_extreme_shapes(H, W):
    """A 4096 x 4096 frame (16.8 M pixels, ~17 GB of state) and extreme aspect
    ratios (a single strip 65536 rows tall: many 256-row restarts of the
    y-recursion; 8 rows by 65536 columns: thousands of strips) at 15 x 15 /
    order 6 / grid +-3, against the oracle on sampled pixels over every frame
    (velocity and the whitened output against the oracle's own)."""
    T = 8
    sc = scenes.small_scene(T=T, H=H, W=W, seed=31, vx=0.8, vy=-0.6, tex_size=512)
    g = P.run_gpu(sc.frames, 15, 6, 3.0, 0.25, debug=False)
    o = oracle.Oracle(15, 6, 3.0, 0.25)
    rng = np.random.default_rng(5)
    pts = [(0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1), (H // 2, W // 2)]
    pts += [(int(rng.integers(0, H)), int(rng.integers(0, W))) for _ in range(11)]
    same, n, wmax = 0, 0, 0.0
    for (y, x) in pts:
        ref = o.run(sc.frames, crop=(y, x, 1, 1))
        gi = g["vel_index"][:, y:y + 1, x:x + 1]
        ri = ref["vel_index"]
        same += int(np.sum(gi[1:] == ri[1:]))
        n += T - 1
        d = np.maximum(np.abs(gi % o.L - ri % o.L), np.abs(gi // o.L - ri // o.L))
        assert np.all(d[1:] <= 1), (y, x, d.ravel())
        wr = P.whitened_report(g["whitened"][:, y:y + 1, x:x + 1], gi, ref["whitened"], ri, sc.frames, o.mpz)
        assert wr["matched"] <= P.WHITE_TOL_REL, (y, x, wr)
        wmax = max(wmax, wr["matched"])
    print(f"\n[parity {H}x{W} sampled] velocity identical {same}/{n}, whitened vs oracle {wmax:.2e} xRMS",
          flush=True)
    assert same >= n - 1


def test_parity_single_velocity_grid():
    """A grid of one point (vmax = 0, L = 1): the search returns it everywhere
    and the filter is the one tuned to v = 0."""
    sc = scenes.small_scene(T=10, H=30, W=44, seed=9, vx=0.2, vy=0.1, tex_size=128)
    g = P.run_gpu(sc.frames, 9, 4, 0.0, 0.25, debug=False)
    assert np.all(g["vel_index"] == 0)
    o = oracle.Oracle(9, 4, 0.0, 0.25)
    assert o.L == 1
    ref = o.run(sc.frames)
    assert P.whitened_err(g["whitened"], ref["whitened"], sc.frames, o.mpz) <= P.WHITE_TOL_REL
