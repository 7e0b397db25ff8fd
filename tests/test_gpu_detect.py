"""Threshold detector on the whitened output (needs a B300): the same pixels,
values and velocity tags as thresholding the read-back frame on the host."""
import numpy as np
import pytest

from paper_1408_3526_b300 import scenes

pytestmark = pytest.mark.gpu


def test_detector_matches_host_threshold():
    from paper_1408_3526_b300.stream import WhitenStream
    sc = scenes.config1_scene(T=24, H=64, W=64, seed=1)
    with WhitenStream(64, 64, 9, 4, 2.0, 0.25) as s:
        for t in range(sc.frames.shape[0]):
            s.push(np.ascontiguousarray(sc.frames[t]))
        e, fi = s.read_whitened()
        vx, vy, _, ti = s.read_velocity()
        det, n, sigma, di = s.detect(k_sigma=4.0, max_det=1024)
        assert di == fi
        ref_sigma = float(np.sqrt(np.mean(e.astype(np.float64) ** 2)))
        assert abs(sigma - ref_sigma) <= 1e-5 * ref_sigma
        ys, xs = np.nonzero(e >= np.float32(4.0) * np.float32(sigma))
        assert n == len(ys)
        assert np.array_equal(det["y"], ys) and np.array_equal(det["x"], xs)     # raster order
        assert np.array_equal(det["value"], e[ys, xs])
        assert np.array_equal(det["vx"], vx[ys, xs]) and np.array_equal(det["vy"], vy[ys, xs])
        # capacity smaller than the count: the first entries in raster order
        det2, n2, _, _ = s.detect(k_sigma=4.0, max_det=1)
        assert n2 == n and len(det2) == min(1, n)
        if n:
            assert det2[0]["y"] == ys[0] and det2[0]["x"] == xs[0]
        # count only
        _, n3, _, _ = s.detect(k_sigma=4.0, max_det=0)
        assert n3 == n


def test_detector_after_pipelined_async_pushes():
    """wh_detect after asynchronous pushes on a pipelined stream sees the last
    frame's whitened output and velocities (the same as the serial stream's)."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    sc = scenes.config1_scene(T=16, H=64, W=80, seed=2)
    fr = sc.frames.astype(np.float32)
    with WhitenStream(64, 80, 9, 4, 2.0, 0.25) as s:
        for t in range(fr.shape[0]):
            s.push(np.ascontiguousarray(fr[t]))
        ref = s.detect(k_sigma=3.0, max_det=4096)
    pin = [torch.from_numpy(fr[t].copy()).pin_memory() for t in range(fr.shape[0])]
    with WhitenStream(64, 80, 9, 4, 2.0, 0.25, pipeline=True) as s:
        for t in range(fr.shape[0]):
            s.push_async(pin[t])
        got = s.detect(k_sigma=3.0, max_det=4096)
    assert got[1] == ref[1] and got[2] == ref[2] and got[3] == ref[3]
    assert np.array_equal(got[0], ref[0])


def test_detector_matches_oracle_detections():
    """The detector's pixel set against the same sigma rule applied to the FP64
    oracle's own whitened frame (Sec. 1: a threshold on the whitened output
    extracts candidate detections).  Sets must agree except at pixels whose
    oracle value lies within the whitened tolerance (1e-3 x input RMS, plus the
    sigma difference times k) of the oracle's threshold; the velocity tag of a
    common detection equals the oracle's velocity there, or a grid step away at
    an oracle near-tie."""
    import oracle
    from paper_1408_3526_b300.stream import WhitenStream
    from tests import _parity as P
    T, H, W, k = 24, 64, 64, 3.0
    sc = scenes.config1_scene(T=T, H=H, W=W, seed=1)
    with WhitenStream(H, W, 9, 4, 2.0, 0.25) as s:
        for t in range(T):
            s.push(np.ascontiguousarray(sc.frames[t]))
        det, n, sigma, di = s.detect(k_sigma=k, max_det=H * W)
        L = s.L
        vmax, step = s.vmax, s.step
    o = oracle.Oracle(9, 4, 2.0, 0.25)
    ref = o.run(sc.frames)
    assert di == T - 1 - o.mpz
    e_ref = ref["whitened"][T - 1]
    sig_ref = float(np.sqrt(np.mean(e_ref ** 2)))
    rms = float(np.sqrt(np.mean(sc.frames.astype(np.float64) ** 2)))
    assert abs(sigma - sig_ref) <= P.WHITE_TOL_REL * rms
    thr = k * sig_ref
    tol = P.WHITE_TOL_REL * rms + k * abs(sigma - sig_ref)
    ref_set = set(zip(*np.nonzero(e_ref >= thr)))
    got_set = set(zip(det["y"].tolist(), det["x"].tolist()))
    assert len(got_set) == n
    for (y, x) in ref_set ^ got_set:
        assert abs(e_ref[y, x] - thr) <= tol, (y, x, e_ref[y, x], thr)
    vi = ref["vel_index"][T - 1]
    for d in det:
        y, x = int(d["y"]), int(d["x"])
        if (y, x) not in ref_set:
            continue
        rx, ry = vi[y, x] % L, vi[y, x] // L
        gx = int(round((float(d["vx"]) + vmax) / step))
        gy = int(round((float(d["vy"]) + vmax) / step))
        assert max(abs(gx - rx), abs(gy - ry)) <= 1
        if (gx, gy) == (rx, ry):
            assert abs(float(d["value"]) - e_ref[y, x]) <= P.WHITE_TOL_REL * rms
    print(f"\n[detect vs oracle] {len(ref_set)} oracle detections, {n} GPU, "
          f"{len(ref_set ^ got_set)} at the threshold edge", flush=True)
    assert len(ref_set) > 0
