"""Learned velocity estimator on the GPU against the FP64 network oracle and
the plain search (needs a B300)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1408_3526_b300 import scenes
from tests import _mlp_bounds as B
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


def _net_with_random_params(n_in, h1, h2, seed):
    from paper_1408_3526_b300.learned import MLP
    net = MLP(n_in, h1, h2, 3, seed=seed)
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 1, net.n_params).astype(np.float32)
    # scale like the default init, keep biases modest
    o = 0
    for (r, c) in [(h1, n_in), (h2, h1), (3, h2)]:
        p[o:o + r * c] *= 1.0 / np.sqrt(c)
        o += r * c
        p[o:o + r] *= 0.1
        o += r
    net.set_params(p)
    return net, p


def _bf16_params(p, n_in, h1, h2):
    W1, b1, W2, b2, W3, b3 = omlp.unpack(p, n_in, h1, h2)
    return omlp.pack([_bf16_round(W1), b1, _bf16_round(W2), b2, _bf16_round(W3), b3])


@pytest.mark.parametrize("n_in,h1,h2", [(1350, 256, 128), (676, 256, 128), (324, 64, 32)])
def test_mlp_forward_matches_oracle(n_in, h1, h2):
    import torch
    net, p = _net_with_random_params(n_in, h1, h2, 3)
    n, ld = 1000, (n_in + 7) // 8 * 8
    rng = np.random.default_rng(4)
    x = np.zeros((n, ld), np.float32)
    x[:, :n_in] = rng.normal(0, 1, (n, n_in))
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    y = net.forward(xb).cpu().numpy()
    yr, e_y, _ = B.forward_bounds(_bf16_params(p, n_in, h1, h2), xb.float().cpu().numpy()[:, :n_in],
                                  n_in, h1, h2)
    # element-wise: every output within twice its propagated rounding bound
    d = np.abs(y[:, :3] - yr)
    print(f"\n[mlp forward {n_in}-{h1}-{h2}] max |dy| / bound {np.max(d / e_y):.3f}, "
          f"median bound / |y| {np.median(e_y / np.maximum(np.abs(yr), 1e-30)):.2e}", flush=True)
    assert np.all(d <= 2 * e_y), np.max(d / e_y)
    net.close()


def test_mlp_gradients_match_oracle():
    import torch
    n_in, h1, h2, n = 1350, 256, 128, 512
    net, p = _net_with_random_params(n_in, h1, h2, 5)
    ld = 1352
    rng = np.random.default_rng(6)
    x = np.zeros((n, ld), np.float32)
    x[:, :n_in] = rng.normal(0, 1, (n, n_in))
    xb = torch.from_numpy(x).to(torch.bfloat16).cuda()
    pb = _bf16_params(p, n_in, h1, h2)
    xr = xb.float().cpu().numpy()[:, :n_in].astype(np.float64)
    yr, e_y, _ = B.forward_bounds(pb, xr, n_in, h1, h2)
    t = rng.uniform(-1, 1, (n, 2))
    for _ in range(40):                 # keep every confidence label away from its flip
        bad = B.threshold_margin(yr, e_y, t, 0.25) < 8
        if not bad.any():
            break
        t[bad] += 0.03
    t = t.astype(np.float32)
    net.train_step(xb, torch.from_numpy(t).cuda(), 0.25, lr=0.0, apply=False)
    g = net.grads().astype(np.float64)
    gr, e, _, _ = B.grad_bounds(pb, xr, t.astype(np.float64), 0.25, n_in, h1, h2)
    # element-wise: every gradient entry within twice its propagated rounding bound
    for name, sl in B.param_slices(n_in, h1, h2).items():
        d = np.abs(g[sl] - gr[sl])
        print(f"\n[mlp grad {name}] max |dg| / bound {np.max(d / e[sl]):.3f}", flush=True)
        assert np.all(d <= 2 * e[sl]), (name, float(np.max(d / e[sl])))
    net.close()


def _unique_bins(M, Mz):
    """Flat [kz][ky][kx] indices of the bins not after their mirror -k."""
    K, J = (M - 1) // 2, (Mz - 1) // 2
    out = []
    for iz in range(Mz):
        kzm = -(iz - J)
        if kzm < -J:
            kzm += Mz
        for iy in range(M):
            for ix in range(M):
                b = (iz * M + iy) * M + ix
                if b <= ((kzm + J) * M + (2 * K - iy)) * M + (2 * K - ix):
                    out.append(b)
    return np.array(out)


@pytest.mark.parametrize("M,Mz", [(9, 4), (15, 6), (15, 4)])
@pytest.mark.parametrize("mode", [1, 2], ids=["all_bins", "one_per_mirror_pair"])
def test_features_match_oracle_power(mode, M, Mz):
    """Features of every bin (mode 1) or of one bin per mirror pair (mode 2)
    against the oracle's power, for window/order shapes whose per-pixel power
    totals are summed by one, four and two lanes per pixel."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    T, H, W = 8, 24, 30
    sc = scenes.small_scene(T=T, H=H, W=W, seed=8, tex_size=128)
    with WhitenStream(H, W, M, Mz, 2.0, 0.25) as s:
        assert s.lib.wh_stream_set_features(s._s, mode) == 0
        fd = torch.from_numpy(sc.frames).cuda()
        for t in range(T):
            s.push(fd[t])
        ld = C.c_int()
        s.lib.wh_read_features(s._s, None, 1, C.byref(ld))
        feat = torch.empty((H * W, ld.value), dtype=torch.bfloat16, device="cuda")
        assert s.lib.wh_read_features(s._s, C.c_void_p(feat.data_ptr()), 1, None) == 0
        f = feat.float().cpu().numpy()
    P = oracle.Oracle(M, Mz, 2.0, 0.25).run(sc.frames, spec_frames=[T - 1], power=True)["power"][0]
    ref = omlp.features_from_power(P).reshape(H * W, -1)
    if mode == 2:
        ref = ref[:, _unique_bins(M, Mz)]
        assert ref.shape[1] == (M * M * Mz + 2) // 2
    nb = ref.shape[1]
    assert np.all(f[:, nb:] == 0)
    err = np.abs(f[:, :nb] - ref)
    assert np.max(err - (2.0 ** -7) * np.abs(ref)) <= 2e-3, np.max(err)


def test_training_gains_and_learned_mode():
    """Train on plain-search labels from small scenes.  Gain over the method
    without it: the trained network decides most pixels itself (the search is
    skipped there) while the learned mode's velocities still agree with the
    plain search within one grid step on >= 95% of pixels; the untrained
    network of the same seed decides (almost) none at the same threshold."""
    import torch

    from paper_1408_3526_b300 import learned
    from paper_1408_3526_b300.stream import WhitenStream
    M, Mz, vmax, step = 9, 4, 2.0, 0.25
    X, V = learned.generate_training_data(n_scenes=240, frames=10, H=64, W=64, M=M, Mz=Mz, vmax=vmax,
                                          step=step, samples=240_000, seed0=200)
    n_in = learned.n_features(M, Mz)          # one input per mirror pair of bins
    trained = learned.MLP(n_in, 256, 128, 3, seed=1)
    untrained = learned.MLP(n_in, 256, 128, 3, seed=1)
    hist = learned.train(trained, X, V, vstep=step, epochs=30, batch=4096, lr=2e-3)
    T, H, W = 12, 96, 96
    frames, _ = next(scenes.training_scene_set(1, T, H, W, seed0=777))
    fd = torch.from_numpy(frames).cuda()
    res = {}
    seq = {}
    for name, net in [("plain", None), ("trained", trained), ("untrained", untrained)]:
        with WhitenStream(H, W, M, Mz, vmax, step) as s:
            if net is not None:
                assert s.lib.wh_stream_set_learned(s._s, net._m, 0.8) == 0
            vel_seq = np.zeros((T, H, W), np.int32)
            wh_seq = np.full((T, H, W), np.nan)
            for t in range(T):
                s.push(fd[t])
                _, _, vi_t, ti = s.read_velocity()
                assert ti == t
                vel_seq[t] = vi_t
                if t >= s.delay_z:
                    wh_seq[t], _ = s.read_whitened()
            seq[name] = (vel_seq, wh_seq, s.delay_z)
            _, _, vi, _ = s.read_velocity()
            fr, fb = C.c_longlong(), C.c_longlong()
            s.lib.wh_stream_learned_stats(s._s, C.byref(fr), C.byref(fb))
            res[name] = (vi.copy(), fb.value / max(fr.value, 1) / (H * W))
    plain = res["plain"][0]
    L = int(round(2 * vmax / step)) + 1
    for name in ("trained", "untrained"):
        vi, fb_frac = res[name]
        d = np.maximum(np.abs(vi % L - plain % L), np.abs(vi // L - plain // L))
        res[name] = (vi, fb_frac, float(np.mean(d <= 1)))
    print(f"\n[learned] trained: accepted {1 - res['trained'][1]:.3f} within-1-step {res['trained'][2]:.3f}; "
          f"untrained: accepted {1 - res['untrained'][1]:.3f} within-1-step {res['untrained'][2]:.3f}; "
          f"loss {hist[0][0]:.3f} -> {hist[-1][0]:.3f}, within-step (train) {hist[-1][3]:.3f}", flush=True)
    assert hist[-1][0] < 0.5 * hist[0][0]
    assert res["trained"][2] >= 0.95
    acc_t, acc_u = 1 - res["trained"][1], 1 - res["untrained"][1]
    assert acc_t >= 0.5 and acc_t > acc_u + 0.3
    # against the FP64 oracle on a 24 x 24 crop: the learned velocities sit
    # within one grid step of the oracle's own argmax, and the whitened output
    # is the oracle's filter on the learned velocity field
    vel_l, wh_l, dz = seq["trained"]
    y0, x0, h, w = 36, 36, 24, 24
    o = oracle.Oracle(M, Mz, vmax, step)
    ref = o.run(frames, crop=(y0, x0, h, w))
    vl = vel_l[:, y0:y0 + h, x0:x0 + w]
    d = np.maximum(np.abs(vl[-1] % L - ref["vel_index"][-1] % L), np.abs(vl[-1] // L - ref["vel_index"][-1] // L))
    ref_l = o.run(frames, crop=(y0, x0, h, w), vel_override=vl)
    werr = P.whitened_err(wh_l[:, y0:y0 + h, x0:x0 + w], ref_l["whitened"], frames, dz)
    print(f"[learned vs oracle] within one step {np.mean(d <= 1):.3f}, whitened on the learned field "
          f"{werr:.2e} x input RMS", flush=True)
    assert np.mean(d <= 1) >= 0.95
    assert werr <= P.WHITE_TOL_REL
    trained.close()
    untrained.close()
