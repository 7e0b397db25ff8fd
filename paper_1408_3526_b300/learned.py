"""Learned velocity estimator: network front end, training and evaluation.

The network (C ABI wh_mlp_*) maps each pixel's log-power spectrum (the
high-passed, Hann-windowed power normalised by its sum, input
(log2(P/sum P + 1e-6) + 10)/10, one value per mirror pair of bins since
P(-k) = P(k): 676 inputs at 15 x 15 x 6) to (vx, vy, confidence).  It is trained on velocities produced by the
plain autocorrelation search of this library, and in a stream's learned mode
replaces that search wherever its confidence reaches a threshold (0.8 by
default); every other pixel still runs the exact search.  All arithmetic runs
in libwhiten.so's kernels (tcgen05 GEMMs with fused epilogues, AdamW);
PyTorch only holds device buffers.
"""
from __future__ import annotations

import ctypes as C
import math
import time

import numpy as np

from . import _abi, scenes
from ._abi import check


def _torch():
    import torch
    return torch


class MLP:
    """n_in -> h1 -> h2 -> 3 network with BF16 weights and FP32 master copy."""

    def __init__(self, n_in=1350, h1=256, h2=128, n_out=3, seed=1, cuda_stream=None):
        torch = _torch()
        self.lib = _abi.load()
        self.n_in, self.h1, self.h2, self.n_out = n_in, h1, h2, n_out
        if cuda_stream is None:
            cuda_stream = torch.cuda.current_stream().cuda_stream
        elif hasattr(cuda_stream, "cuda_stream"):
            cuda_stream = cuda_stream.cuda_stream
        h = C.c_void_p()
        check(self.lib.wh_mlp_create(n_in, h1, h2, n_out, C.c_ulonglong(seed), C.c_void_p(int(cuda_stream)),
                                     C.byref(h)), "wh_mlp_create")
        self._m = h
        self.n_params = int(self.lib.wh_mlp_num_params(self._m))

    def close(self):
        if getattr(self, "_m", None):
            self.lib.wh_mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        check(self.lib.wh_mlp_get_params(self._m, C.c_void_p(out.ctypes.data), self.n_params), "get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.n_params
        check(self.lib.wh_mlp_set_params(self._m, C.c_void_p(p.ctypes.data), self.n_params), "set_params")

    def grads(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        check(self.lib.wh_mlp_get_grads(self._m, C.c_void_p(out.ctypes.data), self.n_params), "get_grads")
        return out

    def save(self, path):
        np.savez(path, params=self.params(), dims=np.array([self.n_in, self.h1, self.h2, self.n_out]))

    def load(self, path):
        d = np.load(path)
        assert tuple(d["dims"]) == (self.n_in, self.h1, self.h2, self.n_out)
        self.set_params(d["params"])

    def forward(self, x, out=None):
        """x: CUDA bf16 [n][ld] (ld % 8 == 0); returns CUDA float32 [n][3]."""
        torch = _torch()
        n, ld = x.shape
        if out is None:
            out = torch.empty((n, self.n_out), dtype=torch.float32, device="cuda")
        check(self.lib.wh_mlp_forward(self._m, C.c_void_p(x.data_ptr()), x.stride(0), n,
                                      C.c_void_p(out.data_ptr()), out.stride(0)), "wh_mlp_forward")
        return out

    def train_step(self, x, target, vstep, lr, weight_decay=0.0, apply=True, stats=True):
        st = (C.c_float * 4)() if stats else None
        check(self.lib.wh_mlp_train_step(self._m, C.c_void_p(x.data_ptr()), x.stride(0), x.shape[0],
                                         C.c_void_p(target.data_ptr()), float(vstep), float(lr),
                                         float(weight_decay), int(bool(apply)),
                                         st if st is not None else None), "wh_mlp_train_step")
        return list(st) if st is not None else None


def n_features(M, Mz, folded=True):
    """Network input width: all M*M*Mz bins, or one per mirror pair (P(-k) = P(k))."""
    nb = M * M * Mz
    return (nb + 2 - Mz % 2) // 2 if folded else nb


def fold_first_layer(W1, M, Mz):
    """Columns of a first layer over all bins ([h1][M*M*Mz], order [kz][ky][kx])
    summed over mirror pairs, in the folded input order: the bins k whose flat
    index is not larger than that of -k.  A network with the folded layer on
    the folded features computes exactly what the original computes on all bins."""
    W1 = np.asarray(W1)
    K, J = (M - 1) // 2, (Mz - 1) // 2
    cols = []
    for iz in range(Mz):
        for iy in range(M):
            for ix in range(M):
                kzm = -(iz - J)
                if kzm < -J:
                    kzm += Mz
                b = (iz * M + iy) * M + ix
                bm = ((kzm + J) * M + (2 * K - iy)) * M + (2 * K - ix)
                if b < bm:
                    cols.append(W1[:, b] + W1[:, bm])
                elif b == bm:
                    cols.append(W1[:, b])
    return np.stack(cols, axis=1)


def generate_training_data(n_scenes=300, frames=12, H=512, W=640, M=15, Mz=6, vmax=3.0, step=0.25,
                           samples=2_000_000, seed0=100, vlim=1.75, folded=True):
    """Scenes -> plain GPU path -> (features, labels) at uniformly sampled
    interior pixels of each scene's last frame.  Returns CUDA tensors
    X bf16 [samples][ld] and V float32 [samples][2].  folded: one feature per
    mirror pair of bins (wh_stream_set_features mode 2), else all bins."""
    torch = _torch()
    from .stream import WhitenStream
    per = int(math.ceil(samples / n_scenes))
    K = (M - 1) // 2
    xs, vs = [], []
    rng = np.random.default_rng(seed0)
    for frames_np, _ in scenes.training_scene_set(n_scenes, frames, H, W, seed0=seed0, vlim=vlim):
        fd = torch.from_numpy(frames_np).cuda()
        with WhitenStream(H, W, M, Mz, vmax, step) as s:
            check(s.lib.wh_stream_set_features(s._s, 2 if folded else 1), "set_features")
            for t in range(frames):
                s.push(fd[t])
            ld = C.c_int()
            check(s.lib.wh_read_features(s._s, None, 1, C.byref(ld)), "read_features")
            feat = torch.empty((H * W, ld.value), dtype=torch.bfloat16, device="cuda")
            check(s.lib.wh_read_features(s._s, C.c_void_p(feat.data_ptr()), 1, None), "read_features")
            vx, vy, _, _ = s.read_velocity(device=True)
        ys = rng.integers(K, H - K, per)
        xs_ = rng.integers(K, W - K, per)
        idx = torch.from_numpy((ys * W + xs_).astype(np.int64)).cuda()
        xs.append(feat[idx])
        vs.append(torch.stack([vx.reshape(-1)[idx], vy.reshape(-1)[idx]], 1))
    X = torch.cat(xs)[:samples].contiguous()
    V = torch.cat(vs)[:samples].contiguous()
    return X, V


def train(mlp: MLP, X, V, vstep=0.25, epochs=3, batch=8192, lr=1e-3, weight_decay=1e-4, seed=0, log=None):
    """Minibatch AdamW over (X, V); returns per-epoch mean statistics."""
    torch = _torch()
    n = X.shape[0] // batch * batch
    g = torch.Generator(device="cuda").manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], generator=g, device="cuda")[:n]
        acc = np.zeros(4)
        nb = 0
        for b0 in range(0, n, batch):
            sel = perm[b0:b0 + batch]
            st = mlp.train_step(X[sel].contiguous(), V[sel].contiguous(), vstep, lr, weight_decay,
                                stats=(b0 // batch) % 20 == 0)
            if st is not None:
                acc += st
                nb += 1
        hist.append((acc / max(nb, 1)).tolist())
        if log:
            log(f"epoch {ep}: loss {hist[-1][0]:.4f} mse {hist[-1][1]:.4f} bce {hist[-1][2]:.4f} "
                f"within-step {hist[-1][3]:.3f}")
    return hist


def detection_snr_db(E, scene, t_frame, radius=1.0, exclude_sigmas=5.0):
    """Detection SNR (dB) of one whitened frame: 20 log10 of the mean over
    targets of the peak |E| within `radius` px of the true position, over the
    standard deviation of E on pixels farther than exclude_sigmas x sigma_psf
    from every target."""
    H, W = E.shape
    py, px = np.mgrid[0:H, 0:W]
    far = np.ones((H, W), bool)
    peaks = []
    for (cx, cy), tg in zip(scene.target_positions(t_frame), scene.targets):
        d = np.hypot(px - cx, py - cy)
        near = d <= radius
        if near.any():
            peaks.append(np.max(np.abs(E[near])))
        far &= d > exclude_sigmas * tg["sigma"]
    if not peaks:
        return float("nan")
    sd = float(np.std(E[far]))
    return 20.0 * math.log10(np.mean(peaks) / max(sd, 1e-30))


def compare_on_sequence(net: MLP, sc, M=15, Mz=6, vmax=3.0, step=0.25, conf=0.8, warmup=12, snr_every=10,
                        modes=("plain", "learned")):
    """Run the plain and the learned mode on the same frames; returns timing
    (device ms per frame), velocity agreement with the plain search, share of
    pixels decided by the network, and the detection SNR of both.  ``modes``
    may restrict the run to one of them (no agreement figures then)."""
    torch = _torch()
    from .stream import WhitenStream
    T, H, W = sc.frames.shape
    L = int(round(2 * vmax / step)) + 1
    out = {}
    vel = {}
    for mode in modes:
        st = torch.cuda.Stream()
        snr = []
        with WhitenStream(H, W, M, Mz, vmax, step, cuda_stream=st) as s:
            if mode == "learned":
                check(s.lib.wh_stream_set_learned(s._s, net._m, float(conf)), "set_learned")
            buf = torch.empty((H, W), dtype=torch.float32, device="cuda")
            ms = 0.0
            agree = []
            for t in range(T):
                buf.copy_(torch.from_numpy(sc.frames[t]))
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                s.push(buf)
                e1.record(st)
                e1.synchronize()
                if t >= warmup:
                    ms += e0.elapsed_time(e1)
                    _, _, vi, _ = s.read_velocity(device=True)
                    if mode == "plain":
                        vel[t] = vi.clone()
                    elif t in vel:
                        p = vel[t]
                        d = torch.maximum((vi % L - p % L).abs(), (vi // L - p // L).abs())
                        agree.append((float((d == 0).float().mean()), float((d <= 1).float().mean())))
                    if (t - warmup) % snr_every == 0:
                        E, fi = s.read_whitened()
                        snr.append(detection_snr_db(E, sc, fi))
            fr, fb = C.c_longlong(), C.c_longlong()
            s.lib.wh_stream_learned_stats(s._s, C.byref(fr), C.byref(fb))
        n = T - warmup
        rec = {"ms_per_frame": ms / n, "mpix_per_s": H * W / (ms / n) / 1e3,
               "snr_db_mean": float(np.nanmean(snr)), "snr_frames": len(snr)}
        if mode == "learned":
            if agree:
                rec["velocity_identical_vs_plain"] = float(np.mean([a[0] for a in agree]))
                rec["velocity_within_one_step_vs_plain"] = float(np.mean([a[1] for a in agree]))
            rec["share_decided_by_network"] = 1.0 - fb.value / max(fr.value, 1) / (H * W)
        out[mode] = rec
    if "plain" in out and "learned" in out:
        out["speedup_learned_over_plain"] = out["plain"]["ms_per_frame"] / out["learned"]["ms_per_frame"]
        out["snr_difference_db"] = out["learned"]["snr_db_mean"] - out["plain"]["snr_db_mean"]
    return out


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="train and evaluate the learned velocity estimator")
    ap.add_argument("--train-scenes", type=int, default=300)
    ap.add_argument("--train-frames", type=int, default=12)
    ap.add_argument("--samples", type=int, default=2_000_000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--eval-frames", type=int, default=500)
    ap.add_argument("--eval-h", type=int, default=1024)
    ap.add_argument("--eval-w", type=int, default=1280)
    ap.add_argument("--conf", type=float, default=0.8)
    ap.add_argument("--ckpt", default=None, help="save the trained weights here")
    ap.add_argument("--load", default=None, help="skip training and load these weights")
    ap.add_argument("--modes", default="plain,learned", help="comma list of plain, learned")
    ap.add_argument("--warmup", type=int, default=12)
    ap.add_argument("--out", default=None)
    ap.add_argument("--all-bins", action="store_true",
                    help="input every M*M*Mz bin (1350) instead of one per mirror pair (676)")
    a = ap.parse_args(argv)
    folded = not a.all_bins
    net = MLP(n_features(15, 6, folded), 256, 128, 3, seed=1)
    if a.load:
        net.load(a.load)
        training = {"loaded": a.load}
    else:
        t0 = time.time()
        X, V = generate_training_data(n_scenes=a.train_scenes, frames=a.train_frames, samples=a.samples,
                                      folded=folded)
        t_data = time.time() - t0
        t0 = time.time()
        hist = train(net, X, V, epochs=a.epochs, lr=1e-3, log=print)
        _torch().cuda.synchronize()
        t_train = time.time() - t0
        del X, V
        training = {"samples": a.samples, "scenes": a.train_scenes, "epochs": a.epochs,
                    "final_loss": hist[-1][0], "final_within_step": hist[-1][3],
                    "data_seconds": t_data, "train_seconds": t_train}
    if a.ckpt:
        net.save(a.ckpt)
    sc = scenes.config1_scene(T=a.eval_frames, H=a.eval_h, W=a.eval_w, seed=4)
    rep = compare_on_sequence(net, sc, conf=a.conf, warmup=min(a.warmup, a.eval_frames - 1),
                              modes=tuple(m for m in a.modes.split(",") if m))
    rep["training"] = training
    rep["eval"] = {"frames": a.eval_frames, "size": [a.eval_h, a.eval_w], "window": 15, "order": 6,
                   "grid": "+-3 step 0.25", "confidence_threshold": a.conf,
                   "network_inputs": net.n_in, "inputs": "one per mirror pair" if folded else "all bins"}
    print(json.dumps(rep))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
