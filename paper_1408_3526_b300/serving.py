"""Multi-stream serving front end (C ABI wh_server_*) and the mixed-stream
load run: many sensor streams of different sizes and parameters, Poisson
frame arrivals, state resident on the device, admission by a memory budget,
p50/p99 latency and served vs offered throughput.

    python -m paper_1408_3526_b300.serving [--streams 64] [--seconds 3] [--out report.json]
"""
from __future__ import annotations

import ctypes as C
import json
import time

import numpy as np

from . import _abi, scenes
from ._abi import check

SIZES = [(128, 128), (256, 320), (512, 640), (1024, 1280)]


class Server:
    def __init__(self, budget_bytes=150e9, max_inflight=16, queue_limit=4, n_cuda_streams=8, keep_results=False):
        self.lib = _abi.load()
        h = C.c_void_p()
        check(self.lib.wh_server_create(float(budget_bytes), max_inflight, queue_limit, n_cuda_streams,
                                        int(keep_results), C.byref(h)), "wh_server_create")
        self._s = h
        self.shapes = {}

    def open(self, h, w, window, order, vmax, step, precision=0, pipeline=False):
        p = _abi.wh_params()
        check(self.lib.wh_default_params(window, order, C.byref(p)), "defaults")
        p.precision = precision
        p.pipeline = int(bool(pipeline))
        sid = C.c_int()
        rc = self.lib.wh_server_open(self._s, h, w, window, order, _abi.wh_vgrid(vmax, step), C.byref(p),
                                     C.byref(sid))
        if rc == _abi.WH_EADMIT:
            return None
        check(rc, "wh_server_open")
        self.shapes[sid.value] = (h, w)
        return sid.value

    def now(self):
        return float(self.lib.wh_server_now(self._s))

    def submit(self, sid, frame, arrival):
        frame = np.ascontiguousarray(frame, np.float32)
        rid = C.c_longlong()
        rc = self.lib.wh_server_submit(self._s, sid, C.c_void_p(frame.ctypes.data), float(arrival), C.byref(rid))
        if rc == _abi.WH_EADMIT:
            return None
        check(rc, "wh_server_submit")
        return rid.value

    def wait(self, rid, sid=None):
        lat = C.c_double()
        out = None
        if sid is not None:
            out = np.empty(self.shapes[sid], np.float32)
        check(self.lib.wh_server_wait(self._s, rid, C.c_void_p(out.ctypes.data) if out is not None else None,
                                      C.byref(lat)), "wh_server_wait")
        return out, lat.value

    def drain(self):
        check(self.lib.wh_server_drain(self._s), "wh_server_drain")

    def stats(self):
        p50, p99, mps = C.c_double(), C.c_double(), C.c_double()
        sv, sh, sb = C.c_longlong(), C.c_longlong(), C.c_longlong()
        check(self.lib.wh_server_stats(self._s, C.byref(p50), C.byref(p99), C.byref(mps), C.byref(sv),
                                       C.byref(sh), C.byref(sb)), "wh_server_stats")
        return {"p50_ms": p50.value, "p99_ms": p99.value, "served_mpix_per_s": mps.value,
                "served": sv.value, "shed": sh.value, "submitted": sb.value}

    def close_stream(self, sid):
        check(self.lib.wh_server_close(self._s, sid), "wh_server_close")

    def close(self):
        if getattr(self, "_s", None):
            self.lib.wh_server_destroy(self._s)
            self._s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def run_mixed_load(n_streams=64, seconds=3.0, seed=1000, budget=150e9, frames_per_stream=4,
                   max_inflight=16, queue_limit=4, n_cuda=8):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n_streams):
        h, w = SIZES[int(rng.integers(len(SIZES)))]
        M = int(rng.choice([9, 15]))
        Mz = int(rng.integers(4, 7))
        rate = float(rng.uniform(30, 200))
        specs.append((h, w, M, Mz, rate))
    # a few frames per stream from the config-1 generator, per-stream seeds, cycled
    frames = {}
    texture_cache = {}
    for i, (h, w, M, Mz, rate) in enumerate(specs):
        sc = scenes.config1_scene(T=frames_per_stream, H=h, W=w, seed=1000 + i, tex_size=1024)
        frames[i] = sc.frames
    with Server(budget, max_inflight, queue_limit, n_cuda) as srv:
        sid = {}
        refused = 0
        for i, (h, w, M, Mz, rate) in enumerate(specs):
            s = srv.open(h, w, M, Mz, 2.0 if M == 9 else 3.0, 0.25)
            if s is None:
                refused += 1
            else:
                sid[i] = s
        # Poisson arrivals
        events = []
        for i, (h, w, M, Mz, rate) in enumerate(specs):
            if i not in sid:
                continue
            t = rng.exponential(1.0 / rate)
            k = 0
            while t < seconds:
                events.append((t, i, k))
                k += 1
                t += rng.exponential(1.0 / rate)
        events.sort()
        offered_px = sum(specs[i][0] * specs[i][1] for _, i, _ in events)
        t0 = srv.now() + 0.2
        late = 0.0
        for (t, i, k) in events:
            target = t0 + t
            now = srv.now()
            if now < target:
                time.sleep(target - now)
            else:
                late = max(late, now - target)
            srv.submit(sid[i], frames[i][k % frames_per_stream], target)
        srv.drain()
        st = srv.stats()
    st.update({"streams": n_streams, "streams_refused_by_budget": refused, "seconds": seconds,
               "offered_frames": len(events), "offered_mpix_per_s": offered_px / seconds / 1e6,
               "max_inflight": max_inflight, "queue_limit": queue_limit, "cuda_streams": n_cuda,
               "budget_gb": budget / 1e9, "driver_max_lateness_s": late,
               "mix": {f"{h}x{w}": sum(1 for s in specs if s[:2] == (h, w)) for (h, w) in SIZES}})
    return st


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--streams", type=int, default=64)
    ap.add_argument("--seconds", type=float, default=3.0)
    ap.add_argument("--max-inflight", type=int, default=16)
    ap.add_argument("--queue-limit", type=int, default=4)
    ap.add_argument("--cuda-streams", type=int, default=8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    rep = run_mixed_load(a.streams, a.seconds, max_inflight=a.max_inflight, queue_limit=a.queue_limit,
                         n_cuda=a.cuda_streams)
    print(json.dumps(rep))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(rep, f, indent=1)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
