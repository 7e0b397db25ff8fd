#!/usr/bin/env python3
"""Benchmark: whitened Mpixel/s on the 512 x 640 stream (15 x 15 window,
temporal order 6, velocity grid +-3 px/frame in 0.25 steps).

One step = one frame through the whole per-pixel path (observer + spatial
SDFT + high-pass + Hann + power + smoothing, autocorrelation search, PEF).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {b300,reference}]

Prints ONE JSON line on rank 0.  Multi-GPU: one process per GPU (torchrun);
every rank runs its own independent 512 x 640 sensor stream (the path shards
by stream with no data exchange), so scaling is weak and the value is the
sum over ranks.  ``--impl reference`` times the FP64 CPU oracle (the only
other implementation of the method) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W, M, MZ, VMAX, VSTEP = 512, 640, 15, 6, 3.0, 0.25
NFRAMES_RESIDENT = 48
WORKLOAD = "512x640 IR stream, 15x15 window, temporal order 6, grid +-3 step 0.25"

# algorithmic bytes per pixel-frame (FP32 accounting): frame in 4, whitened
# out 4, velocity out 8, observer state read+write 2*4*Mz, smoothed
# autocorrelation state read+write 2*4*min(L^2, U), U = (M^2 Mz + 2)/2
L_GRID = int(round(2 * VMAX / VSTEP)) + 1
U_BINS = (M * M * MZ + 2) // 2
BYTES_PER_PX = 4 + 4 + 8 + 2 * 4 * MZ + 2 * 4 * min(L_GRID * L_GRID, U_BINS)
# the same bytes by the kernel that moves them: the spectrum kernel reads the
# frame, updates the observer state and the smoothed state; the search writes
# the velocity; the PEF writes the whitened pixel
KERNEL_BYTES_PER_PX = {
    "spectrum": 4 + 2 * 4 * MZ + 2 * 4 * min(L_GRID * L_GRID, U_BINS),
    "autocorr_argmax": 8,
    "pef": 4,
}
assert sum(KERNEL_BYTES_PER_PX.values()) == BYTES_PER_PX
# ncu summaries with the measured DRAM traffic of one launch at this workload,
# and the kernel sources they were taken from (the figure is reported only
# while those sources are unchanged)
PROFILE_OF = {
    "spectrum": ("profiles/spectrum_512x640_m15_mz6.md", ["k_spectrum.cu", "common.cuh"]),
    "autocorr_argmax": ("profiles/autocorr_512x640_m15.md", ["k_autocorr.cu", "ac_common.cuh", "common.cuh"]),
    "pef": ("profiles/pef_512x640_m15_mz6.md", ["k_pef.cu", "common.cuh"]),
}
# the search kernel's summary for the whole-contraction tensor-core engine (--precision 128)
PROFILE_OF_TCD = ("profiles/autocorr_tcd_512x640_m15.md",
                  ["k_autocorr_tcd.cu", "ac_common.cuh", "common.cuh", "tc_ptx.cuh"])
# the search kernel's summary when the tensor-core separable engine runs (--precision 32)
PROFILE_OF_TCSEP = ("profiles/autocorr_tcsep_512x640_m15.md",
                    ["k_autocorr_tcsep.cu", "ac_common.cuh", "common.cuh", "tc_ptx.cuh"])


def kernel_source_sha256(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_1408_3526_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel):
    """DRAM bytes per launch from the kernel's ncu summary, or None when the
    summary is missing or the kernel's sources changed since it was taken."""
    md, srcs = PROFILE_OF[kernel]
    try:
        with open(os.path.join(ROOT, md)) as f:
            text = f.read()
    except OSError:
        return None
    m1 = re.search(r"^traffic_bytes_per_launch:\s*(\d+)", text, re.M)
    m2 = re.search(r"^kernel_source_sha256:\s*([0-9a-f]{64})", text, re.M)
    if not (m1 and m2) or m2.group(1) != kernel_source_sha256(srcs):
        return None
    return int(m1.group(1))


def measured_limiter(kernel):
    """Issue and DRAM utilisation of the kernel from its ncu summary (same
    validity rule as the traffic), or None."""
    if measured_traffic(kernel) is None:
        return None
    md, _ = PROFILE_OF[kernel]
    with open(os.path.join(ROOT, md)) as f:
        text = f.read()
    m1 = re.search(r"^\| smsp__issue_active \(% of active\) \| ([0-9.]+) \|", text, re.M)
    m2 = re.search(r"^\| gpu__dram_throughput \(% of peak\) \| ([0-9.]+) \|", text, re.M)
    if not (m1 and m2):
        return None
    return {"issue_active_pct": float(m1.group(1)), "dram_throughput_pct": float(m2.group(1)),
            "source": md}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device="cpu"):
    """Largest value of x over the ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def engine_name(precision):
    """The autocorrelation search (and spectrum form) a precision value selects."""
    if precision & 16:
        name = "tensor-core shortlist (F16) + exact FP32 re-rank"
    elif precision & 3:
        name = "tensor-core contraction alone (%s)" % ("BF16" if precision & 2 else "F16")
    elif precision & 32:
        name = "FP32-exact separable search, first stage on tensor cores (TF32 row bounds)"
    elif precision & 128:
        name = ("FP32-exact argmax: whole contraction on tcgen05 tensor cores (F16, F32 accumulation) "
                "with a rigorous error window, near ties re-evaluated in FP32")
    else:
        name = "FP32-exact separable search on CUDA cores"
    if precision & 64:
        name += "; spatial sums in FP64"
    return name


def whole_job_mpx_per_s(world, frames_per_rank, seconds):
    """Pixels processed by all ranks divided by the slowest rank's time."""
    return world * H * W * frames_per_rank / seconds / 1e6


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout_s=3.0):
        """Block until the sampler has printed its first line (or timeout)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout_s:
            time.sleep(0.02)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_frames(seed=2):
    from paper_1408_3526_b300 import scenes
    sc = scenes.config2_scene(T=NFRAMES_RESIDENT, H=H, W=W, seed=seed)
    return sc.frames


def cpu_baseline(frames, seconds_target=12.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    o = oracle.Oracle(M, MZ, VMAX, VSTEP)
    cores = os.cpu_count() or 1
    # a crop of the same scene: every pixel of the crop runs the full method
    h = w = 48
    T = 8
    crop = (232, 296, h, w)
    o.run(frames[:T], crop=crop, nthreads=cores)          # untimed: thread pool and caches
    reps = 0
    t0 = time.perf_counter()
    while True:                                            # whole repetitions, ~seconds_target in all
        o.run(frames[:T], crop=crop, nthreads=cores)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= seconds_target or reps >= 1000:
            break
    px = h * w * T * reps
    return {"value": round(px / dt / 1e6, 6), "unit": "Mpixel/s", "cores": cores, "kind": "oracle",
            "sample": f"{h}x{w} crop x {T} frames x {reps} reps of the 512x640 workload "
                      f"({dt:.1f} s, FP64, OpenMP over rows)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    frames = make_frames()
    o = oracle.Oracle(M, MZ, VMAX, VSTEP)
    cores = os.cpu_count() or 1
    # per-step sample: a fixed 24x32 crop (the oracle also computes its (M - 1)-pixel
    # halo, so the crop is not shrunk, which would bias the rate low) over the most
    # frames, of 6, whose K + W steps fit in about 90 s; every frame costs the same
    h, w = 24, 32
    crop = (240, 300, h, w)
    t0 = time.perf_counter()
    o.run(frames[:6], crop=crop, nthreads=cores)
    t_frame = (time.perf_counter() - t0) / 6
    T = 1
    for cand in (6, 4, 3, 2):
        if t_frame * cand * (args.steps + args.warmup) <= 90.0:
            T = cand
            break

    def step():
        o.run(frames[:T], crop=crop, nthreads=cores)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    px = h * w * T * args.steps
    val = px / dt / 1e6
    line = {"metric": "whitened Mpixel/s (512x640 stream)", "value": round(val, 6),
            "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": f"{h}x{w} crop x {T} frames per step"},
            "cpu_baseline": {"value": round(val, 6), "unit": "Mpixel/s", "cores": cores,
                             "kind": "oracle", "sample": f"{h}x{w} crop x {T} frames per step"},
            "e2e": {"value": round(val, 6), "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="duration of the oracle's CPU-baseline sample")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--profile-steps", type=int, default=20,
                    help="frames of the serial pass that times each kernel alone (roofline)")
    ap.add_argument("--no-tc-engine", action="store_true",
                    help="skip the secondary measurement of the whole-contraction tensor-core search "
                         "(--precision 128) on the same workload")
    ap.add_argument("--no-pipeline", action="store_true",
                    help="serial stream (no overlap of consecutive frames)")
    ap.add_argument("--precision", type=int, default=0,
                    help="wh_params.precision (0: FP32-exact separable search on CUDA cores; 16: "
                         "tensor-core shortlist + exact re-rank; 32: separable search with its first "
                         "stage on tensor cores; 128: FP32-exact argmax with the whole contraction on "
                         "tensor cores)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if (args.precision & 32) and not (args.precision & (16 | 3)):
        PROFILE_OF["autocorr_argmax"] = PROFILE_OF_TCSEP
    elif (args.precision & 128) and not (args.precision & (8 | 16 | 32 | 3)):
        PROFILE_OF["autocorr_argmax"] = PROFILE_OF_TCD

    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1408_3526_b300.stream import WhitenStream, kernel_launch_count
    frames_h = make_frames(seed=2 + rank)
    frames_d = torch.from_numpy(frames_h).cuda()
    stream = torch.cuda.Stream()
    pipeline = not args.no_pipeline
    s = WhitenStream(H, W, M, MZ, VMAX, VSTEP, cuda_stream=stream, precision=args.precision,
                     pipeline=pipeline)
    # warm-up (state evolves; the work per frame is data-independent)
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            s.push(frames_d[i % NFRAMES_RESIDENT])
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    n0 = kernel_launch_count()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        s.push(frames_d[(args.warmup + i) % NFRAMES_RESIDENT])
    s.join()                       # the caller's stream follows the pipeline's internal streams
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = kernel_launch_count() - n0
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, world, "cuda")
    # per-kernel durations for the roofline: the same kernels timed alone (a
    # serial stream, CUDA events around each kernel, same frames)
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, cuda_stream=stream, precision=args.precision) as sk:
        with torch.cuda.stream(stream):
            for i in range(3):
                sk.push(frames_d[i % NFRAMES_RESIDENT])
        torch.cuda.synchronize()
        sk.profile(True)
        sk.profile_read(reset=True)
        with torch.cuda.stream(stream):
            for i in range(args.profile_steps):
                sk.push(frames_d[(3 + i) % NFRAMES_RESIDENT])
        torch.cuda.synchronize()
        kms, nprof = sk.profile_read(reset=True)
    value = whole_job_mpx_per_s(world, args.steps, ms_max * 1e-3)

    # the same step with the whole contraction of Eq. (10) on tcgen05 tensor cores
    # (exact, identical velocities; slower than the default CUDA-core search)
    tc_engine = None
    if not args.no_tc_engine and args.precision == 0:
        nt = min(args.steps, 50)
        with WhitenStream(H, W, M, MZ, VMAX, VSTEP, cuda_stream=stream, precision=128,
                          pipeline=pipeline) as st:
            with torch.cuda.stream(stream):
                for i in range(args.warmup):
                    st.push(frames_d[i % NFRAMES_RESIDENT])
            st.join()
            torch.cuda.synchronize()
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for i in range(nt):
                st.push(frames_d[(args.warmup + i) % NFRAMES_RESIDENT])
            st.join()
            f1.record(stream)
            torch.cuda.synchronize()
            barrier()
            tms = max_over_ranks(f0.elapsed_time(f1), world, "cuda")
            listed, whole = st.search_counts()
        with WhitenStream(H, W, M, MZ, VMAX, VSTEP, cuda_stream=stream, precision=128) as sk:
            with torch.cuda.stream(stream):
                for i in range(3):
                    sk.push(frames_d[i % NFRAMES_RESIDENT])
            torch.cuda.synchronize()
            sk.profile(True)
            sk.profile_read(reset=True)
            with torch.cuda.stream(stream):
                for i in range(args.profile_steps):
                    sk.push(frames_d[(3 + i) % NFRAMES_RESIDENT])
            torch.cuda.synchronize()
            tkms, tn = sk.profile_read(reset=True)
        frames_seen = args.warmup + nt
        tc_engine = {"engine": engine_name(128), "precision": 128,
                     "value": round(whole_job_mpx_per_s(world, nt, tms * 1e-3), 3), "unit": "Mpixel/s",
                     "steps": nt, "ms_per_step": round(tms / nt, 5),
                     "search_ms": round(tkms[1] / max(tn, 1), 5),
                     "pixel_frames_exact_step": round((listed + whole) / (frames_seen * H * W), 4),
                     "profile": PROFILE_OF_TCD[0]}

    # end to end through the C ABI: pinned host frame in, whitened + velocity out
    pin_in = torch.from_numpy(frames_h[:8].copy()).pin_memory()
    out_w = torch.empty((H, W), dtype=torch.float32).pin_memory()
    out_x = torch.empty((H, W), dtype=torch.float32).pin_memory()
    out_y = torch.empty((H, W), dtype=torch.float32).pin_memory()
    import ctypes as C
    lib = s.lib
    idx = C.c_longlong()
    # two sets of pinned outputs; the pipelined push copies each frame in, runs
    # the path and copies whitened + velocity out, overlapping the copies of one
    # frame with the kernels of the next; the timed region ends when the last
    # frame's outputs are on the host
    outs = [(out_w, out_x, out_y)] + [tuple(torch.empty((H, W), dtype=torch.float32).pin_memory()
                                            for _ in range(3))]
    s.sync()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.e2e_steps):
        o = outs[i & 1]
        rc = lib.wh_push_frame_async(s._s, C.c_void_p(pin_in[i % 8].data_ptr()), C.c_void_p(o[0].data_ptr()),
                                     C.c_void_p(o[1].data_ptr()), C.c_void_p(o[2].data_ptr()), C.byref(idx))
        assert rc == 0
    assert lib.wh_stream_sync(s._s) == 0
    e2e_s = time.perf_counter() - t0
    e2e_val = whole_job_mpx_per_s(world, args.e2e_steps, max_over_ranks(e2e_s, world, "cuda"))
    # the clock sampler ran through the timed region, the per-kernel pass and the
    # end-to-end pass (the same kernels back to back), so a short timed region
    # still gets a clock record under the same load
    clk = clocks.stop()
    clk["window"] = ("timed region + per-kernel serial pass + tensor-core search pass + end-to-end pass"
                     if tc_engine is not None else "timed region + per-kernel serial pass + end-to-end pass")

    if rank == 0:
        hbm, src = peaks()
        names = ["spectrum", "autocorr_argmax", "pef"]
        per = [k / max(nprof, 1) for k in kms]
        dom = int(np.argmax(per))
        # roofline of the whole path against HBM (all three kernels in one step)
        step_ms = ms_max / args.steps
        achieved_path = BYTES_PER_PX * H * W / (step_ms * 1e-3) / 1e9
        achieved_dom = KERNEL_BYTES_PER_PX[names[dom]] * H * W / (per[dom] * 1e-3) / 1e9
        line = {
            "metric": "whitened Mpixel/s (512x640 stream)",
            "value": round(value, 3), "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_resident": NFRAMES_RESIDENT,
                       "l2": "inputs larger than L2 (smoothed state 299 MB per buffer, two "
                             "buffers with the frame pipeline)",
                       "parallelism": f"{world} independent streams" if world > 1 else "1 stream",
                       "bytes_per_px_algorithmic": BYTES_PER_PX,
                       "frame_pipeline": pipeline,
                       "engine": engine_name(0)},
            "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": round(achieved_dom, 1),
                         "peak": hbm, "unit": "GB/s", "frac": round(achieved_dom / hbm, 4),
                         "traffic": measured_traffic(names[dom]), "peak_source": src,
                         "limiter": measured_limiter(names[dom]),
                         "bytes_per_launch_algorithmic": KERNEL_BYTES_PER_PX[names[dom]] * H * W,
                         "path_achieved": round(achieved_path, 1),
                         "path_frac": round(achieved_path / hbm, 4),
                         "kernel_ms": {n: round(p, 5) for n, p in zip(names, per)},
                         "kernel_timing": "each kernel alone: serial stream, CUDA events around every kernel"},
            "e2e": {"value": round(e2e_val, 3), "unit": "Mpixel/s",
                    "h2d_bytes_per_step": 4 * H * W, "d2h_bytes_per_step": 12 * H * W},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        line["config"]["engine"] = engine_name(args.precision)
        if tc_engine is not None:
            line["tensor_core_search"] = tc_engine
        if args.precision & 16:
            import ctypes as C
            fb = C.c_longlong()
            s.lib.wh_stream_stats(s._s, C.byref(fb))
            line["config"]["full_grid_fallback_pixel_frames"] = int(fb.value)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(frames_h, args.cpu_seconds)
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
