"""Python front end of the whitening stream (thin layer over the C ABI).

PyTorch supplies device memory and CUDA streams; all computation runs in
libwhiten.so's kernels.  Frames may be CUDA tensors (passed in place) or
host arrays (copied by the library on its stream).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import _abi
from ._abi import check


def _torch():
    import torch
    return torch


def _ptr_of(x):
    """(pointer, is_device) of a contiguous float32/int32 tensor or ndarray."""
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data, 0
    torch = _torch()
    if isinstance(x, torch.Tensor):
        assert x.is_contiguous()
        return x.data_ptr(), int(x.is_cuda)
    raise TypeError(f"unsupported buffer type {type(x)}")


class WhitenStream:
    """One sensor stream: recursive state resident on the GPU.

    Parameters follow ``wh_create_stream``: frame size, spatial window M
    (odd), temporal order Mz, velocity grid (vmax, step), and the optional
    band B, output delay m'_z, smoother pole alpha, precision mode, and
    ``pipeline`` (overlap consecutive frames on two internal CUDA streams;
    identical results).
    """

    def __init__(self, h: int, w: int, window: int, temporal_order: int, vmax: float,
                 step: float, band: int | None = None, delay_z: int | None = None,
                 alpha: float | None = None, precision: int = 0, debug_dump: bool = False,
                 cuda_stream=None, pipeline: bool = False):
        self.lib = _abi.load()
        self.h, self.w, self.M, self.Mz = int(h), int(w), int(window), int(temporal_order)
        p = _abi.wh_params()
        check(self.lib.wh_default_params(self.M, self.Mz, C.byref(p)), "wh_default_params")
        if band is not None:
            p.band = int(band)
        if delay_z is not None:
            p.delay_z = int(delay_z)
        if alpha is not None:
            p.alpha = float(alpha)
        p.precision = int(precision)
        p.debug_dump = int(bool(debug_dump))
        p.pipeline = int(bool(pipeline))
        if cuda_stream is None:
            torch = _torch()
            cuda_stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        elif hasattr(cuda_stream, "cuda_stream"):
            cuda_stream = cuda_stream.cuda_stream
        self.cuda_stream = int(cuda_stream)
        h_out = C.c_void_p()
        check(self.lib.wh_create_stream(self.h, self.w, self.M, self.Mz,
                                        _abi.wh_vgrid(float(vmax), float(step)), C.byref(p),
                                        C.c_void_p(self.cuda_stream), C.byref(h_out)),
              "wh_create_stream")
        self._s = h_out
        L, dz, B, n = C.c_int(), C.c_int(), C.c_int(), C.c_longlong()
        check(self.lib.wh_stream_info(self._s, C.byref(L), C.byref(dz), C.byref(B), C.byref(n)),
              "wh_stream_info")
        self.L, self.delay_z, self.band = L.value, dz.value, B.value
        self.vmax, self.step = float(vmax), float(step)

    # -- lifecycle -----------------------------------------------------------------
    def close(self):
        if getattr(self, "_s", None):
            self.lib.wh_destroy_stream(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def reset(self):
        check(self.lib.wh_reset_stream(self._s), "wh_reset_stream")

    @property
    def frames_pushed(self) -> int:
        n = C.c_longlong()
        check(self.lib.wh_stream_info(self._s, None, None, None, C.byref(n)), "wh_stream_info")
        return n.value

    # -- per frame --------------------------------------------------------------------
    def push(self, frame):
        ptr, dev = _ptr_of(frame)
        check(self.lib.wh_push_frame(self._s, C.c_void_p(ptr), dev), "wh_push_frame")

    def push_async(self, frame, whitened=None, vx=None, vy=None) -> int:
        """Pipelined push from page-locked host memory (wh_push_frame_async).

        frame, whitened, vx, vy: pinned CPU torch tensors of shape (H, W)
        (outputs may be None).  Returns the frame index; the outputs are
        complete after wait_frame(index) or sync()."""
        def p(t):
            if t is None:
                return None
            if not (t.is_pinned() and t.is_contiguous()):
                raise ValueError("asynchronous push needs contiguous pinned host tensors")
            return C.c_void_p(t.data_ptr())
        idx = C.c_longlong()
        check(self.lib.wh_push_frame_async(self._s, p(frame), p(whitened), p(vx), p(vy), C.byref(idx)),
              "wh_push_frame_async")
        return int(idx.value)

    DETECTION_DTYPE = np.dtype([("y", np.int32), ("x", np.int32), ("value", np.float32),
                                ("vx", np.float32), ("vy", np.float32)])

    def detect(self, k_sigma: float = 5.0, max_det: int = 4096):
        """Threshold detector on the latest whitened frame (wh_detect).

        Returns (detections, n_total, sigma, frame_index); detections is a
        structured array (y, x, value, vx, vy) in raster order, at most max_det
        long, n_total the number of pixels above k_sigma * sigma."""
        out = np.zeros(max(max_det, 0), dtype=self.DETECTION_DTYPE)
        n, sig, idx = C.c_int(), C.c_float(), C.c_longlong()
        check(self.lib.wh_detect(self._s, C.c_float(k_sigma), int(max_det),
                                 C.c_void_p(out.ctypes.data if max_det > 0 else 0), C.byref(n),
                                 C.byref(sig), 0, C.byref(idx)), "wh_detect")
        return out[:min(n.value, max_det)], n.value, sig.value, idx.value

    def wait_frame(self, index: int) -> None:
        check(self.lib.wh_stream_query_frame(self._s, C.c_longlong(index), 1), "wh_stream_query_frame")

    def sync(self) -> None:
        check(self.lib.wh_stream_sync(self._s), "wh_stream_sync")

    def join(self) -> None:
        """Order the stream's CUDA stream after all enqueued work (no host wait)."""
        check(self.lib.wh_stream_join(self._s), "wh_stream_join")

    def _alloc(self, shape, dtype, device):
        if device:
            torch = _torch()
            tdt = {np.float32: torch.float32, np.int32: torch.int32,
                   np.complex64: torch.complex64}[dtype]
            return torch.empty(shape, dtype=tdt, device="cuda")
        return np.empty(shape, dtype)

    def read_whitened(self, out=None, device: bool = False):
        """Whitened frame t - m'_z (returns (array, frame_index))."""
        if out is None:
            out = self._alloc((self.h, self.w), np.float32, device)
        ptr, dev = _ptr_of(out)
        idx = C.c_longlong()
        check(self.lib.wh_read_whitened(self._s, C.c_void_p(ptr), dev, C.byref(idx)),
              "wh_read_whitened")
        return out, idx.value

    def read_velocity(self, device: bool = False):
        """(vx, vy, vidx, frame_index) of the last frame."""
        vx = self._alloc((self.h, self.w), np.float32, device)
        vy = self._alloc((self.h, self.w), np.float32, device)
        vi = self._alloc((self.h, self.w), np.int32, device)
        (px, dev), (py, _), (pi, _) = _ptr_of(vx), _ptr_of(vy), _ptr_of(vi)
        idx = C.c_longlong()
        check(self.lib.wh_read_velocity(self._s, C.c_void_p(px), C.c_void_p(py), C.c_void_p(pi),
                                        dev, C.byref(idx)), "wh_read_velocity")
        return vx, vy, vi, idx.value

    def read_spectrum(self, kind: int = _abi.WH_SPEC_RAW):
        """[h][w][Mz][M][M] complex64 (RAW/WINDOWED) or float32 (POWER), on the host."""
        shape = (self.h, self.w, self.Mz, self.M, self.M)
        out = np.empty(shape, np.float32 if kind == _abi.WH_SPEC_POWER else np.complex64)
        check(self.lib.wh_read_spectrum(self._s, int(kind), C.c_void_p(out.ctypes.data), 0),
              "wh_read_spectrum")
        return out

    def read_autocorr(self):
        """Smoothed autocorrelation R' on the grid, [h][w][L][L] float32 (host)."""
        out = np.empty((self.h, self.w, self.L, self.L), np.float32)
        check(self.lib.wh_read_autocorr(self._s, C.c_void_p(out.ctypes.data), 0),
              "wh_read_autocorr")
        return out

    def output_pointers(self):
        wp, xp, yp, ip = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
        check(self.lib.wh_output_pointers(self._s, C.byref(wp), C.byref(xp), C.byref(yp),
                                          C.byref(ip)), "wh_output_pointers")
        return wp.value, xp.value, yp.value, ip.value

    def profile(self, on: bool = True):
        check(self.lib.wh_profile_enable(self._s, int(bool(on))), "wh_profile_enable")

    def profile_read(self, reset: bool = True):
        """(ms per kernel [spectrum, autocorr, pef], timed frames)."""
        ms = (C.c_double * 3)()
        n = (C.c_longlong * 3)()
        check(self.lib.wh_profile_read(self._s, ms, n, int(bool(reset))), "wh_profile_read")
        return list(ms), int(n[0])

    def search_counts(self):
        """(listed, whole_grid) pixel-frames of the default tensor-core search
        since creation (wh_stream_search_counts)."""
        a, b = C.c_longlong(), C.c_longlong()
        check(self.lib.wh_stream_search_counts(self._s, C.byref(a), C.byref(b)), "wh_stream_search_counts")
        return int(a.value), int(b.value)

    def grid_values(self) -> np.ndarray:
        return -self.vmax + self.step * np.arange(self.L)


def kernel_launch_count() -> int:
    return int(_abi.load().wh_kernel_launch_count())
