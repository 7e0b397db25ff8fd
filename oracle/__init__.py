"""FP64 CPU oracle of the recursive clutter-whitening preprocessor.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the
benchmark's CPU-baseline / reference leg are the only callers.  The product
path never imports this package and shares no code with it.

Plain C (``whiten_oracle.c``) built with gcc, no fast-math and no FMA
contraction, OpenMP over rows (the paper's Sec. 5 parallelises its C++ code
over image rows).  Every function follows the paper's steps in order; see the
C source header for the readings taken where the paper is silent.

Pins: every oracle function is checked in ``tests/test_oracle_pins.py``
against brute force or closed forms (direct windowed DFT, deadbeat
convergence, Dirichlet partition of unity, sample-domain FIR of Eq. (1)-(2),
PEF null on translating band-limited textures, autocorrelation of the
windowed block, known-shift peak, conjugate symmetries).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "whiten_oracle.c")
_LIB = os.path.join(_HERE, "_whiten_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (gcc, OpenMP, strict FP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-std=c11", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            lib.orc_dirichlet.restype = C.c_double
            lib.orc_dirichlet.argtypes = [C.c_int, C.c_double]
            lib.orc_observer_run.restype = None
            lib.orc_observer_run.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                             _dp, _dp]
            lib.orc_pef_design.restype = None
            lib.orc_pef_design.argtypes = [C.c_int] * 6 + [C.c_double, C.c_double, _dp, _dp]
            lib.orc_create.restype = C.c_void_p
            lib.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_double, C.c_double, C.c_int]
            lib.orc_destroy.restype = None
            lib.orc_destroy.argtypes = [C.c_void_p]
            lib.orc_grid_len.restype = C.c_int
            lib.orc_grid_len.argtypes = [C.c_void_p]
            lib.orc_run.restype = C.c_int
            lib.orc_run.argtypes = [C.c_void_p, _fp, C.c_int, C.c_int, C.c_int,
                                    C.c_int, C.c_int, C.c_int, C.c_int,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
def default_band(M: int) -> int:
    """PEF half-bandwidth B: the paper's cutoff B/M = 1/3 (B = 3 at M = 9)."""
    return max(1, int(round(M / 3.0)))


def default_delay(Mz: int) -> int:
    """Output delay m'_z = floor((Mz - 1)/2) (2 frames for the paper's Mz = 5)."""
    return (Mz - 1) // 2


def dirichlet(W: int, w) -> np.ndarray:
    """Eq. (3), D_W(w) = sin(pi W w)/(W sin(pi w)), limit value at integers."""
    lib = _load()
    w = np.asarray(w, np.float64)
    return np.vectorize(lambda x: lib.orc_dirichlet(int(W), float(x)))(w)


def observer_run(u: np.ndarray, Mz: int, s0: np.ndarray | None = None) -> np.ndarray:
    """Deadbeat observer over the complex sequence u; returns a-posteriori
    states [n][Mz] (bins kz = -((Mz-1)//2) .. Mz//2)."""
    lib = _load()
    u = np.ascontiguousarray(u, np.complex128)
    n = u.shape[0]
    are = np.zeros(n * Mz)
    aim = np.zeros(n * Mz)
    if s0 is not None:
        s0 = np.ascontiguousarray(s0, np.complex128)
        s0r, s0i = np.ascontiguousarray(s0.real), np.ascontiguousarray(s0.imag)
        lib.orc_observer_run(np.ascontiguousarray(u.real), np.ascontiguousarray(u.imag), n, Mz,
                             _ptr(s0r), _ptr(s0i), are, aim)
    else:
        lib.orc_observer_run(np.ascontiguousarray(u.real), np.ascontiguousarray(u.imag), n, Mz,
                             None, None, are, aim)
    return (are + 1j * aim).reshape(n, Mz)


def pef_design(M: int, Mz: int, B: int, mpz: int, vx: float, vy: float) -> np.ndarray:
    """Eq. (8) at the DFT bins: H[iz][jy][jx], k'x = jx - B, k'y = jy - B."""
    lib = _load()
    W = 2 * B + 1
    hr = np.zeros(Mz * W * W)
    hi = np.zeros(Mz * W * W)
    K = (M - 1) // 2
    lib.orc_pef_design(M, Mz, B, K, K, mpz, float(vx), float(vy), hr, hi)
    return (hr + 1j * hi).reshape(Mz, W, W)


class Oracle:
    """Context for one parameter set (precomputes Eq. (10) phases and the
    Eq. (8) coefficient table for every grid velocity)."""

    def __init__(self, M: int, Mz: int, vmax: float, vstep: float, B: int | None = None,
                 mpz: int | None = None, alpha: float | None = None, hp_lines: bool = False):
        self.lib = _load()
        self.M, self.Mz = int(M), int(Mz)
        self.K = (self.M - 1) // 2
        self.kzlo = -((self.Mz - 1) // 2)
        self.B = default_band(M) if B is None else int(B)
        self.mpz = default_delay(Mz) if mpz is None else int(mpz)
        self.alpha = math.exp(-0.1) if alpha is None else float(alpha)
        self.vmax, self.vstep = float(vmax), float(vstep)
        self._h = self.lib.orc_create(self.M, self.Mz, self.B, self.mpz, self.alpha,
                                      self.vmax, self.vstep, int(bool(hp_lines)))
        self.L = self.lib.orc_grid_len(self._h)
        self.nb = self.M * self.M * self.Mz

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.orc_destroy(h)
            self._h = None

    def grid_values(self) -> np.ndarray:
        return -self.vmax + self.vstep * np.arange(self.L)

    def run(self, frames: np.ndarray, crop=None, *, whitened=True, velocity=True,
            spec_frames=(), spectrum=False, power=False, autocorr=False, windowed=False,
            vel_override: np.ndarray | None = None, fixed_v=None, nthreads: int = 0):
        """Run over frames [T][H][W] (float32) for the crop (y0, x0, h, w).

        Returns a dict with 'whitened' [T][h][w] (E of frame t - m'z at t,
        NaN before), 'vel_index' [T][h][w], and at ``spec_frames``:
        'spectrum' complex [n][h][w][Mz][M][M], 'power' likewise (real),
        'autocorr' [n][h][w][L][L] (smoothed R'), 'windowed' complex like
        'spectrum' (high-passed, Hann-windowed).
        """
        frames = np.ascontiguousarray(frames, np.float32)
        T, H, W = frames.shape
        y0, x0, h, w = (0, 0, H, W) if crop is None else crop
        assert 0 <= y0 and y0 + h <= H and 0 <= x0 and x0 + w <= W
        n = len(spec_frames)
        st = np.ascontiguousarray(np.asarray(spec_frames, np.int32))
        out = {}
        wh = np.zeros((T, h, w)) if whitened else None
        vi = np.zeros((T, h, w), np.int32) if velocity else None
        vo = None
        if vel_override is not None:
            vo = np.ascontiguousarray(vel_override, np.int32)
            assert vo.shape == (T, h, w)
        fv = None if fixed_v is None else np.ascontiguousarray(np.asarray(fixed_v, np.float64))
        sre = np.zeros((n, h, w, self.nb)) if (spectrum and n) else None
        sim = np.zeros((n, h, w, self.nb)) if (spectrum and n) else None
        pw = np.zeros((n, h, w, self.nb)) if (power and n) else None
        rs = np.zeros((n, h, w, self.L * self.L)) if (autocorr and n) else None
        wre = np.zeros((n, h, w, self.nb)) if (windowed and n) else None
        wim = np.zeros((n, h, w, self.nb)) if (windowed and n) else None
        rc = self.lib.orc_run(self._h, frames, T, H, W, y0, x0, h, w, _ptr(wh), _ptr(vi),
                              _ptr(vo), _ptr(fv), _ptr(st), n, _ptr(sre), _ptr(sim), _ptr(pw),
                              _ptr(rs), _ptr(wre), _ptr(wim), int(nthreads))
        if rc != 0:
            raise RuntimeError(f"oracle run failed ({rc})")
        shp = (n, h, w, self.Mz, self.M, self.M)
        if wh is not None:
            out["whitened"] = wh
        if vi is not None:
            out["vel_index"] = vi
        if sre is not None:
            out["spectrum"] = (sre + 1j * sim).reshape(shp)
        if pw is not None:
            out["power"] = pw.reshape(shp)
        if wre is not None:
            out["windowed"] = (wre + 1j * wim).reshape(shp)
        if rs is not None:
            out["autocorr"] = rs.reshape(n, h, w, self.L, self.L)
        return out
