"""ctypes binding of libwhiten.so: the C ABI of include/whiten.h, same names.

Argument marshalling only -- every step of the path runs in the library's
CUDA kernels.  Loading fails loudly (ImportError) if the shared library has
not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwhiten.so")

WH_OK = 0
WH_EINVAL = -1
WH_ENOMEM = -2
WH_EADMIT = -3
WH_ENOTREADY = -4
WH_ECUDA = -5
WH_ETIMEOUT = -6
WH_EUNSUP = -7

WH_PREC_FP32 = 0
WH_PREC_TC_FP16 = 1
WH_PREC_TC_BF16 = 2
WH_PREC_CUDA_CORES = 8
WH_PREC_TC_SHORTLIST = 16
WH_PREC_TC_SEPARABLE = 32
WH_PREC_SPEC_F64 = 64
WH_PREC_TC_DENSE = 128

WH_SPEC_RAW = 0
WH_SPEC_WINDOWED = 1
WH_SPEC_POWER = 2


class wh_vgrid(C.Structure):
    _fields_ = [("vmax", C.c_float), ("step", C.c_float)]


class wh_params(C.Structure):
    _fields_ = [("band", C.c_int), ("delay_z", C.c_int), ("alpha", C.c_double),
                ("precision", C.c_int), ("debug_dump", C.c_int), ("pipeline", C.c_int)]


class WhitenError(RuntimeError):
    def __init__(self, status: int, what: str, lib=None):
        msg = f"{what}: {status}"
        if lib is not None:
            msg += f" ({lib.wh_status_string(status).decode()})"
            if status == WH_ECUDA:
                msg += f": {lib.wh_last_error().decode()}"
        super().__init__(msg)
        self.status = status


# name -> (restype, argtypes)
_VP = C.c_void_p
_SIGS = {
    "wh_default_params": (C.c_int, [C.c_int, C.c_int, C.POINTER(wh_params)]),
    "wh_create_stream": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, wh_vgrid,
                                   C.POINTER(wh_params), _VP, C.POINTER(_VP)]),
    "wh_push_frame": (C.c_int, [_VP, _VP, C.c_int]),
    "wh_push_frame_noalloc": (C.c_int, [_VP, _VP, C.c_int]),
    "wh_push_frame_async": (C.c_int, [_VP, _VP, _VP, _VP, _VP, C.POINTER(C.c_longlong)]),
    "wh_stream_sync": (C.c_int, [_VP]),
    "wh_stream_join": (C.c_int, [_VP]),
    "wh_detect": (C.c_int, [_VP, C.c_float, C.c_int, _VP, C.POINTER(C.c_int), C.POINTER(C.c_float),
                            C.c_int, C.POINTER(C.c_longlong)]),
    "wh_selftest_wait_timeout": (C.c_int, [C.c_int, _VP]),
    "wh_stream_selftest_status": (C.c_int, [_VP, C.c_int]),
    "wh_stream_query_frame": (C.c_int, [_VP, C.c_longlong, C.c_int]),
    "wh_read_whitened": (C.c_int, [_VP, _VP, C.c_int, C.POINTER(C.c_longlong)]),
    "wh_read_velocity": (C.c_int, [_VP, _VP, _VP, _VP, C.c_int, C.POINTER(C.c_longlong)]),
    "wh_read_spectrum": (C.c_int, [_VP, C.c_int, _VP, C.c_int]),
    "wh_read_autocorr": (C.c_int, [_VP, _VP, C.c_int]),
    "wh_stream_info": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                 C.POINTER(C.c_longlong)]),
    "wh_stream_stats": (C.c_int, [_VP, C.POINTER(C.c_longlong)]),
    "wh_stream_search_counts": (C.c_int, [_VP, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "wh_tcsep_operand": (C.c_int, [C.c_int, C.c_int, C.c_double, _VP]),
    "wh_output_pointers": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP),
                                     C.POINTER(_VP)]),
    "wh_profile_enable": (C.c_int, [_VP, C.c_int]),
    "wh_profile_read": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.c_int]),
    "wh_tc_gemm": (C.c_int, [_VP, C.c_int, _VP, C.c_int, _VP, C.c_int, C.c_int, C.c_int, C.c_int,
                             C.c_int, C.c_int, _VP, C.c_int, _VP]),
    "wh_tc_gemm_topk": (C.c_int, [_VP, C.c_int, _VP, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_int, _VP, _VP, _VP]),
    "wh_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, _VP, C.POINTER(_VP)]),
    "wh_mlp_destroy": (C.c_int, [_VP]),
    "wh_mlp_num_params": (C.c_longlong, [_VP]),
    "wh_mlp_get_params": (C.c_int, [_VP, _VP, C.c_longlong]),
    "wh_mlp_set_params": (C.c_int, [_VP, _VP, C.c_longlong]),
    "wh_mlp_get_grads": (C.c_int, [_VP, _VP, C.c_longlong]),
    "wh_mlp_forward": (C.c_int, [_VP, _VP, C.c_int, C.c_int, _VP, C.c_int]),
    "wh_mlp_train_step": (C.c_int, [_VP, _VP, C.c_int, C.c_int, _VP, C.c_float, C.c_float, C.c_float,
                                    C.c_int, _VP]),
    "wh_stream_set_features": (C.c_int, [_VP, C.c_int]),
    "wh_read_features": (C.c_int, [_VP, _VP, C.c_int, C.POINTER(C.c_int)]),
    "wh_stream_set_learned": (C.c_int, [_VP, _VP, C.c_float]),
    "wh_stream_learned_stats": (C.c_int, [_VP, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "wh_stream_device_bytes": (C.c_longlong, [C.c_int, C.c_int, C.c_int, C.c_int, wh_vgrid]),
    "wh_stream_device_bytes_opt": (C.c_longlong, [C.c_int, C.c_int, C.c_int, C.c_int, wh_vgrid,
                                                  C.POINTER(wh_params)]),
    "wh_server_create": (C.c_int, [C.c_double, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_VP)]),
    "wh_server_open": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, C.c_int, wh_vgrid, C.POINTER(wh_params),
                                 C.POINTER(C.c_int)]),
    "wh_server_submit": (C.c_int, [_VP, C.c_int, _VP, C.c_double, C.POINTER(C.c_longlong)]),
    "wh_server_now": (C.c_double, [_VP]),
    "wh_server_wait": (C.c_int, [_VP, C.c_longlong, _VP, C.POINTER(C.c_double)]),
    "wh_server_drain": (C.c_int, [_VP]),
    "wh_server_stats": (C.c_int, [_VP, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "wh_server_close": (C.c_int, [_VP, C.c_int]),
    "wh_server_destroy": (C.c_int, [_VP]),
    "wh_reset_stream": (C.c_int, [_VP]),
    "wh_destroy_stream": (C.c_int, [_VP]),
    "wh_status_string": (C.c_char_p, [C.c_int]),
    "wh_last_error": (C.c_char_p, []),
    "wh_kernel_launch_count": (C.c_longlong, []),
}

_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libwhiten.so (built by paper_1408_3526_b300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"CUDA library not built: {p} (run python -m "
                                  "paper_1408_3526_b300.build)")
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                if hasattr(lib, name):
                    fn = getattr(lib, name)
                    fn.restype = res
                    fn.argtypes = args
            _lib = lib
    return _lib


def check(status: int, what: str):
    if status != WH_OK:
        raise WhitenError(status, what, _lib)
    return status
