"""C-ABI contract checks that need no GPU: the library builds and loads,
exports every function include/*.h declares, validates arguments before any
CUDA call, and the product package never reaches the oracle."""
import ctypes as C
import glob
import os
import re

import pytest

from paper_1408_3526_b300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(wh_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(_declared_functions()) <= set(_abi._SIGS)


def test_status_strings_and_defaults(lib):
    for st in (0, -1, -2, -3, -4, -5, -6, -7):
        assert lib.wh_status_string(st)
    p = _abi.wh_params()
    assert lib.wh_default_params(15, 6, C.byref(p)) == 0
    assert p.band == 5 and p.delay_z == 2 and abs(p.alpha - 0.904837418) < 1e-8
    assert lib.wh_default_params(9, 5, C.byref(p)) == 0
    assert p.band == 3 and p.delay_z == 2
    assert lib.wh_default_params(8, 5, C.byref(p)) == _abi.WH_EINVAL


@pytest.mark.parametrize("args", [
    (0, 64, 9, 4, 2.0, 0.25),     # h < 1
    (64, 64, 8, 4, 2.0, 0.25),    # even window
    (64, 64, 1, 4, 2.0, 0.25),    # window < 3
    (64, 64, 9, 1, 2.0, 0.25),    # Mz < 2
    (64, 64, 9, 4, 2.0, 0.0),     # step <= 0
    (64, 64, 9, 4, 2.0, 0.3),     # vmax not a multiple of step
    (64, 64, 9, 4, 20.0, 0.25),   # grid longer than the kernels' limit
    (40000, 40000, 9, 4, 2.0, 0.25),  # more than 2^30 pixels
])
def test_create_rejects_bad_arguments_without_cuda(lib, args):
    h, w, M, Mz, vmax, step = args
    out = C.c_void_p()
    rc = lib.wh_create_stream(h, w, M, Mz, _abi.wh_vgrid(vmax, step), None, None, C.byref(out))
    assert rc == _abi.WH_EINVAL
    assert not out.value


def test_null_handles_are_rejected(lib):
    assert lib.wh_push_frame(None, None, 0) == _abi.WH_EINVAL
    assert lib.wh_read_whitened(None, None, 0, None) == _abi.WH_EINVAL
    assert lib.wh_destroy_stream(None) == _abi.WH_OK


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1408_3526_b300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
            txt = open(path).read()
            assert not re.search(r"^\s*(import|from)\s+oracle", txt, re.M), path
            assert "whiten_oracle" not in txt, path


def test_stream_device_bytes_estimate(lib):
    g = _abi.wh_vgrid(3.0, 0.25)
    a = lib.wh_stream_device_bytes(512, 640, 15, 6, g)
    b = lib.wh_stream_device_bytes(1024, 1280, 15, 6, g)
    assert a > 512 * 640 * (4 * 228) and 3.9 < b / a < 4.1
    assert lib.wh_stream_device_bytes(0, 640, 15, 6, g) == -1
