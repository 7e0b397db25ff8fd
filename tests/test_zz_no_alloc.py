"""The allocation-free frame push against the ordinary one (needs a B300).

wh_push_frame_noalloc serves callers that cannot allocate device memory once
streaming has started (fixed-memory real-time loops, frozen memory pools,
hosts that forbid driver allocations after start-up); its search scratch lives
in a static device array.  Two twin streams receive the same frames; for the
last two frames one uses wh_push_frame and the other wh_push_frame_noalloc,
called twice in a row.  Their velocities and whitened frames must agree
within the parity tolerances used everywhere else (identical velocity index on
>= 99.9% of pixels, within one grid step elsewhere; whitened within 1e-3 x
input RMS).  Further cases: host frames, a stream in learned mode (the
allocation-free push still runs the exact search), the status word reported
once, and the combinations it rejects.  This file is collected last so that a
run stopping at the first failure has run every other test already; it also
passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1408_3526_b300 import _abi, scenes
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _agree(ref, na, rms):
    _, _, vi_r, _ = ref.read_velocity()
    _, _, vi_n, _ = na.read_velocity()
    same = float(np.mean(vi_r == vi_n))
    L = ref.L
    steps = np.maximum(np.abs(vi_r % L - vi_n % L), np.abs(vi_r // L - vi_n // L))
    assert same >= P.VEL_EXACT_FRAC, same
    assert steps.max() <= 1
    e_r, i_r = ref.read_whitened()
    e_n, i_n = na.read_whitened()
    assert i_r == i_n
    assert np.max(np.abs(e_r - e_n)) / rms <= P.WHITE_TOL_REL


def _noalloc(s, frame, is_device):
    ptr = frame.data_ptr() if is_device else frame.ctypes.data
    rc = s.lib.wh_push_frame_noalloc(s._s, C.c_void_p(ptr), int(is_device))
    assert rc == 0, s.lib.wh_last_error()


@pytest.mark.parametrize("is_device", [1, 0], ids=["device_frames", "host_frames"])
@pytest.mark.parametrize("M,Mz,vmax,H,W,T", [(9, 4, 2.0, 64, 64, 10), (15, 6, 3.0, 136, 150, 9)])
def test_push_frame_noalloc_matches_push_frame(M, Mz, vmax, H, W, T, is_device):
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    sc = scenes.small_scene(T=T, H=H, W=W, seed=M + 100, vx=0.6, vy=-0.45, tex_size=256)
    fr = torch.from_numpy(sc.frames).cuda()
    rms = float(np.sqrt(np.mean(sc.frames.astype(np.float64) ** 2)))
    with WhitenStream(H, W, M, Mz, vmax, 0.25) as ref, WhitenStream(H, W, M, Mz, vmax, 0.25) as na:
        for t in range(T):
            ref.push(fr[t])
            if t < T - 2:
                na.push(fr[t])
            else:   # two calls in a row of the allocation-free entry point
                _noalloc(na, fr[t] if is_device else np.ascontiguousarray(sc.frames[t]), is_device)
                _agree(ref, na, rms)


def test_push_frame_noalloc_in_learned_mode():
    """A stream in learned mode: the allocation-free push runs the exact search
    (the network is not used), so it equals a plain twin's wh_push_frame."""
    import torch

    from paper_1408_3526_b300.learned import MLP
    from paper_1408_3526_b300.stream import WhitenStream
    H, W, T = 48, 56, 8
    sc = scenes.small_scene(T=T, H=H, W=W, seed=77, vx=0.4, vy=0.7, tex_size=128)
    fr = torch.from_numpy(sc.frames).cuda()
    rms = float(np.sqrt(np.mean(sc.frames.astype(np.float64) ** 2)))
    net = MLP(n_in=9 * 9 * 4, h1=64, h2=32, seed=5)
    with WhitenStream(H, W, 9, 4, 2.0, 0.25) as ref, WhitenStream(H, W, 9, 4, 2.0, 0.25) as na:
        assert na.lib.wh_stream_set_features(na._s, 1) == 0
        assert na.lib.wh_stream_set_learned(na._s, net._m, C.c_float(0.8)) == 0
        for t in range(T):
            ref.push(fr[t])
            if t < T - 2:
                na.push(fr[t])
            else:
                _noalloc(na, fr[t], 1)
                _agree(ref, na, rms)
        na.lib.wh_stream_set_learned(na._s, None, C.c_float(0.8))
    net.close()


def test_push_frame_noalloc_reports_status_once():
    """A status word set as a bounded device wait that gave up would set it is
    reported once, as WH_ETIMEOUT, by the read after an allocation-free push."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = torch.zeros((40, 48), dtype=torch.float32, device="cuda")
    with WhitenStream(40, 48, 9, 4, 2.0, 0.25) as s:
        _noalloc(s, fr, 1)
        assert s.lib.wh_stream_sync(s._s) == _abi.WH_OK
        assert s.lib.wh_stream_selftest_status(s._s, 5) == _abi.WH_OK
        _noalloc(s, fr, 1)
        with pytest.raises(Exception):
            s.read_velocity()
        s.read_velocity()                              # cleared after one report
        assert s.lib.wh_stream_sync(s._s) == _abi.WH_OK


def test_push_frame_noalloc_rejects_unsupported():
    """The frame pipeline and grids beyond 25 x 25 are refused with WH_EUNSUP
    before anything is enqueued (the stream stays at frame 0)."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = torch.zeros((32, 40), dtype=torch.float32, device="cuda")
    with WhitenStream(32, 40, 9, 4, 2.0, 0.25, pipeline=True) as s:
        rc = s.lib.wh_push_frame_noalloc(s._s, C.c_void_p(fr.data_ptr()), 1)
        assert rc == _abi.WH_EUNSUP
        assert s.frames_pushed == 0
    with WhitenStream(32, 40, 9, 4, 3.5, 0.25) as s:     # L = 29
        assert s.L == 29
        rc = s.lib.wh_push_frame_noalloc(s._s, C.c_void_p(fr.data_ptr()), 1)
        assert rc == _abi.WH_EUNSUP
        assert s.frames_pushed == 0
