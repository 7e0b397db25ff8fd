"""The allocation-free frame push against the ordinary one (needs a B300).

wh_push_frame_noalloc serves callers that cannot allocate device memory once
streaming has started; its search scratch lives in a static device array.
Two twin streams receive the same frames; for the last two frames one uses
wh_push_frame and the other wh_push_frame_noalloc, called twice in a row.
Their velocities and whitened frames must agree within the parity tolerances
used everywhere else (identical velocity index on >= 99.9% of pixels, within
one grid step elsewhere; whitened within 1e-3 x input RMS).  This file is
collected last so that a run stopping at the first failure has run every
other test already; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1408_3526_b300 import scenes
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,Mz,vmax,H,W,T", [(9, 4, 2.0, 64, 64, 10), (15, 6, 3.0, 136, 150, 9)])
def test_push_frame_noalloc_matches_push_frame(M, Mz, vmax, H, W, T):
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    sc = scenes.small_scene(T=T, H=H, W=W, seed=M + 100, vx=0.6, vy=-0.45, tex_size=256)
    fr = torch.from_numpy(sc.frames).cuda()
    rms = float(np.sqrt(np.mean(sc.frames.astype(np.float64) ** 2)))
    with WhitenStream(H, W, M, Mz, vmax, 0.25) as ref, WhitenStream(H, W, M, Mz, vmax, 0.25) as na:
        lib = na.lib
        for t in range(T):
            ref.push(fr[t])
            if t < T - 2:
                na.push(fr[t])
            else:   # two calls in a row of the allocation-free entry point
                rc = lib.wh_push_frame_noalloc(na._s, C.c_void_p(fr[t].data_ptr()), 1)
                assert rc == 0, lib.wh_last_error()
                _, _, vi_r, _ = ref.read_velocity()
                _, _, vi_n, _ = na.read_velocity()
                same = float(np.mean(vi_r == vi_n))
                L = ref.L
                steps = np.maximum(np.abs(vi_r % L - vi_n % L), np.abs(vi_r // L - vi_n // L))
                assert same >= P.VEL_EXACT_FRAC, same
                assert steps.max() <= 1
                e_r, i_r = ref.read_whitened()
                e_n, i_n = na.read_whitened()
                assert i_r == i_n == t - ref.delay_z
                assert np.max(np.abs(e_r - e_n)) / rms <= P.WHITE_TOL_REL
