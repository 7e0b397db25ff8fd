"""The search engine with the whole contraction of Eq. (10) on tcgen05 tensor
cores (WH_PREC_TC_DENSE) against the CUDA-core search (needs a B300).

The tensor-core product decides a pixel only where a single grid point lies
within the rigorous F16 error window of its maximum; every other pixel's
listed points (or its whole grid) are evaluated in FP32 with the CUDA-core
search's operation sequence.  The velocity indices must therefore equal the
CUDA-core search's bit for bit, and so must the whitened output: on the full
512 x 640 stream in the benchmark's configuration, with the frame pipeline, on
frame sizes that leave partial 128-pixel tiles and partial 32-pixel staging
slots, for every built window size, on the widest grid, and after a reset.
"""
import numpy as np
import pytest

from paper_1408_3526_b300 import _abi, scenes

pytestmark = pytest.mark.gpu


def _twin(frames, M, Mz, vmax, step, pipeline=False, reset_at=None):
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    T, H, W = frames.shape
    fd = torch.from_numpy(np.ascontiguousarray(frames)).cuda()
    out = {}
    for prec in (_abi.WH_PREC_CUDA_CORES, _abi.WH_PREC_TC_DENSE):
        vel = np.zeros((T, H, W), np.int32)
        white = np.zeros((T, H, W), np.float32)
        with WhitenStream(H, W, M, Mz, vmax, step, precision=prec,
                          pipeline=pipeline and prec == _abi.WH_PREC_TC_DENSE) as s:
            for t in range(T):
                if reset_at is not None and t == reset_at:
                    s.reset()
                s.push(fd[t])
                vel[t] = s.read_velocity()[2]
                if s.frames_pushed > s.delay_z:
                    white[t] = s.read_whitened()[0]
        out[prec] = (vel, white)
    return out[_abi.WH_PREC_CUDA_CORES], out[_abi.WH_PREC_TC_DENSE]


@pytest.mark.parametrize("pipeline", [False, True], ids=["serial", "pipelined"])
def test_tc_dense_equals_cuda_cores_full_size(pipeline):
    """512 x 640, 15 x 15, order 6, grid +-3 step 1/4, 12 frames."""
    sc = scenes.config2_scene(T=12)
    (v0, w0), (v1, w1) = _twin(sc.frames, 15, 6, 3.0, 0.25, pipeline=pipeline)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_array_equal(w0, w1)


@pytest.mark.parametrize("M,Mz,vmax", [(5, 3, 1.0), (7, 5, 1.5), (9, 4, 3.75), (9, 6, 2.0), (15, 4, 3.0),
                                       (15, 6, 3.75)])
def test_tc_dense_equals_cuda_cores_shapes(M, Mz, vmax):
    """Every window size the spectrum kernel is built for, grids up to 31 x 31
    (4 chunks of the half grid), a pixel count that leaves a partial last tile
    and a partial staging slot."""
    sc = scenes.small_scene(T=9, H=37, W=53, seed=M + 30, vx=0.9, vy=-1.3, tex_size=128)
    (v0, w0), (v1, w1) = _twin(sc.frames, M, Mz, vmax, 0.25)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_array_equal(w0, w1)


@pytest.mark.parametrize("pipeline", [False, True], ids=["serial", "pipelined"])
def test_tc_dense_partial_tile_and_reset(pipeline):
    """A reset in the middle of the sequence; 31 x 31 grid."""
    sc = scenes.small_scene(T=10, H=41, W=67, seed=21, vx=0.9, vy=-1.3, tex_size=128)
    (v0, w0), (v1, w1) = _twin(sc.frames, 9, 4, 3.75, 0.25, pipeline=pipeline, reset_at=5)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_array_equal(w0, w1)


def test_tc_dense_degenerate_states():
    """Constant frames (all-zero state: R = 0 everywhere, index 0), frames scaled
    to 1e-30 and 1e-19 (states that underflow to zero or sit near FP32's
    subnormal range, where the whole grid is evaluated), frames scaled to 1e15,
    and a NaN pixel (non-finite state)."""
    rng = np.random.default_rng(5)
    T, H, W = 8, 24, 40
    base = rng.standard_normal((T, H, W)).astype(np.float32)
    nan = base.copy()
    nan[T // 2, H // 3, W // 4] = np.nan
    for fr in (np.full((T, H, W), 3.25, np.float32), base * np.float32(1e-30), base * np.float32(1e-19),
               base * np.float32(1e15), nan):
        (v0, _), (v1, _) = _twin(fr, 9, 4, 2.0, 0.25)
        np.testing.assert_array_equal(v0, v1)
