"""The tensor-core separable search against the CUDA-core search (needs a
B300): both evaluate Eq. (10) exactly in FP32 on the rows their bounds keep,
with the same operation sequence, so the velocity indices must be identical
bit for bit: on the full 512 x 640 stream in the benchmark's launch
configuration, on a frame size that leaves a partial last tile, with the
frame pipeline, and after a reset."""
import numpy as np
import pytest

from paper_1408_3526_b300 import _abi, scenes

pytestmark = pytest.mark.gpu


def _twin_velocities(frames, M, Mz, vmax, step, pipeline=False, reset_at=None):
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    T, H, W = frames.shape
    fd = torch.from_numpy(np.ascontiguousarray(frames)).cuda()
    out = {}
    for prec in (_abi.WH_PREC_CUDA_CORES, _abi.WH_PREC_TC_SEPARABLE):
        vel = np.zeros((T, H, W), np.int32)
        white = np.zeros((T, H, W), np.float32)
        with WhitenStream(H, W, M, Mz, vmax, step, precision=prec,
                          pipeline=pipeline and prec == _abi.WH_PREC_TC_SEPARABLE) as s:
            for t in range(T):
                if reset_at is not None and t == reset_at:
                    s.reset()
                s.push(fd[t])
                vel[t] = s.read_velocity()[2]
                if s.frames_pushed > s.delay_z:
                    white[t] = s.read_whitened()[0]
        out[prec] = (vel, white)
    return out[_abi.WH_PREC_CUDA_CORES], out[_abi.WH_PREC_TC_SEPARABLE]


def test_tc_separable_equals_cuda_cores_full_size():
    """512 x 640, 15 x 15, order 6, grid +-3 step 1/4, 12 frames."""
    sc = scenes.config2_scene(T=12)
    (v0, w0), (v1, w1) = _twin_velocities(sc.frames, 15, 6, 3.0, 0.25)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_array_equal(w0, w1)


@pytest.mark.parametrize("pipeline", [False, True], ids=["serial", "pipelined"])
def test_tc_separable_partial_tile_and_reset(pipeline):
    """A pixel count that is not a multiple of the 64-pixel tile, the widest
    grid (31 points), and a reset in the middle of the sequence."""
    sc = scenes.small_scene(T=10, H=37, W=53, seed=21, vx=0.9, vy=-1.3, tex_size=128)
    (v0, w0), (v1, w1) = _twin_velocities(sc.frames, 9, 4, 3.75, 0.25, pipeline=pipeline, reset_at=5)
    np.testing.assert_array_equal(v0, v1)
    np.testing.assert_array_equal(w0, w1)
