"""Pipelined push (wh_push_frame_async) gives the same outputs as the
synchronous push-and-read sequence, frame by frame (needs a B300)."""
import numpy as np
import pytest

from paper_1408_3526_b300 import scenes

pytestmark = pytest.mark.gpu

H, W, M, MZ, VMAX, VSTEP, T = 64, 80, 9, 4, 2.0, 0.25, 14
DELAY = (MZ - 1) // 2


@pytest.mark.parametrize("pipeline,precision", [(False, 0), (True, 0), (True, 16)],
                         ids=["serial", "pipelined", "pipelined_tc_engine"])
def test_async_push_matches_sync(pipeline, precision):
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = scenes.config1_scene(T=T, H=H, W=W, seed=5).frames.astype(np.float32)
    ref_w, ref_x, ref_y = [], [], []
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, precision=precision) as s:
        for t in range(T):
            s.push(np.ascontiguousarray(fr[t]))
            vx, vy, _, _ = s.read_velocity()
            ref_x.append(vx.copy())
            ref_y.append(vy.copy())
            ref_w.append(s.read_whitened()[0].copy() if t >= DELAY else np.zeros((H, W), np.float32))
    pin = [torch.from_numpy(fr[t].copy()).pin_memory() for t in range(T)]
    outs = [[torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(3)] for _ in range(T)]
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, precision=precision, pipeline=pipeline) as s:
        idx = []
        for t in range(T):
            idx.append(s.push_async(pin[t], *outs[t]))
            if t >= 3:
                s.wait_frame(idx[t - 3])          # an older frame completes on request
        s.sync()
        assert idx == list(range(T))
        for t in range(T):
            w, x, y = (o.numpy() for o in outs[t])
            assert np.array_equal(x, ref_x[t]), t
            assert np.array_equal(y, ref_y[t]), t
            if t >= DELAY:
                assert np.array_equal(w, ref_w[t]), t
        # a synchronous push after asynchronous ones continues the same sequence
        s.push(np.ascontiguousarray(fr[T - 1]))
        vx = s.read_velocity()[0]
        assert vx.shape == (H, W)


def test_async_query_before_and_after():
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = scenes.config1_scene(T=4, H=H, W=W, seed=6).frames.astype(np.float32)
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP) as s:
        pin = torch.from_numpy(fr[0].copy()).pin_memory()
        out = torch.empty((H, W), dtype=torch.float32).pin_memory()
        i0 = s.push_async(pin, None, out, None)
        s.wait_frame(i0)
        rc = s.lib.wh_stream_query_frame(s._s, i0, 0)
        assert rc == 0
        assert s.lib.wh_stream_query_frame(s._s, i0 + 5, 0) != 0     # never pushed
        with pytest.raises(ValueError):
            s.push_async(torch.from_numpy(fr[1].copy()))             # pageable memory refused
