"""Frame pipeline (wh_params.pipeline): the spectrum kernel of frame t+1 overlaps
the search and PEF of frame t on two internal CUDA streams, with the smoothed
state double-buffered.  Results must be bit-identical to the serial stream,
for device and host frames, the synchronous and the pipelined host push, and
both search engines (needs a B300)."""
import numpy as np
import pytest

from paper_1408_3526_b300 import scenes

pytestmark = pytest.mark.gpu

H, W, M, MZ, VMAX, VSTEP, T = 96, 120, 9, 4, 2.0, 0.25, 16
DELAY = (MZ - 1) // 2


def _run(frames, pipeline, precision=0, device=True, debug=False):
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    out = []
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, precision=precision, pipeline=pipeline,
                      debug_dump=debug) as s:
        dev = torch.from_numpy(frames).cuda()
        for t in range(frames.shape[0]):
            s.push(dev[t] if device else np.ascontiguousarray(frames[t]))
            vx, vy, vi, _ = s.read_velocity()
            w = s.read_whitened()[0] if t >= DELAY else None
            out.append((vx, vy, vi, w))
        if debug:
            from paper_1408_3526_b300 import _abi
            out.append(s.read_spectrum(_abi.WH_SPEC_WINDOWED))
            out.append(s.read_autocorr())
    return out


def _same(a, b):
    for x, y in zip(a, b):
        if isinstance(x, tuple):
            for u, v in zip(x, y):
                if u is None:
                    assert v is None
                else:
                    assert np.array_equal(u, v)
        else:
            assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", [0, 128, 16], ids=["cuda_cores", "tc_dense", "tc_shortlist_rerank"])
def test_pipeline_identical_to_serial(precision):
    fr = scenes.config1_scene(T=T, H=H, W=W, seed=9).frames.astype(np.float32)
    _same(_run(fr, False, precision), _run(fr, True, precision))


def test_pipeline_host_frames_and_debug_reads():
    fr = scenes.config1_scene(T=10, H=H, W=W, seed=10).frames.astype(np.float32)
    _same(_run(fr, False, device=False, debug=True), _run(fr, True, device=False, debug=True))


def test_pipeline_unread_frames_then_async_push():
    """Frames pushed back to back without reads (the overlapped case), then the
    pipelined host push with double-buffered outputs."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = scenes.config1_scene(T=T, H=H, W=W, seed=11).frames.astype(np.float32)
    ref = []
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP) as s:
        for t in range(T):
            s.push(np.ascontiguousarray(fr[t]))
            ref.append((s.read_velocity()[0].copy(), s.read_whitened()[0].copy() if t >= DELAY else None))
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, pipeline=True) as s:
        dev = torch.from_numpy(fr).cuda()
        for t in range(T // 2):
            s.push(dev[t])
        vx = s.read_velocity()[0]
        assert np.array_equal(vx, ref[T // 2 - 1][0])
        pin = [torch.from_numpy(fr[t].copy()).pin_memory() for t in range(T)]
        outs = [[torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(2)]
                for _ in range(T)]
        for t in range(T // 2, T):
            s.push_async(pin[t], outs[t][0], outs[t][1], None)
        s.sync()
        for t in range(T // 2, T):
            assert np.array_equal(outs[t][1].numpy(), ref[t][0]), t
            assert np.array_equal(outs[t][0].numpy(), ref[t][1]), t


@pytest.mark.parametrize("conf", [0.0, 0.8])
def test_pipeline_learned_mode_identical_to_serial(conf):
    """Learned velocity mode with the frame pipeline: the spectrum kernel of
    frame t+1 writes the feature buffer that the network of frame t reads, so
    it must wait for that search; frames are pushed back to back (no reads in
    between) and the results must equal the serial stream's."""
    import ctypes as C

    import torch

    from paper_1408_3526_b300 import learned
    from paper_1408_3526_b300.stream import WhitenStream
    net = learned.MLP(M * M * MZ, 256, 128, 3, seed=3)
    fr = scenes.config1_scene(T=T, H=H, W=W, seed=11).frames.astype(np.float32)
    dev = torch.from_numpy(fr).cuda()
    res = []
    for pipeline in (False, True):
        with WhitenStream(H, W, M, MZ, VMAX, VSTEP, pipeline=pipeline) as s:
            assert s.lib.wh_stream_set_learned(s._s, net._m, conf) == 0
            for t in range(T):
                s.push(dev[t])
            vx, vy, vi, _ = s.read_velocity()
            w, _ = s.read_whitened()
            nfr, nfb = C.c_longlong(), C.c_longlong()
            assert s.lib.wh_stream_learned_stats(s._s, C.byref(nfr), C.byref(nfb)) == 0
            res.append((vx, vy, vi, w, np.array([nfr.value, nfb.value])))
    net.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_pipeline_reset_orders_after_the_callers_stream():
    """wh_reset_stream clears the state on the caller's CUDA stream; with the
    pipeline the next push (a host frame, which needs nothing else from that
    stream) must still start after it.  The caller's stream is kept busy across
    the reset, then the results must equal a fresh stream's."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = scenes.config1_scene(T=12, H=H, W=W, seed=12).frames.astype(np.float32)
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP) as s:
        for t in range(4, 12):
            s.push(np.ascontiguousarray(fr[t]))
        ref = (s.read_velocity()[2], s.read_whitened()[0])
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, pipeline=True) as s:
        for t in range(4):
            s.push(np.ascontiguousarray(fr[t]))
        s.sync()
        torch.cuda._sleep(100_000_000)           # ~50 ms of work queued on the caller's stream
        s.reset()
        for t in range(4, 12):
            s.push(np.ascontiguousarray(fr[t]))
        got = (s.read_velocity()[2], s.read_whitened()[0])
    assert np.array_equal(got[0], ref[0])
    assert np.array_equal(got[1], ref[1])


@pytest.mark.parametrize("pipeline", [False, True])
def test_learned_mode_async_push_equals_sync(pipeline):
    """Learned mode through the asynchronous host push (copies overlapped with
    the kernels) gives the synchronous push's velocities and whitened frames."""
    import ctypes as C

    import torch

    from paper_1408_3526_b300 import learned
    from paper_1408_3526_b300.stream import WhitenStream
    net = learned.MLP(M * M * MZ, 256, 128, 3, seed=4)
    fr = scenes.config1_scene(T=T, H=H, W=W, seed=13).frames.astype(np.float32)
    ref = []
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP) as s:
        assert s.lib.wh_stream_set_learned(s._s, net._m, 0.5) == 0
        for t in range(T):
            s.push(np.ascontiguousarray(fr[t]))
            vx, vy, _, _ = s.read_velocity()
            w = s.read_whitened()[0] if t >= DELAY else np.zeros((H, W), np.float32)
            ref.append((vx.copy(), vy.copy(), w.copy()))
    pin = [torch.from_numpy(fr[t].copy()).pin_memory() for t in range(T)]
    outs = [[torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(3)] for _ in range(T)]
    with WhitenStream(H, W, M, MZ, VMAX, VSTEP, pipeline=pipeline) as s:
        assert s.lib.wh_stream_set_learned(s._s, net._m, 0.5) == 0
        for t in range(T):
            s.push_async(pin[t], *outs[t])
        s.sync()
    net.close()
    for t in range(T):
        w, x, y = (o.numpy() for o in outs[t])
        assert np.array_equal(x, ref[t][0]) and np.array_equal(y, ref[t][1]), t
        if t >= DELAY:
            assert np.array_equal(w, ref[t][2]), t


def _random_shapes():
    from tests.test_gpu_parity_random import _cases
    return [c[:7] for c in _cases()][:6]


@pytest.mark.parametrize("i,Mw,Mzw,vmax,step,Hh,Ww", _random_shapes())
def test_pipeline_identical_to_serial_random_shapes(i, Mw, Mzw, vmax, step, Hh, Ww):
    """Frames pushed back to back (no reads in between, so consecutive frames
    overlap on the device) on seeded random shapes: the pipelined stream's last
    outputs equal the serial stream's bit for bit."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = scenes.small_scene(T=10, H=Hh, W=Ww, seed=300 + i, tex_size=128).frames.astype(np.float32)
    dev = torch.from_numpy(fr).cuda()
    res = []
    for pipeline in (False, True):
        with WhitenStream(Hh, Ww, Mw, Mzw, vmax, step, pipeline=pipeline) as s:
            for t in range(fr.shape[0]):
                s.push(dev[t])
            vx, vy, vi, _ = s.read_velocity()
            w, _ = s.read_whitened()
            res.append((vx, vy, vi, w))
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_pipeline_identical_to_serial_full_size():
    """The benchmark's configuration (512 x 640, 15 x 15, order 6, grid +-3/0.25),
    frames pushed back to back: pipelined and serial streams agree bit for bit."""
    import torch

    from paper_1408_3526_b300.stream import WhitenStream
    fr = scenes.config2_scene(T=10, H=512, W=640, seed=2).frames.astype(np.float32)
    dev = torch.from_numpy(fr).cuda()
    res = []
    for pipeline in (False, True):
        with WhitenStream(512, 640, 15, 6, 3.0, 0.25, pipeline=pipeline) as s:
            for t in range(fr.shape[0]):
                s.push(dev[t])
            vx, vy, vi, _ = s.read_velocity()
            w, _ = s.read_whitened()
            res.append((vx, vy, vi, w))
    for a, b in zip(*res):
        assert np.array_equal(a, b)
