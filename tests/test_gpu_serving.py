"""Serving runtime on the GPU: every stream's result in a concurrent mix of
streams (different sizes, windows, orders; overlapping on several CUDA
streams) equals its result alone, and admission honours the memory budget."""
import numpy as np
import pytest

from paper_1408_3526_b300 import _abi, scenes
from tests import _parity as P

pytestmark = pytest.mark.gpu

SPECS = [(128, 128, 9, 4, 2.0), (96, 160, 15, 6, 3.0), (64, 64, 9, 5, 2.0), (128, 96, 15, 4, 3.0),
         (40, 72, 7, 6, 1.5)]


def test_results_in_the_mix_equal_results_alone():
    import torch

    from paper_1408_3526_b300.serving import Server
    from paper_1408_3526_b300.stream import WhitenStream
    T = 7
    frames = [scenes.small_scene(T=T, H=h, W=w, seed=50 + i, tex_size=256).frames
              for i, (h, w, M, Mz, vm) in enumerate(SPECS)]
    alone = []
    for (h, w, M, Mz, vm), fr in zip(SPECS, frames):
        out = []
        with WhitenStream(h, w, M, Mz, vm, 0.25) as s:
            for t in range(T):
                s.push(fr[t])
                out.append(s.read_whitened()[0].copy() if t >= s.delay_z else None)
        alone.append(out)
    with Server(budget_bytes=8e9, max_inflight=4, queue_limit=T, n_cuda_streams=3, keep_results=True) as srv:
        sids = [srv.open(h, w, M, Mz, vm, 0.25) for (h, w, M, Mz, vm) in SPECS]
        assert all(s is not None for s in sids)
        rids = []
        for t in range(T):                       # interleaved submission: all streams in flight together
            for i, s in enumerate(sids):
                rids.append((i, t, srv.submit(s, frames[i][t], srv.now())))
        for i, t, rid in rids:
            assert rid is not None
            e, lat = srv.wait(rid, sids[i])
            assert lat >= 0
            if alone[i][t] is not None:
                rms = float(np.sqrt(np.mean(frames[i].astype(np.float64) ** 2)))
                assert np.max(np.abs(e - alone[i][t])) <= P.WHITE_TOL_REL * rms
                assert np.array_equal(e, alone[i][t])   # same kernels, same inputs: bit-identical
        st = srv.stats()
        assert st["served"] == len(rids) and st["shed"] == 0


def test_admission_by_memory_budget_and_release():
    from paper_1408_3526_b300.serving import Server
    lib = _abi.load()
    need = lib.wh_stream_device_bytes(256, 320, 15, 6, _abi.wh_vgrid(3.0, 0.25))
    assert need > 256 * 320 * 900
    with Server(budget_bytes=2.5 * need, max_inflight=2, queue_limit=2, n_cuda_streams=2) as srv:
        a = srv.open(256, 320, 15, 6, 3.0, 0.25)
        b = srv.open(256, 320, 15, 6, 3.0, 0.25)
        c = srv.open(256, 320, 15, 6, 3.0, 0.25)
        assert a is not None and b is not None and c is None     # third does not fit
        srv.close_stream(a)
        c = srv.open(256, 320, 15, 6, 3.0, 0.25)                 # memory freed: admitted now
        assert c is not None


def test_back_pressure_sheds_when_a_stream_queue_is_full():
    from paper_1408_3526_b300.serving import Server
    fr = scenes.small_scene(T=1, H=512, W=640, seed=3, tex_size=256).frames[0]
    with Server(budget_bytes=8e9, max_inflight=1, queue_limit=2, n_cuda_streams=1) as srv:
        s = srv.open(512, 640, 15, 6, 3.0, 0.25)
        got = [srv.submit(s, fr, srv.now()) for _ in range(20)]   # far faster than it is served
        srv.drain()
        st = srv.stats()
        assert st["shed"] >= 1 and st["shed"] + st["served"] == 20
        assert sum(r is None for r in got) == st["shed"]


def test_admission_charges_the_stream_parameters():
    """A stream with the frame pipeline (a second smoothed-state buffer) is
    refused at a budget that admits the serial stream of the same shape."""
    import ctypes as C

    from paper_1408_3526_b300.serving import Server
    lib = _abi.load()
    g = _abi.wh_vgrid(3.0, 0.25)
    serial = lib.wh_stream_device_bytes(256, 320, 15, 6, g)
    p = _abi.wh_params()
    assert lib.wh_default_params(15, 6, C.byref(p)) == 0
    p.pipeline = 1
    piped = lib.wh_stream_device_bytes_opt(256, 320, 15, 6, g, C.byref(p))
    assert piped >= serial + 256 * 320 * 228 * 4
    with Server(budget_bytes=serial + 1, max_inflight=1, queue_limit=1, n_cuda_streams=1) as srv:
        assert srv.open(256, 320, 15, 6, 3.0, 0.25, pipeline=True) is None
        assert srv.open(256, 320, 15, 6, 3.0, 0.25) is not None


def test_requests_are_forgotten_once_returned():
    """The request table stays bounded: a request id is returned once."""
    from paper_1408_3526_b300.serving import Server
    fr = scenes.small_scene(T=3, H=48, W=64, seed=9, tex_size=128).frames
    with Server(budget_bytes=2e9, max_inflight=2, queue_limit=4, n_cuda_streams=1, keep_results=True) as srv:
        s = srv.open(48, 64, 9, 4, 2.0, 0.25)
        rids = [srv.submit(s, fr[t], srv.now()) for t in range(3)]
        for r in rids:
            e, lat = srv.wait(r, s)
            assert e.shape == (48, 64) and lat >= 0
        with pytest.raises(Exception):
            srv.wait(rids[0], s)
