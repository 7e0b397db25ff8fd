"""Failure detection without a GPU fault (needs a B300): a bounded device
wait that nothing completes gives up, the host reads WH_ETIMEOUT, and the
context and the stream stay usable."""
import numpy as np
import pytest

from paper_1408_3526_b300 import _abi

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    from paper_1408_3526_b300.stream import WhitenStream
    lib = _abi.load()
    assert lib.wh_selftest_wait_timeout(2000, None) == _abi.WH_ETIMEOUT
    # the same context keeps working: a stream runs and a second self-test passes too
    with WhitenStream(32, 40, 5, 3, 1.0, 0.25) as s:
        for _ in range(3):
            s.push(np.random.default_rng(0).standard_normal((32, 40)).astype(np.float32))
        vx = s.read_velocity()[0]
        assert np.isfinite(vx).all()
    assert lib.wh_selftest_wait_timeout(1000, None) == _abi.WH_ETIMEOUT


def test_stream_status_word_reported_once():
    from paper_1408_3526_b300.stream import WhitenStream
    with WhitenStream(32, 40, 5, 3, 1.0, 0.25) as s:
        s.push(np.zeros((32, 40), np.float32))
        assert s.lib.wh_stream_sync(s._s) == _abi.WH_OK
        assert s.lib.wh_stream_selftest_status(s._s, 7) == _abi.WH_OK
        assert s.lib.wh_stream_sync(s._s) == _abi.WH_ETIMEOUT
        assert s.lib.wh_stream_sync(s._s) == _abi.WH_OK          # cleared after the report
        assert s.lib.wh_stream_selftest_status(s._s, 3) == _abi.WH_OK
        with pytest.raises(Exception):
            s.read_velocity()                                      # a host read reports it too
        s.push(np.zeros((32, 40), np.float32))
        s.read_velocity()
