"""The pruned velocity search equals the full evaluation, bit for bit (needs a B300).

The search evaluates only the rows of the velocity grid whose upper bound
t0 + 2 sum_kx |T(kx, ly)| reaches the value of the most promising row.
`wh_read_autocorr` re-runs the search on the same smoothed state with every
grid value evaluated (and written out), overwriting the velocity field, so
reading the velocity before and after it compares the two on identical
inputs.  The full result is also checked against the dumped R: its flat index
is the lowest one holding the maximum.

Both pruned engines are covered: the CUDA-core search and the tensor-core
separable search (WH_PREC_TC_SEPARABLE), whose row bounds come from a TF32
tensor-core product widened by its rigorous error bound.

Scenes cover structured spectra (texture under flow, the paper's sinusoids,
an impulse), flat spectra (white noise: weak pruning), an all-tie state
(constant frames: R = 0 everywhere) and a non-finite state (a NaN frame: the
bound is NaN and every row is evaluated).
"""
import numpy as np
import pytest

from paper_1408_3526_b300 import scenes
from paper_1408_3526_b300.stream import WhitenStream

pytestmark = pytest.mark.gpu


def _frames(kind, T, H, W):
    rng = np.random.default_rng(17)
    if kind == "flow":
        sc = scenes.config2_scene(T=T, H=512, W=640)
        return np.ascontiguousarray(sc.frames[:, 100:100 + H, 200:200 + W])
    if kind == "paper_sim":
        return np.ascontiguousarray(scenes.paper_sim_scene(T=T, H=H, W=W).frames)
    if kind == "noise":
        return rng.standard_normal((T, H, W)).astype(np.float32)
    if kind == "constant":
        return np.full((T, H, W), 3.25, np.float32)
    if kind == "impulse":
        f = np.zeros((T, H, W), np.float32)
        for t in range(T):
            f[t, H // 2, (W // 3 + t) % W] = 100.0
        return f
    if kind == "nan":
        f = rng.standard_normal((T, H, W)).astype(np.float32)
        f[T // 2, H // 3, W // 4] = np.nan
        return f
    raise ValueError(kind)


def _lowest_argmax(R):
    """Flat index iy*L + ix of the first maximum of R [H][W][L][L] per pixel."""
    H, W = R.shape[:2]
    flat = R.reshape(H, W, -1)
    return np.argmax(flat, axis=-1)      # numpy returns the first occurrence


@pytest.mark.parametrize("precision", [0, 128, 32], ids=["cuda_cores", "tc_dense", "tc_separable"])
@pytest.mark.parametrize("kind", ["flow", "paper_sim", "noise", "constant", "impulse", "nan"])
@pytest.mark.parametrize("M,Mz,vmax,step", [(15, 6, 3.0, 0.25), (9, 4, 2.0, 0.25), (7, 5, 3.75, 0.25),
                                             (15, 6, 3.75, 0.25)])
def test_pruned_search_equals_full_evaluation(kind, M, Mz, vmax, step, precision):
    """Both pruned engines: the CUDA-core search (exact row bounds) and the
    tensor-core separable search (row bounds from the TF32 product, widened by
    its error bound): the velocity equals the full FP32 evaluation's bit for bit."""
    T, H, W = 10, 24, 40
    frames = _frames(kind, T, H, W)
    with WhitenStream(H, W, M, Mz, vmax, step, precision=precision) as s:
        for t in range(T):
            s.push(frames[t])
            if t < 1:
                continue
            _, _, vi_pruned, _ = s.read_velocity()
            R = s.read_autocorr()
            _, _, vi_full, _ = s.read_velocity()
            np.testing.assert_array_equal(vi_pruned, vi_full, err_msg=f"{kind} frame {t}")
            finite = np.isfinite(R).all(axis=(2, 3))
            ref = _lowest_argmax(R)
            np.testing.assert_array_equal(vi_full[finite], ref[finite], err_msg=f"{kind} frame {t}")
            if kind == "constant":
                assert (vi_full == 0).all()
