"""GPU path vs the FP64 oracle on seeded random shapes (needs a B300).

Each case draws a window and temporal order the kernels support, a grid
inside the unambiguous range |v| <= (M - 1)/2 (R is M-periodic in l) and the
search's length limit, a frame size from a few pixels to several
tiles with ragged edges, and a translating texture inside the grid, then
applies the same acceptance bar as the other parity tests (spectra, power,
autocorrelation, velocity within one grid step with mismatches only at near
ties, whitened output).  The velocity agreement fraction is not asserted:
on frames this small one near tie is a large fraction.
"""
import numpy as np
import pytest

from paper_1408_3526_b300 import scenes
from tests.test_gpu_parity import _compare

pytestmark = pytest.mark.gpu

SUPPORTED = {5: (3, 4, 5, 6), 7: (3, 4, 5, 6), 9: (3, 4, 5, 6), 15: (4, 5, 6)}


def _cases(n=10, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = int(rng.choice(list(SUPPORTED)))
        Mz = int(rng.choice(SUPPORTED[M]))
        step = float(rng.choice([0.25, 0.5]))
        # R is periodic in l with period M, so a grid spanning M or more holds
        # exact duplicates of its maximum (decided by rounding): stay inside
        # |v| <= (M - 1) / 2, the unambiguous range
        lmax = min(31, int(2 * ((M - 1) / 2) / step) + 1)
        L = int(rng.choice(np.arange(5, lmax + 1, 2)))
        vmax = (L - 1) / 2 * step
        H, W = int(rng.integers(6, 49)), int(rng.integers(6, 61))
        vx, vy = (float(v) for v in rng.uniform(-0.8, 0.8, 2) * min(vmax, 2.0))
        out.append((i, M, Mz, vmax, step, H, W, vx, vy))
    return out


@pytest.mark.parametrize("precision", [0, 128, 16, 32],
                         ids=["cuda_cores", "tc_dense", "tc_shortlist_rerank", "tc_separable"])
@pytest.mark.parametrize("i,M,Mz,vmax,step,H,W,vx,vy", _cases(),
                         ids=lambda v: str(v) if isinstance(v, int) else None)
def test_parity_random_shape(i, M, Mz, vmax, step, H, W, vx, vy, precision):
    """The three FP32-exact search engines (the tensor-core shortlist takes
    grids up to 25 points per axis)."""
    if precision == 16 and 2 * vmax / step + 1 > 25:
        pytest.skip("tensor-core search: grid longer than 25")
    T = 8
    sc = scenes.small_scene(T=T, H=H, W=W, seed=100 + i, vx=vx, vy=vy, tex_size=128)
    _compare(sc.frames, M, Mz, vmax, step, spec_frames=(T - 1,), check_vel_frac=False,
             precision=precision)


@pytest.mark.parametrize("M,Mz", [(M, Mz) for M in SUPPORTED for Mz in SUPPORTED[M]])
def test_parity_every_window_and_order(M, Mz):
    """Every compiled (window, temporal order) of the spectrum kernel against
    the oracle on a frame of several strips with a ragged last strip: each has
    its own compile-time tile width, x-DFT split, observer-row stride and lane
    order (Eq. (6)-(10), Eq. (1)-(2))."""
    T = 8
    sc = scenes.small_scene(T=T, H=20, W=67, seed=300 + 10 * M + Mz, vx=0.6, vy=-0.4, tex_size=128)
    _compare(sc.frames, M, Mz, 1.5, 0.5, spec_frames=(T - 1,), check_vel_frac=False)
