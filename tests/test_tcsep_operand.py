"""The constant operand of the tensor-core separable search (host logic, no
GPU): multiplied with a pixel's Q sums it gives T(kx, l) = sum_ky Q(kx, ky)
e^{j2pi ky l/M} on every grid row (the separable form of Eq. (10)), within the
TF32 rounding of its entries; the error of the whole tensor-core product with
TF32 operands stays inside the bound widening the search uses, and the
entries sit in the 128-byte-swizzled layout the tensor cores read."""
import ctypes as C

import numpy as np
import pytest

from paper_1408_3526_b300 import _abi, build

WIDEN = 4.5e-3      # the search's bound widening per unit of sum |Q sums|


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def _operand(lib, M, L, step):
    out = np.zeros(64 * 32, np.float32)
    assert lib.wh_tcsep_operand(M, L, step, C.c_void_p(out.ctypes.data)) == 0
    B = np.zeros((64, 32))
    for n in range(64):
        for k in range(32):
            B[n, k] = out[n * 32 + (((k >> 2) ^ (n & 7)) << 2) + (k & 3)]
    return out, B


def _qsums(Q, K):
    """Row of the A operand of one (pixel, kx): Q over ky = -K..K (index ky + K)."""
    a = np.zeros(32)
    for ky in range(1, K + 1):
        p, m = Q[K + ky], Q[K - ky]
        a[4 * (ky - 1):4 * ky] = [p.real + m.real, p.real - m.real, p.imag + m.imag, p.imag - m.imag]
    a[28], a[29] = Q[K].real, Q[K].imag
    return a


def _tf32(x):
    """Truncation to 10 explicit mantissa bits (the worst a TF32 operand can lose)."""
    u = np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return u.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("M,L,step", [(15, 25, 0.25), (9, 17, 0.25), (5, 31, 0.1), (7, 1, 0.5)])
def test_operand_gives_T_on_every_row(lib, M, L, step):
    K, gc = (M - 1) // 2, (L - 1) // 2
    raw, B = _operand(lib, M, L, step)
    # TF32 values: the low 13 bits of every entry are zero; rows past 2L and
    # columns 30, 31 (and ky > K) are zero
    assert np.all(raw.view(np.uint32) & np.uint32(0x1FFF) == 0)
    assert np.all(B[2 * L:] == 0) and np.all(B[:, 30:] == 0) and np.all(B[:, 4 * K:28] == 0)
    rng = np.random.default_rng(M * 100 + L)
    ky = np.arange(-K, K + 1)
    lv = (np.arange(L) - gc) * step
    for trial in range(20):
        Q = rng.normal(0, 1, 2 * K + 1) + 1j * rng.normal(0, 1, 2 * K + 1)
        Q *= 10.0 ** rng.uniform(-3, 3)
        if trial % 4 == 0:               # kx = 0: Hermitian in ky
            Q[K] = Q[K].real
            Q[:K] = np.conj(Q[K + 1:][::-1])
        a = _qsums(Q, K)
        T = np.array([np.sum(Q * np.exp(2j * np.pi * ky * l / M)) for l in lv])
        got = B[:2 * L] @ a
        s1 = np.sum(np.abs(a))
        err = np.abs((got[0::2] + 1j * got[1::2]) - T)
        assert np.max(err) <= 2 ** -10 * s1, (np.max(err), s1)        # B entries rounded to TF32
        # the tensor-core product: A entries truncated to TF32 as well
        got_tc = B[:2 * L] @ _tf32(a)
        err_tc = np.abs((got_tc[0::2] + 1j * got_tc[1::2]) - T)
        assert np.max(err_tc) <= np.sqrt(2) * 1.53 * 2 ** -10 * s1
        if trial % 4 == 0:
            assert np.max(np.abs(got[1::2])) <= 2 ** -10 * s1         # T(0, l) is real


def test_widening_covers_the_row_bound_error(lib):
    """Per pixel, W = 4.5e-3 x sum |Q sums| covers the error of the row bound
    t0 + 2 sum_{kx >= 1} |T(kx, l)| computed from TF32 products."""
    M, L, step = 15, 25, 0.25
    K, gc = (M - 1) // 2, (L - 1) // 2
    _, B = _operand(lib, M, L, step)
    rng = np.random.default_rng(5)
    ky = np.arange(-K, K + 1)
    lv = (np.arange(L) - gc) * step
    for _ in range(30):
        Qs = [rng.normal(0, 1, 2 * K + 1) + 1j * rng.normal(0, 1, 2 * K + 1) for _ in range(K + 1)]
        Qs[0][K] = Qs[0][K].real
        Qs[0][:K] = np.conj(Qs[0][K + 1:][::-1])
        rows = [_qsums(Q, K) for Q in Qs]
        S = sum(np.sum(np.abs(a)) for a in rows)
        T = np.array([[np.sum(Q * np.exp(2j * np.pi * ky * l / M)) for l in lv] for Q in Qs])
        ub = T[0].real + 2 * np.abs(T[1:]).sum(0)
        Tt = np.array([B[:2 * L] @ _tf32(a) for a in rows])
        Tt = Tt[:, 0::2] + 1j * Tt[:, 1::2]
        ubt = Tt[0].real + 2 * np.abs(Tt[1:]).sum(0)
        assert np.max(np.abs(ubt - ub)) <= WIDEN * S
