"""tcgen05 GEMM through the C ABI vs a plain PyTorch FP32 reference (needs a B300)."""
import ctypes as C

import numpy as np
import pytest

from paper_1408_3526_b300 import _abi

pytestmark = pytest.mark.gpu


def _gemm(A, B, out_bf16=False, bias=None, gelu=False):
    import torch
    lib = _abi.load()
    M, K = A.shape
    N = B.shape[0]
    Cm = torch.empty((M, N), dtype=torch.bfloat16 if out_bf16 else torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = lib.wh_tc_gemm(C.c_void_p(A.data_ptr()), A.stride(0), C.c_void_p(B.data_ptr()), B.stride(0),
                        C.c_void_p(Cm.data_ptr()), N, M, N, K, int(A.dtype == torch.bfloat16),
                        int(out_bf16), C.c_void_p(bias.data_ptr()) if bias is not None else None,
                        int(gelu), C.c_void_p(st))
    assert rc == 0, rc
    return Cm


@pytest.mark.parametrize("M,N,K,bf16", [(256, 128, 256, False), (300, 200, 1350, True),
                                        (130, 16, 128, True), (512, 640, 232, False),
                                        (1000, 256, 64, True), (128, 3, 128, False),
                                        # many output tiles: the persistent, double-buffered kernel
                                        (76837, 128, 1350, True), (80000, 100, 232, False),
                                        (80000, 40, 256, True),
                                        # tall and wide: 256 x 256 tiles (two 128-row sub-tiles)
                                        (40000, 256, 1350, True), (45001, 200, 232, False)])
def test_tc_gemm_matches_torch(M, N, K, bf16):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N)
    dt = torch.bfloat16 if bf16 else torch.float16
    ld = (K + 7) // 8 * 8
    Abuf = torch.randn((M, ld), generator=g, device="cuda").to(dt)
    Bbuf = torch.randn((N, ld), generator=g, device="cuda").to(dt)
    A, B = Abuf[:, :K], Bbuf[:, :K]
    Cm = _gemm(A, B)
    ref = A.float() @ B.float().T
    err = (Cm - ref).abs().max().item()
    assert err <= 1e-4 * K ** 0.5 * ref.abs().max().item() + 1e-3, err


def test_tc_gemm_bias_gelu_bf16_out():
    import torch
    g = torch.Generator(device="cuda").manual_seed(3)
    M, N, K = 777, 256, 1352
    A = torch.randn((M, K), generator=g, device="cuda").to(torch.bfloat16) * 0.05
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16) * 0.05
    bias = torch.randn((N,), generator=g, device="cuda")
    Cm = _gemm(A, B, out_bf16=True, bias=bias, gelu=True)
    ref = torch.nn.functional.gelu(A.float() @ B.float().T + bias, approximate="tanh")
    assert (Cm.float() - ref).abs().max().item() < 2e-2


def test_tc_gemm_persistent_bias_gelu_preact():
    """Many tiles (persistent kernel), ragged M and N, bias + GELU, BF16 output."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(11)
    M, N, K = 150 * 128 * 4 + 77, 120, 256
    A = torch.randn((M, K), generator=g, device="cuda").to(torch.bfloat16) * 0.05
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16) * 0.05
    bias = torch.randn((N,), generator=g, device="cuda")
    Cm = _gemm(A, B, out_bf16=True, bias=bias, gelu=True)
    ref = torch.nn.functional.gelu(A.float() @ B.float().T + bias, approximate="tanh")
    assert (Cm.float() - ref).abs().max().item() < 2e-2


def test_tc_gemm_tall_wide_bias_gelu_bf16_out():
    """256 x 256 tiles (M above two tile rows per SM), ragged M, bias + GELU,
    BF16 output: the first layer's shape."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(21)
    M, N, K = 148 * 256 + 1234, 256, 1352
    A = torch.randn((M, K), generator=g, device="cuda").to(torch.bfloat16) * 0.05
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.bfloat16) * 0.05
    bias = torch.randn((N,), generator=g, device="cuda")
    Cm = _gemm(A, B, out_bf16=True, bias=bias, gelu=True)
    ref = torch.nn.functional.gelu(A.float() @ B.float().T + bias, approximate="tanh")
    assert (Cm.float() - ref).abs().max().item() < 2e-2


def test_tc_gemm_topk_epilogue():
    import torch
    lib = _abi.load()
    g = torch.Generator(device="cuda").manual_seed(5)
    M, N, K, nvalid = 1000, 640, 232, 625
    A = torch.randn((M, K), generator=g, device="cuda").to(torch.float16)
    B = torch.randn((N, K), generator=g, device="cuda").to(torch.float16)
    nt = (N + 127) // 128
    cv = torch.empty((M, nt, 4), device="cuda")
    ci = torch.empty((M, nt, 4), dtype=torch.int32, device="cuda")
    rc = lib.wh_tc_gemm_topk(C.c_void_p(A.data_ptr()), K, C.c_void_p(B.data_ptr()), K, M, N, K, 0,
                             nvalid, C.c_void_p(cv.data_ptr()), C.c_void_p(ci.data_ptr()),
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    ref = (A.float() @ B.float().T)[:, :nvalid]
    best = cv.reshape(M, -1).argmax(1)
    got = ci.reshape(M, -1).gather(1, best[:, None])[:, 0]
    agree = (got == ref.argmax(1)).float().mean().item()
    assert agree > 0.999, agree
    top4 = torch.topk(ref[:, :128], 4, dim=1)
    assert (ci[:, 0, :] == top4.indices).float().mean().item() > 0.995
