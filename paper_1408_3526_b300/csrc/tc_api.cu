// C ABI of the tensor-core GEMM (used by the learned velocity estimator and
// the autocorrelation contraction; exported for direct use and testing).
#include <cstdio>

#include "../../include/whiten.h"
#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

using namespace wh;

namespace {
// Self-test of the bounded device-side wait: one thread arms an mbarrier that
// expects two arrivals, arrives once, and waits with the production helper;
// the phase never completes, so the wait gives up after limit_ns and the
// kernel records it in *flag and returns (no hang, no fault).
__global__ void wait_selftest_kernel(uint64_t limit_ns, int* flag) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 2);
  tc::fence_mbar_init();
  tc::mbar_arrive(&bar);
  if (!tc::mbar_wait(&bar, 0, limit_ns)) atomicExch(flag, 1);
}

thread_local char g_err2[256] = "";
// One error flag per (host thread, device): concurrent calls from different
// threads never share a flag.  (Allocated once per thread and device; freed at
// process exit with the context.)
int* device_err_flag() {
  thread_local int* flags[64] = {nullptr};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!flags[dev]) {
    if (cudaMalloc(&flags[dev], sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(flags[dev], 0, sizeof(int));
  }
  return flags[dev];
}
}  // namespace

extern "C" int wh_tc_gemm(const void* A, int lda, const void* B, int ldb, void* C, int ldc, int M, int N,
                          int K, int bf16, int out_bf16, const float* bias, int gelu, void* cuda_stream) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N) return WH_EINVAL;
  int* err = device_err_flag();
  if (!err) return WH_ENOMEM;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.bf16 = bf16 ? 1 : 0;
  g.epi = out_bf16 ? EPI_BF16 : EPI_F32; g.act = gelu ? 1 : 0; g.bias = bias;
  g.C = C; g.ldc = ldc; g.err = err;
  const int bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  cudaError_t e = tc_gemm(g, A, lda, B, ldb, bn, st);
  if (e != cudaSuccess) return WH_EINVAL;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WH_ECUDA;
  if (h) {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    return WH_ETIMEOUT;
  }
  return WH_OK;
}

extern "C" int wh_tc_gemm_topk(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                               int bf16, int n_valid, float* cand_val, int* cand_idx, void* cuda_stream) {
  if (!A || !B || !cand_val || !cand_idx || M < 1 || N < 1 || K < 1) return WH_EINVAL;
  int* err = device_err_flag();
  if (!err) return WH_ENOMEM;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.bf16 = bf16 ? 1 : 0; g.epi = EPI_TOPK;
  g.cand_val = cand_val; g.cand_idx = cand_idx; g.n_valid = n_valid; g.err = err;
  cudaError_t e = tc_gemm(g, A, lda, B, ldb, 128, st);
  if (e != cudaSuccess) return WH_EINVAL;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WH_ECUDA;
  if (h) {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    return WH_ETIMEOUT;
  }
  return WH_OK;
}

extern "C" int wh_selftest_wait_timeout(int limit_us, void* cuda_stream) {
  if (limit_us < 1 || limit_us > 1000000) return WH_EINVAL;
  int* err = device_err_flag();
  if (!err) return WH_ENOMEM;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(err, 0, sizeof(int), st) != cudaSuccess) return WH_ECUDA;
  wait_selftest_kernel<<<1, 32, 0, st>>>(uint64_t(limit_us) * 1000ull, err);
  if (cudaGetLastError() != cudaSuccess) return WH_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return WH_ECUDA;
  if (h) {
    cudaMemsetAsync(err, 0, sizeof(int), st);
    return WH_ETIMEOUT;
  }
  return WH_OK;
}
