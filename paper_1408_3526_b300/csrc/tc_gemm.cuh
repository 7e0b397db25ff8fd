// Host interface of the tcgen05 GEMM (see tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>

namespace wh {

enum { EPI_F32 = 0, EPI_BF16 = 1, EPI_TOPK = 2 };

struct GemmArgs {
  int M, N, K;
  int bf16;             // 1: BF16 operands, 0: F16
  int epi;              // EPI_*
  int act;              // 1: GELU (tanh form) after the bias
  const float* bias;    // [N] or null
  void* C;              // EPI_F32: float [M][ldc]; EPI_BF16: bf16 [M][ldc]
  int ldc;
  float* preact;        // optional float [M][ldp] pre-activation (acc + bias)
  int ldp;
  float* cand_val;      // EPI_TOPK: [M][N tiles][4]
  int* cand_idx;
  int n_valid;          // EPI_TOPK: columns >= n_valid are ignored
  int* err;             // device error flag (0 = ok)
  int vec;              // set by tc_gemm: C (and preact) rows allow 16-byte vector stores
};

// A: [M][lda] K-major, B: [N][ldb] K-major (2-byte elements, 16-byte aligned rows).
// bn: N tile (64, 128 or 256).
cudaError_t tc_gemm(const GemmArgs& g, const void* A, int lda, const void* B, int ldb, int bn,
                    cudaStream_t st);

// Persistent autocorrelation shortlist (tc_rgemm.cu): per row of a16 [M][lda]
// (K <= 256), the 8 largest a16 . table[l] over l < n_valid, table
// [ntile*128][ldb]; candidates cval/cidx [M][8].  With l1 (per-row sum |a16|)
// given, values more than the re-rank's window below their 32-column chunk's
// maximum are skipped (they cannot matter to the exact re-rank).
cudaError_t tc_autocorr_shortlist(const void* a16, int lda, const void* table, int ldb, int M, int K,
                                  int ntile, int n_valid, bool bf16, const float* l1, float* cval,
                                  int* cidx, int* err, cudaStream_t st);

}  // namespace wh
