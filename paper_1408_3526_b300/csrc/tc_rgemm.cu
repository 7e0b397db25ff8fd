// Persistent tcgen05 contraction for the autocorrelation shortlist:
//   D[p][l] = sum_k a16[p][k] B[l][k]   (K <= 256, N = ntile * 128 grid columns)
// and, per pixel p, the 8 largest D[p][l] over l < n_valid (ties -> lowest l).
//
// One CTA per SM loops over 128-pixel tiles.  A tile's operand rows (K = 4
// blocks of 64 F16 = 64 KB, 128-byte swizzle) are loaded once and stay in
// shared memory (double-buffered across tiles) while every 128-column block of
// the grid table streams through a 4-stage ring.  Two TMEM accumulators
// (2 x 128 columns) let the epilogue of column block n overlap the MMAs of
// block n + 1; the epilogue keeps each row's top 8 across all column blocks, so
// the shortlist leaves the kernel complete.  Warp 0: TMA producer; warp 1: MMA
// issuer; warps 2-5: epilogue (one TMEM lane quadrant each).  Every wait is
// bounded (~1 s) and a timeout sets *err and stops the CTA's work.
#include <cuda.h>

#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace wh {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;
constexpr int kKB = 4;            // K blocks resident (K <= 256)
constexpr int kBS = 4;            // B ring stages
constexpr int kTop = 8;
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint32_t kTileBytes = kBM * kBK * 2;   // 16 KB per 128 x 64 F16 block

struct RGemmArgs {
  int M, ntile, nkb, n_valid, bf16;
  const float* l1;      // per-row sum |a16| (error window), may be null
  float* cval;
  int* cidx;
  int* err;
};

__global__ void __launch_bounds__(192, 1)
    rgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                 const RGemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
  uint8_t* sA = smem;                                   // [2][kKB][16 KB]
  uint8_t* sB = sA + 2 * kKB * kTileBytes;              // [kBS][16 KB]
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + kBS * kTileBytes);
  uint64_t* a_full = bar;            // [2]
  uint64_t* a_empty = bar + 2;       // [2]
  uint64_t* b_full = bar + 4;        // [kBS]
  uint64_t* b_empty = bar + 4 + kBS; // [kBS]
  uint64_t* c_full = bar + 4 + 2 * kBS;     // [2]
  uint64_t* c_empty = bar + 6 + 2 * kBS;    // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 8 + 2 * kBS);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nm = (g.M + kBM - 1) / kBM;
  const int G = gridDim.x;

  if (warp == 0) {
    if (lane == 0) {
      for (int i = 0; i < 2; ++i) {
        tc::mbar_init(&a_full[i], 1);
        tc::mbar_init(&a_empty[i], 1);
        tc::mbar_init(&c_full[i], 1);
        tc::mbar_init(&c_empty[i], 4);
      }
      for (int s = 0; s < kBS; ++s) {
        tc::mbar_init(&b_full[s], 1);
        tc::mbar_init(&b_empty[s], 1);
      }
      *abort_flag = 0;
      tc::fence_mbar_init();
      tc::tma_prefetch_desc(&tmA);
      tc::tma_prefetch_desc(&tmB);
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, 2 * kBN);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  auto fail = [&](int code) {
    atomicExch(g.err, code);
    *abort_flag = 1;
  };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int bc = 0;
    for (int j = 0; !*abort_flag; ++j) {
      const int m = blockIdx.x + j * G;
      if (m >= nm) break;
      const int ab = j & 1;
      if (j >= 2 && !tc::mbar_wait(&a_empty[ab], ((j >> 1) - 1) & 1, kWaitNs)) { fail(11); break; }
      tc::mbar_expect_tx(&a_full[ab], g.nkb * kTileBytes);
      for (int kb = 0; kb < g.nkb; ++kb)
        tc::tma_load_2d(sA + (ab * kKB + kb) * kTileBytes, &tmA, &a_full[ab], kb * kBK, m * kBM);
      bool ok = true;
      for (int n = 0; n < g.ntile && ok; ++n)
        for (int kb = 0; kb < g.nkb; ++kb, ++bc) {
          const int s = bc % kBS;
          if (bc >= kBS && !tc::mbar_wait(&b_empty[s], ((bc / kBS) - 1) & 1, kWaitNs)) {
            fail(12);
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&b_full[s], kTileBytes);
          tc::tma_load_2d(sB + s * kTileBytes, &tmB, &b_full[s], kb * kBK, n * kBN);
        }
      if (!ok) break;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = tc::idesc_f16(kBM, kBN, g.bf16 != 0);
    int bc = 0, tcount = 0;
    bool ok = true;
    for (int j = 0; ok; ++j) {
      const int m = blockIdx.x + j * G;
      if (m >= nm) break;
      const int ab = j & 1;
      if (!tc::mbar_wait(&a_full[ab], (j >> 1) & 1, kWaitNs)) { fail(13); ok = false; break; }
      tc::tc_fence_after();
      for (int n = 0; n < g.ntile && ok; ++n, ++tcount) {
        const int acc = tcount & 1;
        if (tcount >= 2 && !tc::mbar_wait(&c_empty[acc], ((tcount >> 1) - 1) & 1, kWaitNs)) {
          fail(14);
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const uint32_t d = tmem + uint32_t(acc * kBN);
        for (int kb = 0; kb < g.nkb; ++kb, ++bc) {
          const int s = bc % kBS;
          if (!tc::mbar_wait(&b_full[s], (bc / kBS) & 1, kWaitNs)) { fail(15); ok = false; break; }
          tc::tc_fence_after();
          const uint32_t a0 = tc::smem_u32(sA + (ab * kKB + kb) * kTileBytes);
          const uint32_t b0 = tc::smem_u32(sB + s * kTileBytes);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            tc::mma_f16(d, tc::sdesc_sw128(a0 + 32 * k), tc::sdesc_sw128(b0 + 32 * k), idesc,
                        (kb > 0 || k > 0) ? 1u : 0u);
          tc::mma_commit(&b_empty[s]);
        }
        if (ok) tc::mma_commit(&c_full[acc]);
      }
      if (ok) tc::mma_commit(&a_empty[ab]);
    }
    if (!ok) {                       // release the epilogue so it can see the flag and stop
      tc::mbar_arrive(&c_full[0]);
      tc::mbar_arrive(&c_full[1]);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue: running top-8 per row ----------------
    const int q = warp & 3;
    int tcount = 0;
    bool ok = true;
    for (int j = 0; ok; ++j) {
      const int m = blockIdx.x + j * G;
      if (m >= nm) break;
      const int row = m * kBM + q * 32 + lane;
      // twice the error bound of the re-rank (must match ac_rerank_kernel)
      const float win2 = (g.l1 && row < g.M) ? 2.f * (2.05e-3f * g.l1[row] + 2e-5f) : INFINITY;
      float tv[kTop];
      int ti[kTop];
#pragma unroll
      for (int t = 0; t < kTop; ++t) { tv[t] = -INFINITY; ti[t] = 0x7fffffff; }
      for (int n = 0; n < g.ntile; ++n, ++tcount) {
        const int acc = tcount & 1;
        const bool w = tc::mbar_wait(&c_full[acc], (tcount >> 1) & 1, 4 * kWaitNs);
        if (!w) fail(16);
        tc::tc_fence_after();
        if (!w || *abort_flag) { ok = false; break; }
#pragma unroll 1
        for (int c = 0; c < kBN / 32; ++c) {
          uint32_t r[32];
          tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * kBN + c * 32), r);
          tc::tmem_ld_wait();
          const int col0 = n * kBN + c * 32;
          // Values below (chunk max - 2E) cannot be within the re-rank window of
          // the row's maximum (which is >= the chunk max): skip them cheaply.
          float cm = -INFINITY;
#pragma unroll
          for (int jj = 0; jj < 32; ++jj)
            if (col0 + jj < g.n_valid) cm = fmaxf(cm, __uint_as_float(r[jj]));
          const float thr = fmaxf(tv[kTop - 1], cm - win2);
          if (cm <= tv[kTop - 1]) continue;
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            float cv = __uint_as_float(r[jj]);
            int ci = col0 + jj;
            if (ci < g.n_valid && cv >= thr && cv > tv[kTop - 1]) {
#pragma unroll
              for (int t = 0; t < kTop; ++t) {
                if (cv > tv[t]) {
                  const float fv = tv[t];
                  const int fi = ti[t];
                  tv[t] = cv; ti[t] = ci;
                  cv = fv; ci = fi;
                }
              }
            }
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&c_empty[acc]);
      }
      if (ok && row < g.M) {
#pragma unroll
        for (int t = 0; t < kTop; ++t) {
          g.cval[size_t(row) * kTop + t] = tv[t];
          g.cidx[size_t(row) * kTop + t] = ti[t];
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * kBN);
  }
}

}  // namespace

bool make_map_2b(CUtensorMap* m, const void* ptr, int rows, int K, int ld, int box_rows, bool bf16);

// a16: [M][lda] (K <= 256 valid columns), table: [ntile*128][ldb]; candidates [M][8].
cudaError_t tc_autocorr_shortlist(const void* a16, int lda, const void* table, int ldb, int M, int K,
                                  int ntile, int n_valid, bool bf16, const float* l1, float* cval,
                                  int* cidx, int* err, cudaStream_t st) {
  if (K > kKB * kBK || M < 1 || ntile < 1) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map_2b(&ma, a16, M, K, lda, kBM, bf16) || !make_map_2b(&mb, table, ntile * kBN, K, ldb, kBN, bf16))
    return cudaErrorInvalidValue;
  RGemmArgs g{};
  g.M = M; g.ntile = ntile; g.nkb = (K + kBK - 1) / kBK; g.n_valid = n_valid; g.bf16 = bf16 ? 1 : 0;
  g.l1 = l1; g.cval = cval; g.cidx = cidx; g.err = err;
  const size_t smem = 1024 + size_t(2 * kKB + kBS) * kTileBytes + (8 + 2 * kBS) * 8 + 16;
  cudaError_t e = cudaFuncSetAttribute(rgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int nm = (M + kBM - 1) / kBM;
  const int grid = nm < nsm ? nm : nsm;
  rgemm_kernel<<<grid, 192, smem, st>>>(ma, mb, g);
  return cudaGetLastError();
}

}  // namespace wh
