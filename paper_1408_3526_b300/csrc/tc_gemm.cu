// Tensor-core GEMM on tcgen05 (sm_103a): C[M x N] = A[M x K] * B[N x K]^T
// with F16 or BF16 operands (both K-major in HBM), F32 accumulation in TMEM.
//
// One CTA computes a 128 x BN tile.  Warp roles:
//   warp 0  TMA producer (one lane): A and B 64-wide K blocks into a 4-stage
//           ring of 128-byte-swizzled shared-memory tiles (mbarrier full/empty)
//   warp 1  MMA issuer (one lane): 4 x tcgen05.mma (K = 16 each) per K block,
//           tcgen05.commit frees the stage; a final commit signals the epilogue
//   warps 2-5  epilogue: tcgen05.ld of their 32-lane TMEM quadrant, 32 columns
//           at a time, then the selected epilogue.
// Every wait is bounded (about one second); on timeout the CTA records an
// error code in *err, stops issuing work, and still frees its TMEM.
//
// Epilogues:
//   EPI_F32    C (float) = acc (+ bias[col]) (GELU if act)
//   EPI_BF16   C (bf16)  = GELU?(acc + bias[col]); optional pre-activation (float)
//   EPI_TOPK   per row, the 4 largest columns (value, index) of this N tile among
//              the first n_valid columns, ties to the lowest index, written to
//              cand_val/cand_idx[row][tile][4]
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "tc_gemm.cuh"
#include "tc_ptx.cuh"

namespace wh {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;          // 64 two-byte elements = one 128-byte swizzle row
constexpr int kStages = 4;
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s

// GELU, tanh form, through the identity 0.5 z (1 + tanh u) = z / (1 + e^{-2u}),
// u = sqrt(2/pi) (z + 0.044715 z^3): one hardware exponential and one fast
// divide per value instead of the branchy library tanh (the epilogue of a
// 256 x 256 tile evaluates 65536 of them while no MMA of the CTA can run).
// Where e^{-2u} overflows (z below about -10) the quotient is -0, the limit.
__device__ __forceinline__ float gelu_tanh(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float u = k0 * fmaf(k1 * x, x * x, x);
  return __fdividef(x, 1.f + __expf(-2.f * u));
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
  uint8_t* sA = smem;                                    // kStages x 16 KB
  uint8_t* sB = smem + kStages * kBM * kBK * 2;          // kStages x BN*128 B
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * BN * kBK * 2);
  uint64_t* empty = full + kStages;
  uint64_t* accum = empty + kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* bias_s = reinterpret_cast<float*>(tmem_slot + 4);      // [BN] bias of this N tile

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int nk = (g.K + kBK - 1) / kBK;
  constexpr uint32_t kStageBytes = (kBM + BN) * kBK * 2;

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < kStages; ++s) {
        tc::mbar_init(&full[s], 1);
        tc::mbar_init(&empty[s], 1);
      }
      tc::mbar_init(accum, 1);
      *abort_flag = 0;
      tc::fence_mbar_init();
      tc::tma_prefetch_desc(&tmA);
      tc::tma_prefetch_desc(&tmB);
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, BN);
    tc::tmem_relinquish();
  }
  if (warp >= 2)
    for (int i = threadIdx.x - 64; i < BN; i += 128)
      bias_s[i] = (g.bias && n0 + i < g.N) ? g.bias[n0 + i] : 0.f;
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      const uint32_t use = kb / kStages;
      if (kb >= kStages && !tc::mbar_wait(&empty[s], (use & 1) ^ 1, kWaitNs)) {
        atomicExch(g.err, 1);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      tc::mbar_expect_tx(&full[s], kStageBytes);
      tc::tma_load_2d(sA + s * kBM * kBK * 2, &tmA, &full[s], kb * kBK, m0);
      tc::tma_load_2d(sB + s * BN * kBK * 2, &tmB, &full[s], kb * kBK, n0);
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = tc::idesc_f16(kBM, BN, g.bf16 != 0);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      const uint32_t use = kb / kStages;
      if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
        atomicExch(g.err, 2);
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t a0 = tc::smem_u32(sA + s * kBM * kBK * 2);
      const uint32_t b0 = tc::smem_u32(sB + s * BN * kBK * 2);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k) {
        tc::mma_f16(tmem, tc::sdesc_sw128(a0 + 32 * k), tc::sdesc_sw128(b0 + 32 * k), idesc,
                    (kb > 0 || k > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[s]);
    }
    if (ok) tc::mma_commit(accum);
    else tc::mbar_arrive(accum);          // release the epilogue (it checks the flag)
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                   // TMEM lane quadrant of this warp
    const int row = m0 + q * 32 + lane;
    const bool waited = tc::mbar_wait(accum, 0, 4 * kWaitNs);
    if (!waited) atomicExch(g.err, 3);
    tc::tc_fence_after();
    const bool live = waited && (*abort_flag == 0);
    float tv[4];
    int ti[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) { tv[t] = -INFINITY; ti[t] = 0x7fffffff; }
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      uint32_t r[32];
      if (live) {
        tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c * 32), r);
        tc::tmem_ld_wait();
      }
      if (!live || row >= g.M) continue;
      const int col0 = n0 + c * 32;
      if (g.epi == EPI_TOPK) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = col0 + j;
          const float v = __uint_as_float(r[j]);
          if (col < g.n_valid && v > tv[3]) {
            // insert keeping descending order (earlier columns win ties)
            if (v > tv[0]) { tv[3] = tv[2]; ti[3] = ti[2]; tv[2] = tv[1]; ti[2] = ti[1]; tv[1] = tv[0]; ti[1] = ti[0]; tv[0] = v; ti[0] = col; }
            else if (v > tv[1]) { tv[3] = tv[2]; ti[3] = ti[2]; tv[2] = tv[1]; ti[2] = ti[1]; tv[1] = v; ti[1] = col; }
            else if (v > tv[2]) { tv[3] = tv[2]; ti[3] = ti[2]; tv[2] = v; ti[2] = col; }
            else { tv[3] = v; ti[3] = col; }
          }
        }
      } else if (g.vec && col0 + 32 <= g.N) {
        // a full 32-column chunk of this thread's row: 16-byte vector stores
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + bias_s[c * 32 + j];
        if (g.preact) {
          float4* pp = reinterpret_cast<float4*>(g.preact + size_t(row) * g.ldp + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q) pp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        if (g.act) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = gelu_tanh(v[j]);
        }
        if (g.epi == EPI_F32) {
          float4* cp = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.C) + size_t(row) * g.ldc + col0);
#pragma unroll
          for (int q = 0; q < 8; ++q) cp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
          uint4* cp = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.C) + size_t(row) * g.ldc + col0);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
              w[e] = *reinterpret_cast<const uint32_t*>(&h2);
            }
            cp[q] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = col0 + j;
          if (col >= g.N) break;
          float v = __uint_as_float(r[j]) + bias_s[c * 32 + j];
          if (g.preact) g.preact[size_t(row) * g.ldp + col] = v;
          if (g.act) v = gelu_tanh(v);
          if (g.epi == EPI_F32) reinterpret_cast<float*>(g.C)[size_t(row) * g.ldc + col] = v;
          else reinterpret_cast<__nv_bfloat16*>(g.C)[size_t(row) * g.ldc + col] = __float2bfloat16(v);
        }
      }
    }
    if (live && g.epi == EPI_TOPK && row < g.M) {
      const size_t o = (size_t(row) * gridDim.y + blockIdx.y) * 4;
#pragma unroll
      for (int t = 0; t < 4; ++t) { g.cand_val[o + t] = tv[t]; g.cand_idx[o + t] = ti[t]; }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, BN);
  }
}

// Persistent variant for many output tiles (EPI_F32 / EPI_BF16): one CTA per
// SM walks the 128 x BN tiles t = blockIdx.x, +gridDim.x, ... (N tiles
// fastest).  A and B K-blocks stream through one 4-stage ring whose counters
// run on across tiles; the accumulator is double-buffered in TMEM (2 x BN
// columns), so the epilogue of one tile overlaps the loads and MMAs of the
// next.  Same warp roles, bounded waits and error flag as tc_gemm_kernel.
template <int BN>
__device__ __forceinline__ void epilogue_chunk(const GemmArgs& g, const uint32_t (&r)[32], int row, int col0,
                                               const float* bias) {
  if (row >= g.M) return;
  if (g.vec && col0 + 32 <= g.N) {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + (bias ? __ldg(bias + col0 + j) : 0.f);
    if (g.preact) {
      float4* pp = reinterpret_cast<float4*>(g.preact + size_t(row) * g.ldp + col0);
#pragma unroll
      for (int q = 0; q < 8; ++q) pp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (g.act) {
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = gelu_tanh(v[j]);
    }
    if (g.epi == EPI_F32) {
      float4* cp = reinterpret_cast<float4*>(reinterpret_cast<float*>(g.C) + size_t(row) * g.ldc + col0);
#pragma unroll
      for (int q = 0; q < 8; ++q) cp[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
      uint4* cp = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(g.C) + size_t(row) * g.ldc + col0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * q + 2 * e], v[8 * q + 2 * e + 1]);
          w[e] = *reinterpret_cast<const uint32_t*>(&h2);
        }
        cp[q] = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int col = col0 + j;
      if (col >= g.N) break;
      float v = __uint_as_float(r[j]) + (bias ? __ldg(bias + col) : 0.f);
      if (g.preact) g.preact[size_t(row) * g.ldp + col] = v;
      if (g.act) v = gelu_tanh(v);
      if (g.epi == EPI_F32) reinterpret_cast<float*>(g.C)[size_t(row) * g.ldc + col] = v;
      else reinterpret_cast<__nv_bfloat16*>(g.C)[size_t(row) * g.ldc + col] = __float2bfloat16(v);
    }
  }
}

template <int BN>
__global__ void __launch_bounds__(192, 1)
    tc_pgemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const GemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
  uint8_t* sA = smem;                                    // kStages x 16 KB
  uint8_t* sB = smem + kStages * kBM * kBK * 2;          // kStages x BN*128 B
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kStages * BN * kBK * 2);
  uint64_t* empty = full + kStages;
  uint64_t* acc_full = empty + kStages;                  // [2]
  uint64_t* acc_empty = acc_full + 2;                    // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = (g.K + kBK - 1) / kBK;
  const int nN = (g.N + BN - 1) / BN, nM = (g.M + kBM - 1) / kBM;
  const int ntiles = nM * nN, G = gridDim.x;
  constexpr uint32_t kStageBytes = (kBM + BN) * kBK * 2;

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < kStages; ++s) {
        tc::mbar_init(&full[s], 1);
        tc::mbar_init(&empty[s], 1);
      }
      for (int b = 0; b < 2; ++b) {
        tc::mbar_init(&acc_full[b], 1);
        tc::mbar_init(&acc_empty[b], 4);
      }
      *abort_flag = 0;
      tc::fence_mbar_init();
      tc::tma_prefetch_desc(&tmA);
      tc::tma_prefetch_desc(&tmB);
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, 2 * BN);
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
    int sc = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += G) {
      const int m = t / nN, n = t - m * nN;
      for (int kb = 0; kb < nk; ++kb, ++sc) {
        const int s = sc % kStages;
        if (sc >= kStages && !tc::mbar_wait(&empty[s], ((sc / kStages) - 1) & 1, kWaitNs)) {
          fail(21);
          ok = false;
          break;
        }
        if (*abort_flag) { ok = false; break; }
        tc::mbar_expect_tx(&full[s], kStageBytes);
        tc::tma_load_2d(sA + s * kBM * kBK * 2, &tmA, &full[s], kb * kBK, m * kBM);
        tc::tma_load_2d(sB + s * BN * kBK * 2, &tmB, &full[s], kb * kBK, n * BN);
      }
    }
    if (*abort_flag)   // let the copies still in flight land before the CTA exits (bounded)
      for (int i = sc > kStages ? sc - kStages : 0; i < sc; ++i)
        tc::mbar_wait(&full[i % kStages], (i / kStages) & 1, kWaitNs);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = tc::idesc_f16(kBM, BN, g.bf16 != 0);
    int sc = 0, tcount = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += G, ++tcount) {
      const int acc = tcount & 1;
      if (tcount >= 2 && !tc::mbar_wait(&acc_empty[acc], ((tcount >> 1) - 1) & 1, kWaitNs)) {
        fail(22);
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t d = tmem + uint32_t(acc * BN);
      for (int kb = 0; kb < nk; ++kb, ++sc) {
        const int s = sc % kStages;
        if (!tc::mbar_wait(&full[s], (sc / kStages) & 1, kWaitNs)) { fail(23); ok = false; break; }
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(sA + s * kBM * kBK * 2);
        const uint32_t b0 = tc::smem_u32(sB + s * BN * kBK * 2);
#pragma unroll
        for (int k = 0; k < kBK / 16; ++k)
          tc::mma_f16(d, tc::sdesc_sw128(a0 + 32 * k), tc::sdesc_sw128(b0 + 32 * k), idesc,
                      (kb > 0 || k > 0) ? 1u : 0u);
        tc::mma_commit(&empty[s]);
      }
      if (ok) tc::mma_commit(&acc_full[acc]);
    }
    if (!ok) {                       // release the epilogue so it can see the flag and stop
      tc::mbar_arrive(&acc_full[0]);
      tc::mbar_arrive(&acc_full[1]);
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                   // TMEM lane quadrant of this warp
    int tcount = 0;
    for (int t = blockIdx.x; t < ntiles; t += G, ++tcount) {
      const int acc = tcount & 1;
      const bool w = tc::mbar_wait(&acc_full[acc], (tcount >> 1) & 1, 4 * kWaitNs);
      if (!w) fail(24);
      tc::tc_fence_after();
      if (!w || *abort_flag) break;
      const int m = t / nN, n = t - m * nN;
      const int row = m * kBM + q * 32 + lane;
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        uint32_t r[32];
        tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(acc * BN + c * 32), r);
        tc::tmem_ld_wait();
        epilogue_chunk<BN>(g, r, row, n * BN + c * 32, g.bias);
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acc_empty[acc]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * BN);
  }
}

// 256 x 256 output tile per CTA for wide, tall products (EPI_F32 / EPI_BF16):
// two 128-row sub-tiles share each K block of B, so the B block (the weights
// of a network layer) is read from L2 once per 256 rows instead of once per
// 128; the two accumulators take all 512 TMEM columns.  Three stages of
// (2 x 16 KB of A + 32 KB of B); same warp roles, bounded waits and error flag
// as tc_gemm_kernel.
constexpr int kS2 = 3;

__global__ void __launch_bounds__(192, 1)
    tc_gemm2_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const GemmArgs g) {
  constexpr int BN = 256;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
  uint8_t* sA = smem;                                     // kS2 x 2 x 16 KB
  uint8_t* sB = smem + kS2 * 2 * kBM * kBK * 2;           // kS2 x 32 KB
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + kS2 * BN * kBK * 2);
  uint64_t* empty = full + kS2;
  uint64_t* accum = empty + kS2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * 2 * kBM, n0 = blockIdx.y * BN;
  const int nk = (g.K + kBK - 1) / kBK;
  constexpr uint32_t kStageBytes = (2 * kBM + BN) * kBK * 2;
  constexpr uint32_t kATile = kBM * kBK * 2;

  if (warp == 0) {
    if (lane == 0) {
      for (int s = 0; s < kS2; ++s) {
        tc::mbar_init(&full[s], 1);
        tc::mbar_init(&empty[s], 1);
      }
      tc::mbar_init(accum, 1);
      *abort_flag = 0;
      tc::fence_mbar_init();
      tc::tma_prefetch_desc(&tmA);
      tc::tma_prefetch_desc(&tmB);
    }
    __syncwarp();
    tc::tmem_alloc(tmem_slot, 2 * BN);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kS2;
      const uint32_t use = kb / kS2;
      if (kb >= kS2 && !tc::mbar_wait(&empty[s], (use & 1) ^ 1, kWaitNs)) {
        atomicExch(g.err, 31);
        *abort_flag = 1;
        break;
      }
      if (*abort_flag) break;
      tc::mbar_expect_tx(&full[s], kStageBytes);
      tc::tma_load_2d(sA + (2 * s) * kATile, &tmA, &full[s], kb * kBK, m0);
      tc::tma_load_2d(sA + (2 * s + 1) * kATile, &tmA, &full[s], kb * kBK, m0 + kBM);
      tc::tma_load_2d(sB + s * BN * kBK * 2, &tmB, &full[s], kb * kBK, n0);
      issued = kb + 1;
    }
    if (*abort_flag)   // let the copies still in flight land before the CTA exits (bounded)
      for (int i = issued > kS2 ? issued - kS2 : 0; i < issued; ++i)
        tc::mbar_wait(&full[i % kS2], (i / kS2) & 1, kWaitNs);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t idesc = tc::idesc_f16(kBM, BN, g.bf16 != 0);
    bool ok = true;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kS2;
      const uint32_t use = kb / kS2;
      if (!tc::mbar_wait(&full[s], use & 1, kWaitNs)) {
        atomicExch(g.err, 32);
        *abort_flag = 1;
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const uint32_t a0 = tc::smem_u32(sA + (2 * s) * kATile);
      const uint32_t a1 = tc::smem_u32(sA + (2 * s + 1) * kATile);
      const uint32_t b0 = tc::smem_u32(sB + s * BN * kBK * 2);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k) {
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        tc::mma_f16(tmem, tc::sdesc_sw128(a0 + 32 * k), tc::sdesc_sw128(b0 + 32 * k), idesc, acc);
        tc::mma_f16(tmem + uint32_t(BN), tc::sdesc_sw128(a1 + 32 * k), tc::sdesc_sw128(b0 + 32 * k), idesc, acc);
      }
      tc::mma_commit(&empty[s]);
    }
    if (ok) tc::mma_commit(accum);
    else tc::mbar_arrive(accum);          // release the epilogue (it checks the flag)
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;                   // TMEM lane quadrant of this warp
    const bool waited = tc::mbar_wait(accum, 0, 4 * kWaitNs);
    if (!waited) atomicExch(g.err, 33);
    tc::tc_fence_after();
    if (waited && *abort_flag == 0) {
#pragma unroll 1
      for (int sub = 0; sub < 2; ++sub) {
        const int row = m0 + sub * kBM + q * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
          uint32_t r[32];
          tc::tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(sub * BN + c * 32), r);
          tc::tmem_ld_wait();
          epilogue_chunk<BN>(g, r, row, n0 + c * 32, g.bias);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 2 * BN);
  }
}

// ---- host side: tensor maps through the driver entry point -----------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// K-major [rows][ld] 2-byte matrix, box 64 x box_rows, 128-byte swizzle, OOB -> 0.
bool make_map(CUtensorMap* m, const void* ptr, int rows, int K, int ld, int box_rows, bool bf16) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((size_t(ld) * 2) & 15)) return false;
  cuuint64_t gdim[2] = {cuuint64_t(K), cuuint64_t(rows)};
  cuuint64_t gstride[1] = {cuuint64_t(ld) * 2};
  cuuint32_t box[2] = {cuuint32_t(kBK), cuuint32_t(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                  const_cast<void*>(ptr), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_bn(const GemmArgs& g, const void* A, int lda, const void* B, int ldb, cudaStream_t st) {
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, g.M, g.K, lda, kBM, g.bf16) || !make_map(&mb, B, g.N, g.K, ldb, BN, g.bf16))
    return cudaErrorInvalidValue;
  const long long ntiles = (long long)((g.M + kBM - 1) / kBM) * ((g.N + BN - 1) / BN);
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (BN == 256 && g.epi != EPI_TOPK && (long long)g.M >= 2LL * kBM * nsm) {
    // tall and wide: 256 x 256 tiles, the B block read once per 256 rows
    const size_t smem2 = 1024 + size_t(kS2) * (2 * kBM + 256) * kBK * 2 + (2 * kS2 + 1) * 8 + 16;
    ResidentShape rs{};
    cudaError_t e = resident_shape(tc_gemm2_kernel, 192, smem2, &rs);
    if (e != cudaSuccess) return e;
    dim3 grid2((g.M + 2 * kBM - 1) / (2 * kBM), (g.N + 255) / 256);
    tc_gemm2_kernel<<<grid2, 192, smem2, st>>>(ma, mb, g);
    return cudaGetLastError();
  }
  if (g.epi != EPI_TOPK && BN <= 128 && ntiles >= 4LL * nsm) {
    // many tiles: one persistent CTA per SM with a double-buffered accumulator
    // (at BN = 256 the per-tile kernel measured faster: the loads, not the
    // epilogue, bound that shape)
    const size_t psmem = 1024 + size_t(kStages) * (kBM + BN) * kBK * 2 + (2 * kStages + 4) * 8 + 16;
    ResidentShape rs{};
    cudaError_t e = resident_shape(tc_pgemm_kernel<BN>, 192, psmem, &rs);
    if (e != cudaSuccess) return e;
    const long long grid = ntiles < (long long)nsm ? ntiles : (long long)nsm;
    tc_pgemm_kernel<BN><<<unsigned(grid), 192, psmem, st>>>(ma, mb, g);
    return cudaGetLastError();
  }
  const size_t smem = 1024 + size_t(kStages) * (kBM + BN) * kBK * 2 + (2 * kStages + 1) * 8 + 16 + 4 * BN;
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  dim3 grid((g.M + kBM - 1) / kBM, (g.N + BN - 1) / BN);
  tc_gemm_kernel<BN><<<grid, 192, smem, st>>>(ma, mb, g);
  return cudaGetLastError();
}

}  // namespace

bool make_map_2b(CUtensorMap* m, const void* ptr, int rows, int K, int ld, int box_rows, bool bf16) {
  return make_map(m, ptr, rows, K, ld, box_rows, bf16);
}

cudaError_t tc_gemm(const GemmArgs& g_in, const void* A, int lda, const void* B, int ldb, int bn,
                    cudaStream_t st) {
  if (g_in.M < 1 || g_in.N < 1 || g_in.K < 1 || !g_in.err) return cudaErrorInvalidValue;
  GemmArgs g = g_in;
  const auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  g.vec = g.epi != EPI_TOPK && g.C && a16(g.C) &&
          (g.epi == EPI_F32 ? (g.ldc % 4 == 0) : (g.ldc % 8 == 0)) &&
          (!g.preact || (a16(g.preact) && g.ldp % 4 == 0));
  switch (bn) {
    case 64: return launch_bn<64>(g, A, lda, B, ldb, st);
    case 128: return launch_bn<128>(g, A, lda, B, ldb, st);
    case 256: return launch_bn<256>(g, A, lda, B, ldb, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wh
