// Autocorrelation search with the whole contraction of Eq. (10) on tcgen05
// tensor cores (lz = 1 slice), exact FP32 argmax.
//
// In the basis of the stream state a = [A_c(0), A_c(h), A_s(h)] (h over the
// half plane, a_h(l) = 2pi (hx lx + hy ly)/M)
//   R(l) = A_c(0) + 2 sum_h [A_c(h) cos a_h(l) - A_s(h) sin a_h(l)].
// The grid is symmetric and a_h(-l) = -a_h(l), so with
//   C(l) = A_c(0) + 2 sum_h A_c(h) cos a_h(l),   S(l) = -2 sum_h A_s(h) sin a_h(l)
// both R(l) = C + S and R(-l) = C - S follow from one evaluation of C and S on
// the half grid g <= (L^2-1)/2 (flat index g = iy L + ix; -l is L^2-1-g).  C and
// S are two dense products, [pixels x (NH+1)] x [(NH+1) x half grid] and
// [pixels x NH] x [NH x half grid] (half the work of the full-grid product).
//
// Per 128-pixel tile (one CTA per SM walks its tiles):
//   - a producer warp streams the tile's FP32 state rows (contiguous, 912 B per
//     pixel at M = 15) into a ring of 32-pixel slots with bulk copies;
//   - four converter warps (one pixel per thread) scale each row by a power of
//     two (max |a| in [1/2, 1): exact, and the argmax does not depend on it),
//     round it to F16 into the tensor cores' K-major 128-byte-swizzled operand,
//     and form the pixel's error window (below);
//   - a second producer streams the constant F16 cos/sin operand (one 16 KB block
//     of 128 half-grid rows x 64 k per stage) from L2;
//   - one thread issues the MMAs (M = 128 pixels, N = 128 half-grid points per
//     chunk, F32 accumulation) into one of two TMEM buffers [C | S];
//   - four epilogue warps (one pixel per TMEM lane) read C and S, keep the
//     running maximum of R~ = C + |S| = max(R~(l), R~(-l)), and list every grid
//     point whose R~ lies within the pixel's window of that maximum.
// Error window.  With F16 rounding of both operands (2^-11 relative each),
// exact products and F32 accumulation (2^-22 per term allowed), F16 subnormals
// (2^-25 absolute) and the FP32 rounding of the exact evaluation below,
//   |R~(l) - R32(l)| <= E = 1.0125e-3 Bnd + 6.2e-5 (scaled units),
//   Bnd = |A_c(0)| + 2 sum_h oct(A_c(h), A_s(h)) >= sum_k |a_k| |B_k(l)|,
//   oct(x, y) = max(|x|,|y|) + (sqrt(2)-1) min(|x|,|y|) >= sqrt(x^2 + y^2),
// so every grid point whose FP32 value can be the largest satisfies
// R~(l) >= max R~ - 2E.  A pixel with one such point is decided by the tensor
// cores; its index is the FP32 argmax.  Pixels with 2..8 points get them
// evaluated exactly in FP32 (ac::exact_R, the CUDA-core search's operation
// sequence) after the last tile, by 8-lane groups with the state row prefetched
// by cp.async, and the largest wins (ties to the lowest flat index).  Pixels
// with more points, a non-finite or subnormal-range state evaluate the whole
// grid exactly; an all-zero state is R = 0 everywhere (index 0).  The result
// equals the CUDA-core search's bit for bit.
//
// Every wait is bounded (~1 s); a timeout sets the stream's status word and
// the CTA stops.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ac_common.cuh"
#include "common.cuh"
#include "tc_ptx.cuh"

namespace wh {
namespace {

constexpr int kTile = 128;                 // pixels per tile (MMA M, TMEM lanes)
constexpr int kQPx = 32;                   // pixels per staging slot (one converter warp)
constexpr int kSlots = 3;                  // staging ring slots
constexpr int kBSt = 4;                    // constant-operand ring stages
constexpr int kCN = 128;                   // half-grid points per chunk (MMA N)
constexpr uint32_t kTmemCols = 512;        // 2 buffers x [C 128 | S 128]
constexpr int kWarps = 15;                 // producer, B producer, MMA, 8 converters, 4 epilogue
constexpr int kThreads = kWarps * 32;
constexpr int kWConv = 3;
constexpr int kWEpi = 11;
constexpr int kMaxCand = 8;
constexpr int kGroups = kThreads / 8;      // 8-lane groups of the exact evaluation
constexpr int kBatchTiles = 16;            // tiles whose listed pixels are gathered at once
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr uint32_t kBlk = 16384;           // one operand block: 128 rows x 64 F16
constexpr float kWinRel = 1.0125e-3f;      // E per unit of Bnd
constexpr float kWinAbs = 6.2e-5f;         // E absolute part (scaled units)
constexpr float kThrRel = 2.384185791e-7f; // 2^-22: rounding of the threshold itself
constexpr float kTiny = 2.3509887e-38f;    // 2^-125: below this max |a| the state takes the full path
constexpr float kOct = 0.41421357f;        // >= sqrt(2) - 1
enum : int { kFlagNone = 0, kFlagZero = 1, kFlagFull = 2 };

__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

template <int M>
struct TD {
  static constexpr int K = (M - 1) / 2;
  static constexpr int NH = 2 * K * (K + 1);      // (M^2 - 1)/2, a multiple of 4
  static constexpr int KP = ac::Geo<M>::KP;
  static constexpr int QN = ac::Geo<M>::QN;
  static constexpr int NE = ac::Geo<M>::NE;
  static constexpr int QIT = (NE + 7) / 8;
  static constexpr int KSC = (NH + 1 + 15) / 16;  // MMA K steps (16) of C
  static constexpr int KSS = (NH + 15) / 16;      // ... of S
  static constexpr int KBC = (KSC + 3) / 4;       // 64-wide K blocks of C
  static constexpr int KBS = (KSS + 3) / 4;
  static constexpr int KBW = 64 * (KBC > KBS ? KBC : KBS);   // constant operand row length
  static constexpr size_t SLOT = size_t(kQPx) * KP * 4;
  static constexpr size_t O_A = 0;                                   // [KBC + KBS][16 KB]
  static constexpr size_t O_B = O_A + size_t(KBC + KBS) * kBlk;      // [kBSt][16 KB]
  static constexpr size_t O_ST = O_B + size_t(kBSt) * kBlk;          // [kSlots][SLOT]
  static constexpr int QS = QN + 4;               // phase-2 Q-sum stride (the 4 groups of a warp in distinct banks)
  static constexpr size_t P2 = al16(size_t(kGroups) * QS * 4) + 8ull * kBatchTiles * kTile;
  static constexpr size_t O_W = O_ST + (kSlots * SLOT > P2 ? kSlots * SLOT : P2);   // float [2][128] windows
  static constexpr size_t O_F = O_W + 2 * kTile * 4;                 // int [2][128] flags
  static constexpr size_t O_X = O_F + 2 * kTile * 4;                 // float [4][2][2][32] stop flags, maxima
  static constexpr size_t O_TAB = O_X + 4 * 4 * 32 * 4;               // float2 [kMaxL][K+1]
  static constexpr size_t O_BAR = al16(O_TAB + 8ull * kMaxL * (K + 1));
  static constexpr size_t SMEM = O_BAR + 8 * 24 + 32 + 1024;        // + 1024-byte alignment slack
  // after the last tile: Q sums per group and the pixel list in the staging
  // area, two state-row buffers per group in the operand area
  static constexpr size_t O_Q2 = O_ST;
  static constexpr size_t O_L2 = O_ST + al16(size_t(kGroups) * QS * 4);
  static_assert(O_L2 + 8ull * kBatchTiles * kTile <= O_W, "phase-2 Q sums and list fit the staging area");
  static_assert(size_t(kGroups) * 2 * (KP + 8) * 4 <= O_ST, "phase-2 row buffers fit the operand area");
  static_assert(NH % 4 == 0, "state halves start on a float4");
  static_assert(KBC <= 2 && KBS <= 2, "M <= 15");
};

// single-thread roles wait with a back-off so they do not take issue slots
__device__ __forceinline__ bool wait_backoff(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    __nanosleep(64);
    if (tc::mbar_try_wait(bar, parity)) return true;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// maximum of three, NaN if any input is NaN
__device__ __forceinline__ float max3nan(float a, float b, float c) {
  float d;
  asm("max.NaN.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// x[j] for a lane-dependent j in [0, 32) by a tree of selects (no local memory)
__device__ __forceinline__ float mux32(const float (&x)[32], int j) {
  float y[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) y[i] = (j & 1) ? x[2 * i + 1] : x[2 * i];
#pragma unroll
  for (int i = 0; i < 8; ++i) y[i] = (j & 2) ? y[2 * i + 1] : y[2 * i];
#pragma unroll
  for (int i = 0; i < 4; ++i) y[i] = (j & 4) ? y[2 * i + 1] : y[2 * i];
#pragma unroll
  for (int i = 0; i < 2; ++i) y[i] = (j & 8) ? y[2 * i + 1] : y[2 * i];
  return (j & 16) ? y[1] : y[0];
}

// byte offset of 16-byte chunk cj (0..7) of row r in a 128-byte-swizzled K-major block
__device__ __forceinline__ uint32_t sw128(int r, int cj) {
  return uint32_t(r) * 128u + (uint32_t(cj ^ (r & 7)) << 4);
}

template <int M>
__global__ void __launch_bounds__(kThreads, 1)
    autocorr_tcd_kernel(const __grid_constant__ CUtensorMap tmB, const TcDenseArgs a) {
  using G = TD<M>;
  constexpr int K = G::K, NH = G::NH, KP = G::KP;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
  uint8_t* sA = sm + G::O_A;
  uint8_t* sB = sm + G::O_B;
  float* stage = reinterpret_cast<float*>(sm + G::O_ST);
  float* wbuf = reinterpret_cast<float*>(sm + G::O_W);
  int* fbuf = reinterpret_cast<int*>(sm + G::O_F);
  float2* tabs = reinterpret_cast<float2*>(sm + G::O_TAB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + G::O_BAR);
  uint64_t* st_full = bar;            // [kSlots]
  uint64_t* st_empty = bar + 3;       // [kSlots]
  uint64_t* a_full = bar + 6;
  uint64_t* a_empty = bar + 7;
  uint64_t* b_full = bar + 8;         // [kBSt]
  uint64_t* b_empty = bar + 12;       // [kBSt]
  uint64_t* c_full = bar + 16;        // [2]
  uint64_t* c_empty = bar + 18;       // [2]
  uint64_t* e_full = bar + 20;        // [2]
  uint64_t* e_empty = bar + 22;       // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 24);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* list_n = reinterpret_cast<int*>(tmem_slot + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npix = a.npix, L = a.L, L2 = L * L;
  const int NHG = (L2 + 1) / 2;
  const int NCH = (NHG + kCN - 1) / kCN;
  const int ntiles = (npix + kTile - 1) / kTile;
  const int nct = gridDim.x;
  const int mytiles = int(blockIdx.x) < ntiles ? (ntiles - 1 - int(blockIdx.x)) / nct + 1 : 0;
  auto fail = [&](int code) {
    if (a.err) atomicExch(a.err, code);
    *abort_flag = 1;
  };

  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) {
      tc::mbar_init(&st_full[s], 1);
      tc::mbar_init(&st_empty[s], 2);
    }
    tc::mbar_init(a_full, 8);
    tc::mbar_init(a_empty, 1);
    for (int s = 0; s < kBSt; ++s) {
      tc::mbar_init(&b_full[s], 1);
      tc::mbar_init(&b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&c_full[b], 1);
      tc::mbar_init(&c_empty[b], 4);
      tc::mbar_init(&e_full[b], 8);
      tc::mbar_init(&e_empty[b], 4);
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
    tc::tma_prefetch_desc(&tmB);
  }
  if (warp == 2) {
    tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  for (int i = tid; i < L * (K + 1); i += kThreads) tabs[i] = a.tab_x[i];
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- staging producer: 32-pixel slots of FP32 state rows ----------------
    if (lane == 0) {
      for (int i = 0; i < mytiles && !*abort_flag; ++i) {
        const int tile = int(blockIdx.x) + i * nct;
        bool ok = true;
        for (int q = 0; q < 4; ++q) {
          const int u = 4 * i + q, s = u % kSlots;
          if (u >= kSlots && !wait_backoff(&st_empty[s], uint32_t(((u / kSlots) - 1) & 1), kWaitNs)) {
            fail(41);
            ok = false;
            break;
          }
          const int p0 = tile * kTile + q * kQPx;
          const int n = npix - p0 < kQPx ? (npix - p0 > 0 ? npix - p0 : 0) : kQPx;
          if (n > 0) {
            const uint32_t bytes = uint32_t(n) * KP * 4u;          // KP % 4 == 0: a multiple of 16
            tc::mbar_expect_tx(&st_full[s], bytes);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                ::"r"(tc::smem_u32(reinterpret_cast<uint8_t*>(stage) + s * G::SLOT)),
                  "l"(a.Astate + size_t(p0) * KP), "r"(bytes), "r"(tc::smem_u32(&st_full[s]))
                : "memory");
          } else {
            tc::mbar_arrive(&st_full[s]);
          }
        }
        if (!ok) break;
      }
    }
  } else if (warp == 1) {
    // ---------------- constant-operand producer ----------------
    if (lane == 0) {
      int bc = 0;
      bool ok = true;
      for (int i = 0; i < mytiles && ok && !*abort_flag; ++i)
        for (int c = 0; c < NCH && ok; ++c)
          for (int part = 0; part < 2 && ok; ++part)
            for (int kb = 0; kb < (part ? G::KBS : G::KBC); ++kb, ++bc) {
              const int s = bc % kBSt;
              if (bc >= kBSt && !wait_backoff(&b_empty[s], uint32_t(((bc / kBSt) - 1) & 1), kWaitNs)) {
                fail(42);
                ok = false;
                break;
              }
              tc::mbar_expect_tx(&b_full[s], kBlk);
              tc::tma_load_2d(sB + s * kBlk, &tmB, &b_full[s], 64 * kb, (part * NCH + c) * kCN);
            }
    }
  } else if (warp == 2) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      int bc = 0, cc = 0, issued = 0;
      bool ok = true;
      for (int i = 0; i < mytiles && ok; ++i) {
        if (!wait_backoff(a_full, uint32_t(i & 1), kWaitNs)) { fail(43); ok = false; break; }
        if (*abort_flag) { ok = false; break; }
        tc::tc_fence_after();
        for (int c = 0; c < NCH && ok; ++c, ++cc) {
          const int b = cc & 1;
          if (cc >= 2 && !wait_backoff(&c_empty[b], uint32_t(((cc >> 1) - 1) & 1), kWaitNs)) {
            fail(44);
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const int nc = NHG - c * kCN < kCN ? NHG - c * kCN : kCN;
          const uint32_t idesc = tc::idesc_f16(128, (nc + 15) & ~15, false);
          for (int part = 0; part < 2 && ok; ++part) {
            const uint32_t d = tmem + uint32_t(b * 256 + part * 128);
            const int nkb = part ? G::KBS : G::KBC, nks = part ? G::KSS : G::KSC;
            for (int kb = 0; kb < nkb; ++kb, ++bc) {
              const int s = bc % kBSt;
              if (!wait_backoff(&b_full[s], uint32_t((bc / kBSt) & 1), kWaitNs)) { fail(45); ok = false; break; }
              tc::tc_fence_after();
              const uint32_t a0 = tc::smem_u32(sA + (part ? G::KBC + kb : kb) * kBlk);
              const uint32_t b0 = tc::smem_u32(sB + s * kBlk);
#pragma unroll
              for (int k = 0; k < 4; ++k)
                if (kb * 4 + k < nks)
                  tc::mma_f16(d, tc::sdesc_sw128(a0 + 32 * k), tc::sdesc_sw128(b0 + 32 * k), idesc,
                              (kb > 0 || k > 0) ? 1u : 0u);
              tc::mma_commit(&b_empty[s]);
            }
          }
          if (ok) tc::mma_commit(&c_full[b]);
        }
        if (ok) {
          tc::mma_commit(a_empty);
          issued = cc;
        }
      }
      if (!ok) {            // let the epilogue see the flag instead of waiting for its chunks
        tc::mbar_arrive(&c_full[0]);
        tc::mbar_arrive(&c_full[1]);
      }
      if (issued > 0)       // the last MMAs finish before TMEM is freed
        wait_backoff(&c_full[(issued - 1) & 1], uint32_t(((issued - 1) >> 1) & 1), kWaitNs);
    }
  } else if (warp < kWEpi) {
    // ---------------- converters: two threads per pixel ----------------
    // Warp q (quarter of the tile, 32 pixels) and half hf: half 0 takes the first
    // half of the row's maximum and the C operand row, half 1 the second half of
    // the maximum, the S operand row and the error window.
    const int q = (warp - kWConv) & 3, hf = (warp - kWConv) >> 2;
    const int r = q * kQPx + lane;
    float* xbuf = reinterpret_cast<float*>(sm + G::O_X) + q * 128;   // [0, 64): stop flags, [64, 128): maxima
    for (int i = 0; i < mytiles; ++i) {
      const int tile = int(blockIdx.x) + i * nct;
      const int u = 4 * i + q, s = u % kSlots;
      // Four quarters consume a ring of three slots, so a parity wait is safe only
      // when the barrier is at most one phase behind the awaited one.  The order
      // below guarantees that: the operand of tile i-1 released (every slot use
      // of tile i-1 and earlier consumed), then the previous use of this slot
      // released, then this use filled; the window buffer of tile i-2 read.
      bool bad = i >= 1 && !tc::mbar_wait(a_empty, uint32_t((i - 1) & 1), kWaitNs);
      if (!bad && u >= kSlots) bad = !tc::mbar_wait(&st_empty[s], uint32_t(((u / kSlots) - 1) & 1), kWaitNs);
      if (!bad) bad = !tc::mbar_wait(&st_full[s], uint32_t((u / kSlots) & 1), kWaitNs);
      if (!bad && i >= 2) bad = !tc::mbar_wait(&e_empty[i & 1], uint32_t(((i >> 1) - 1) & 1), kWaitNs);
      if (bad) fail(46);
      // both halves of the quarter take the same decision before their shared barriers
      const bool stop_now = __any_sync(0xffffffffu, bad || *abort_flag);
      xbuf[hf * 32 + lane] = stop_now ? 1.f : 0.f;
      asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");
      if (xbuf[lane] != 0.f || xbuf[32 + lane] != 0.f) break;
      const int pix = tile * kTile + r;
      const float* src = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(stage) + s * G::SLOT) +
                         lane * KP;
      const float4* s4 = reinterpret_cast<const float4*>(src);
      uint8_t* aC = sA;
      uint8_t* aS = sA + G::KBC * kBlk;
      const bool valid = pix < npix;
      // pass 1: this half's part of max |a|, NaN if any value is NaN
      constexpr int NV = (2 * NH + 4) / 4, NV0 = NV / 2;
      float mx0 = 0.f, mx1 = 0.f;
      if (valid) {
        const int v0 = hf ? NV0 : 0, v1 = hf ? NV : NV0;
#pragma unroll 4
        for (int v = v0; v < v1; ++v) {
          const float4 x = s4[v];
          const float e3 = (4 * v + 3 <= 2 * NH) ? x.w : 0.f;
          const float e2 = (4 * v + 2 <= 2 * NH) ? x.z : 0.f;
          const float e1 = (4 * v + 1 <= 2 * NH) ? x.y : 0.f;
          mx0 = max3nan(mx0, fabsf(x.x), fabsf(e1));
          mx1 = max3nan(mx1, fabsf(e2), fabsf(e3));
        }
      }
      xbuf[64 + hf * 32 + lane] = max3nan(mx0, mx1, 0.f);
      asm volatile("bar.sync %0, 64;" ::"r"(1 + q) : "memory");
      const float mx = max3nan(xbuf[64 + lane], xbuf[96 + lane], 0.f);
      int flag = kFlagNone;
      if (!valid) flag = kFlagZero;
      else if (!(mx <= 3.402823466e38f)) flag = kFlagFull;
      else if (mx == 0.f) flag = kFlagZero;
      else if (mx < kTiny) flag = kFlagFull;
      float sc = 1.f;
      if (flag == kFlagNone) {
        int e;
        frexpf(mx, &e);                     // mx = f 2^e, f in [1/2, 1); e in [-124, 128]
        sc = ldexpf(1.f, -e);
      }
      if (!valid) sc = 0.f;                 // rows past the frame: zeros
      const float2 sc2 = make_float2(sc, sc);
      // pass 2: scaled values -> F16 operand rows.  Half 0 writes C chunk j (A_c(0) ..
      // elements 8j .. 8j+7); half 1 writes S chunk j (A_s(h), h = 8j+1 .. 8j+8) and
      // forms Bnd: with NH % 4 == 0 the pair (A_c(h), A_s(h)) sits in the same
      // component of float4s h/4 and NH/4 + h/4.
      auto ldx = [&](int v) { return (valid && 4 * v <= NH) ? s4[v] : make_float4(0.f, 0.f, 0.f, 0.f); };
      auto ldy = [&](int v) { return (valid && 4 * v <= NH) ? s4[NH / 4 + v] : make_float4(0.f, 0.f, 0.f, 0.f); };
      if (hf == 0) {
#pragma unroll
        for (int j = 0; j < 2 * G::KSC; ++j) {
          const float4 x0 = ldx(2 * j), x1 = ldx(2 * j + 1);
          float2 v[4] = {make_float2(x0.x, x0.y), make_float2(x0.z, x0.w), make_float2(x1.x, x1.y),
                         make_float2(x1.z, x1.w)};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            v[t] = __fmul2_rn(v[t], sc2);
            if (8 * j + 2 * t > NH) v[t].x = 0.f;
            if (8 * j + 2 * t + 1 > NH) v[t].y = 0.f;
          }
          const uint4 w = make_uint4(pack_h2(v[0].x, v[0].y), pack_h2(v[1].x, v[1].y),
                                     pack_h2(v[2].x, v[2].y), pack_h2(v[3].x, v[3].y));
          *reinterpret_cast<uint4*>(aC + (j >> 3) * kBlk + sw128(r, j & 7)) = w;
        }
      } else {
        float2 bsq2 = make_float2(0.f, 0.f);
        float4 x0 = ldx(0), y0 = ldy(0);
#pragma unroll
        for (int j = 0; j < 2 * G::KSS; ++j) {
          const float4 x1 = ldx(2 * j + 1), x2 = ldx(2 * j + 2);
          const float4 y1 = ldy(2 * j + 1), y2 = ldy(2 * j + 2);
          float2 c[4] = {make_float2(x0.y, x0.z), make_float2(x0.w, x1.x), make_float2(x1.y, x1.z),
                         make_float2(x1.w, x2.x)};
          float2 sn[4] = {make_float2(y0.y, y0.z), make_float2(y0.w, y1.x), make_float2(y1.y, y1.z),
                          make_float2(y1.w, y2.x)};
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            c[t] = __fmul2_rn(c[t], sc2);
            sn[t] = __fmul2_rn(sn[t], sc2);
            if (8 * j + 2 * t + 1 > NH) { c[t].x = 0.f; sn[t].x = 0.f; }
            if (8 * j + 2 * t + 2 > NH) { c[t].y = 0.f; sn[t].y = 0.f; }
            // |(c, s)| <= max(|c|,|s|) + (sqrt(2) - 1) min(|c|,|s|) (exact on the axes and diagonals)
            const float2 hi = make_float2(fmaxf(fabsf(c[t].x), fabsf(sn[t].x)), fmaxf(fabsf(c[t].y), fabsf(sn[t].y)));
            const float2 lo = make_float2(fminf(fabsf(c[t].x), fabsf(sn[t].x)), fminf(fabsf(c[t].y), fabsf(sn[t].y)));
            bsq2 = __fadd2_rn(bsq2, __ffma2_rn(make_float2(kOct, kOct), lo, hi));
          }
          const uint4 w = make_uint4(pack_h2(sn[0].x, sn[0].y), pack_h2(sn[1].x, sn[1].y),
                                     pack_h2(sn[2].x, sn[2].y), pack_h2(sn[3].x, sn[3].y));
          *reinterpret_cast<uint4*>(aS + (j >> 3) * kBlk + sw128(r, j & 7)) = w;
          x0 = x2;
          y0 = y2;
        }
        const float a0 = valid ? src[0] * sc : 0.f;
        const float bnd = fmaf(2.f, bsq2.x + bsq2.y, fabsf(a0));
        if (flag == kFlagNone && !(bnd <= 3.0e38f)) flag = kFlagFull;
        wbuf[(i & 1) * kTile + r] = 2.f * fmaf(kWinRel, bnd, kWinAbs);
        fbuf[(i & 1) * kTile + r] = flag;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operand writes -> tensor cores
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&st_empty[s]);
        tc::mbar_arrive(a_full);
        tc::mbar_arrive(&e_full[i & 1]);
      }
    }
  } else {
    // ---------------- epilogue: one pixel per TMEM lane ----------------
    // Per chunk, pass 1 reads C and S and keeps the maximum of R~ = C + |S| of
    // each 32-point piece.  Pass 2 of chunk c runs after pass 1 of chunk c+1 (both
    // TMEM buffers hold data then), so its threshold max - window already covers
    // two chunks (the whole half grid for the last two): it re-reads only the
    // pieces whose maximum reaches the threshold and lists their points at or
    // above it.
    const int qd = warp & 3;
    const int r = qd * 32 + lane;
    const uint32_t lane_base = tmem + (uint32_t(qd * 32) << 16);
    int cc = 0;
    bool stop = false;
    for (int i = 0; i < mytiles && !stop; ++i) {
      const int tile = int(blockIdx.x) + i * nct;
      bool bad = !tc::mbar_wait(&e_full[i & 1], uint32_t((i >> 1) & 1), kWaitNs);
      if (bad) fail(47);
      if (__any_sync(0xffffffffu, bad) || *abort_flag) break;
      const float win = wbuf[(i & 1) * kTile + r];
      const int flag = fbuf[(i & 1) * kTile + r];
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&e_empty[i & 1]);
      float m = -INFINITY;
      bool ovf = false;
      // pieces holding points at or above their threshold: first point g0 and the
      // bit masks of R(l) = C + S (mp) and R(-l) = C - S (mm) at or above it
      constexpr int kRec = 4;
      int nrec = 0;
      int rg0[kRec];
      uint32_t rmp[kRec], rmm[kRec];
#pragma unroll
      for (int k = 0; k < kRec; ++k) { rg0[k] = 0; rmp[k] = 0u; rmm[k] = 0u; }
      auto wait_chunk = [&](int c) -> bool {
        const int gcc = cc + c;
        bool b2 = !tc::mbar_wait(&c_full[gcc & 1], uint32_t((gcc >> 1) & 1), 4 * kWaitNs);
        if (b2) fail(48);
        tc::tc_fence_after();
        return !(__any_sync(0xffffffffu, b2) || *abort_flag);
      };
      // pass 1 of chunk c: piece maxima
      auto pass1 = [&](int c, float (&pmx)[4]) {
        const int nc = NHG - c * kCN < kCN ? NHG - c * kCN : kCN;
        const uint32_t col = uint32_t(((cc + c) & 1) * 256);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          pmx[p] = -INFINITY;
          if (p * 32 < nc) {
            uint32_t vc[32], vs[32];
            __syncwarp();                      // tcgen05.ld is warp-collective
            tc::tmem_ld32(lane_base + col + uint32_t(p * 32), vc);
            tc::tmem_ld32(lane_base + col + uint32_t(128 + p * 32), vs);
            tc::tmem_ld_wait();
            const int nv = nc - p * 32;
            float a0 = -INFINITY, a1 = -INFINITY, a2 = -INFINITY, a3 = -INFINITY;
            if (nv >= 32) {
#pragma unroll
              for (int jj = 0; jj < 32; jj += 4) {
                a0 = max3f(a0, __uint_as_float(vc[jj]) + fabsf(__uint_as_float(vs[jj])),
                           __uint_as_float(vc[jj + 1]) + fabsf(__uint_as_float(vs[jj + 1])));
                a1 = max3f(a1, __uint_as_float(vc[jj + 2]) + fabsf(__uint_as_float(vs[jj + 2])),
                           __uint_as_float(vc[jj + 3]) + fabsf(__uint_as_float(vs[jj + 3])));
              }
            } else {
#pragma unroll
              for (int jj = 0; jj < 32; jj += 2) {
                const float t0 = jj < nv ? __uint_as_float(vc[jj]) + fabsf(__uint_as_float(vs[jj])) : -INFINITY;
                const float t1 =
                    jj + 1 < nv ? __uint_as_float(vc[jj + 1]) + fabsf(__uint_as_float(vs[jj + 1])) : -INFINITY;
                if (jj & 2) a2 = max3f(a2, t0, t1); else a3 = max3f(a3, t0, t1);
              }
            }
            pmx[p] = fmaxf(fmaxf(a0, a1), fmaxf(a2, a3));
          }
        }
      };
      // pass 2 of chunk c: record the points at or above thr in the pieces that can
      // hold one (thr only rises later, so the records hold every final candidate)
      auto pass2 = [&](int c, const float (&pmx)[4], float thr) {
        const int nc = NHG - c * kCN < kCN ? NHG - c * kCN : kCN;
        const uint32_t col = uint32_t(((cc + c) & 1) * 256);
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const bool need = flag == kFlagNone && pmx[p] >= thr;
          if (p * 32 < nc && __any_sync(0xffffffffu, need)) {
            uint32_t vc[32], vs[32];
            __syncwarp();
            tc::tmem_ld32(lane_base + col + uint32_t(p * 32), vc);
            tc::tmem_ld32(lane_base + col + uint32_t(128 + p * 32), vs);
            tc::tmem_ld_wait();
            if (need) {
              const int nv = nc - p * 32, g0 = c * kCN + p * 32;
              uint32_t mp = 0, mm = 0;
#pragma unroll
              for (int jj = 0; jj < 32; jj += 2) {
                const float2 cv2 = make_float2(__uint_as_float(vc[jj]), __uint_as_float(vc[jj + 1]));
                const float2 sv2 = make_float2(__uint_as_float(vs[jj]), __uint_as_float(vs[jj + 1]));
                const float2 p2 = __fadd2_rn(cv2, sv2);
                const float2 m2 = __fadd2_rn(cv2, make_float2(-sv2.x, -sv2.y));
                mp |= (p2.x >= thr ? 1u : 0u) << jj;
                mp |= (p2.y >= thr ? 1u : 0u) << (jj + 1);
                mm |= (m2.x >= thr ? 1u : 0u) << jj;
                mm |= (m2.y >= thr ? 1u : 0u) << (jj + 1);
              }
              if (nv < 32) {
                const uint32_t valid = (1u << nv) - 1u;
                mp &= valid;
                mm &= valid;
              }
              // the centre of the grid is its own mirror: listed once (as +l)
              const int jc = (L2 - 1) / 2 - g0;
              if (jc >= 0 && jc < 32) mm &= ~(1u << jc);
              if (mp | mm) {
                if (nrec < kRec) {
#pragma unroll
                  for (int k = 0; k < kRec; ++k)
                    if (k == nrec) { rg0[k] = g0; rmp[k] = mp; rmm[k] = mm; }
                  ++nrec;
                } else {
                  ovf = true;
                }
              }
            }
          }
        }
      };
      float pmA[4], pmB[4];
      if (!wait_chunk(0)) { stop = true; break; }
      pass1(0, pmA);
      m = fmaxf(fmaxf(pmA[0], pmA[1]), fmaxf(pmA[2], pmA[3]));
      for (int c = 0; c < NCH; ++c) {
        if (c + 1 < NCH) {
          if (!wait_chunk(c + 1)) { stop = true; break; }
          pass1(c + 1, pmB);
          m = fmaxf(m, fmaxf(fmaxf(pmB[0], pmB[1]), fmaxf(pmB[2], pmB[3])));
        }
        pass2(c, pmA, m - fmaf(kThrRel, fabsf(m), win));
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&c_empty[(cc + c) & 1]);
#pragma unroll
        for (int p = 0; p < 4; ++p) pmA[p] = pmB[p];
      }
      if (stop) break;
      cc += NCH;
      const int pix = tile * kTile + r;
      if (pix < npix) {
        int res = -1;                          // resolved grid index, else listed
        int code = 0;                          // 0 resolved, n > 1 listed points, -1 whole grid
        int nlist = 0;
#pragma unroll
        for (int k = 0; k < kRec; ++k) nlist += __popc(rmp[k]) + __popc(rmm[k]);

        if (flag == kFlagZero) {
          res = 0;
        } else if (flag == kFlagFull || ovf || nlist < 1 || nlist > kMaxCand) {
          code = -1;                           // (no point listed cannot happen: the maximum is)
        } else if (nlist == 1) {
#pragma unroll
          for (int k = 0; k < kRec; ++k) {
            if (rmp[k]) res = rg0[k] + __ffs(int(rmp[k])) - 1;
            if (rmm[k]) res = L2 - 1 - (rg0[k] + __ffs(int(rmm[k])) - 1);
          }
        } else {
          code = nlist;
          int n = 0;

#pragma unroll
          for (int k = 0; k < kRec; ++k) {
            for (uint32_t mk = rmp[k]; mk; mk &= mk - 1)
              a.cand[size_t(pix) * kMaxCand + n++] = rg0[k] + __ffs(int(mk)) - 1;
            for (uint32_t mk = rmm[k]; mk; mk &= mk - 1)
              a.cand[size_t(pix) * kMaxCand + n++] = L2 - 1 - (rg0[k] + __ffs(int(mk)) - 1);
          }
        }
        if (res >= 0) {
          const int iy = int((float(res) + 0.5f) * (1.0f / float(L))), ix = res - iy * L;
          a.vidx[pix] = res;
          a.vx[pix] = -a.vmax + ix * a.vstep;
          a.vy[pix] = -a.vmax + iy * a.vstep;
        }
        a.ccount[pix] = code;
      }
    }
  }

  // ---------------- after the last tile: exact FP32 evaluation of listed pixels ----------------
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 2) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
  if (*abort_flag) return;
  const int grp = tid >> 3, j = lane & 7;
  const unsigned gmask = 0xFFu << (lane & 24);
  const int gc = (L - 1) / 2;
  constexpr int RB = KP + 8;                       // row buffer: state row, then the listed points
  float* qbuf = reinterpret_cast<float*>(sm + G::O_Q2) + grp * G::QS;
  int* list = reinterpret_cast<int*>(sm + G::O_L2);
  int* lcode = list + kBatchTiles * kTile;
  float* rowbuf = reinterpret_cast<float*>(sm + G::O_A) + grp * 2 * RB;
  int qoff[G::QIT];
  ac::qsum_offsets<M, G::QIT, 8>(j, qoff);
  const float invL = 1.0f / float(L);
  // the state row (KP floats) and the listed points (8 ints) of list entry e
  auto fetch = [&](float* dst, int e) {
    const int pix = list[e];
    const float* src = a.Astate + size_t(pix) * KP;
    for (int c = j; c < KP / 4; c += 8) ac::cp_async16(dst + 4 * c, src + 4 * c);
    if (j < 2 && lcode[e] > 0) ac::cp_async16(dst + KP + 4 * j, a.cand + size_t(pix) * kMaxCand + 4 * j);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if (tid == 0) { list_n[1] = 0; list_n[2] = 0; }
  for (int t0 = 0; t0 < mytiles; t0 += kBatchTiles) {
    const int nb = mytiles - t0 < kBatchTiles ? mytiles - t0 : kBatchTiles;
    if (tid == 0) *list_n = 0;
    __syncthreads();
    for (int idx = tid; idx < nb * kTile; idx += kThreads) {
      const int tile = int(blockIdx.x) + (t0 + idx / kTile) * nct;
      const int pix = tile * kTile + (idx % kTile);
      const int code = pix < npix ? a.ccount[pix] : 0;
      if (code != 0) {
        const int e = atomicAdd(list_n, 1);
        list[e] = pix;
        lcode[e] = code;
        atomicAdd(&list_n[code > 0 ? 1 : 2], 1);
      }
    }
    __syncthreads();
    const int n = *list_n;
    int k = 0;
    if (grp < n) fetch(rowbuf, grp);
    else asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int e = grp; e < n; e += kGroups, ++k) {
      const int en = e + kGroups;
      if (en < n) fetch(rowbuf + ((k + 1) & 1) * RB, en);
      else asm volatile("cp.async.commit_group;\n" ::: "memory");
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      __syncwarp(gmask);
      const int pix = list[e], code = lcode[e];
      const float* row = rowbuf + (k & 1) * RB;
      ac::build_qsums<M, G::QIT, 8>(row, qbuf, qoff, j);
      __syncwarp(gmask);
      float best = -INFINITY;
      int bi = 0x7fffffff;
      if (code > 0) {
        if (j < code) {
          const int g = reinterpret_cast<const int*>(row + KP)[j];
          const float rv = ac::exact_R<M>(qbuf, tabs, L, g);
          if (rv > best) { best = rv; bi = g; }
        }
      } else {
        for (int g = j; g < L2; g += 8) {
          const float rv = ac::exact_R<M>(qbuf, tabs, L, g);
          if (rv > best) { best = rv; bi = g; }     // g increases in this lane: first of equals kept
        }
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(gmask, best, off);
        const int oi = __shfl_xor_sync(gmask, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (!(best > -INFINITY)) {
        // no value above -inf (non-finite state): the CUDA-core search then
        // resolves each grid column value in row 0 and takes the lowest index
        int lo = 0x7fffffff;
        for (int l = j; l <= gc; l += 8) {
          int idx = gc;
          if (l > 0) idx = ac::exact_R<M>(qbuf, tabs, L, gc - l) >= ac::exact_R<M>(qbuf, tabs, L, gc + l) ? gc - l
                                                                                                      : gc + l;
          lo = min(lo, idx);
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) lo = min(lo, __shfl_xor_sync(gmask, lo, off));
        bi = lo;
      }
      if (j == 0) {
        const int b = (bi >= 0 && bi < L2) ? bi : 0;
        const int iy = int((float(b) + 0.5f) * invL), ix = b - iy * L;
        a.vidx[pix] = b;
        a.vx[pix] = -a.vmax + ix * a.vstep;
        a.vy[pix] = -a.vmax + iy * a.vstep;
      }
      __syncwarp(gmask);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
  }
  if (tid == 0 && a.counts && (list_n[1] | list_n[2])) {
    atomicAdd(&a.counts[0], (unsigned long long)list_n[1]);
    atomicAdd(&a.counts[1], (unsigned long long)list_n[2]);
  }
}

template <int M>
cudaError_t launch_tcd_m(const TcDenseArgs& a, const CUtensorMap& tm, cudaStream_t st) {
  using G = TD<M>;
  if (a.kpad != G::KP) return cudaErrorInvalidValue;
  ResidentShape rs{};
  cudaError_t e = resident_shape(autocorr_tcd_kernel<M>, kThreads, G::SMEM, &rs);
  if (e != cudaSuccess) return e;
  if (rs.per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = (a.npix + kTile - 1) / kTile;
  const int grid = ntiles < rs.nsm ? ntiles : rs.nsm;
  if (grid < 1) return cudaSuccess;
  autocorr_tcd_kernel<M><<<grid, kThreads, G::SMEM, st>>>(tm, a);
  return cudaGetLastError();
}

template <int M>
constexpr int tcd_kbw() { return TD<M>::KBW; }

int kbw_of(int M) {
  switch (M) {
    case 5: return tcd_kbw<5>();
    case 7: return tcd_kbw<7>();
    case 9: return tcd_kbw<9>();
    case 11: return tcd_kbw<11>();
    case 13: return tcd_kbw<13>();
    case 15: return tcd_kbw<15>();
    default: return 0;
  }
}

}  // namespace

bool make_map_2b(CUtensorMap* m, const void* ptr, int rows, int K, int ld, int box_rows, bool bf16);

bool autocorr_tcd_supported(int M, int L) {
  return M >= 5 && M <= 15 && (M % 2) == 1 && L >= 1 && L <= kMaxL && (L % 2) == 1 &&
         TD<15>::SMEM <= 227 * 1024;
}

int tcd_table_rows(int L) {
  const int nhg = (L * L + 1) / 2;
  return 2 * ((nhg + kCN - 1) / kCN) * kCN;
}
int tcd_table_ld(int M) { return kbw_of(M); }

// Constant operand: rows [2][nch * 128] (C part, then S part) of tcd_table_ld(M) F16.
//   C row g (half-grid point, l = grid point g): k = 0 -> 1, k = h -> 2 cos a_h(l);
//   S row g: k = h - 1 -> -2 sin a_h(l); zero elsewhere and for g >= (L^2+1)/2.
void build_tcd_table(int M, int L, double vmax, double vstep, uint16_t* out) {
  const int K = (M - 1) / 2, nh = (M * M - 1) / 2;
  const int nhg = (L * L + 1) / 2, nch = (nhg + kCN - 1) / kCN;
  const int kbw = kbw_of(M);
  std::memset(out, 0, sizeof(uint16_t) * size_t(tcd_table_rows(L)) * kbw);
  std::vector<int> hx(nh + 1), hy(nh + 1);
  int hi = 1;
  for (int ky = 1; ky <= K; ++ky) { hx[hi] = 0; hy[hi] = ky; ++hi; }
  for (int kx = 1; kx <= K; ++kx)
    for (int ky = -K; ky <= K; ++ky) { hx[hi] = kx; hy[hi] = ky; ++hi; }
  auto h16 = [](double v) {
    const __half h = __float2half_rn(float(v));
    uint16_t u;
    std::memcpy(&u, &h, 2);
    return u;
  };
  const double pi = 3.14159265358979323846;
  for (int g = 0; g < nhg; ++g) {
    const double lx = -vmax + (g % L) * vstep, ly = -vmax + (g / L) * vstep;
    uint16_t* rc = out + size_t(g) * kbw;
    uint16_t* rs = out + size_t(nch * kCN + g) * kbw;
    rc[0] = h16(1.0);
    for (int h = 1; h <= nh; ++h) {
      const double ph = 2.0 * pi * (hx[h] * lx + hy[h] * ly) / M;
      rc[h] = h16(2.0 * std::cos(ph));
      rs[h - 1] = h16(-2.0 * std::sin(ph));
    }
  }
}

cudaError_t launch_autocorr_tcd(const TcDenseArgs& a, const void* table, cudaStream_t st) {
  if (!autocorr_tcd_supported(a.M, a.L)) return cudaErrorInvalidValue;
  const int nhg = (a.L * a.L + 1) / 2, nch = (nhg + kCN - 1) / kCN;
  CUtensorMap tm;
  const int kbw = kbw_of(a.M);
  if (!make_map_2b(&tm, table, 2 * nch * kCN, kbw, kbw, kCN, false)) return cudaErrorInvalidValue;
  switch (a.M) {
    case 5: return launch_tcd_m<5>(a, tm, st);
    case 7: return launch_tcd_m<7>(a, tm, st);
    case 9: return launch_tcd_m<9>(a, tm, st);
    case 11: return launch_tcd_m<11>(a, tm, st);
    case 13: return launch_tcd_m<13>(a, tm, st);
    case 15: return launch_tcd_m<15>(a, tm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wh
