// Autocorrelation search with the separable stage on tcgen05 tensor cores
// (Eq. (10) on the lz = 1 slice, exact FP32 argmax).
//
// Separable form (as in k_autocorr.cu):
//   T(kx, ly) = sum_ky Q(kx, ky) e^{j2pi ky ly/M},
//   R(lx, ly) = Re T(0, ly) + 2 sum_{kx>=1} Re(e^{j2pi kx lx/M} T(kx, ly)).
// Stage 1 gives T for every grid row.  Per pixel and kx it is the product of
// the row of Q sums [sr, dr, si, di (ky = 1..K), Qr(kx,0), Qi(kx,0)] with a
// fixed [32 x 2L] matrix (both signs of ly at once:
//   T(kx, +|ly|) = (a - b, c + d), T(kx, -|ly|) = (a + b, d - c),
//   a = Qr0 + sum sr cos, b = sum di sin, c = sum dr sin, d = Qi0 + sum si cos),
// a dense contraction that runs here on the tensor cores in TF32 (kind::tf32,
// F32 accumulation in tensor memory).  Its only use is the row bound
//   R(lx, ly) <= t0(ly) + 2 sum_{kx>=1} |T(kx, ly)|      (Cauchy-Schwarz per kx)
// which is formed from the tensor-core T~ and widened by the TF32 error:
// operands rounded to 10 explicit mantissa bits and |B| <= 1 give
// |T~ - T| <= sqrt(2) 1.53 2^-10 S1(kx), S1 = sum of |Q sums| of (pixel, kx),
// so the widening W = 1.53 2^-10 (S1(0) + 2 sqrt(2) sum_{kx>=1} S1(kx))
// <= 4.23e-3 S, S = the sum over all of a pixel's Q sums (4.5e-3 S is used).
// Stage 2 then evaluates in exact FP32 on CUDA cores, with the operation
// sequence of ac::exact_R and of the CUDA-core search, only the rows whose
// widened bound reaches the exact value of the row with the largest bound;
// a row below it holds neither the maximum nor a tie, so the argmax (ties to
// the lowest flat index iy*L + ix) equals that of the full FP32 evaluation.
//
// Organisation: one CTA per SM walks 64-pixel tiles.  Warp 9 copies a tile's
// smoothed state (64 contiguous rows of KP floats) into shared memory with one
// bulk copy.  Worker warps 0-7 build the tile's Q sums directly in the tensor
// cores' operand layout: K-major, 128-byte swizzle, 128-byte rows (kx, pixel),
// one 8 KB block of 64 rows per kx.  Warp 8 issues the MMAs: M = 128 rows
// (kx even and kx odd of the 64 pixels, two adjacent blocks), N = 64 columns
// (2 gy + re/im), four K = 8 steps per kx pair, into one of two TMEM buffers of
// 4 x 64 columns.  The workers read T~ (TMEM lanes 0-63: kx even, 64-127: kx
// odd), form the bounds, and run stage 2 with 8 lanes per pixel (lane j owns
// the grid columns l_j, l_{j+8} and computes T(kx = j, +-|ly|) of the rows it
// needs).  Q sums and TMEM are double-buffered, so the MMAs of tile i+1 run
// while the workers finish tile i.  Every wait is bounded (~1 s); a timeout
// sets the stream's status word and the CTA stops.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "ac_common.cuh"
#include "common.cuh"
#include "tc_ptx.cuh"

namespace wh {
namespace {

constexpr int kTP = 64;                       // pixels per tile
constexpr int kWorkers = 16;                  // worker warps
constexpr int kWT = kWorkers * 32;            // worker threads
constexpr int kThreads = kWT + 64;            // + MMA warp + producer warp
constexpr int kGroups = kWT / 8;              // 8-lane groups (one pixel each per tile)
constexpr int kUS = kTP + 1;                  // row stride of the bound arrays [gy][pixel] (bank spread)
constexpr uint32_t kTmemCols = 512;           // 2 buffers x 4 kx pairs x 64 columns
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr float kUbRel = 1.0f / 4096.0f;      // relative margin for FP32 rounding (as k_autocorr.cu)
constexpr float kUbAbs = 1.3877788e-17f;      // 2^-56: squares that underflow, subnormal rounding, TF32 flush
constexpr size_t kQBuf = 8ull * kTP * 128;    // one tile's operand: 8 kx blocks of 64 rows x 128 B

__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) & ~size_t(15); }

template <int M>
struct TG {
  static constexpr int K = (M - 1) / 2;
  static constexpr int KP = ac::Geo<M>::KP;
  static constexpr int NH = ac::Geo<M>::NH;
  static constexpr int NE = ac::Geo<M>::NE;
  static constexpr int QIT = (NE + 7) / 8;
  static constexpr int NQ = (K + 2) / 2;                     // kx pairs holding kx <= K
  static constexpr size_t O_Q = 0;                           // [2][8][64][128 B]
  static constexpr size_t O_B = O_Q + 2 * kQBuf;             // [64][32] floats (8 KB)
  static constexpr size_t O_ST = O_B + 8192;                 // [64][KP] floats
  static constexpr size_t O_UB = al16(O_ST + 4ull * kTP * KP);   // [32][kUS] floats
  static constexpr size_t O_PART = al16(O_UB + 4ull * 32 * kUS);  // [32][kUS] floats
  static constexpr size_t O_S = al16(O_PART + 4ull * 32 * kUS);   // [2][64] floats (per operand buffer)
  static constexpr size_t O_PB = O_S + 8ull * kTP;               // [kGroups][2][8] float2
  static constexpr size_t O_TAB = O_PB + 16ull * 8 * kGroups;    // [kMaxL][K+1] float2
  static constexpr size_t O_BAR = al16(O_TAB + 8ull * kMaxL * (K + 1));
  static constexpr size_t SMEM = O_BAR + 8 * 8 + 16 + 1024;      // + 1024-byte alignment slack
  static_assert(K + 1 <= 8, "one lane per kx");
};

// Bounded wait for the single-thread producer and MMA roles: they wait on the
// workers most of the time, so they back off between polls instead of taking
// issue slots from them.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    __nanosleep(200);
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

// Named barrier over the worker warps returning the OR of a predicate (uniform).
__device__ __forceinline__ bool workers_bar_or(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(uint32_t(v)), "n"(kWT)
      : "memory");
  return r != 0;
}

template <int M>
__global__ void __launch_bounds__(kThreads, 1) autocorr_tcsep_kernel(const TcSepArgs a) {
  using G = TG<M>;
  constexpr int K = G::K, KP = G::KP, NH = G::NH, QIT = G::QIT, NQ = G::NQ;
  extern __shared__ uint8_t smem_raw[];
  const uint32_t base_u32 = tc::smem_u32(smem_raw);
  uint8_t* sm = smem_raw + ((1024u - (base_u32 & 1023u)) & 1023u);
  uint8_t* qbuf = sm + G::O_Q;
  float* bop = reinterpret_cast<float*>(sm + G::O_B);
  float* stage = reinterpret_cast<float*>(sm + G::O_ST);
  float* ub = reinterpret_cast<float*>(sm + G::O_UB);
  float* part = reinterpret_cast<float*>(sm + G::O_PART);
  float* sbuf = reinterpret_cast<float*>(sm + G::O_S);
  float2* pbuf = reinterpret_cast<float2*>(sm + G::O_PB);
  float2* tabs = reinterpret_cast<float2*>(sm + G::O_TAB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + G::O_BAR);
  uint64_t* qfull = bar;          // [2] Q sums of the buffer built
  uint64_t* tfull = bar + 2;      // [2] MMAs into the TMEM buffer done
  uint64_t* tempty = bar + 4;     // [2] TMEM buffer read
  uint64_t* sfull = bar + 6;      // staged state landed
  uint64_t* sempty = bar + 7;     // staged state consumed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int npix = a.npix, L = a.L, gc = (L - 1) / 2;
  const int ntiles = (npix + kTP - 1) / kTP;
  const int nct = gridDim.x;
  const int mytiles = int(blockIdx.x) < ntiles ? (ntiles - 1 - int(blockIdx.x)) / nct + 1 : 0;
  auto fail = [&](int code) {
    if (a.err) atomicExch(a.err, code);
    *abort_flag = 1;
  };

  // ---- set-up: barriers, TMEM, the constant operand, zeroed operand buffers
  // (chunks and rows the builders never write stay zero), twiddle table
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&qfull[b], 1);
      tc::mbar_init(&tfull[b], 1);
      tc::mbar_init(&tempty[b], 1);
    }
    tc::mbar_init(sfull, 1);
    tc::mbar_init(sempty, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == kWorkers) {
    tc::tmem_alloc(tmem_slot, kTmemCols);
    tc::tmem_relinquish();
  }
  for (int i = tid; i < 2048; i += kThreads) bop[i] = a.bop[i];
  for (int i = tid; i < int(2 * kQBuf / 16); i += kThreads)
    reinterpret_cast<uint4*>(qbuf)[i] = make_uint4(0u, 0u, 0u, 0u);
  for (int i = tid; i < L * (K + 1); i += kThreads) tabs[i] = a.tab_x[i];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == kWorkers + 1) {
    // ---------------- producer: one bulk copy of a tile's state ----------------
    if (lane == 0) {
      for (int i = 0; i < mytiles && !*abort_flag; ++i) {
        const int tile = int(blockIdx.x) + i * nct;
        if (i > 0 && !mbar_wait_backoff(sempty, uint32_t((i - 1) & 1), kWaitNs)) { fail(31); break; }
        const int n = min(kTP, npix - tile * kTP);
        const uint32_t bytes = uint32_t(n) * KP * 4u;       // KP % 4 == 0: a multiple of 16
        tc::mbar_expect_tx(sfull, bytes);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(tc::smem_u32(stage)), "l"(a.Astate + size_t(tile) * kTP * KP), "r"(bytes),
              "r"(tc::smem_u32(sfull))
            : "memory");
      }
    }
  } else if (warp == kWorkers) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_tf32(128, 64);
      const uint32_t b0 = tc::smem_u32(bop);
      int issued = 0;
      for (int i = 0; i < mytiles; ++i) {
        const int b = i & 1;
        if (!mbar_wait_backoff(&qfull[b], uint32_t((i >> 1) & 1), kWaitNs)) { fail(32); break; }
        if (i >= 2 && !mbar_wait_backoff(&tempty[b], uint32_t(((i >> 1) - 1) & 1), kWaitNs)) { fail(33); break; }
        if (*abort_flag) break;
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(qbuf + b * kQBuf);
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
          for (int k = 0; k < 4; ++k)
            tc::mma_tf32(tmem + uint32_t(b * 256 + q * 64), tc::sdesc_sw128(a0 + q * 2 * 8192 + 32 * k),
                         tc::sdesc_sw128(b0 + 32 * k), idesc, k > 0 ? 1u : 0u);
        tc::mma_commit(&tfull[b]);
        issued = i + 1;
      }
      if (issued > 0)   // the last MMAs finish before TMEM is freed (a no-wait after normal completion)
        mbar_wait_backoff(&tfull[(issued - 1) & 1], uint32_t(((issued - 1) >> 1) & 1), kWaitNs);
    }
  } else {
    // ---------------- workers ----------------
    const int grp = tid >> 3, j = lane & 7;
    const unsigned gmask = 0xFFu << (lane & 24);
    const int Lh = (L + 1) / 2;
    const int l0 = j, l1 = j + 8;
    const bool act0 = l0 < Lh, act1 = l1 < Lh;
    float2 c0[K], c1[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      c0[k] = act0 ? tabs[(gc + l0) * (K + 1) + k + 1] : make_float2(0.f, 0.f);
      c1[k] = act1 ? tabs[(gc + l1) * (K + 1) + k + 1] : make_float2(0.f, 0.f);
    }
    int qoff[QIT];
    ac::qsum_offsets<M, QIT, 8>(j, qoff);
    const float wcoef = a.wcoef;

    // Q sums of tile i (from the staged state) into operand buffer i & 1, and
    // per pixel the sum S of their absolute values
    auto build = [&](int i) -> bool {
      const int b = i & 1, tile = int(blockIdx.x) + i * nct;
      bool bad = !tc::mbar_wait(sfull, uint32_t(i & 1), kWaitNs);
      if (bad) fail(34);
      bad = __any_sync(0xffffffffu, bad);        // warp-uniform: the group shuffles below
      uint8_t* qb = qbuf + b * kQBuf;
      if (!bad) {
        const int pl = grp;
        const bool valid = tile * kTP + pl < npix;
        float s = 0.f;
        if (valid) {
          const float* A = stage + pl * KP;
          const int sw = pl & 7;
#pragma unroll
          for (int r = 0; r < QIT; ++r) {
            const int t = qoff[r];
            if (t >= 0) {
              const int e = j + 8 * r, kx = e / K, ky = e - kx * K;
              const int hp = t & 0xff, hm = (t >> 8) & 0xff;
              const float rp = A[hp], rm = A[hm], ip = A[NH + hp];
              const float im = __int_as_float(__float_as_int(A[NH + hm]) ^ (unsigned(t >> 16) << 31));
              const float4 v = make_float4(rp + rm, rp - rm, ip + im, ip - im);
              *reinterpret_cast<float4*>(qb + kx * 8192 + pl * 128 + ((ky ^ sw) << 4)) = v;
              s += (fabsf(v.x) + fabsf(v.y)) + (fabsf(v.z) + fabsf(v.w));
            }
          }
          if (j <= K) {
            const int h0 = j == 0 ? 0 : K + (j - 1) * M + K + 1;
            const float zr = A[h0], zi = j == 0 ? 0.f : A[NH + h0];
            *reinterpret_cast<float4*>(qb + j * 8192 + pl * 128 + ((7 ^ sw) << 4)) = make_float4(zr, zi, 0.f, 0.f);
            s += fabsf(zr) + fabsf(zi);
          }
        }
        s += __shfl_xor_sync(gmask, s, 4);
        s += __shfl_xor_sync(gmask, s, 2);
        s += __shfl_xor_sync(gmask, s, 1);
        if (j == 0) sbuf[b * kTP + pl] = s;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // operand writes -> tensor cores
      bad = workers_bar_or(bad || *abort_flag);
      if (!bad && tid == 0) {
        tc::mbar_arrive(sempty);
        tc::mbar_arrive(&qfull[b]);
      }
      return !bad;
    };

    // T~ of tile i from TMEM -> widened row bounds ub[pixel][gy]
    auto bounds = [&](int i) -> bool {
      const int b = i & 1;
      bool bad = !tc::mbar_wait(&tfull[b], uint32_t((i >> 1) & 1), kWaitNs);
      if (bad) fail(35);
      bad = __any_sync(0xffffffffu, bad);        // warp-uniform: tcgen05.ld is warp-collective
      tc::tc_fence_after();
      const int qd = warp & 3, par = qd >> 1;
      const int pl = 32 * (qd & 1) + lane;
      const int gy0 = 8 * (warp >> 2);
      float acc[8], t0v[8];
#pragma unroll
      for (int g = 0; g < 8; ++g) { acc[g] = 0.f; t0v[g] = 0.f; }
      if (!bad && gy0 < L) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int kx = 2 * q + par;
          if (kx > K) continue;
          uint32_t r[16];
          tc::tmem_ld16(tmem + (uint32_t(32 * qd) << 16) + uint32_t(b * 256 + q * 64 + 2 * gy0), r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            const float tr = __uint_as_float(r[2 * g]), ti = __uint_as_float(r[2 * g + 1]);
            if (kx == 0) t0v[g] = tr;
            else acc[g] += sqrt_approx(fmaf(tr, tr, ti * ti));
          }
        }
      }
      if (par == 1) {
#pragma unroll
        for (int g = 0; g < 8; ++g) part[(gy0 + g) * kUS + pl] = acc[g];
      }
      tc::tc_fence_before();
      bad = workers_bar_or(bad || *abort_flag);
      if (bad) return false;
      if (tid == 0) tc::mbar_arrive(&tempty[b]);
      if (par == 0) {
        const float W = fmaf(wcoef, sbuf[b * kTP + pl], kUbAbs);
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const int gy = gy0 + g;
          const float t0 = t0v[g], rs = acc[g] + part[gy * kUS + pl];
          ub[gy * kUS + pl] = fmaf(2.f * rs, 1.f + kUbRel, fmaf(kUbRel, fabsf(t0), t0)) + W;
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kWT) : "memory");
      return true;
    };

    // exact stage 2 of tile i (8 lanes per pixel)
    auto stage2 = [&](int i) {
      const int b = i & 1, tile = int(blockIdx.x) + i * nct;
      const uint8_t* qb = qbuf + b * kQBuf;
      float2* pb = pbuf + grp * 16;
      {
        const int pl = grp;
        const int pix = tile * kTP + pl;
        if (pix >= npix) goto done;
        const float* u = ub + pl;     // u[gy * kUS]
        const int sw = pl & 7;
        // T(kx = j, gc +- p) into pb[0][j] (row gc + p) and pb[1][j] (row gc - p)
        auto tpair = [&](int p) {
          __syncwarp(gmask);                         // the previous pair has been read
          if (j <= K) {
            const uint8_t* row = qb + j * 8192 + pl * 128;
            const float4 z = *reinterpret_cast<const float4*>(row + ((7 ^ sw) << 4));
            const float2* cy = tabs + (gc + p) * (K + 1) + 1;
            float2 ac = make_float2(z.x, 0.f), db = make_float2(z.y, 0.f);
#pragma unroll
            for (int ky = 0; ky < K; ++ky) {
              const float4 q = *reinterpret_cast<const float4*>(row + ((ky ^ sw) << 4));
              const float2 c = cy[ky];
              ac = __ffma2_rn(make_float2(q.x, q.y), c, ac);
              db = __ffma2_rn(make_float2(q.z, q.w), c, db);
            }
            pb[j] = make_float2(ac.x - db.y, ac.y + db.x);
            pb[8 + j] = make_float2(ac.x + db.y, db.x - ac.y);
          }
          __syncwarp(gmask);
        };
        float best0 = -INFINITY, best1 = -INFINITY;
        int bi0 = 0x7fffffff, bi1 = 0x7fffffff;
        int fb0 = gc + l0, fb1 = gc + l1;            // row 0's resolution if nothing is taken
        // R(+-l, gy) for this lane's values from the pair slot holding row gy
        auto eval_row = [&](int gy, int slot) {
          const float2* T = pb + 8 * slot;
          const float r0 = T[0].x;
          auto one = [&](const float2 (&cs)[K], int l, float& bb, int& bi, int& fb) {
            float2 v = make_float2(0.f, 0.f);
#pragma unroll
            for (int kx = 1; kx <= K; ++kx) v = __ffma2_rn(cs[kx - 1], T[kx], v);
            const float rp = fmaf(2.f, v.x - v.y, r0), rm = fmaf(2.f, v.x + v.y, r0);
            const bool minus = rm >= rp;             // -l has the lower index
            const float m = minus ? rm : rp;
            const int idx = gy * L + (minus ? gc - l : gc + l);
            if (gy == 0) fb = idx;
            if (m > bb || (m == bb && m > -INFINITY && idx < bi)) { bb = m; bi = idx; }
          };
          if (act0) one(c0, l0, best0, bi0, fb0);
          if (act1) one(c1, l1, best1, bi1, fb1);
        };
        // seed: the row with the largest bound (lowest gy on ties)
        float bu = -INFINITY;
        int bg = 0x7fffffff;
        for (int gy = j; gy < L; gy += 8) {
          const float v = u[gy * kUS];
          if (v > bu || (v == bu && gy < bg)) { bu = v; bg = gy; }
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
          const float ov = __shfl_xor_sync(gmask, bu, off);
          const int og = __shfl_xor_sync(gmask, bg, off);
          if (ov > bu || (ov == bu && og < bg)) { bu = ov; bg = og; }
        }
        if (bg >= L) bg = gc;                        // every bound NaN
        const int ps = bg >= gc ? bg - gc : gc - bg;
        tpair(ps);
        eval_row(bg, bg >= gc ? 0 : 1);
        float seed = fmaxf(best0, best1);
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) seed = fmaxf(seed, __shfl_xor_sync(gmask, seed, off));
        // rows whose widened bound reaches the seed value (every row if it is not finite)
        unsigned need = 0;
        if (isfinite(seed)) {
          for (int gy = j; gy < L; gy += 8)
            if (u[gy * kUS] >= seed) need |= 1u << gy;
#pragma unroll
          for (int off = 4; off > 0; off >>= 1) need |= __shfl_xor_sync(gmask, need, off);
        } else {
          need = (1u << L) - 1u;
        }
        need &= ~(1u << bg);
        const int partner = 2 * gc - bg;
        if (partner != bg && ((need >> partner) & 1u)) {
          eval_row(partner, bg >= gc ? 1 : 0);
          need &= ~(1u << partner);
        }
        while (need) {
          const int gy = __ffs(int(need)) - 1;
          const int p = gy >= gc ? gy - gc : gc - gy;
          tpair(p);
          if ((need >> (gc + p)) & 1u) { eval_row(gc + p, 0); need &= ~(1u << (gc + p)); }
          if (p > 0 && ((need >> (gc - p)) & 1u)) { eval_row(gc - p, 1); need &= ~(1u << (gc - p)); }
        }
        if (bi0 == 0x7fffffff) bi0 = fb0;
        if (bi1 == 0x7fffffff) bi1 = fb1;
        float best = act0 ? best0 : -INFINITY;
        int bidx = act0 ? bi0 : 0x7fffffff;
        if (act1 && (best1 > best || (best1 == best && bi1 < bidx))) { best = best1; bidx = bi1; }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
          const float ob = __shfl_xor_sync(gmask, best, off);
          const int oi = __shfl_xor_sync(gmask, bidx, off);
          if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
        }
        if (j == 0) {
          const int iy = int((float(bidx) + 0.5f) * (1.0f / float(L))), ix = bidx - iy * L;
          a.vidx[pix] = bidx;
          a.vx[pix] = -a.vmax + ix * a.vstep;
          a.vy[pix] = -a.vmax + iy * a.vstep;
        }
      }
    done:
      __syncwarp();
    };

    bool ok = true;
    for (int i = 0; i < mytiles && ok; ++i) {
      ok = build(i);
      if (ok && i > 0) {
        ok = bounds(i - 1);
        if (ok) stage2(i - 1);
      }
    }
    if (ok && mytiles > 0 && bounds(mytiles - 1)) stage2(mytiles - 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == kWorkers) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

template <int M>
cudaError_t launch_tcsep_m(const TcSepArgs& a, cudaStream_t st) {
  using G = TG<M>;
  if (a.kpad != G::KP) return cudaErrorInvalidValue;
  ResidentShape rs{};
  cudaError_t e = resident_shape(autocorr_tcsep_kernel<M>, kThreads, G::SMEM, &rs);
  if (e != cudaSuccess) return e;
  if (rs.per_sm < 1) return cudaErrorInvalidConfiguration;
  const int ntiles = (a.npix + kTP - 1) / kTP;
  const int grid = ntiles < rs.nsm ? ntiles : rs.nsm;
  if (grid < 1) return cudaSuccess;
  autocorr_tcsep_kernel<M><<<grid, kThreads, G::SMEM, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool autocorr_tcsep_supported(int M, int L) {
  return M >= 5 && M <= 15 && (M % 2) == 1 && L >= 1 && L <= 31 && (L % 2) == 1 &&
         TG<15>::SMEM <= 227 * 1024;
}

cudaError_t launch_autocorr_tcsep(const TcSepArgs& a, cudaStream_t st) {
  if (!autocorr_tcsep_supported(a.M, a.L)) return cudaErrorInvalidValue;
  switch (a.M) {
    case 5: return launch_tcsep_m<5>(a, st);
    case 7: return launch_tcsep_m<7>(a, st);
    case 9: return launch_tcsep_m<9>(a, st);
    case 11: return launch_tcsep_m<11>(a, st);
    case 13: return launch_tcsep_m<13>(a, st);
    case 15: return launch_tcsep_m<15>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wh

namespace wh {

// Host: the stage-1 operand.  Row n = 2 gy + c (c = 0: Re T, 1: Im T of grid
// row gy, jy = gy - gc), column k = 4 (ky - 1) + {0: sr, 1: dr, 2: si, 3: di},
// k = 28: Qr(kx, 0), k = 29: Qi(kx, 0); with theta = 2 pi ky |l(jy)| / M:
//   Re T: sr cos, di (jy >= 0 ? -sin : +sin), Qr0 1;
//   Im T: dr (jy >= 0 ? +sin : -sin), si cos, Qi0 1.
// Values rounded to the nearest TF32 (10 explicit mantissa bits), stored in the
// 128-byte-swizzled K-major layout (16-byte chunk k/4 of row n at k/4 ^ (n % 8)).
void build_tcsep_operand(int M, int L, double vstep, float* out) {
  const int K = (M - 1) / 2, gc = (L - 1) / 2;
  const double vmax = gc * vstep, pi = 3.14159265358979323846;
  for (int i = 0; i < 64 * 32; ++i) out[i] = 0.f;
  auto put = [&](int n, int k, double v) {
    float f = float(v);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) {
      u += 0xfffu + ((u >> 13) & 1u);
      u &= 0xffffe000u;
    }
    std::memcpy(&f, &u, 4);
    out[n * 32 + (((k >> 2) ^ (n & 7)) << 2) + (k & 3)] = f;
  };
  for (int gy = 0; gy < L; ++gy) {
    const int jy = gy - gc, p = jy < 0 ? -jy : jy;
    const double l = -vmax + (gc + p) * vstep;
    const double sg = jy >= 0 ? 1.0 : -1.0;
    for (int ky = 1; ky <= K; ++ky) {
      const double th = 2.0 * pi * ky * l / M, c = std::cos(th), s = std::sin(th);
      const int k0 = 4 * (ky - 1);
      put(2 * gy, k0 + 0, c);
      put(2 * gy, k0 + 3, -sg * s);
      put(2 * gy + 1, k0 + 1, sg * s);
      put(2 * gy + 1, k0 + 2, c);
    }
    put(2 * gy, 28, 1.0);
    put(2 * gy + 1, 29, 1.0);
  }
}

}  // namespace wh

// C ABI: the stage-1 operand as the tensor-core search uses it (host only).
extern "C" int wh_tcsep_operand(int window, int grid_len, double step, float* out) {
  if (!out || window < 5 || window > 15 || (window % 2) == 0 || grid_len < 1 || grid_len > 31 ||
      (grid_len % 2) == 0 || !(step > 0.0))
    return -1;
  wh::build_tcsep_operand(window, grid_len, step, out);
  return 0;
}
