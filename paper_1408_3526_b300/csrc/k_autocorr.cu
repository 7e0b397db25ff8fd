// Autocorrelation on the velocity grid + argmax, exact FP32 on CUDA cores.
//
// Eq. (10) on the lz = 1 slice: R(l) = sum_k P(k) cos(2pi(kx lx/M + ky ly/M + kz/Mz)).
// With A_c/A_s the kz-reduced (and smoothed) power held in the stream state,
// Q(kx,ky) = A_c + j A_s satisfies Q(-k) = conj(Q(k)) and
//   R(lx,ly) = Re T(0,ly) + 2 sum_{kx=1..K} Re(e^{j2pi kx lx/M} T(kx,ly)),
//   T(kx,ly) = sum_{ky=-K..K} Q(kx,ky) e^{j2pi ky ly/M}.
// The grid is symmetric (l and -l both on it), so with
//   a = Qr(kx,0) + sum_{ky>0} (Qr(ky)+Qr(-ky)) cos,  b = sum_{ky>0} (Qi(ky)-Qi(-ky)) sin,
//   c = sum_{ky>0} (Qr(ky)-Qr(-ky)) sin,             d = Qi(kx,0) + sum_{ky>0} (Qi(ky)+Qi(-ky)) cos
// one pass gives T(kx,+ly) = (a-b, c+d) and T(kx,-ly) = (a+b, d-c); likewise
// one pass over kx gives R(+lx,ly) and R(-lx,ly).  The velocity is the grid
// point of the largest R (v = l/lz, lz = 1); ties go to the lowest flat
// index iy*L + ix.
//
// Mapping: a warp works on four pixels, one per 8-lane group, and lane j owns
// two grid values l_j and l_{j+8} (twiddles for both in registers), so every
// broadcast shared-memory load feeds four packed FMAs.  Stage 1: lane j
// computes T(kx, +-ly) for its two ly from the pixel's Q sums.  Stage 2: lane
// j computes R(+-lx, ly) for its two lx, reading T(., ly) two ly rows per
// 16-byte load.  The (cos, sin) x (re, im) products run as packed FP32x2 FMAs,
// each component rounded exactly as fmaf, in the same order as ac::exact_R.
// Stage 2 evaluates only the rows whose upper bound reaches the value of the
// most promising row (exact pruning, see the row bounds below).
#include "ac_common.cuh"
#include "common.cuh"

namespace wh {
namespace {

constexpr int kWarps4 = 4;

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr int kGrp = 8;       // lanes per pixel; each owns two grid values, so (L+1)/2 <= 16

template <int M, bool RS, int LP>
__global__ void __launch_bounds__(kWarps4 * 32) autocorr_kernel(const AutocorrArgs a) {
  using GE = ac::Geo<M>;
  constexpr int K = GE::K, KP = GE::KP;
  constexpr int QS = GE::QN + 4;                // Q-sum stride: the four groups' broadcasts in distinct banks
  constexpr int TS = (K + 1) * LP + 2;          // T stride (float2): likewise
  const int L = a.L, Lh = (L + 1) / 2, gc = (L - 1) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int grp = lane >> 3, j = lane & 7;
  const int slot = wid * 4 + grp;               // pixel slot in the block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sbase = reinterpret_cast<float*>(smem_raw);
  constexpr int NSLOT = kWarps4 * 4;
  // one state-row buffer per pixel slot: the next pixel's row is fetched into
  // it as soon as the Q sums of this one are built (it lands during the stages)
  float* abuf = sbase + slot * KP;                                              // [KP]
  float* qbuf = sbase + NSLOT * KP + slot * QS;                                 // [QN]
  // T buffers in the order (group, warp), groups 2 and 3 shifted by 4 words: the
  // two groups of a half warp then sit 4 TS 8-byte words apart, 8 (mod 16)
  // whenever TS = 2 (mod 4) (M = 7, 11, 15, or LP = 32), so their stage-1
  // stores of 8 consecutive words fall on complementary banks, and the four
  // groups' 4-byte broadcast reads of T(0, row) fall on four distinct banks
  const int tslot = grp * kWarps4 + wid;
  float2* tbuf = reinterpret_cast<float2*>(sbase + NSLOT * (KP + QS)) + tslot * TS + ((grp & 2) ? 4 : 0);   // [K+1][LP]
  const bool act0 = j < Lh, act1 = j + kGrp < Lh;
  const int l0 = j, l1 = j + kGrp;
  float2 c0[K], c1[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    c0[k] = act0 ? a.tab_x[(gc + l0) * (K + 1) + k + 1] : make_float2(0.f, 0.f);
    c1[k] = act1 ? a.tab_x[(gc + l1) * (K + 1) + k + 1] : make_float2(0.f, 0.f);
  }
  constexpr int QIT = (GE::NE + kGrp - 1) / kGrp;
  int qoff[QIT];
  ac::qsum_offsets<M, QIT, kGrp>(j, qoff);
  const float invL = 1.0f / float(L);
  const long long npix = a.pix_list ? (long long)*a.n_list : (long long)a.H * a.W;
  const long long stride = (long long)gridDim.x * NSLOT;
  auto pixel_of = [&](long long b) -> long long { return a.pix_list ? (long long)a.pix_list[b] : b; };
  auto prefetch = [&](long long b) {
    ac::prefetch_row<M, kGrp>(abuf, a.Astate + (b < npix ? pixel_of(b) : 0) * KP, j, b < npix);
  };
  long long base = ((long long)blockIdx.x * kWarps4 + wid) * 4;
  prefetch(base + grp);
  for (; base < npix; base += stride) {
    const bool valid = base + grp < npix;
    const long long pix = valid ? pixel_of(base + grp) : 0;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    if (valid) ac::build_qsums<M, QIT, kGrp>(abuf, qbuf, qoff, j);
    __syncwarp();                       // every lane's reads of abuf are done
    prefetch(base + stride + grp);
    // ---- stage 1: T(kx, +-ly) for ly = l_j, l_{j+8} ---------------------------
    // Each lane also accumulates, for its four rows gc +- l_j, gc +- l_{j+8},
    // t0 = Re T(0, ly) and sum_{kx>=1} |T(kx, ly)| for the row bounds below.
    float rt0[4], rsa[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) { rt0[t] = 0.f; rsa[t] = 0.f; }
    if (valid && act0) {
      const float4* q4 = reinterpret_cast<const float4*>(qbuf);
      const float2* q0 = reinterpret_cast<const float2*>(qbuf + 4 * (K + 1) * K);
      auto acc = [&](int kx, int t, float2 tv) {
        if (kx == 0) rt0[t] = tv.x;
        else if (!RS) rsa[t] += sqrt_approx(fmaf(tv.x, tv.x, tv.y * tv.y));
      };
#pragma unroll
      for (int kx = 0; kx <= K; ++kx) {
        const float2 z = q0[kx];
        float2 ac0 = make_float2(z.x, 0.f), db0 = make_float2(z.y, 0.f);
        float2 ac1 = ac0, db1 = db0;
#pragma unroll
        for (int ky = 0; ky < K; ++ky) {
          const float4 q = q4[kx * K + ky];
          ac0 = __ffma2_rn(make_float2(q.x, q.y), c0[ky], ac0);
          db0 = __ffma2_rn(make_float2(q.z, q.w), c0[ky], db0);
          ac1 = __ffma2_rn(make_float2(q.x, q.y), c1[ky], ac1);
          db1 = __ffma2_rn(make_float2(q.z, q.w), c1[ky], db1);
        }
        const float2 tp0 = make_float2(ac0.x - db0.y, ac0.y + db0.x);
        const float2 tm0 = make_float2(ac0.x + db0.y, db0.x - ac0.y);
        tbuf[kx * LP + gc + l0] = tp0;
        tbuf[kx * LP + gc - l0] = tm0;
        acc(kx, 0, tp0);
        acc(kx, 1, tm0);
        if (act1) {
          const float2 tp1 = make_float2(ac1.x - db1.y, ac1.y + db1.x);
          const float2 tm1 = make_float2(ac1.x + db1.y, db1.x - ac1.y);
          tbuf[kx * LP + gc + l1] = tp1;
          tbuf[kx * LP + gc - l1] = tm1;
          acc(kx, 2, tp1);
          acc(kx, 3, tm1);
        }
      }
    }
    __syncwarp();
    // ---- stage 2: R(+-lx, ly) for lx = l_j, l_{j+8}, and the argmax -----------
    // R(+lx) = t0 + 2(v1 - v2), R(-lx) = t0 + 2(v1 + v2); their larger one is
    // exactly t0 + 2(v1 + |v2|) (the same rounded operations).  Per owned value
    // the rows arrive in increasing flat index, so the first row reaching the
    // value's maximum is kept and its -lx / +lx resolved at the end; values and
    // lanes then combine by (largest R, lowest flat index).
    auto row_v = [&](const float2 (&cs)[K], int gy) {
      float2 v = make_float2(0.f, 0.f);
#pragma unroll
      for (int kx = 1; kx <= K; ++kx) v = __ffma2_rn(cs[kx - 1], tbuf[kx * LP + gy], v);
      return v;
    };
    auto mval = [](float r0, float2 v) { return fmaf(2.f, v.x + fabsf(v.y), r0); };
    // Row bounds: R(lx, ly) <= t0 + 2 sum_kx |T(kx, ly)| (Cauchy-Schwarz per kx,
    // |(cos, sin)| = 1).  The relative margin 2^-12 covers every FP32 rounding
    // of the evaluated R (~1e-6) and of the bound, whose square roots are the
    // hardware approximation (relative error ~2^-22).  The row with the largest
    // bound is evaluated first; a row whose bound is below that value holds no
    // maximum (nor a tie), so only the row pairs with a row reaching it are
    // evaluated, in increasing order, and the argmax is exactly that of the
    // full evaluation.
    // An absolute floor of 2^-56 covers |T| whose square underflows (|T| below
    // 2^-63 per kx) and the absolute rounding of R in the subnormal range.
    constexpr float kUbRel = 1.0f / 4096.0f, kUbAbs = 1.3877788e-17f;
    const unsigned all_pairs = (1u << ((L + 1) / 2)) - 1u;
    unsigned pairs = all_pairs;
    if (!RS) {
      // this lane's rows gc + l_j, gc - l_j, gc + l_{j+8}, gc - l_{j+8} (the
      // second copy of row gc for l_j = 0 left out)
      const int rows[4] = {gc + l0, gc - l0, gc + l1, gc - l1};
      const bool own[4] = {valid && act0, valid && act0 && l0 > 0, valid && act1, valid && act1};
      float u[4];
      float um = -INFINITY;
      int ur = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        u[t] = own[t] ? fmaf(2.f * rsa[t], 1.f + kUbRel, fmaf(kUbRel, fabsf(rt0[t]), rt0[t])) + kUbAbs
                      : -INFINITY;
        if (u[t] > um || (u[t] == um && own[t] && rows[t] < ur)) { um = u[t]; ur = rows[t]; }
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        const float ou = __shfl_xor_sync(0xffffffffu, um, off);
        const int orow = __shfl_xor_sync(0xffffffffu, ur, off);
        if (ou > um || (ou == um && orow < ur)) { um = ou; ur = orow; }
      }
      float seed = -INFINITY;
      if (valid && act0) {
        const float r0 = tbuf[ur].x;
        seed = mval(r0, row_v(c0, ur));
        if (act1) seed = fmaxf(seed, mval(r0, row_v(c1, ur)));
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) seed = fmaxf(seed, __shfl_xor_sync(0xffffffffu, seed, off));
      unsigned need = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (own[t] && u[t] >= seed) need |= 1u << (rows[t] >> 1);
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) need |= __shfl_xor_sync(0xffffffffu, need, off);
      if (isfinite(seed)) pairs = need & all_pairs;
    }
    float best = -INFINITY;
    int bidx = 0x7fffffff;
    if (valid && act0) {
      float b0 = -INFINITY, b1 = -INFINITY;
      int g0 = 0, g1 = 0;
      auto take = [&](float r0, float2 v, int gy, int l, float& bb, int& bg) {
        if (RS) {
          a.rs_out[pix * (L * L) + gy * L + gc + l] = fmaf(2.f, v.x - v.y, r0);
          if (l) a.rs_out[pix * (L * L) + gy * L + gc - l] = fmaf(2.f, v.x + v.y, r0);
        }
        const float m = fmaf(2.f, v.x + fabsf(v.y), r0);
        if (m > bb) { bb = m; bg = gy; }
      };
      for (unsigned pm = pairs; pm; pm &= pm - 1) {
        const int gy = 2 * (__ffs(pm) - 1);
        if (gy + 1 >= L) {                 // the last row of an odd grid
          take(tbuf[gy].x, row_v(c0, gy), gy, l0, b0, g0);
          if (act1) take(tbuf[gy].x, row_v(c1, gy), gy, l1, b1, g1);
          continue;
        }
        float2 v00 = make_float2(0.f, 0.f), v01 = v00, v10 = v00, v11 = v00;
#pragma unroll
        for (int kx = 1; kx <= K; ++kx) {
          const float4 t = *reinterpret_cast<const float4*>(tbuf + kx * LP + gy);
          v00 = __ffma2_rn(c0[kx - 1], make_float2(t.x, t.y), v00);
          v01 = __ffma2_rn(c0[kx - 1], make_float2(t.z, t.w), v01);
          v10 = __ffma2_rn(c1[kx - 1], make_float2(t.x, t.y), v10);
          v11 = __ffma2_rn(c1[kx - 1], make_float2(t.z, t.w), v11);
        }
        const float4 t0 = *reinterpret_cast<const float4*>(tbuf + gy);
        take(t0.x, v00, gy, l0, b0, g0);
        take(t0.z, v01, gy + 1, l0, b0, g0);
        if (act1) {
          take(t0.x, v10, gy, l1, b1, g1);
          take(t0.z, v11, gy + 1, l1, b1, g1);
        }
      }
      // resolve -lx / +lx within each value's best row (-lx has the lower index)
      auto resolve = [&](const float2 (&cs)[K], int bg, int l) {
        const float2 v = row_v(cs, bg);
        const float r0 = tbuf[bg].x;
        const float rp = fmaf(2.f, v.x - v.y, r0), rm = fmaf(2.f, v.x + v.y, r0);
        return bg * L + (rm >= rp ? gc - l : gc + l);
      };
      best = b0;
      bidx = resolve(c0, g0, l0);
      if (act1) {
        const int i1 = resolve(c1, g1, l1);
        if (b1 > best || (b1 == best && i1 < bidx)) { best = b1; bidx = i1; }
      }
    }
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (valid && j == 0) {
      const int iy = int((float(bidx) + 0.5f) * invL), ix = bidx - iy * L;   // exact: bidx < 31^2
      a.vidx[pix] = bidx;
      a.vx[pix] = -a.vmax + ix * a.vstep;
      a.vy[pix] = -a.vmax + iy * a.vstep;
    }
    __syncwarp();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int M, int LP>
cudaError_t launch_mp(const AutocorrArgs& a, cudaStream_t st) {
  using GE = ac::Geo<M>;
  constexpr int K = GE::K, NSLOT = kWarps4 * 4;
  const size_t smem = sizeof(float) * size_t(NSLOT) * (GE::KP + GE::QN + 4) +
                      sizeof(float2) * (size_t(NSLOT) * ((K + 1) * LP + 2) + 4);
  const long long npix = (long long)a.H * a.W;   // a pixel list is at most this long
  auto kern = a.rs_out ? autocorr_kernel<M, true, LP> : autocorr_kernel<M, false, LP>;
  // all of the SM's unified L1/shared storage as shared memory: four blocks
  // (16 warps) fit at M = 15, L <= 25 (the kernel re-reads nothing through L1)
  ResidentShape rs{};
  cudaError_t e = resident_shape(kern, kWarps4 * 32, smem, &rs, 100);
  if (e != cudaSuccess) return e;
  const int nsm = rs.nsm, per_sm = rs.per_sm < 1 ? 1 : rs.per_sm;
  long long blocks = (npix + NSLOT - 1) / NSLOT;
  if (blocks > (long long)nsm * per_sm) blocks = (long long)nsm * per_sm;
  kern<<<unsigned(blocks), kWarps4 * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_m(const AutocorrArgs& a, cudaStream_t st) {
  if (a.kpad != ac::Geo<M>::KP) return cudaErrorInvalidValue;
  return a.L <= 25 ? launch_mp<M, 26>(a, st) : launch_mp<M, 32>(a, st);
}

}  // namespace

cudaError_t launch_autocorr(const AutocorrArgs& a, cudaStream_t st) {
  if ((a.L + 1) / 2 > 2 * kGrp || (a.L % 2) == 0) return cudaErrorInvalidValue;
  switch (a.M) {
    case 5: return launch_m<5>(a, st);
    case 7: return launch_m<7>(a, st);
    case 9: return launch_m<9>(a, st);
    case 11: return launch_m<11>(a, st);
    case 13: return launch_m<13>(a, st);
    case 15: return launch_m<15>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wh
