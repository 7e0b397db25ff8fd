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
// Mapping: a warp works on two pixels, one per half-warp.  Stage 1: lane j
// owns ly = +-l_j (twiddles for its ly in registers) and reads the pixel's
// Q sums from shared memory by broadcast.  Stage 2: lane j owns lx = +-l_j
// and reads T(., ly) by broadcast, two ly rows per 16-byte load.  The
// (cos, sin) x (re, im) products run as packed FP32x2 FMAs, each component
// rounded exactly as fmaf.
#include "ac_common.cuh"
#include "common.cuh"

namespace wh {
namespace {

constexpr int kWarps = 8;
constexpr int kHalf = 16;   // lanes per pixel; the grid half-length (L+1)/2 must fit

template <int M>
struct AcSmem {
  static constexpr int kQ = ac::Geo<M>::QN;
  static constexpr int kPad = ac::Geo<M>::KP;
};

// LP: row stride of the T buffer (even, >= L): 26 covers the common grids up
// to L = 25 and lets three blocks share an SM; 32 covers L <= 31.
template <int M, bool RS, int LP>
__global__ void __launch_bounds__(kWarps * 32) autocorr_kernel(const AutocorrArgs a) {
  constexpr int K = (M - 1) / 2;
  constexpr int QN = AcSmem<M>::kQ, KP = AcSmem<M>::kPad;
  const int L = a.L, Lh = (L + 1) / 2, gc = (L - 1) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int half = lane >> 4, j = lane & 15;
  const int hw = wid * 2 + half;                        // half-warp (pixel slot) in the block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sbase = reinterpret_cast<float*>(smem_raw);
  float* abuf = sbase + hw * 2 * KP;                                                    // [2][KP]
  float* qbuf = sbase + kWarps * 2 * 2 * KP + hw * QN;                                  // [QN]
  constexpr int Lp = LP;          // row stride (>= L, even: rows gy, gy+1 load as one float4)
  // per half-warp T buffer, padded by 64 bytes so the two half-warps' broadcast
  // loads fall in different shared-memory banks
  constexpr int TS = (K + 1) * Lp + 8;
  float2* tbuf = reinterpret_cast<float2*>(sbase + kWarps * 2 * (2 * KP + QN)) + hw * TS;   // [K+1][Lp]
  // lane-owned twiddles (cos, sin)(2pi k l_j / M), k = 1..K, l_j = j-th grid value >= 0
  float2 cs[K];
  const bool act = j < Lh;
#pragma unroll
  for (int k = 0; k < K; ++k) cs[k] = act ? a.tab_x[(gc + j) * (K + 1) + k + 1] : make_float2(0.f, 0.f);
  constexpr int QIT = (ac::Geo<M>::NE + kHalf - 1) / kHalf;
  int qoff[QIT];
  ac::qsum_offsets<M, QIT>(j, qoff);
  const float invL = 1.0f / float(L);
  const long long npix = a.pix_list ? (long long)*a.n_list : (long long)a.H * a.W;
  const long long stride = (long long)gridDim.x * kWarps * 2;
  auto pixel_of = [&](long long b) -> long long {
    return a.pix_list ? (long long)a.pix_list[b] : b;
  };
  // the state row of this half-warp's pixel at b -> abuf slot (16-byte copies)
  auto prefetch = [&](long long b, int slot) {
    ac::prefetch_row<M>(abuf + slot * KP, a.Astate + (b < npix ? pixel_of(b) : 0) * KP, j, b < npix);
  };
  long long base = ((long long)blockIdx.x * kWarps + wid) * 2;
  prefetch(base + half, 0);
  for (int it = 0; base < npix; base += stride, ++it) {
    const bool valid = base + half < npix;
    const long long pix = valid ? pixel_of(base + half) : 0;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    prefetch(base + stride + half, (it + 1) & 1);
    // ---- Q sums of this half-warp's pixel ----------------------------------
    if (valid) ac::build_qsums<M, QIT>(abuf + (it & 1) * KP, qbuf, qoff, j);
    __syncwarp();
    // ---- stage 1: T(kx, +-ly_j) ---------------------------------------------
    if (valid && act) {
      const float4* q4 = reinterpret_cast<const float4*>(qbuf);
      const float2* q0 = reinterpret_cast<const float2*>(qbuf + 4 * (K + 1) * K);
#pragma unroll 2
      for (int kx = 0; kx <= K; ++kx) {
        const float2 z = q0[kx];
        float2 ac = make_float2(z.x, 0.f);   // (a, c)
        float2 db = make_float2(z.y, 0.f);   // (d, b)
#pragma unroll
        for (int ky = 0; ky < K; ++ky) {
          const float4 q = q4[kx * K + ky];
          ac = __ffma2_rn(make_float2(q.x, q.y), cs[ky], ac);
          db = __ffma2_rn(make_float2(q.z, q.w), cs[ky], db);
        }
        tbuf[kx * Lp + gc + j] = make_float2(ac.x - db.y, ac.y + db.x);
        tbuf[kx * Lp + gc - j] = make_float2(ac.x + db.y, db.x - ac.y);
      }
    }
    __syncwarp();
    // ---- stage 2: R(+-lx_j, ly) and argmax ------------------------------------
    // R(+lx) = t0 + 2(v1 - v2), R(-lx) = t0 + 2(v1 + v2); their larger one is
    // exactly t0 + 2(v1 + |v2|) (the same rounded operations).  Candidates reach
    // this lane in increasing flat index (R(-lx) before R(+lx), row by row), so
    // the first row reaching the maximum is kept and resolved at the end.
    float best = -INFINITY;
    int bidx = 0x7fffffff;
    if (valid && act) {
      int bgy = 0;
      auto row_v = [&](int gy) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int kx = 1; kx <= K; ++kx) v = __ffma2_rn(cs[kx - 1], tbuf[kx * Lp + gy], v);
        return v;
      };
      auto take = [&](float r0, float2 v, int gy) {
        if (RS) {
          a.rs_out[pix * (L * L) + gy * L + gc + j] = fmaf(2.f, v.x - v.y, r0);
          if (j) a.rs_out[pix * (L * L) + gy * L + gc - j] = fmaf(2.f, v.x + v.y, r0);
        }
        const float m = fmaf(2.f, v.x + fabsf(v.y), r0);
        if (m > best) { best = m; bgy = gy; }
      };
      int gy = 0;
      for (; gy + 1 < L; gy += 2) {
        float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
#pragma unroll
        for (int kx = 1; kx <= K; ++kx) {
          const float4 t = *reinterpret_cast<const float4*>(tbuf + kx * Lp + gy);
          v0 = __ffma2_rn(cs[kx - 1], make_float2(t.x, t.y), v0);
          v1 = __ffma2_rn(cs[kx - 1], make_float2(t.z, t.w), v1);
        }
        const float4 t0 = *reinterpret_cast<const float4*>(tbuf + gy);
        take(t0.x, v0, gy);
        take(t0.z, v1, gy + 1);
      }
      if (gy < L) take(tbuf[gy].x, row_v(gy), gy);
      // which of R(-lx), R(+lx) of the best row holds the maximum (-lx first)
      const float2 v = row_v(bgy);
      const float r0 = tbuf[bgy].x;
      const float rp = fmaf(2.f, v.x - v.y, r0), rm = fmaf(2.f, v.x + v.y, r0);
      bidx = bgy * L + (rm >= rp ? gc - j : gc + j);
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
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
  constexpr int K = (M - 1) / 2;
  const size_t smem = sizeof(float) * size_t(kWarps) * 2 * (2 * AcSmem<M>::kPad + AcSmem<M>::kQ) +
                      sizeof(float2) * size_t(kWarps) * 2 * ((K + 1) * LP + 8);
  const long long npix = (long long)a.H * a.W;
  auto kern = a.rs_out ? autocorr_kernel<M, true, LP> : autocorr_kernel<M, false, LP>;
  // one resident wave (blocks per SM from the occupancy of this shape), the
  // pixel pairs strided over it, so no partial last wave idles SMs
  ResidentShape rs{};
  cudaError_t e = resident_shape(kern, kWarps * 32, smem, &rs);
  if (e != cudaSuccess) return e;
  const int nsm = rs.nsm, per_sm = rs.per_sm < 1 ? 1 : rs.per_sm;
  long long blocks = (npix + 2 * kWarps - 1) / (2 * kWarps);
  if (blocks > (long long)nsm * per_sm) blocks = (long long)nsm * per_sm;
  kern<<<unsigned(blocks), kWarps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_m(const AutocorrArgs& a, cudaStream_t st) {
  if (a.kpad != AcSmem<M>::kPad) return cudaErrorInvalidValue;
  return a.L <= 25 ? launch_mp<M, 26>(a, st) : launch_mp<M, 2 * kHalf>(a, st);
}

}  // namespace

cudaError_t launch_autocorr(const AutocorrArgs& a, cudaStream_t st) {
  if ((a.L + 1) / 2 > kHalf || (a.L % 2) == 0) return cudaErrorInvalidValue;
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
