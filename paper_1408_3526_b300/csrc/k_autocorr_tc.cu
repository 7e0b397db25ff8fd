// Autocorrelation search with the contraction on tcgen05 tensor cores.
//
// R(l) = sum_k a_k B(l,k) (Eq. (10) on the lz = 1 slice, in the kz-reduced
// basis of the stream state: a = [A_c(0), A_c(h), A_s(h)], B(l,.) = [1,
// 2 cos a_h(l), -2 sin a_h(l)]) is a dense [pixels x M^2] x [M^2 x L^2]
// contraction.  Three steps:
//   1. ac_convert: per pixel, scale a by a power of two so max|a| < 1 (the
//      argmax is scale-invariant and the scaling is exact) and round to F16
//      (or BF16); also keep sum|a~| for the error bound.
//   2. tcgen05 contraction [pixels x 232] x [232 x 640] (persistent, the
//      pixel block resident while the grid table streams; tc_rgemm.cu) whose
//      epilogue keeps each pixel's 8 largest R~(l) over the whole grid.
//   3. ac_rerank (FP32-exact mode): every shortlisted l with R~(l) >= max R~ -
//      2E is re-evaluated exactly in FP32 on CUDA cores (separable form, as in
//      the CUDA-core search) and the largest wins (ties -> lowest index).  E
//      bounds |R~ - R| from the operand rounding (2^-11 relative per F16
//      operand, 2^-25 absolute below the normal range, |B| <= 2) and F32
//      accumulation of 225 terms.  If the last entry of a shortlist group is
//      inside the window the shortlist may be incomplete and the whole grid is
//      evaluated exactly for that pixel.  The result equals the exact FP32 argmax.
//      Precision-study modes (F16 / BF16 alone) take the GEMM's best directly.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace wh {
namespace {

constexpr int kWarpsR = 8;

template <int M, bool BF16>
__global__ void __launch_bounds__(256) ac_convert_kernel(const AutocorrTcArgs a) {
  const int lane = threadIdx.x & 31;
  const long long npix = (long long)a.H * a.W;
  const int nk = M * M;
  for (long long pix = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pix < npix;
       pix += ((long long)gridDim.x * blockDim.x) >> 5) {
    const float* src = a.Astate + pix * a.kpad;
    float v[8];
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = lane + 32 * i;
      v[i] = k < nk ? src[k] : 0.f;
      mx = fmaxf(mx, fabsf(v[i]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    // power-of-two scale: max |a| * s in [0.5, 1)
    int e = 0;
    if (mx > 0.f) frexpf(mx, &e);
    const float s = mx > 0.f ? ldexpf(1.f, -e) : 1.f;
    float l1 = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = lane + 32 * i;
      if (k < a.kg) {
        const float x = v[i] * s;
        if (BF16) {
          const __nv_bfloat16 h = __float2bfloat16(x);
          reinterpret_cast<__nv_bfloat16*>(a.a16)[pix * a.kg + k] = h;
          l1 += fabsf(__bfloat162float(h));
        } else {
          const __half h = __float2half_rn(x);
          reinterpret_cast<__half*>(a.a16)[pix * a.kg + k] = h;
          l1 += fabsf(__half2float(h));
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
    if (lane == 0) a.l1[pix] = l1;
  }
}

// Exact FP32 R at flat grid index g from the pixel's Q sums (layout as in
// the CUDA-core search: [K+1][K] x (sr, dr, si, di), then Q(kx,0)).
template <int M>
__device__ __forceinline__ float exact_R(const float* qbuf, const float2* tabx, int L, int g) {
  constexpr int K = (M - 1) / 2;
  const int gc = (L - 1) / 2;
  const int gy = g / L, gx = g % L;
  const int jy = gy - gc, jx = gx - gc;
  const float2* ty = tabx + (gc + (jy < 0 ? -jy : jy)) * (K + 1);   // cos/sin(2pi k |ly|/M)
  const float2* tx = tabx + (gc + (jx < 0 ? -jx : jx)) * (K + 1);
  const float4* q4 = reinterpret_cast<const float4*>(qbuf);
  const float2* q0 = reinterpret_cast<const float2*>(qbuf + 4 * (K + 1) * K);
  float ry[K], iy[K];                 // cos/sin(2pi ky |ly|/M), ky = 1..K
#pragma unroll
  for (int ky = 0; ky < K; ++ky) { const float2 w = ty[ky + 1]; ry[ky] = w.x; iy[ky] = w.y; }
  float t0r = 0.f, v1 = 0.f, v2 = 0.f;
#pragma unroll 1
  for (int kx = 0; kx <= K; ++kx) {
    const float2 z = q0[kx];
    float va = z.x, vb = 0.f, vc = 0.f, vd = z.y;
#pragma unroll
    for (int ky = 0; ky < K; ++ky) {
      const float4 q = q4[kx * K + ky];
      va = fmaf(q.x, ry[ky], va);
      vb = fmaf(q.w, iy[ky], vb);
      vc = fmaf(q.y, iy[ky], vc);
      vd = fmaf(q.z, ry[ky], vd);
    }
    const float tr = jy >= 0 ? va - vb : va + vb;
    const float ti = jy >= 0 ? vc + vd : vd - vc;
    if (kx == 0) t0r = tr;
    else {
      const float2 w = tx[kx];
      v1 = fmaf(w.x, tr, v1);
      v2 = fmaf(w.y, ti, v2);
    }
  }
  return jx >= 0 ? fmaf(2.f, v1 - v2, t0r) : fmaf(2.f, v1 + v2, t0r);
}

template <int M>
__global__ void __launch_bounds__(kWarpsR * 32, 4) ac_rerank_kernel(const AutocorrTcArgs a) {
  constexpr int K = (M - 1) / 2;
  constexpr int QN = (4 * (K + 1) * K + 2 * (K + 1) + 3) & ~3;
  const int L = a.L, nh = (M * M - 1) / 2, ncand = a.ncand, og = a.ovf_group;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tabx = reinterpret_cast<float2*>(smem_raw);                            // [L][K+1]
  float* qbuf = reinterpret_cast<float*>(tabx + ((L * (K + 1) + 1) & ~1)) + wid * QN;
  for (int i = threadIdx.x; i < L * (K + 1); i += blockDim.x) tabx[i] = a.tab_x[i];
  __syncthreads();
  const long long npix = (long long)a.H * a.W;
  for (long long pix = (long long)blockIdx.x * kWarpsR + wid; pix < npix;
       pix += (long long)gridDim.x * kWarpsR) {
    // shortlist
    float cv = -INFINITY;
    int ci = 0x7fffffff;
    if (lane < ncand) {
      cv = a.cand_val[pix * ncand + lane];
      ci = a.cand_idx[pix * ncand + lane];
    }
    float vmax = cv;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    int best_i;
    if (a.mode != 0) {
      // precision study: the tensor-core value decides (ties -> lowest index)
      int bi = (cv == vmax) ? ci : 0x7fffffff;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) bi = min(bi, __shfl_xor_sync(0xffffffffu, bi, off));
      best_i = bi;
    } else {
      // |R~ - R| <= sum_k (|da_k||B| + |a_k||dB|) + accumulation <= 2^-9 sum|a~| (F16
      // operands, |B| <= 2) + 225 * 2^-23 * 2 sum|a~| + subnormal flush of a~ (2^-25 each)
      const float E = 2.05e-3f * a.l1[pix] + 2e-5f;
      const float thr = vmax - 2.f * E;
      // a group whose last entry is inside the window may hide further candidates
      const bool ovf_lane = (lane < ncand) && ((lane % og) == og - 1) && (cv >= thr);
      const bool overflow = __any_sync(0xffffffffu, ovf_lane);
      // Q sums of the pixel (exact FP32 state)
      const float* A = a.Astate + pix * a.kpad;
      for (int e = lane; e < (K + 1) * K; e += 32) {
        const int kx = e / K, ky = e % K + 1;
        float sr, dr, si, di;
        if (kx == 0) {
          sr = 2.f * A[ky]; dr = 0.f; si = 0.f; di = 2.f * A[nh + ky];
        } else {
          const int hp = K + (kx - 1) * M + (ky + K) + 1, hm = K + (kx - 1) * M + (-ky + K) + 1;
          const float rp = A[hp], rm = A[hm], ip = A[nh + hp], im = A[nh + hm];
          sr = rp + rm; dr = rp - rm; si = ip + im; di = ip - im;
        }
        qbuf[4 * e + 0] = sr; qbuf[4 * e + 1] = dr; qbuf[4 * e + 2] = si; qbuf[4 * e + 3] = di;
      }
      if (lane <= K) {
        float qr, qi;
        if (lane == 0) { qr = A[0]; qi = 0.f; }
        else { const int h0 = K + (lane - 1) * M + K + 1; qr = A[h0]; qi = A[nh + h0]; }
        qbuf[4 * (K + 1) * K + 2 * lane] = qr;
        qbuf[4 * (K + 1) * K + 2 * lane + 1] = qi;
      }
      __syncwarp();
      float bv = -INFINITY;
      int bi = 0x7fffffff;
      if (!overflow) {
        if (lane < ncand && cv >= thr && ci < L * L) {
          bv = exact_R<M>(qbuf, tabx, L, ci);
          bi = ci;
        }
      } else {
        if (lane == 0 && a.n_fallback) atomicAdd(a.n_fallback, 1);
        for (int g = lane; g < L * L; g += 32) {
          const float r = exact_R<M>(qbuf, tabx, L, g);
          if (r > bv) { bv = r; bi = g; }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, bv, off);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ob > bv || (ob == bv && oi < bi)) { bv = ob; bi = oi; }
      }
      best_i = bi;
      __syncwarp();
    }
    if (lane == 0) {
      const int b = (best_i >= 0 && best_i < L * L) ? best_i : 0;
      a.vidx[pix] = b;
      a.vx[pix] = -a.vmax + (b % L) * a.vstep;
      a.vy[pix] = -a.vmax + (b / L) * a.vstep;
    }
  }
}

template <int M>
cudaError_t launch_conv_m(const AutocorrTcArgs& a, cudaStream_t st) {
  const long long npix = (long long)a.H * a.W;
  long long blocks = (npix + 7) / 8;
  if (blocks > 148LL * 16) blocks = 148LL * 16;
  if (a.bf16) ac_convert_kernel<M, true><<<unsigned(blocks), 256, 0, st>>>(a);
  else ac_convert_kernel<M, false><<<unsigned(blocks), 256, 0, st>>>(a);
  return cudaGetLastError();
}

template <int M>
cudaError_t launch_rerank_m(const AutocorrTcArgs& a, cudaStream_t st) {
  constexpr int K = (M - 1) / 2;
  constexpr int QN = (4 * (K + 1) * K + 2 * (K + 1) + 3) & ~3;
  const size_t smem = sizeof(float2) * size_t((a.L * (K + 1) + 1) & ~1) + sizeof(float) * kWarpsR * QN;
  const long long npix = (long long)a.H * a.W;
  long long blocks = (npix + kWarpsR - 1) / kWarpsR;
  if (blocks > 148LL * 8) blocks = 148LL * 8;
  ac_rerank_kernel<M><<<unsigned(blocks), kWarpsR * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool autocorr_tc_supported(int M) { return M == 5 || M == 7 || M == 9 || M == 15; }

cudaError_t launch_autocorr_convert(const AutocorrTcArgs& a, cudaStream_t st) {
  switch (a.M) {
    case 5: return launch_conv_m<5>(a, st);
    case 7: return launch_conv_m<7>(a, st);
    case 9: return launch_conv_m<9>(a, st);
    case 15: return launch_conv_m<15>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_autocorr_rerank(const AutocorrTcArgs& a, cudaStream_t st) {
  switch (a.M) {
    case 5: return launch_rerank_m<5>(a, st);
    case 7: return launch_rerank_m<7>(a, st);
    case 9: return launch_rerank_m<9>(a, st);
    case 15: return launch_rerank_m<15>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace wh
