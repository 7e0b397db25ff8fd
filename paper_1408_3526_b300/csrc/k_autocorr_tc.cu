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

#include "ac_common.cuh"
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

// Re-rank: two pixels per warp (a half-warp each).  The pixel's state row
// arrives by cp.async one pixel ahead (double buffer), its Q sums are built in
// shared memory, and lane j evaluates shortlist entries j, j + 16, ... exactly
// (ac::exact_R: the same FP32 sequence as the CUDA-core search, so the result
// equals that search's whenever the shortlist holds its argmax).
template <int M>
__global__ void __launch_bounds__(kWarpsR * 32) ac_rerank_kernel(const AutocorrTcArgs a) {
  using G = ac::Geo<M>;
  constexpr int QN = G::QN, KP = G::KP, K = G::K;
  constexpr int QIT = (G::NE + 15) / 16;
  const int L = a.L, ncand = a.ncand, og = a.ovf_group;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int half = lane >> 4, j = lane & 15;
  const int hw = wid * 2 + half;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sbase = reinterpret_cast<float*>(smem_raw);
  float* abuf = sbase + hw * 2 * KP;                                   // [2][KP]
  float* qbuf = sbase + kWarpsR * 2 * 2 * KP + hw * QN;                // [QN]
  float2* tabx = reinterpret_cast<float2*>(sbase + kWarpsR * 2 * (2 * KP + QN));   // [L][K+1]
  for (int i = threadIdx.x; i < L * (K + 1); i += blockDim.x) tabx[i] = a.tab_x[i];
  __syncthreads();
  int qoff[QIT];
  ac::qsum_offsets<M, QIT>(j, qoff);
  const float invL = 1.0f / float(L);
  const long long npix = (long long)a.H * a.W;
  const long long stride = (long long)gridDim.x * kWarpsR * 2;
  long long base = ((long long)blockIdx.x * kWarpsR + wid) * 2;
  ac::prefetch_row<M>(abuf, a.Astate + (base + half < npix ? base + half : 0) * KP, j, base + half < npix);
  for (int it = 0; base < npix; base += stride, ++it) {
    const long long pix = base + half;
    const bool valid = pix < npix;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    {
      const long long nb = base + stride + half;
      ac::prefetch_row<M>(abuf + ((it + 1) & 1) * KP, a.Astate + (nb < npix ? nb : 0) * KP, j, nb < npix);
    }
    // shortlist of this pixel: the largest tensor-core value over the entries
    float vmax = -INFINITY;
    for (int c = j; c < ncand; c += 16)
      if (valid) vmax = fmaxf(vmax, a.cand_val[pix * ncand + c]);
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    if (a.mode != 0) {
      // precision study: the tensor-core value decides (ties -> lowest index)
      for (int c = j; c < ncand; c += 16)
        if (valid && a.cand_val[pix * ncand + c] == vmax) bi = min(bi, a.cand_idx[pix * ncand + c]);
      bv = vmax;
    } else {
      // |R~ - R| <= sum_k (|da_k||B| + |a_k||dB|) + accumulation <= 2^-9 sum|a~| (F16
      // operands, |B| <= 2) + 225 * 2^-23 * 2 sum|a~| + subnormal flush of a~ (2^-25 each)
      const float E = valid ? 2.05e-3f * a.l1[pix] + 2e-5f : 0.f;
      const float thr = vmax - 2.f * E;
      // a group whose last entry is inside the window may hide further candidates
      bool ovf = false;
      for (int c = j; c < ncand; c += 16)
        if (valid && (c % og) == og - 1 && a.cand_val[pix * ncand + c] >= thr) ovf = true;
      const bool overflow = ((__ballot_sync(0xffffffffu, ovf) >> (16 * half)) & 0xffffu) != 0;
      if (valid) ac::build_qsums<M, QIT>(abuf + (it & 1) * KP, qbuf, qoff, j);
      __syncwarp();
      if (valid) {
        if (!overflow) {
          for (int c = j; c < ncand; c += 16) {
            const float cv = a.cand_val[pix * ncand + c];
            const int ci = a.cand_idx[pix * ncand + c];
            if (cv >= thr && ci >= 0 && ci < L * L) {
              const float r = ac::exact_R<M>(qbuf, tabx, L, ci);
              if (r > bv || (r == bv && ci < bi)) { bv = r; bi = ci; }
            }
          }
        } else {
          if (j == 0 && a.n_fallback) atomicAdd(a.n_fallback, 1);
          for (int g = j; g < L * L; g += 16) {
            const float r = ac::exact_R<M>(qbuf, tabx, L, g);
            if (r > bv) { bv = r; bi = g; }       // g increases in this lane: first of equals kept
          }
        }
      }
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, bv, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
      if (ob > bv || (ob == bv && oi < bi)) { bv = ob; bi = oi; }
    }
    if (valid && j == 0) {
      const int b = (bi >= 0 && bi < L * L) ? bi : 0;
      const int iy = int((float(b) + 0.5f) * invL), ix = b - iy * L;   // exact: b < 31^2
      a.vidx[pix] = b;
      a.vx[pix] = -a.vmax + ix * a.vstep;
      a.vy[pix] = -a.vmax + iy * a.vstep;
    }
    __syncwarp();
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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
  using G = ac::Geo<M>;
  constexpr int K = G::K;
  if (a.kpad != G::KP) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * size_t(kWarpsR) * 2 * (2 * G::KP + G::QN) +
                      sizeof(float2) * size_t(a.L) * (K + 1);
  const long long npix = (long long)a.H * a.W;
  ResidentShape rs{};
  cudaError_t e = resident_shape(ac_rerank_kernel<M>, kWarpsR * 32, smem, &rs);
  if (e != cudaSuccess) return e;
  const int nsm = rs.nsm, per_sm = rs.per_sm < 1 ? 1 : rs.per_sm;
  long long blocks = (npix + 2 * kWarpsR - 1) / (2 * kWarpsR);
  if (blocks > (long long)nsm * per_sm) blocks = (long long)nsm * per_sm;
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
