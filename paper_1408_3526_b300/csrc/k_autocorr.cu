// Autocorrelation on the velocity grid + argmax, FP32 on CUDA cores.
//
// Eq. (10) on the lz = 1 slice: R(l) = sum_k P(k) cos(2pi(kx lx/M + ky ly/M + kz/Mz)).
// With A_c/A_s the kz-reduced (and smoothed) power held in the stream state,
// Q(kx,ky) = A_c + j A_s satisfies Q(-k) = conj(Q(k)) and
//   R(lx,ly) = Re sum_{kx,ky} Q(kx,ky) e^{j2pi(kx lx + ky ly)/M}
//            = Re T(0,ly) + 2 sum_{kx=1..K} Re(e^{j2pi kx lx/M} T(kx,ly)),
//   T(kx,ly) = sum_{ky=-K..K} Q(kx,ky) e^{j2pi ky ly/M},
// evaluated separably (two small complex contractions per pixel).  The
// velocity is the grid point of the largest R (Sec. 2: v = l/lz, lz = 1);
// ties go to the lowest flat index iy*L + ix.
//
// One warp per pixel; Q and T live in shared memory.
#include "common.cuh"

namespace wh {
namespace {

constexpr int kWarps = 8;

__global__ void __launch_bounds__(kWarps * 32) autocorr_kernel(const AutocorrArgs a) {
  const int M = a.M, K = (a.M - 1) / 2, L = a.L, nh = (a.M * a.M - 1) / 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* ty = reinterpret_cast<float2*>(smem_raw);     // [L][M]
  float2* tx = ty + L * M;                               // [L][K+1]
  float2* Qall = tx + L * (K + 1);                       // [warps][K+1][M]
  float2* Tall = Qall + kWarps * (K + 1) * M;            // [warps][K+1][L]
  for (int i = threadIdx.x; i < L * M; i += blockDim.x) ty[i] = a.tab_y[i];
  for (int i = threadIdx.x; i < L * (K + 1); i += blockDim.x) tx[i] = a.tab_x[i];
  __syncthreads();

  const long long npix = (long long)a.H * a.W;
  float2* Q = Qall + wid * (K + 1) * M;
  float2* T = Tall + wid * (K + 1) * L;
  for (long long pix = (long long)blockIdx.x * kWarps + wid; pix < npix;
       pix += (long long)gridDim.x * kWarps) {
    const float* A = a.Astate + pix * a.kpad;
    // Q(kx, ky) for kx = 0..K, ky = -K..K
    for (int e = lane; e < (K + 1) * M; e += 32) {
      const int kx = e / M, iy = e % M, ky = iy - K;
      float2 q;
      if (kx == 0) {
        if (ky == 0) q = make_float2(A[0], 0.f);
        else {
          const int hi = ky > 0 ? ky : -ky;
          q = make_float2(A[hi], ky > 0 ? A[nh + hi] : -A[nh + hi]);
        }
      } else {
        const int hi = K + (kx - 1) * M + iy + 1;
        q = make_float2(A[hi], A[nh + hi]);
      }
      Q[e] = q;
    }
    __syncwarp();
    for (int e = lane; e < (K + 1) * L; e += 32) {
      const int kx = e / L, gl = e % L;
      const float2* qr = Q + kx * M;
      const float2* tr = ty + gl * M;
      float re = 0.f, im = 0.f;
      for (int iy = 0; iy < M; ++iy) {
        const float2 q = qr[iy], w = tr[iy];
        re = fmaf(q.x, w.x, fmaf(-q.y, w.y, re));
        im = fmaf(q.x, w.y, fmaf(q.y, w.x, im));
      }
      T[kx * L + gl] = make_float2(re, im);
    }
    __syncwarp();
    float best = -INFINITY;
    int bidx = 0x7fffffff;
    for (int g = lane; g < L * L; g += 32) {
      const int gy = g / L, gx = g % L;
      float acc = 0.f;
      const float2* txr = tx + gx * (K + 1);
      for (int kx = 1; kx <= K; ++kx) {
        const float2 t = T[kx * L + gy], w = txr[kx];
        acc = fmaf(w.x, t.x, fmaf(-w.y, t.y, acc));
      }
      const float R = fmaf(2.f, acc, T[gy].x);
      if (a.rs_out) a.rs_out[pix * (L * L) + g] = R;
      if (R > best) { best = R; bidx = g; }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, off);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (lane == 0) {
      a.vidx[pix] = bidx;
      a.vx[pix] = -a.vmax + (bidx % L) * a.vstep;
      a.vy[pix] = -a.vmax + (bidx / L) * a.vstep;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_autocorr(const AutocorrArgs& a, cudaStream_t st) {
  const int K = (a.M - 1) / 2;
  const size_t smem = sizeof(float2) * (size_t(a.L) * a.M + size_t(a.L) * (K + 1) +
                                        size_t(kWarps) * (K + 1) * (a.M + a.L));
  long long npix = (long long)a.H * a.W;
  long long blocks = (npix + kWarps - 1) / kWarps;
  if (blocks > 148LL * 16) blocks = 148LL * 16;
  cudaError_t e = cudaFuncSetAttribute(autocorr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e != cudaSuccess) return e;
  autocorr_kernel<<<unsigned(blocks), kWarps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace wh
