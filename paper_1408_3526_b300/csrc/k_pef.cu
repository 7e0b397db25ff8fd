// Velocity-tuned prediction-error filter (PEF) and subtraction.
//
// Eq. (4) with the coefficients of Eq. (8) equals, exactly (Parseval over the
// M x M x Mz window; the band-limited FIR of Eq. (2) has no DFT content
// outside |kx|,|ky| <= B), the direct convolution of Eq. (1):
//   Ihat(n - m') = sum_m H(m; m', v) I(n - m),
//   H = W^2/(Mx My Mz) D_W((mx - m'x - vx(mz - m'z))/M) D_W((my - m'y - vy(mz - m'z))/M),
// which is separable in x and y for each frame mz.  With the spatial delay
// m' = (K, K) and the offset d = K - m of a neighbour from the output pixel,
// each frame contributes sum_dy hy(dy) sum_dx hx(dx) I(p + d, t - mz), with
// h(d; v, mz) = D_W((d + v (mz - m'z))/M) tabulated per grid velocity.
//
// The last Mz frames are not stored: the observer state T_t(kz) is the DFT of
// the last Mz samples of every pixel, so x(t - m) = sum_kz T_t(kz) e^{-j2pi kz m/Mz}
// recovers them (exactly, up to rounding).  The output is
//   E(p, t - m'z) = I(p, t - m'z) - Ihat.
//
// One CTA per 16 x 16 output tile: the (16+2K)^2 x Mz history tile is rebuilt
// in shared memory, then every thread filters one pixel with its own velocity.
#include "common.cuh"

namespace wh {
namespace {

constexpr int kT = 16;

__global__ void __launch_bounds__(kT * kT) pef_kernel(const PefArgs a) {
  const int M = a.M, K = (M - 1) / 2, Mz = a.Mz, L = a.L, H = a.H, W = a.W;
  const int J = (Mz - 1) / 2;
  const bool even = (Mz % 2) == 0;
  const int RT = kT + 2 * K;
  const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* hist = reinterpret_cast<float*>(smem_raw);      // [Mz][RT][RT]
  float* hw = hist + Mz * RT * RT;                         // [L][Mz][M]
  float* cs = hw + L * Mz * M;                             // [J+1][Mz] cos, then sin
  float* sn = cs + (J + 1) * Mz;
  const int tid = threadIdx.y * kT + threadIdx.x, nthr = kT * kT;
  for (int i = tid; i < L * Mz * M; i += nthr) hw[i] = a.hw[i];
  for (int i = tid; i < (J + 1) * Mz; i += nthr) {
    const int j = i / Mz, m = i % Mz;
    float s, c;
    sincospif(2.0f * float((j * m) % Mz) / float(Mz), &s, &c);
    cs[i] = c;
    sn[i] = s;
  }
  __syncthreads();
  const size_t plane = size_t(H) * W;
  for (int i = tid; i < RT * RT; i += nthr) {
    const int yy = i / RT, xx = i % RT;
    int ys = y0 - K + yy, xs = x0 - K + xx;
    ys = ys < 0 ? 0 : (ys >= H ? H - 1 : ys);
    xs = xs < 0 ? 0 : (xs >= W ? W - 1 : xs);
    const size_t o = size_t(ys) * W + xs;
    float st[kMaxMz];
    for (int f = 0; f < Mz; ++f) st[f] = __ldg(a.obs + f * plane + o);
    for (int m = 0; m < Mz; ++m) {
      float v = st[0];
      for (int j = 1; j <= J; ++j)
        v += 2.f * (st[2 * j - 1] * cs[j * Mz + m] + st[2 * j] * sn[j * Mz + m]);
      if (even) v += (m & 1) ? -st[Mz - 1] : st[Mz - 1];
      hist[(m * RT + yy) * RT + xx] = v;
    }
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int px = x0 + tx, py = y0 + ty;
  if (px >= W || py >= H) return;
  const size_t pix = size_t(py) * W + px;
  const int g = a.vidx[pix];
  const int gx = g % L, gy = g / L;
  float Ihat = 0.f;
  for (int m = 0; m < Mz; ++m) {
    const float* hxr = hw + (gx * Mz + m) * M;
    const float* hyr = hw + (gy * Mz + m) * M;
    const float* hb = hist + (m * RT + ty) * RT + tx;
    float acc = 0.f;
    for (int dy = 0; dy < M; ++dy) {
      const float* row = hb + dy * RT;
      float r = 0.f;
      for (int dx = 0; dx < M; ++dx) r = fmaf(hxr[dx], row[dx], r);
      acc = fmaf(hyr[dy], r, acc);
    }
    Ihat += acc;
  }
  a.whitened[pix] = hist[(a.mpz * RT + ty + K) * RT + tx + K] - Ihat;
}

// Raw spectrum S(k; n) of Eq. (6)-(7) from the observer state, by direct
// 2-D DFT of the Mz temporal planes (debug and parity checks only).
__global__ void raw_spectrum_kernel(const RawSpecArgs a) {
  const int M = a.M, K = (M - 1) / 2, Mz = a.Mz, H = a.H, W = a.W;
  const int J = (Mz - 1) / 2, kzlo = -J;
  const long long nb = (long long)M * M * Mz;
  const long long total = (long long)H * W * nb;
  const size_t plane = size_t(H) * W;
  const float scale = float(Mz) / sqrtf(float(M * M * Mz));
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long pix = idx / nb;
    const int b = int(idx % nb);
    const int iz = b / (M * M), iy = (b / M) % M, ix = b % M;
    const int kx = ix - K, ky = iy - K, kz = iz + kzlo;
    const int px = int(pix % W), py = int(pix / W);
    float2 acc = make_float2(0.f, 0.f);
    for (int my = 0; my < M; ++my) {
      int ys = py + K - my;
      ys = ys < 0 ? 0 : (ys >= H ? H - 1 : ys);
      for (int mx = 0; mx < M; ++mx) {
        int xs = px + K - mx;
        xs = xs < 0 ? 0 : (xs >= W ? W - 1 : xs);
        const size_t o = size_t(ys) * W + xs;
        float2 T;
        const int akz = kz < 0 ? -kz : kz;
        if (akz == 0) T = make_float2(a.obs[o], 0.f);
        else if ((Mz % 2) == 0 && akz == Mz / 2) T = make_float2(a.obs[(Mz - 1) * plane + o], 0.f);
        else T = make_float2(a.obs[(2 * akz - 1) * plane + o], a.obs[(2 * akz) * plane + o]);
        if (kz < 0) T.y = -T.y;
        float s, c;
        sincospif(2.0f * float(((kx * mx + ky * my) % M + M) % M) / float(M), &s, &c);
        acc = cadd(acc, cmul(make_float2(c, s), T));
      }
    }
    a.out[idx] = cscale(acc, scale);
  }
}

}  // namespace

cudaError_t launch_pef(const PefArgs& a, cudaStream_t st) {
  const int K = (a.M - 1) / 2, RT = kT + 2 * K, J = (a.Mz - 1) / 2;
  const size_t smem = sizeof(float) * (size_t(a.Mz) * RT * RT + size_t(a.L) * a.Mz * a.M +
                                       2 * size_t(J + 1) * a.Mz);
  cudaError_t e = cudaFuncSetAttribute(pef_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + kT - 1) / kT, (a.H + kT - 1) / kT);
  pef_kernel<<<grid, dim3(kT, kT), smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_raw_spectrum(const RawSpecArgs& a, cudaStream_t st) {
  const long long total = (long long)a.H * a.W * a.M * a.M * a.Mz;
  long long blocks = (total + 255) / 256;
  if (blocks > 148LL * 32) blocks = 148LL * 32;
  raw_spectrum_kernel<<<unsigned(blocks), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace wh
