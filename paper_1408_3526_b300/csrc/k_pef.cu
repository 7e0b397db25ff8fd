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
#include <atomic>
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace wh {
namespace {

constexpr int kT = 16;

// cos / sin(2pi ((j m) mod Mz) / Mz) per temporal order (index Mz - 3), j = 0..Mz/2,
// m = 0..Mz-1: the inverse temporal DFT that recovers the last Mz samples from
// the observer state, read as constant-bank operands
__constant__ float c_pcs[kMaxMz - 2][kMaxPlanes][kMaxMz], c_psn[kMaxMz - 2][kMaxPlanes][kMaxMz];

template <int M>
struct PefGeo {
  static constexpr int K = (M - 1) / 2;
  static constexpr int RT = kT + 2 * K;   // history tile edge
};

// One CTA per 16 x 16 output tile, 128 threads: thread (tx2, ty) filters the
// two pixels (2 tx2, ty) and (2 tx2 + 1, ty).  The history tile is kept as
// pairs of consecutive rows, hp[m][r][x] = (x(r), x(r+1)), so one 8-byte value
// feeds a packed FP32x2 FMA over the taps dy = 2i, 2i+1 of the y-sum, and one
// 16-byte load of two adjacent columns serves both pixels (the second pixel's
// window is the first's shifted by one column).  The x-weights of each pixel's
// velocity come duplicated, (h, h), from the L1-cached table.
template <int M, int MZ>
__global__ void __launch_bounds__(kT * kT / 2) pef_kernel(const PefArgs a) {
  constexpr int K = PefGeo<M>::K, RT = PefGeo<M>::RT;
  constexpr int J = (MZ - 1) / 2;
  constexpr bool EVEN = (MZ % 2) == 0;
  constexpr int NQ = (M + 2) / 2;            // 16-byte column pairs covering M + 1 columns
  const int L = a.L, H = a.H, W = a.W;
  const int x0 = blockIdx.x * kT, y0 = blockIdx.y * kT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* hp = reinterpret_cast<float2*>(smem_raw);        // [MZ][RT][RT]
  const int tid = threadIdx.y * (kT / 2) + threadIdx.x, nthr = kT * kT / 2;
  constexpr int ZI = MZ - 3;
  const size_t plane = size_t(H) * W;
  for (int i = tid; i < RT * RT; i += nthr) {
    const int yy = i / RT, xx = i % RT;
    int ys = y0 - K + yy, xs = x0 - K + xx;
    ys = ys < 0 ? 0 : (ys >= H ? H - 1 : ys);
    xs = xs < 0 ? 0 : (xs >= W ? W - 1 : xs);
    const size_t o = size_t(ys) * W + xs;
    float st[MZ];
#pragma unroll
    for (int f = 0; f < MZ; ++f) st[f] = __ldg(a.obs + f * plane + o);
#pragma unroll
    for (int m = 0; m < MZ; ++m) {
      float v = st[0];
#pragma unroll
      for (int j = 1; j <= J; ++j)
        v += 2.f * (st[2 * j - 1] * c_pcs[ZI][j][m] + st[2 * j] * c_psn[ZI][j][m]);
      if (EVEN) v += (m & 1) ? -st[MZ - 1] : st[MZ - 1];
      float2* row = hp + (m * RT + yy) * RT + xx;
      row->x = v;
      if (yy > 0) row[-RT].y = v;
      if (yy == RT - 1) row->y = 0.f;
    }
  }
  __syncthreads();
  const int tx = 2 * threadIdx.x, ty = threadIdx.y;
  const int px = x0 + tx, py = y0 + ty;
  if (px >= W || py >= H) return;
  const bool has_b = px + 1 < W;
  const size_t pix = size_t(py) * W + px;
  // grid indices of the two pixels, clamped before they index any table
  int ga = a.vidx[pix], gb = has_b ? a.vidx[pix + 1] : ga;
  ga = ga < 0 ? 0 : (ga >= L * L ? L * L - 1 : ga);
  gb = gb < 0 ? 0 : (gb >= L * L ? L * L - 1 : gb);
  const float2* hw2 = reinterpret_cast<const float2*>(a.hw + pef_hw2_offset(L, MZ, M));
  const float2* hwp = reinterpret_cast<const float2*>(a.hw + pef_hwp_offset(L, MZ, M));
  const int gxa = ga % L, gya = ga / L, gxb = gb % L, gyb = gb / L;
  float Ia = 0.f, Ib = 0.f;
#pragma unroll 1
  for (int m = 0; m < MZ; ++m) {
    float2 wa[M], wb[M];
#pragma unroll
    for (int dx = 0; dx < M; ++dx) {
      wa[dx] = __ldg(hw2 + (size_t(gxa) * MZ + m) * M + dx);
      wb[dx] = __ldg(hw2 + (size_t(gxb) * MZ + m) * M + dx);
    }
    const float4* hb = reinterpret_cast<const float4*>(hp + (m * RT + ty) * RT + tx);
    float2 acca = make_float2(0.f, 0.f), accb = make_float2(0.f, 0.f);   // (even dy, odd dy)
    float rla = 0.f, rlb = 0.f;
#pragma unroll
    for (int i = 0; i <= K; ++i) {
      // row pair (2i, 2i+1) (i < K), or the last row 2K in .x (i == K); columns tx .. tx+M
      float2 d[2 * NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const float4 v = hb[(2 * i) * (RT / 2) + q];
        d[2 * q] = make_float2(v.x, v.y);
        d[2 * q + 1] = make_float2(v.z, v.w);
      }
      if (i < K) {
        float2 ra = make_float2(0.f, 0.f), rb = make_float2(0.f, 0.f);
#pragma unroll
        for (int dx = 0; dx < M; ++dx) {
          ra = __ffma2_rn(wa[dx], d[dx], ra);
          rb = __ffma2_rn(wb[dx], d[dx + 1], rb);
        }
        acca = __ffma2_rn(__ldg(hwp + (size_t(gya) * MZ + m) * K + i), ra, acca);
        accb = __ffma2_rn(__ldg(hwp + (size_t(gyb) * MZ + m) * K + i), rb, accb);
      } else {
#pragma unroll
        for (int dx = 0; dx < M; ++dx) {
          rla = fmaf(wa[dx].x, d[dx].x, rla);
          rlb = fmaf(wb[dx].x, d[dx + 1].x, rlb);
        }
      }
    }
    Ia += fmaf(__ldg(a.hw + (size_t(gya) * MZ + m) * M + 2 * K), rla, acca.x + acca.y);
    Ib += fmaf(__ldg(a.hw + (size_t(gyb) * MZ + m) * M + 2 * K), rlb, accb.x + accb.y);
  }
  const float2 c = hp[(a.mpz * RT + ty + K) * RT + tx + K];   // (x(row), x(row+1)): need row's two columns
  a.whitened[pix] = c.x - Ia;
  if (has_b) a.whitened[pix + 1] = hp[(a.mpz * RT + ty + K) * RT + tx + K + 1].x - Ib;
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

// Upload the inverse-DFT tables (all temporal orders) once per device.
cudaError_t pef_init_constants() {
  static std::atomic<bool> done[64];
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < 64 && done[dev].load()) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev].load()) return cudaSuccess;
  static float cs[kMaxMz - 2][kMaxPlanes][kMaxMz], sn[kMaxMz - 2][kMaxPlanes][kMaxMz];
  const double two_pi = 6.283185307179586476925286766559;
  for (int z = 3; z <= kMaxMz; ++z)
    for (int j = 0; j < kMaxPlanes; ++j)
      for (int m = 0; m < kMaxMz; ++m) {
        const double ang = two_pi * double((j * m) % z) / double(z);
        cs[z - 3][j][m] = float(std::cos(ang));
        sn[z - 3][j][m] = float(std::sin(ang));
      }
  e = cudaMemcpyToSymbol(c_pcs, cs, sizeof(cs));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_psn, sn, sizeof(sn));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev].store(true);
  return e;
}

template <int M, int MZ>
static cudaError_t launch_pef_t(const PefArgs& a, cudaStream_t st) {
  constexpr int RT = PefGeo<M>::RT;
  cudaError_t ce = pef_init_constants();
  if (ce != cudaSuccess) return ce;
  const size_t smem = sizeof(float2) * size_t(MZ) * RT * RT;
  ResidentShape rs{};
  cudaError_t e = resident_shape(pef_kernel<M, MZ>, kT * kT / 2, smem, &rs);   // sets the smem attribute once
  if (e != cudaSuccess) return e;
  dim3 grid((a.W + kT - 1) / kT, (a.H + kT - 1) / kT);
  pef_kernel<M, MZ><<<grid, dim3(kT / 2, kT), smem, st>>>(a);
  return cudaGetLastError();
}

#define WH_PEF_CASES(X) \
  X(5, 3) X(5, 4) X(5, 5) X(5, 6) \
  X(7, 3) X(7, 4) X(7, 5) X(7, 6) \
  X(9, 3) X(9, 4) X(9, 5) X(9, 6) \
  X(15, 4) X(15, 5) X(15, 6)

cudaError_t launch_pef(const PefArgs& a, cudaStream_t st) {
#define X(m, z) if (a.M == m && a.Mz == z) return launch_pef_t<m, z>(a, st);
  WH_PEF_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_raw_spectrum(const RawSpecArgs& a, cudaStream_t st) {
  const long long total = (long long)a.H * a.W * a.M * a.M * a.Mz;
  long long blocks = (total + 255) / 256;
  if (blocks > 148LL * 32) blocks = 148LL * 32;
  raw_spectrum_kernel<<<unsigned(blocks), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace wh
