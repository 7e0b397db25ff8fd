// Device helpers shared by the autocorrelation kernels (k_autocorr.cu and the
// exact re-rank of k_autocorr_tc.cu): per-pixel state row prefetch, the Q sums
// of a pixel, and R at one grid point with the same FP32 operation sequence as
// the separable search (so both give bit-identical R).
//
// State row of a pixel (kpad floats): A_c(0), A_c(h), A_s(h) over the half
// plane h = 1..nh (h = (0,1..K), then (kx>=1, ky=-K..K)).  Q(kx,ky) = A_c + jA_s.
// Q sums per (kx = 0..K, ky = 1..K): sr = Qr(ky)+Qr(-ky), dr = Qr(ky)-Qr(-ky),
// si = Qi(ky)+Qi(-ky), di = Qi(ky)-Qi(-ky) (float4), then Q(kx,0) (float2).
#pragma once
#include "common.cuh"

namespace wh {
namespace ac {

template <int M>
struct Geo {
  static constexpr int K = (M - 1) / 2;
  static constexpr int NH = (M * M - 1) / 2;
  static constexpr int QN = (4 * (K + 1) * K + 2 * (K + 1) + 3) & ~3;   // Q-sum floats (16-byte multiple)
  static constexpr int KP = (M * M + 3) & ~3;                            // state row floats
  static constexpr int NE = (K + 1) * K;                                 // Q-sum float4 elements
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Copy the KP-float state row at src into dst with the lanes j = 0..G-1 of a
// lane group (16-byte copies), and commit one group.
template <int M, int G = 16>
__device__ __forceinline__ void prefetch_row(float* dst, const float* src, int j, bool valid) {
  if (valid)
    for (int c = j; c < Geo<M>::KP / 4; c += G) cp_async16(dst + 4 * c, src + 4 * c);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Q-sum elements e = j + G r handled by lane j of a G-lane group: offsets hp,
// hm of A(kx, +ky) and A(kx, -ky) and a sign bit conjugating the second for
// kx = 0 (A(0, -ky) = conj A(0, ky) is stored as A(0, ky)); -1 past the end.
template <int M, int QIT, int G = 16>
__device__ __forceinline__ void qsum_offsets(int j, int (&qoff)[QIT]) {
  constexpr int K = Geo<M>::K, NE = Geo<M>::NE;
#pragma unroll
  for (int r = 0; r < QIT; ++r) {
    const int e = j + G * r;
    const int kx = e / K, ky = e % K + 1;
    int hp, hm, neg;
    if (kx == 0) { hp = ky; hm = ky; neg = 1; }
    else { hp = K + (kx - 1) * M + (ky + K) + 1; hm = K + (kx - 1) * M + (-ky + K) + 1; neg = 0; }
    qoff[r] = e < NE ? (hp | (hm << 8) | (neg << 16)) : -1;
  }
}

// Q sums of the state row A (shared) into qbuf (shared), by the G lanes of a
// lane group (G >= K + 1).
template <int M, int QIT, int G = 16>
__device__ __forceinline__ void build_qsums(const float* A, float* qbuf, const int (&qoff)[QIT], int j) {
  constexpr int K = Geo<M>::K, NH = Geo<M>::NH;
  static_assert(G >= K + 1, "one lane per Q(kx, 0)");
#pragma unroll
  for (int r = 0; r < QIT; ++r) {
    const int t = qoff[r];
    if (t >= 0) {
      const int hp = t & 0xff, hm = (t >> 8) & 0xff;
      const float rp = A[hp], rm = A[hm], ip = A[NH + hp];
      const float im = __int_as_float(__float_as_int(A[NH + hm]) ^ (unsigned(t >> 16) << 31));
      reinterpret_cast<float4*>(qbuf)[j + G * r] = make_float4(rp + rm, rp - rm, ip + im, ip - im);
    }
  }
  if (j <= K) {
    const int h0 = j == 0 ? 0 : K + (j - 1) * M + K + 1;
    reinterpret_cast<float2*>(qbuf + 4 * (K + 1) * K)[j] = make_float2(A[h0], j == 0 ? 0.f : A[NH + h0]);
  }
}

// R at flat grid index g (iy * L + ix) from the Q sums, tab = (cos, sin)(2pi k l / M)
// [L][K+1] for the grid coordinates l; the same per-component fmaf sequence
// as the two stages of the separable search.
template <int M>
__device__ __forceinline__ float exact_R(const float* qbuf, const float2* tab, int L, int g) {
  constexpr int K = Geo<M>::K;
  const int gc = (L - 1) / 2;
  const int gy = g / L, gx = g - gy * L;
  const int jy = gy - gc, jx = gx - gc;
  const float2* ty = tab + (gc + (jy < 0 ? -jy : jy)) * (K + 1);
  const float2* tx = tab + (gc + (jx < 0 ? -jx : jx)) * (K + 1);
  const float4* q4 = reinterpret_cast<const float4*>(qbuf);
  const float2* q0 = reinterpret_cast<const float2*>(qbuf + 4 * (K + 1) * K);
  float2 cy[K];
#pragma unroll
  for (int ky = 0; ky < K; ++ky) cy[ky] = ty[ky + 1];
  float t0r = 0.f;
  float2 v = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int kx = 0; kx <= K; ++kx) {
    const float2 z = q0[kx];
    float2 ac = make_float2(z.x, 0.f), db = make_float2(z.y, 0.f);
#pragma unroll
    for (int ky = 0; ky < K; ++ky) {
      const float4 q = q4[kx * K + ky];
      ac = __ffma2_rn(make_float2(q.x, q.y), cy[ky], ac);
      db = __ffma2_rn(make_float2(q.z, q.w), cy[ky], db);
    }
    const float2 t = jy >= 0 ? make_float2(ac.x - db.y, ac.y + db.x) : make_float2(ac.x + db.y, db.x - ac.y);
    if (kx == 0) t0r = t.x;
    else v = __ffma2_rn(tx[kx], t, v);
  }
  return jx >= 0 ? fmaf(2.f, v.x - v.y, t0r) : fmaf(2.f, v.x + v.y, t0r);
}

}  // namespace ac
}  // namespace wh
