// Spectrum kernel: observer bank + spatial SDFT + high-pass + Hann + power +
// reduction to the autocorrelation basis + first-order smoothing, fused.
//
// Method (Kennedy, arXiv:1408.3526, Sec. 1-2):
//   S(k;n) = 1/sqrt(Mx My Mz) sum_m e^{j2pi k.m/M} I(n-m)          Eq. (6)-(7)
// estimated recursively: a deadbeat observer over time and a sliding DFT
// (comb + resonator) over space.  The observer bank is linear and
// time-invariant with the same coefficients for every input, so it is run
// per raw pixel (Mz states) before the spatial SDFT instead of per spatial
// bin after it; the result is identical and the state is M^2 times smaller.
// Then the high-passed (kx = ky = 0 removed), Hann-windowed spectrum S'' gives
// P = |S''|^2 (Eq. (9)) and, summing over kz with the lz = 1 phase,
//   A_c(h) = sum_kz P(h,kz) cos(2pi kz/Mz),  A_s(h) = sum_kz P(h,kz) sin(2pi kz/Mz)
// from which R(l) = A_c(0) + 2 sum_{h in half plane} [A_c(h) cos a_h(l) -
// A_s(h) sin a_h(l)] exactly (Eq. (10), a_h(l) = 2pi(hx lx + hy ly)/M).  The
// smoother R'_t = (1-alpha) R_t + alpha R'_{t-1} is linear, so it is applied
// to the M^2 numbers A instead of the L^2 values of R (identical result).
//
// Organisation: one CTA owns a strip of TW output columns x TH output rows and
// walks down it one input row at a time (TH + 2K rows, clamped at the frame
// edge):
//   A  observer update of the row segment (TW + 2K pixels), Hann along kz;
//   B  x-DFT of the row: every (channel, column) as a direct M-tap sum with the
//      Hann(x) window and the centring phase folded into its weights;
//   C  y-SDFT: one thread per (channel, column) carries the M ky-resonators
//      of that column (comb input from a ring of the last M+1 x-DFT rows),
//      then Hann along ky (real 3 taps in the centred basis), the high-pass
//      correction and the power of the output row;
//   D  per output pixel, reduce P over kz into A, smooth, store.
// Register prefetch hides the HBM latency of the next row's frame/observer
// state (phase A) and of the next output row's smoother state (phase D).
#include <cuda_bf16.h>

#include <cmath>

#include "common.cuh"

namespace wh {

namespace {

constexpr int kPrefA = kMaxMz + 1;   // frame + Mz state floats per phase-A pixel
constexpr int kMaxDTasks = 4;        // phase-D tasks per thread (checked on the host)
constexpr int kSpecMaxThreads = 384;   // y-SDFT threads rounded to warps + one observer warp
constexpr int kMaxBTasks = 2;        // phase-B tasks per thread (checked on the host)

template <int M, int MZ>
struct Geo {
  static constexpr int K = (M - 1) / 2;
  static constexpr int J = (MZ - 1) / 2;                 // complex planes 1..J
  static constexpr bool EVEN = (MZ % 2) == 0;
  static constexpr int NPL = J + 1 + (EVEN ? 1 : 0);     // stored planes
};

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// Resonator twiddles e^{+j2pi ky/M} and centring phases e^{-j2pi ky K/M} per
// window size (index (M-3)/2, ky+K); indexed at compile time in the kernel, so
// they are read as constant-bank operands.
__constant__ float2 c_wres[7][kMaxM];
__constant__ float2 c_cph[7][kMaxM];

// Per-thread asynchronous 4-byte copies global -> shared (each thread later
// consumes only what it copied, so a wait on its own groups suffices).
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__host__ __device__ inline int spec_threads_for(int M, int Mz, int tw) {
  const int K = (M - 1) / 2, J = (Mz - 1) / 2;
  const int nchy = (1 + ((Mz % 2) == 0 ? 1 : 0)) * (K + 1) + J * M;
  return ((tw * nchy + 31) / 32) * 32 + 32;      // + the observer warp
}

// Byte offsets of the shared-memory arrays (16-byte aligned each); the same
// function sizes the launch on the host.
struct SpecSmem {
  size_t twr, ring, xc, pbuf, hg, wres, cph, off, dbuf, abuf, dpre, total;
};
__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline SpecSmem spec_smem_layout(int M, int Mz, int tw) {
  const int K = (M - 1) / 2, J = (Mz - 1) / 2;
  const bool even = (Mz % 2) == 0;
  const int npl = J + 1 + (even ? 1 : 0);
  const int nchy = (1 + (even ? 1 : 0)) * (K + 1) + J * M;
  const int nch = nchy + npl;
  const int nh = (M * M - 1) / 2;
  const int nslot = 1 + 2 * J + (even ? 1 : 0);
  const int PS = (nchy * M) | 1;
  const int RW = tw + 2 * K;
  SpecSmem L;
  size_t o = 0;
  L.twr = o;  o = align16(o + sizeof(float2) * size_t(npl) * RW);
  L.ring = o; o = align16(o + sizeof(float2) * size_t(M + 1) * nch * tw);
  L.xc = o;   o = align16(o + sizeof(float2) * size_t(nch) * M);
  L.pbuf = o; o = align16(o + sizeof(float) * size_t(tw) * PS);
  L.hg = o;   o = align16(o + sizeof(int) * size_t(nh + 1) * nslot);
  L.wres = o; o = align16(o + sizeof(float2) * M);
  L.cph = o;  o = align16(o + sizeof(float2) * M);
  L.off = o;  o = align16(o + sizeof(float2) * npl);
  L.dbuf = o; o = align16(o + sizeof(float2) * size_t(npl) * tw);
  L.abuf = o; o = align16(o + sizeof(float) * size_t(RW) * kPrefA);
  L.dpre = o; o = align16(o + sizeof(float) * size_t(kMaxDTasks) * 2 * spec_threads_for(M, Mz, tw));
  L.total = o;
  return L;
}

// Observer update of one pixel (frame value pa[0], packed T_{t-1} in pa[1..Mz])
// -> T_t (packed, written back into T) and its Hann-windowed planes Tw.
template <int M, int MZ>
__device__ __forceinline__ void observer_hann(const float* pa, const float2* lam, float2 hz,
                                              float2 (&T)[Geo<M, MZ>::NPL],
                                              float2 (&Tw)[Geo<M, MZ>::NPL]) {
  using G = Geo<M, MZ>;
  constexpr int J = G::J, NPL = G::NPL;
  constexpr bool EVEN = G::EVEN;
  const float xin = pa[0];
  T[0] = make_float2(pa[1], 0.f);
#pragma unroll
  for (int j = 1; j <= J; ++j) T[j] = make_float2(pa[2 * j], pa[2 * j + 1]);
  if (EVEN) T[NPL - 1] = make_float2(pa[MZ], 0.f);
  // prior s = lambda T_{t-1}; prediction = sum over all Mz bins (Hermitian)
  float2 s[NPL];
  float yhat = 0.f;
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    s[p] = cmul(lam[p], T[p]);
    const bool real = (p == 0) || (EVEN && p == NPL - 1);
    yhat += real ? s[p].x : 2.f * s[p].x;
  }
  const float e = (xin - yhat) * (1.0f / MZ);
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    T[p] = make_float2(s[p].x + e, s[p].y);
    const bool real = (p == 0) || (EVEN && p == NPL - 1);
    if (real) T[p].y = 0.f;
  }
  // Hann along kz: Tw(p) = 1/2 T(p) + 1/4 hz T(p+1) + 1/4 conj(hz) T(p-1), bins mod Mz
  float2 Tf[MZ];
  Tf[0] = T[0];
#pragma unroll
  for (int j = 1; j <= J; ++j) { Tf[j] = T[j]; Tf[MZ - j] = conjf2(T[j]); }
  if (EVEN) Tf[MZ / 2] = T[NPL - 1];
#pragma unroll
  for (int p = 0; p < NPL; ++p) {
    const float2 up = Tf[(p + 1) % MZ], dn = Tf[(p + MZ - 1) % MZ];
    float2 tw = cadd(cscale(Tf[p], 0.5f),
                     cadd(cscale(cmul(hz, up), 0.25f), cscale(cmul(conjf2(hz), dn), 0.25f)));
    const bool real = (p == 0) || (EVEN && p == NPL - 1);
    if (real) tw.y = 0.f;
    Tw[p] = tw;
  }
}

template <int M, int MZ>
__global__ void __launch_bounds__(kSpecMaxThreads, 2) spectrum_kernel(const SpecArgs a) {
  using G = Geo<M, MZ>;
  constexpr int K = G::K, J = G::J, NPL = G::NPL;
  constexpr bool EVEN = G::EVEN;
  const SpecTables& tb = *a.tables;
  const int TW = a.tw, H = a.H, W = a.W;
  const int RW = TW + 2 * K;
  const int nch = tb.nch, nchy = tb.nchy, nh = tb.nh, nslot = tb.nslot;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int PS = (nchy * M) | 1;                          // odd pixel stride of pbuf

  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SpecSmem SL = spec_smem_layout(M, MZ, TW);
  float2* twr = reinterpret_cast<float2*>(smem_raw + SL.twr);         // [NPL][RW]
  float2* ring = reinterpret_cast<float2*>(smem_raw + SL.ring);       // [M+1][nch][TW]
  float2* xc = reinterpret_cast<float2*>(smem_raw + SL.xc);           // [nch][M]
  float* pbuf = reinterpret_cast<float*>(smem_raw + SL.pbuf);         // [TW][PS]
  int* hg = reinterpret_cast<int*>(smem_raw + SL.hg);                 // [(nh+1)][nslot]
  float2* offs = reinterpret_cast<float2*>(smem_raw + SL.off);        // [NPL]
  float2* dbuf = reinterpret_cast<float2*>(smem_raw + SL.dbuf);       // [NPL][TW]
  float* abuf = reinterpret_cast<float*>(smem_raw + SL.abuf);         // [RW][kPrefA]
  float* dpre = reinterpret_cast<float*>(smem_raw + SL.dpre);         // [kMaxDTasks][2][nthr]
  constexpr int MI = (M - 3) / 2;

  for (int i = tid; i < nch * M; i += nthr) xc[i] = tb.xcoef[i / M][i % M];
  for (int i = tid; i < (nh + 1) * nslot; i += nthr) hg[i] = a.hgather[i];
  float2 lam[NPL];
#pragma unroll
  for (int p = 0; p < NPL; ++p) lam[p] = tb.lam[p];
  const float2 hz = tb.hann_z;
  const float alpha = a.alpha, oma = 1.0f - alpha;
  const float sP = float(MZ) * float(MZ) / float(M * M * MZ);   // (Mz/sqrt(N))^2

  // ---- static task assignment (identical for every row) -----------------------
  // B: (channel, column) x-DFT tasks, packed: c | x << 8 | plane << 16 | real << 20 | dc << 21
  int btask[kMaxBTasks];
#pragma unroll
  for (int q = 0; q < kMaxBTasks; ++q) {
    const int task = tid + q * nthr;
    if (task < nch * TW) {
      const int c = task / TW, x = task % TW, p = tb.ch_plane[c];
      const int real = (p == 0) || (EVEN && p == NPL - 1);
      btask[q] = c | (x << 8) | (p << 16) | (real << 20) | (int(c >= nchy) << 21);
    } else {
      btask[q] = -1;
    }
  }
  // C: one (channel, column) y-SDFT per thread
  const bool yth = tid < TW * nchy;
  const int cy = yth ? tid / TW : 0;
  const int xy = yth ? tid % TW : 0;
  const int kxc = tb.ch_kx[cy];
  const int plc = tb.ch_plane[cy];
  // D: (pixel column, h) reduction tasks, packed: hi | x << 16
  const int ntD = TW * (nh + 1);
  int dtask[kMaxDTasks];
#pragma unroll
  for (int q = 0; q < kMaxDTasks; ++q) {
    const int task = tid + q * nthr;
    dtask[q] = task < ntD ? ((task % (nh + 1)) | ((task / (nh + 1)) << 16)) : -1;
  }

  // ---- this CTA's share of the (strip, row) units -------------------------------
  const int nstrip = (W + TW - 1) / TW;
  const long long total = (long long)nstrip * H;
  const long long u0 = total * blockIdx.x / gridDim.x;
  const long long u1 = total * (blockIdx.x + 1) / gridDim.x;
  __syncthreads();

  for (long long u = u0; u < u1;) {
    const int strip = int(u / H);
    const int y0 = int(u % H);
    const int y1 = int(min((long long)H, (long long)y0 + (u1 - u)));
    u += y1 - y0;
    const int x0 = strip * TW;
    const int TH = y1 - y0;

    float2 Y[M];
#pragma unroll
    for (int k = 0; k < M; ++k) Y[k] = make_float2(0.f, 0.f);
    float2 drun[kMaxBTasks];
#pragma unroll
    for (int q = 0; q < kMaxBTasks; ++q) drun[q] = make_float2(0.f, 0.f);
    const int nrows = TH + 2 * K;

    // The last warp runs the observer update of the next input row while the
    // other warps run the y-recursion of the current one.
    const int ua = tid - (nthr - 32);
    const bool athr = ua >= 0 && ua < RW;
    float pa[kPrefA];
    auto loadA = [&](int i) {             // prefetch input row i into this lane's abuf slot
      if (athr) {
        const int rs = clampi(y0 - K + i, H), xs = clampi(x0 - K + ua, W);
        const size_t o = size_t(rs) * W + xs, plane = size_t(H) * W;
        float* dst = abuf + ua * kPrefA;
        cp_async4(dst, a.frame + o);
#pragma unroll
        for (int f = 0; f < MZ; ++f) cp_async4(dst + 1 + f, a.obs_old + f * plane + o);
      }
      cp_async_commit();
    };
    auto doA = [&](int i) {               // observer update + Hann(kz) of input row i
      if (!athr) return;
      const int r = y0 - K + i;
#pragma unroll
      for (int f = 0; f <= MZ; ++f) pa[f] = abuf[ua * kPrefA + f];
      float2 T[NPL], Tw[NPL];
      observer_hann<M, MZ>(pa, lam, hz, T, Tw);
      const int xs = x0 - K + ua;
      if (r >= y0 && r < y1 && ua >= K && ua < K + TW && xs < W) {   // owner writes the new state
        const size_t o = size_t(r) * W + xs, plane = size_t(H) * W;
        a.obs_new[o] = T[0].x;
#pragma unroll
        for (int j = 1; j <= J; ++j) {
          a.obs_new[(2 * j - 1) * plane + o] = T[j].x;
          a.obs_new[(2 * j) * plane + o] = T[j].y;
        }
        if (EVEN) a.obs_new[(MZ - 1) * plane + o] = T[NPL - 1].x;
      }
#pragma unroll
      for (int p = 0; p < NPL; ++p) twr[p * RW + ua] = csub(Tw[p], offs[p]);
    };
    // phase-D prefetch of the smoother state of an output row (own slots of dpre)
    auto loadD = [&](int yo) {
#pragma unroll
      for (int q = 0; q < kMaxDTasks; ++q) {
        const int x = dtask[q] >> 16, hi = dtask[q] & 0xffff;
        if (dtask[q] >= 0 && yo < y1 && x0 + x < W) {
          const float* src = a.Astate + (size_t(yo) * W + x0 + x) * a.kpad;
          cp_async4(dpre + (q * 2 + 0) * nthr + tid, src + hi);
          if (hi > 0) cp_async4(dpre + (q * 2 + 1) * nthr + tid, src + nh + hi);
        }
      }
      cp_async_commit();
    };
    auto doB = [&](int i) {               // x-DFT of input row i into ring slot i mod (M+1)
      const int slot = i % (M + 1);
      const int oslot = (i + 1) % (M + 1);    // holds row i - M
#pragma unroll
      for (int q = 0; q < kMaxBTasks; ++q) {
        const int bt = btask[q];
        if (bt < 0) continue;
        const int c = bt & 0xff, x = (bt >> 8) & 0xff, pl = (bt >> 16) & 0xf;
        const float2* row = twr + pl * RW + x + 2 * K;       // u = x + 2K - mx
        const float2* w = xc + c * M;
        float2 acc = make_float2(0.f, 0.f);
        if (bt & (1 << 20)) {
#pragma unroll
          for (int mx = 0; mx < M; ++mx) {
            const float v = row[-mx].x;
            const float2 cw = w[mx];
            acc.x = fmaf(cw.x, v, acc.x);
            acc.y = fmaf(cw.y, v, acc.y);
          }
        } else {
#pragma unroll
          for (int mx = 0; mx < M; ++mx) {
            const float2 v = row[-mx], cw = w[mx];
            acc.x = fmaf(cw.x, v.x, fmaf(-cw.y, v.y, acc.x));
            acc.y = fmaf(cw.x, v.y, fmaf(cw.y, v.x, acc.y));
          }
        }
        if (bt & (1 << 21)) {                  // running box sum for the high-pass
          drun[q] = cadd(drun[q], acc);
          if (i >= M) drun[q] = csub(drun[q], ring[(oslot * nch + c) * TW + x]);
          dbuf[pl * TW + x] = drun[q];
        }
        ring[(slot * nch + c) * TW + x] = acc;
      }
    };
    auto doC = [&](int i) {               // y-SDFT, Hann(ky), high-pass, power of row i
      if (!yth) return;
      const int slot = i % (M + 1), oslot = (i + 1) % (M + 1);
      const int yo = y0 + i - 2 * K;
      const float2 xn = ring[(slot * nch + cy) * TW + xy];
      float2 d = xn;
      if (i >= M) d = csub(xn, ring[(oslot * nch + cy) * TW + xy]);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const float2 w = c_wres[MI][k], c = c_cph[MI][k];
        Y[k] = make_float2(fmaf(w.x, Y[k].x, fmaf(-w.y, Y[k].y, fmaf(c.x, d.x, -c.y * d.y))),
                           fmaf(w.x, Y[k].y, fmaf(w.y, Y[k].x, fmaf(c.x, d.y, c.y * d.x))));
      }
      if (!(i >= 2 * K && yo < y1)) return;
      // 4 x [Hann along ky (taps 1/4, 1/2, 1/4 in the centred basis), minus
      // Hann_x Hann_y of the removed (0,0) bin]; the factor 16 is in the power scale
      float2 D = make_float2(0.f, 0.f);
      float wxh = 0.f;
      if (kxc >= -1 && kxc <= 1) {
        D = dbuf[plc * TW + xy];
        wxh = (kxc == 0) ? 0.5f : 0.25f;
      }
      float* pb = pbuf + xy * PS + cy * M;
      const bool dump = (a.dump_win != nullptr) && (x0 + xy < W);
      const float sP16 = sP * (1.f / 16.f);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        float2 z = cadd(cscale(Y[k], 2.f), cadd(Y[(k + 1) % M], Y[(k + M - 1) % M]));
        if (k == K) z = csub(z, cscale(D, wxh * 2.f));
        if (k == K - 1 || k == K + 1) z = csub(z, cscale(D, wxh));
        const float pw = sP16 * fmaf(z.x, z.x, z.y * z.y);
        pb[k] = pw;
        if (dump) {
          // uncentred S'' = e^{+j2pi (kx+ky)K/M} Z, and its conjugate partner at -k
          const size_t pix = size_t(yo) * W + x0 + xy;
          const int izp = plc + J, izm = ((-plc) + J + MZ) % MZ;
          const float2 sv = cscale(cmul(cmul(tb.uncenter[kxc + K], tb.uncenter[k]), z),
                                   0.25f * float(MZ) / sqrtf(float(M * M * MZ)));
          const size_t op = ((pix * MZ + izp) * M + k) * M + (kxc + K);
          const size_t om = ((pix * MZ + izm) * M + (M - 1 - k)) * M + (K - kxc);
          a.dump_win[op] = sv;
          a.dump_win[om] = conjf2(sv);
          if (a.dump_pow) { a.dump_pow[op] = pw; a.dump_pow[om] = pw; }
        }
      }
    };
    auto doD = [&](int i) {               // reduce over kz, smooth, store (output row of i)
      const int yo = y0 + i - 2 * K;
      if (!(i >= 2 * K && yo < y1)) return;
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
#pragma unroll
      for (int q = 0; q < kMaxDTasks; ++q) {
        const int x = dtask[q] >> 16, hi = dtask[q] & 0xffff;
        if (dtask[q] < 0 || x0 + x >= W) continue;
        const int* g = hg + hi * nslot;
        const float* pb = pbuf + x * PS;
        float Ac = pb[g[0]], As = 0.f;
#pragma unroll
        for (int j = 1; j <= J; ++j) {
          const float pp = pb[g[j]], pm = pb[g[J + j]];
          Ac = fmaf(pp + pm, tb.cz[j], Ac);
          As = fmaf(pp - pm, tb.sz[j], As);
        }
        if (EVEN) Ac -= pb[g[2 * J + 1]];
        float* dst = a.Astate + (size_t(yo) * W + x0 + x) * a.kpad;
        dst[hi] = fmaf(oma, Ac, alpha * dpre[(q * 2 + 0) * nthr + tid]);
        if (hi > 0) dst[nh + hi] = fmaf(oma, As, alpha * dpre[(q * 2 + 1) * nthr + tid]);
      }
      loadD(yo + 1);
      // learned-estimator features of this output row: one warp per pixel
      if (a.feat != nullptr) {
        const int lane = tid & 31, wid = tid >> 5, nw = nthr >> 5;
        const int nbins = M * M * MZ;
        for (int x = wid; x < TW; x += nw) {
          if (x0 + x >= W) continue;
          const float* pb = pbuf + x * PS;
          float tot = 0.f;
          for (int b = lane; b < nbins; b += 32) tot += pb[a.feat_gather[b]];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
          const float inv = tot > 0.f ? 1.f / tot : 0.f;
          __nv_bfloat16* dst = reinterpret_cast<__nv_bfloat16*>(a.feat) + (size_t(yo) * W + x0 + x) * a.feat_ld;
          for (int b = lane; b < a.feat_ld; b += 32)
            dst[b] = __float2bfloat16(
                b < nbins ? 0.1f * (__log2f(fmaf(pb[a.feat_gather[b]], inv, 1e-6f)) + 10.f) : 0.f);
        }
      }
    };

    // ---- prologue: offsets, observer of row 0, x-DFT of row 0 ----------------
    loadA(0);
    // Per-plane offset removed from every Tw of this segment before the spatial
    // sums.  The high-passed, Hann-windowed spectrum is exactly invariant to a
    // spatially constant offset per temporal plane (it only feeds the removed
    // kx = ky = 0 bin and the correction that cancels its window leakage), so
    // subtracting one constant per segment leaves the result unchanged while
    // keeping the FP32 sums at the scale of the texture instead of the DC level.
    if (ua == 0) {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      for (int f = 0; f <= MZ; ++f) pa[f] = abuf[f];
      float2 Tn[NPL], Tw0[NPL];
      observer_hann<M, MZ>(pa, lam, hz, Tn, Tw0);
#pragma unroll
      for (int p = 0; p < NPL; ++p) offs[p] = Tw0[p];
    }
    loadD(y0);
    __syncthreads();
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    doA(0);
    if (nrows > 1) loadA(1);
    __syncthreads();
    doB(0);
    __syncthreads();

    // ---- pipelined rows: X = {y-SDFT(i), observer(i+1)}, Y = {reduce(i), x-DFT(i+1)}
    for (int i = 0; i < nrows; ++i) {
      doC(i);
      if (i + 1 < nrows) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        doA(i + 1);
        if (i + 2 < nrows) loadA(i + 2);
      }
      __syncthreads();
      doD(i);
      if (i + 1 < nrows) doB(i + 1);
      __syncthreads();
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();   // before the next segment rewrites offs
  }
}

}  // namespace

// Shared-memory bytes and block size for a configuration (host side).
struct SpecLaunch { int threads; size_t smem; };

static SpecLaunch spec_launch_shape(int M, int Mz, int tw) {
  return {spec_threads_for(M, Mz, tw), spec_smem_layout(M, Mz, tw).total};
}

template <int M, int MZ>
static cudaError_t launch_spec_t(const SpecArgs& a, cudaStream_t st) {
  SpecLaunch L = spec_launch_shape(M, MZ, a.tw);
  auto kern = spectrum_kernel<M, MZ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(L.smem));
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 148, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, L.threads, L.smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // one wave of CTAs, each with an equal share of the (strip, row) units
  const long long units = (long long)((a.W + a.tw - 1) / a.tw) * a.H;
  long long grid = (long long)nsm * per_sm;
  if (grid > units) grid = units;
  kern<<<unsigned(grid), L.threads, L.smem, st>>>(a);
  return cudaGetLastError();
}

#define WH_SPEC_CASES(X) \
  X(5, 3) X(5, 4) X(5, 5) X(5, 6) \
  X(7, 3) X(7, 4) X(7, 5) X(7, 6) \
  X(9, 3) X(9, 4) X(9, 5) X(9, 6) \
  X(15, 4) X(15, 5) X(15, 6)

// Upload the constant twiddle tables for window M (all sizes at once, per device).
cudaError_t spectrum_init_constants() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && done[dev]) return cudaSuccess;
  float2 w[7][kMaxM], c[7][kMaxM];
  for (int mi = 0; mi < 7; ++mi) {
    const int M = 2 * mi + 3, K = (M - 1) / 2;
    for (int i = 0; i < kMaxM; ++i) {
      const int k = i - K;
      const double pi = 3.14159265358979323846;
      w[mi][i] = make_float2(float(std::cos(2 * pi * k / M)), float(std::sin(2 * pi * k / M)));
      c[mi][i] = make_float2(float(std::cos(-2 * pi * k * K / M)), float(std::sin(-2 * pi * k * K / M)));
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_wres, w, sizeof(w));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cph, c, sizeof(c));
  if (e == cudaSuccess && dev < 64) done[dev] = true;
  return e;
}

bool spectrum_supported(int M, int Mz) {
#define X(m, z) if (M == m && Mz == z) return true;
  WH_SPEC_CASES(X)
#undef X
  return false;
}

int spectrum_threads(int M, int Mz, int tw) { return spec_launch_shape(M, Mz, tw).threads; }
size_t spectrum_smem(int M, int Mz, int tw) { return spec_launch_shape(M, Mz, tw).smem; }

cudaError_t launch_spectrum(const SpecArgs& a, cudaStream_t st) {
#define X(m, z) if (a.M == m && a.Mz == z) return launch_spec_t<m, z>(a, st);
  WH_SPEC_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace wh
