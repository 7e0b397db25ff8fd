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
// Organisation: one CTA owns a strip of TW output columns and walks down its
// share of rows one input row at a time (2K halo rows first); all geometry is
// fixed at compile time by (M, Mz).  Per input row:
//   A  (observer warp) observer update of the TW + 2K pixels of the row and
//      Hann along kz; in the next phase the same warp forms the M-pixel box
//      sums along x of every plane (warp shuffles) and their running sum over
//      the last M rows, the removed (0,0) bin the high-pass correction needs;
//   B  x-DFT units (x, kx >= 0, plane group): a direct M-tap sum with the
//      Hann(x) window, the centring phase and the power scale folded into the
//      weights; a complex plane's +kx and -kx outputs come from the same four
//      accumulators (the -kx weights are the conjugates);
//   C  y-SDFT: one thread per (channel, column) carries the M ky-resonators
//      (comb input from a ring of the last M+1 x-DFT rows), then Hann along ky
//      (real 3 taps in the centred basis), the high-pass correction and the
//      power of the output row;
//   D  per (output pixel, h): the kz reduction into A_c/A_s read at fixed
//      offsets of the power block (+-h plus constants, no index table), the
//      smoother update and the store; the next row's smoother state is
//      prefetched with cp.async.
// Two barriers per row: {C(i), A(i+1)} then {D(i), B(i+1), box sums(i+1)}.  With
// the learned estimator's features on, phase C also leaves each channel's power
// sum, the observer warp turns them into the pixels' totals at the start of the
// second phase, and the feature threads wait for those (a named barrier) only
// after their reduction tasks.
#include <cuda_bf16.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace wh {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

namespace {

constexpr int kZN = kMaxMz - 2;     // temporal orders Mz = 3 .. kMaxMz
constexpr int kSegRows = 256;       // longest run of the y-recursion (output rows)

// Resonator twiddles w_k = e^{+j2pi ky/M} and centring phases c_k =
// e^{-j2pi ky K/M} (k = ky + K) per window size (index (M-3)/2), packed for
// the bin pairs (p, p+K+1), p = 0..K-1: x, y and -y components of w (rw*) and
// of c (rc*); the centre bin k = K has w = c = 1.  Observer rotations, Hann(kz)
// phase and the kz reduction's cos/sin per temporal order (index Mz-3).  All
// indexed at compile time in the kernel, so read as constant-bank operands.
constexpr int kMaxK = (kMaxM - 1) / 2;
__constant__ float2 c_rwx[7][kMaxK], c_rwy[7][kMaxK], c_rnwy[7][kMaxK];
__constant__ float2 c_rcx[7][kMaxK], c_rcy[7][kMaxK], c_rncy[7][kMaxK];
// x-DFT weights Hann(mx) e^{j2pi kx (mx-K)/M}, kx = 0..K, per window size, as
// (wr, wr) and (wi, wi) pairs for the packed sums over a complex row (FP32 form)
__constant__ float2 c_xrr[7][kMaxK + 1][kMaxM], c_xii[7][kMaxK + 1][kMaxM];
__constant__ double2 c_dw[7][kMaxM], c_dc[7][kMaxM];   // the same twiddles in double (index ky + K)
__constant__ float2 c_lam[kZN][kMaxPlanes];
__constant__ float2 c_hz[kZN];
__constant__ float c_cz[kZN][kMaxPlanes];
__constant__ float c_sz[kZN][kMaxPlanes];

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr size_t al16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

// Extra shared-memory wavefronts of the y-SDFT power stores (thread t writes
// float (t % tw) * ps + (t / tw) * M + k) summed over the warps, for a pixel
// stride ps of the power block.
__host__ __device__ constexpr int pstore_conflicts(int tw, int nct, int M, int ps) {
  int tot = 0;
  for (int w0 = 0; w0 < nct; w0 += 32) {
    int cnt[32] = {};
    int mx = 0;
    for (int t = w0; t < w0 + 32 && t < nct; ++t) {
      const int b = ((t % tw) * ps + (t / tw) * M) % 32;
      ++cnt[b];
      if (cnt[b] > mx) mx = cnt[b];
    }
    tot += mx - 1;
  }
  return tot;
}
// Smallest conflict-free (else least-conflicting) stride >= the block size.
__host__ __device__ constexpr int pick_pstride(int tw, int nct, int M, int minps) {
  int best = minps, bc = 1 << 30;
  for (int ps = minps; ps < minps + 32; ++ps) {
    const int c = pstore_conflicts(tw, nct, M, ps);
    if (c < bc) { bc = c; best = ps; }
  }
  return best;
}

// Compile-time geometry of one (M, Mz) configuration.  F64: the spatial sums
// (x-DFT, comb differences, y-resonators, box sums, Hann and high-pass
// correction) in double precision, the precision form; element sizes of
// their buffers double.
template <int M, int MZ, bool F64 = false>
struct SG {
  static constexpr int K = (M - 1) / 2;
  static constexpr int J = (MZ - 1) / 2;                  // complex planes 1..J
  static constexpr bool EVEN = (MZ % 2) == 0;
  static constexpr int NREAL = EVEN ? 2 : 1;              // real planes 0 (and Mz/2)
  static constexpr int NPL = J + NREAL;                   // stored planes
  static constexpr int NCHY = NREAL * (K + 1) + J * M;    // y-SDFT channels
  static constexpr int NH = (M * M - 1) / 2;
  static constexpr int NH1 = NH + 1;
  static constexpr int TW = spec_tile_w(M, MZ);
  static constexpr int RW = TW + 2 * K;
  static constexpr int NCT = TW * NCHY;                   // y-SDFT threads
  static constexpr int NTHR = cdiv(NCT, 32) * 32 + 32;    // + the observer warp
  static constexpr int PS = pick_pstride(TW, NCT, M, NCHY * M);   // pixel stride of pbuf
  static constexpr int KPAD = (M * M + 3) & ~3;
  // x-DFT, precision form: units (group, kx, x), group 0 = the real planes,
  // j = complex plane j; each group padded to whole warps so a warp runs one
  // code path
  static constexpr int GU = TW * (K + 1);
  static constexpr int GP = cdiv(GU, 32) * 32;
  // x-DFT, FP32: one lane per (slot, column), slot 0 = both real planes as one
  // complex row (v0, v_Mz/2), slot j = complex plane j, so every lane runs the
  // same sums; the K+1 values kx >= 0 split into NXC chunks of KC, one chunk
  // per warp (WPC warps when the units exceed a warp), so the weights are
  // compile-time constant-bank operands and each tap loaded once serves KC kx
  static constexpr int XG = J + 1;
  static constexpr int XU = XG * TW;
  static constexpr int WPC = cdiv(XU, 32);
  // FP32: slot stride SW of the observer rows and the lane order (unit =
  // (lane + ROT) mod XU) picked so that the 8-byte tap loads of a half warp, and
  // each of its ring stores, fall on distinct banks (fewest extra wavefronts)
  static constexpr int base_of(int p) { return p == 0 ? 0 : (K + 1) + (p - 1) * M; }
  static constexpr int spread(const int* w, int n) {   // extra wavefronts of 8-byte words w[0..n)
    int cnt[16] = {}, mx = 0;
    for (int i = 0; i < n; ++i) { const int b = ((w[i] % 16) + 16) % 16; if (++cnt[b] > mx) mx = cnt[b]; }
    return mx > 0 ? mx - 1 : 0;
  }
  static constexpr int xdft_conflicts(int sw, int rot) {
    int tot = 0;
    for (int w0 = 0; w0 < WPC * 32; w0 += 16) {
      int ld[16] = {}, r0[16] = {}, r1[16] = {}, c0[16] = {}, c1[16] = {};
      int n = 0;
      for (int t = w0; t < w0 + 16 && t < XU; ++t) ++n;
      if (n == 0) break;
      for (int kx = -1; kx <= K; ++kx) {   // kx = -1: the tap loads (weight M)
        int nr = 0, nc = 0;
        for (int t = w0; t < w0 + n; ++t) {
          const int u = (t + rot) % XU, g = u / TW, bx = u % TW;
          if (kx < 0) { ld[t - w0] = g * sw + bx; continue; }
          if (g == 0) {
            r0[nr] = kx * TW + bx;
            r1[nr] = (base_of(NPL - 1) + kx) * TW + bx;
            ++nr;
          } else {
            c0[nc] = (base_of(g) + K + kx) * TW + bx;
            c1[nc] = (base_of(g) + K - kx) * TW + bx;
            ++nc;
          }
        }
        if (kx < 0) tot += M * spread(ld, n);
        else tot += spread(r0, nr) + (EVEN ? spread(r1, nr) : 0) + spread(c0, nc) + (kx > 0 ? spread(c1, nc) : 0);
      }
    }
    return tot;
  }
  static constexpr int pick_swrot() {   // first conflict-free pair, else the least conflicting
    int best = RW * 64, bc = 1 << 30;
    for (int rot = 0; rot < (XU <= 32 ? XU : 1); ++rot)
      for (int sw = RW; sw < RW + 16; ++sw) {
        const int c = xdft_conflicts(sw, rot);
        if (c < bc) { bc = c; best = sw * 64 + rot; }
        if (bc == 0) return best;
      }
    return best;
  }
  static constexpr int SWROT = F64 ? RW * 64 : pick_swrot();
  static constexpr int SW = SWROT / 64;
  static constexpr int ROT = SWROT % 64;
  static constexpr int NDT = TW * NH1;                    // reduction tasks per row
  // Reduction tasks: RD rounds on each thread without x-DFT work and RB rounds
  // on each x-DFT thread, with the x-DFT split (NXC) and RB chosen for the
  // shortest estimated critical path (instructions: x-DFT ~5.5 per tap and unit
  // in the precision form, M loads + KC (2M + 8) + 8 per FP32 x-DFT lane,
  // reduction task ~25); never on the observer warp, which runs the box sums
  // meanwhile.
  static constexpr int NTW = NTHR - 32;                   // threads other than the observer warp
  static constexpr int DCOST = 25;
  static constexpr int nbt_of(int nxc) { return F64 ? (J + 1) * GP : nxc * WPC * 32; }
  static constexpr int bcost_of(int nxc) { return F64 ? 11 * M / 2 + 12 : M + cdiv(K + 1, nxc) * (2 * M + 8) + 8; }
  static constexpr int rd_for(int nxc, int rb) {
    return NTW - nbt_of(nxc) > 0 ? cdiv(imax(0, NDT - nbt_of(nxc) * rb), NTW - nbt_of(nxc))
                                 : (nbt_of(nxc) * rb >= NDT ? 0 : (1 << 20));
  }
  static constexpr int cost_for(int nxc, int rb) {
    return imax(bcost_of(nxc) + rb * DCOST, rd_for(nxc, rb) * DCOST);
  }
  // best (NXC, RB) packed as NXC * 64 + RB; NXC = 1 in the precision form
  static constexpr int pick_split() {
    int best = -1, bc = 1 << 30;
    for (int nxc = 1; nxc <= (F64 ? 1 : K + 1); nxc *= 2) {
      if (nbt_of(nxc) > NTW) break;
      for (int rb = 0; rb <= 16; ++rb)
        if (cost_for(nxc, rb) < bc) { bc = cost_for(nxc, rb); best = nxc * 64 + rb; }
    }
    return best;
  }
  static constexpr int NXC = pick_split() / 64;
  static constexpr int KC = cdiv(K + 1, NXC);
  static constexpr int NBT = nbt_of(NXC);                 // x-DFT threads
  static constexpr int NOB = NTW - NBT;                   // threads without x-DFT work
  static constexpr int RB = pick_split() % 64;
  static constexpr int RD = rd_for(NXC, RB);
  static constexpr int SROW = TW * KPAD;                  // smoothed state of one output row segment
  // first channel of plane p (channel order: plane 0 kx = 0..K, complex planes
  // kx = -K..K, Nyquist plane kx = 0..K)
  __host__ __device__ static constexpr int base(int p) { return p == 0 ? 0 : (K + 1) + (p - 1) * M; }
  // shared-memory layout (bytes); E2 = bytes of a complex element of the sums
  static constexpr size_t E2 = F64 ? 16 : 8;
  static constexpr size_t O_TWR = 0;                          // [NPL][RW] (precision form), [XG][SW] (FP32)
  static constexpr size_t O_RING = al16(O_TWR + E2 * imax(NPL * RW, XG * SW));  // [M+1][NCHY][TW]
  static constexpr size_t O_DCR = al16(O_RING + E2 * (M + 1) * NCHY * TW);     // [M+1][NPL][TW]
  // x-DFT weights in double, precision form only (FP32: constant bank)
  static constexpr size_t O_XW = al16(O_DCR + E2 * (M + 1) * NPL * TW);        // [K+1][M]
  static constexpr size_t O_PBUF = al16(O_XW + (F64 ? E2 * (K + 1) * M : 0));  // float  [TW][PS]
  static constexpr size_t O_DBUF = al16(O_PBUF + 4ull * TW * PS);              // [2][NPL][TW]
  static constexpr size_t O_ABUF = al16(O_DBUF + E2 * 2 * NPL * TW);           // float  [RW][MZ+1]
  static constexpr size_t O_SROW = al16(O_ABUF + 4ull * RW * (MZ + 1));        // float  [3][SROW]
  static constexpr size_t O_MBAR = al16(O_SROW + 4ull * 3 * SROW);             // uint64 [3]
  static constexpr size_t O_OFFS = al16(O_MBAR + 8ull * 3);                    // float2 [NPL]
  // learned-estimator features (used only when they are requested)
  static constexpr int NBINS = M * M * MZ;
  static constexpr size_t O_FGS = al16(O_OFFS + 8ull * NPL);                   // int   [NBINS] gather
  static constexpr size_t O_FCH = al16(O_FGS + 4ull * NBINS);                  // float [TW][NCHY]
  static constexpr size_t O_FTOT = al16(O_FCH + 4ull * TW * NCHY);             // float [TW] 1/sum P
  static constexpr size_t SMEM = al16(O_FTOT + 4ull * TW);
  static_assert(RW <= 32, "the observer warp covers the row segment");
  static_assert(NBT <= NTW, "one x-DFT unit per thread, none on the observer warp");
  static_assert(F64 || (NXC <= 8 && NXC * KC >= K + 1), "x-DFT chunks cover kx = 0..K");
  static_assert(NBT * RB + NOB * RD >= NDT, "every reduction task has a thread");
};

__device__ __forceinline__ int clampi(int v, int n) { return v < 0 ? 0 : (v >= n ? n - 1 : v); }

// Per-thread asynchronous 4-byte copies global -> shared (each thread later
// consumes only what it copied, so a wait on its own groups suffices).
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Sum of M consecutive lanes' values starting at this lane (lanes + M - 1 <= 31
// are exact; the rest are unused), by doubling windows.
template <int M, typename T = float>
__device__ __forceinline__ T lane_box_sum(T v) {
  static_assert(M < 16, "window");
  const unsigned full = 0xffffffffu;
  const T s1 = v;
  const T s2 = s1 + __shfl_down_sync(full, s1, 1);
  const T s4 = s2 + __shfl_down_sync(full, s2, 2);
  const T s8 = s4 + __shfl_down_sync(full, s4, 4);
  T r = 0;
  int off = 0;
  if (M & 8) { r = s8; off = 8; }
  if (M & 4) { r += off ? __shfl_down_sync(full, s4, off) : s4; off += 4; }
  if (M & 2) { r += off ? __shfl_down_sync(full, s2, off) : s2; off += 2; }
  if (M & 1) { r += off ? __shfl_down_sync(full, s1, off) : s1; }
  return r;
}

// Observer update of one pixel (frame value pa[0], packed T_{t-1} in pa[1..Mz])
// -> T_t (packed) and its Hann-windowed planes Tw.
template <int M, int MZ>
__device__ __forceinline__ void observer_hann(const float* pa, float2 (&T)[SG<M, MZ>::NPL],
                                              float2 (&Tw)[SG<M, MZ>::NPL]) {
  using G = SG<M, MZ>;
  constexpr int J = G::J, NPL = G::NPL, ZI = MZ - 3;
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
    s[p] = cmul(c_lam[ZI][p], T[p]);
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
  const float2 hz = c_hz[ZI];
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

// FP32 x-DFT of one lane's (slot bg, column bx) for the kx of chunk CH: direct
// M-tap sums over the complex row (row[-mx], mx = 0..M-1) with the weights as
// constant-bank operands, each tap loaded once for the chunk's kx.  Slot 0
// holds the two real planes as (v0, v_Mz/2), whose spectra are (ac.x, db.x)
// and (ac.y, db.y); a complex plane's +kx and -kx outputs come from the same
// accumulators (the -kx weights are the conjugates).
template <int M, int MZ, int CH>
__device__ __forceinline__ void xdft_chunk(const float2* __restrict__ row, float2* __restrict__ rs, int bg, int bx) {
  using G = SG<M, MZ>;
  constexpr int K = G::K, TW = G::TW, NPL = G::NPL, KC = G::KC, MI = (M - 3) / 2;
  constexpr int KX0 = CH * KC;
  constexpr int NK = KX0 >= K + 1 ? 0 : (KX0 + KC <= K + 1 ? KC : K + 1 - KX0);
  if constexpr (NK > 0) {
    float2 ac[NK], db[NK];   // (sum wr vr, sum wr vi), (sum wi vr, sum wi vi)
#pragma unroll
    for (int c = 0; c < NK; ++c) { ac[c] = make_float2(0.f, 0.f); db[c] = make_float2(0.f, 0.f); }
#pragma unroll
    for (int mx = 0; mx < M; ++mx) {
      const float2 v = row[-mx];
#pragma unroll
      for (int c = 0; c < NK; ++c) {
        ac[c] = __ffma2_rn(c_xrr[MI][KX0 + c][mx], v, ac[c]);
        db[c] = __ffma2_rn(c_xii[MI][KX0 + c][mx], v, db[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < NK; ++c) {
      const int kx = KX0 + c;
      if (bg == 0) {
        rs[kx * TW + bx] = make_float2(ac[c].x, db[c].x);                                   // channel (0, kx)
        if (G::EVEN) rs[(G::base(NPL - 1) + kx) * TW + bx] = make_float2(ac[c].y, db[c].y);  // (Mz/2, kx)
      } else {
        const int c0 = G::base(bg) + K;                                                       // channel (bg, 0)
        rs[(c0 + kx) * TW + bx] = make_float2(ac[c].x - db[c].y, ac[c].y + db[c].x);
        if (kx > 0) rs[(c0 - kx) * TW + bx] = make_float2(ac[c].x + db[c].y, ac[c].y - db[c].x);
      }
    }
  }
}

// MODE 0: the plain path (no dump, no features, both compiled out); 1: debug
// dump of the windowed spectrum and power (features if requested); 2: the
// learned estimator's features.  F64: the precision form, spatial sums in
// double precision (one CTA per SM; the observer, the kz reduction and the
// smoothed state stay FP32, the power is rounded to FP32 once).
template <int M, int MZ, int MODE, bool F64 = false>
__global__ void __launch_bounds__(SG<M, MZ, F64>::NTHR, F64 ? 1 : 2) spectrum_kernel(const SpecArgs a) {
  constexpr bool DUMP = MODE == 1;
  using G = SG<M, MZ, F64>;
  using C2 = typename std::conditional<F64, double2, float2>::type;
  constexpr int K = G::K, J = G::J, NPL = G::NPL, NCHY = G::NCHY;
  constexpr int TW = G::TW, RW = G::RW, NTHR = G::NTHR, PS = G::PS, KPAD = G::KPAD;
  constexpr int NH = G::NH, NH1 = G::NH1, NDT = G::NDT, NTW = G::NTW, NBT = G::NBT, NOB = G::NOB;
  constexpr int RB = G::RB, RD = G::RD;
  constexpr bool EVEN = G::EVEN;
  constexpr int MI = (M - 3) / 2, ZI = MZ - 3;
  constexpr int RING_SLOT = NCHY * TW, DC_SLOT = NPL * TW;
  const int H = a.H, W = a.W;
  const int tid = threadIdx.x, lane = tid & 31;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* twr = reinterpret_cast<C2*>(smem_raw + G::O_TWR);
  C2* ring = reinterpret_cast<C2*>(smem_raw + G::O_RING);
  C2* dcr = reinterpret_cast<C2*>(smem_raw + G::O_DCR);
  C2* xw = reinterpret_cast<C2*>(smem_raw + G::O_XW);
  float* pbuf = reinterpret_cast<float*>(smem_raw + G::O_PBUF);
  C2* dbuf = reinterpret_cast<C2*>(smem_raw + G::O_DBUF);
  float* abuf = reinterpret_cast<float*>(smem_raw + G::O_ABUF);
  float* srow = reinterpret_cast<float*>(smem_raw + G::O_SROW);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + G::O_MBAR);
  float2* offs = reinterpret_cast<float2*>(smem_raw + G::O_OFFS);
  int* fgs = reinterpret_cast<int*>(smem_raw + G::O_FGS);
  float* fch = reinterpret_cast<float*>(smem_raw + G::O_FCH);
  float* ftot = reinterpret_cast<float*>(smem_raw + G::O_FTOT);
  const bool feat = MODE != 0 && !F64 && a.feat != nullptr;
  if (feat)
    for (int i = tid; i < a.feat_n; i += NTHR) fgs[i] = a.feat_gather[i];

  // Power scale (Mz/sqrt(N))^2 and the 1/16 of the 4x Hann taps, as sig^2 on
  // the x-DFT weights and box sums (everything before the power is linear).
  const float sig = sqrtf(float(MZ) / float(16 * M * M));
  const double sigd = sqrt(double(MZ) / double(16 * M * M));
  if constexpr (F64) {   // Hann(mx) e^{j2pi kx (mx-K)/M} sig, in double (FP32: constant bank, sig on the rows)
    for (int i = tid; i < (K + 1) * M; i += NTHR) {
      const int kx = i / M, mx = i % M;
      const double hann = 0.5 + 0.5 * cospi(2.0 * (mx - K) / M);
      double sn, cs;
      sincospi(2.0 * kx * (mx - K) / M, &sn, &cs);
      xw[i] = make_double2(hann * cs * sigd, hann * sn * sigd);
    }
  }
  const float alpha = a.alpha, oma = 1.0f - alpha;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(&mbar[b], 1);
    tc::fence_mbar_init();
  }

  // ---- static roles ---------------------------------------------------------
  // C: y-SDFT channel cy (plane plc, kx kxc) of column xy
  const bool cthr = tid < G::NCT;
  const int cy = cthr ? tid / TW : 0, xy = cthr ? tid % TW : 0;
  int plc, kxc;
  if (cy < K + 1) { plc = 0; kxc = cy; }
  else if (cy < K + 1 + J * M) { plc = 1 + (cy - (K + 1)) / M; kxc = (cy - (K + 1)) % M - K; }
  else { plc = NPL - 1; kxc = cy - (K + 1) - J * M; }
  const float wxh = kxc == 0 ? 0.5f : ((kxc == 1 || kxc == -1) ? 0.25f : 0.f);
  // B: x-DFT unit.  Precision form: (group bg, kx bkx, column bx); FP32:
  // (slot bg, column bx) for the kx of chunk bch (one chunk per warp)
  int bg, bkx = 0, bx, bch = 0;
  bool bthr;
  if constexpr (F64) {
    const int br = tid % G::GP;
    bg = tid / G::GP;
    bthr = tid < NBT && br < G::GU;
    bkx = br / TW;
    bx = br % TW;
  } else {
    const int wq = tid >> 5, t = (wq % G::WPC) * 32 + lane;
    const int u = (t + G::ROT) % G::XU;
    bch = wq / G::WPC;
    bthr = tid < NBT && t < G::XU;
    bg = bthr ? u / TW : 0;
    bx = bthr ? u % TW : 0;
  }
  // A: observer lane ua of the last warp
  const bool owarp = tid >= NTHR - 32;
  const int ua = lane;
  const bool athr = owarp && ua < RW;
  // D: reduction tasks d = dbase + q * dstride, q < (x-DFT thread ? RB : RD)
  const bool bown = tid < NBT;
  const int dbase = bown ? NOB * RD + tid : tid - NBT;
  const int dstride = bown ? NBT : NOB;
  const bool dthr = tid < NTW;
  // this thread's reduction tasks, fixed for the whole kernel: column x in the
  // low byte (0xff: no task), h above it
  constexpr int RQ = RB > RD ? RB : RD;
  uint32_t dtask[RQ];
#pragma unroll
  for (int q = 0; q < RQ; ++q) {
    const int d = dbase + q * dstride;
    const bool ok = dthr && q < (bown ? RB : RD) && d < NDT;
    dtask[q] = ok ? uint32_t(d / NH1) | (uint32_t(d % NH1) << 8) : 0xffu;
  }

  // ---- this CTA's share of the (strip, row) units -------------------------------
  // Units (strip, output row) in strip-major order; every segment a CTA walks
  // costs its rows plus 2K warm-up rows.  The split is uniform in a cost
  // coordinate that charges 2K rows at each strip start (cost c -> unit
  // s*H + max(0, o - 2K), s = c / (H + 2K), o = c mod (H + 2K)), so CTAs
  // whose range crosses a strip boundary get fewer output rows.
  const int nstrip = (W + TW - 1) / TW;
  const long long cstrip = (long long)H + 2 * K;
  const long long ctot = (long long)nstrip * cstrip;
  auto unit_of = [&](long long c) -> long long {
    const long long sidx = c / cstrip, o = c - sidx * cstrip;
    return sidx * H + (o > 2 * K ? o - 2 * K : 0);
  };
  const long long u0 = unit_of(ctot * blockIdx.x / gridDim.x);
  const long long u1 = unit_of(ctot * (blockIdx.x + 1) / gridDim.x);
  __syncthreads();

  // Smoothed state of output rows: ring of 3 row segments in shared memory,
  // moved by bulk copies issued by thread 0 (load two rows ahead, update in
  // place, store back); the n-th use of slot b completes mbarrier phase n & 1.
  int gbase = 0;                          // output rows this CTA finished in earlier segments
  bool timed_out = false;
  for (long long u = u0; u < u1;) {
    const int strip = int(u / H);
    const int y0 = int(u % H);
    // at most kSegRows output rows per recursion: the y-SDFT restarts from zero
    // (with its 2K-row warm-up) so rounding that the comb/resonator pole-zero
    // cancellation leaves behind cannot accumulate along an arbitrarily long column
    const int y1 = int(min(min((long long)H, (long long)y0 + (u1 - u)), (long long)y0 + kSegRows));
    u += y1 - y0;
    const int x0 = strip * TW;
    const int nrows = y1 - y0 + 2 * K;

    // y-resonator state: bins (p, p+K+1) packed as (re, re) and (im, im) pairs,
    // and the centre bin K
    float2 YR[K], YI[K], Yc = make_float2(0.f, 0.f);
#pragma unroll
    for (int p = 0; p < K; ++p) { YR[p] = make_float2(0.f, 0.f); YI[p] = make_float2(0.f, 0.f); }
    double2 Yd[F64 ? M : 1];      // the precision form: the M bins in double (index ky + K)
#pragma unroll
    for (int k = 0; k < (F64 ? M : 1); ++k) Yd[k] = make_double2(0.0, 0.0);

    auto loadA = [&](int i) {             // prefetch input row i into this lane's abuf slot
      if (athr) {
        const int rs = clampi(y0 - K + i, H), xs = clampi(x0 - K + ua, W);
        const size_t o = size_t(rs) * W + xs, plane = size_t(H) * W;
        float* dst = abuf + ua * (MZ + 1);
        cp_async4(dst, a.frame + o);
#pragma unroll
        for (int f = 0; f < MZ; ++f) cp_async4(dst + 1 + f, a.obs_old + f * plane + o);
      }
      cp_async_commit();
    };
    auto doA = [&](int i) {               // observer update + Hann(kz) of input row i
      if (!athr) return;
      const int r = y0 - K + i;
      float pa[MZ + 1];
#pragma unroll
      for (int f = 0; f <= MZ; ++f) pa[f] = abuf[ua * (MZ + 1) + f];
      float2 T[NPL], Tw[NPL];
      observer_hann<M, MZ>(pa, T, Tw);
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
      if constexpr (F64) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) {   // exact difference in double, real planes as (v, v)
          const bool real = (p == 0) || (EVEN && p == NPL - 1);
          const double vx = double(Tw[p].x) - double(offs[p].x), vy = double(Tw[p].y) - double(offs[p].y);
          twr[p * RW + ua] = real ? make_double2(vx, vx) : make_double2(vx, vy);
        }
      } else {
        // scaled by sig; slot 0 = the real planes as one complex row (v0, v_Mz/2), slot j = plane j
        const float vn = EVEN ? Tw[NPL - 1].x - offs[NPL - 1].x : 0.f;
        twr[ua] = make_float2((Tw[0].x - offs[0].x) * sig, vn * sig);
#pragma unroll
        for (int j = 1; j <= J; ++j) twr[j * G::SW + ua] = cscale(csub(Tw[j], offs[j]), sig);
      }
    };
    // whole observer warp: box sums along x of input row i (the (0,0) bin of
    // the row window at column ua), their running sum over the last M rows and
    // a ring of the last M+1 rows' sums
    auto doA2 = [&](int i) {
      C2 bs[NPL];
      if constexpr (F64) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) {
          const bool real = (p == 0) || (EVEN && p == NPL - 1);
          C2 v;
          v.x = 0; v.y = 0;
          if (ua < RW) v = twr[p * RW + ua];
          bs[p].x = lane_box_sum<M>(v.x);
          bs[p].y = real ? decltype(v.y)(0) : lane_box_sum<M>(v.y);
        }
      } else {   // slots: (plane 0, plane Mz/2), then the complex planes
#pragma unroll
        for (int s = 0; s <= J; ++s) {
          float2 v = make_float2(0.f, 0.f);
          if (ua < RW) v = twr[s * G::SW + ua];
          const float bx_ = lane_box_sum<M>(v.x);
          const float by_ = (s == 0 && !EVEN) ? 0.f : lane_box_sum<M>(v.y);
          if (s == 0) {
            bs[0] = make_float2(bx_, 0.f);
            if (EVEN) bs[NPL - 1] = make_float2(by_, 0.f);
          } else {
            bs[s] = make_float2(bx_, by_);
          }
        }
      }
      if (ua < TW) {
        const int slot = i % (M + 1), oslot = (i + 1) % (M + 1);   // oslot holds row i - M
        C2* dnew = dbuf + (i & 1) * DC_SLOT;
        const C2* dold = dbuf + ((i + 1) & 1) * DC_SLOT;
#pragma unroll
        for (int p = 0; p < NPL; ++p) {
          C2 val = bs[p];                 // FP32: the rows already carry sig
          if constexpr (F64) val = cscale(bs[p], sigd);
          C2 run = i > 0 ? cadd(dold[p * TW + ua], val) : val;
          if (i >= M) run = csub(run, dcr[oslot * DC_SLOT + p * TW + ua]);
          dcr[slot * DC_SLOT + p * TW + ua] = val;
          dnew[p * TW + ua] = run;
        }
      }
    };
    // bulk copies of the smoothed state of output row r (relative to y0)
    const int ncols = min(TW, W - x0);
    const uint32_t row_bytes = uint32_t(ncols) * KPAD * 4u;   // a multiple of 16
    auto row_slot = [&](int r) { return (gbase + r) % 3; };
    auto load_row = [&](int r) {          // thread 0
      const int b = row_slot(r);
      const float* src = a.Astate + (size_t(y0 + r) * W + x0) * KPAD;
      tc::mbar_expect_tx(&mbar[b], row_bytes);
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          ::"r"(tc::smem_u32(srow + b * G::SROW)), "l"(src), "r"(row_bytes), "r"(tc::smem_u32(&mbar[b]))
          : "memory");
    };
    auto store_row = [&](int r) {         // thread 0, after a CTA barrier
      const int b = row_slot(r);
      float* dst = (a.Astate_out ? a.Astate_out : a.Astate) + (size_t(y0 + r) * W + x0) * KPAD;
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                   ::"l"(dst), "r"(tc::smem_u32(srow + b * G::SROW)), "r"(row_bytes) : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    };
    const int TH = y1 - y0;
    auto doB = [&](int i) {               // x-DFT of input row i into ring slot i mod (M+1)
      if (!bthr) return;
      C2* rs = ring + (i % (M + 1)) * RING_SLOT;
      if constexpr (F64) {
        const double2* w = xw + bkx * M;
        if (bg == 0) {                    // real planes (stored (v, v))
          const double2* r0 = twr + bx + 2 * K;
          const double2* r1 = twr + (NPL - 1) * RW + bx + 2 * K;
          double2 c0 = make_double2(0.0, 0.0), c1 = make_double2(0.0, 0.0);
#pragma unroll
          for (int mx = 0; mx < M; ++mx) {
            const double2 cw = w[mx];
            c0.x = fma(cw.x, r0[-mx].x, c0.x);
            c0.y = fma(cw.y, r0[-mx].x, c0.y);
            if (EVEN) {
              c1.x = fma(cw.x, r1[-mx].x, c1.x);
              c1.y = fma(cw.y, r1[-mx].x, c1.y);
            }
          }
          rs[bkx * TW + bx] = c0;
          if (EVEN) rs[(G::base(NPL - 1) + bkx) * TW + bx] = c1;
        } else {                          // complex plane bg: +kx and -kx together
          const double2* row = twr + bg * RW + bx + 2 * K;
          double2 ac = make_double2(0.0, 0.0), db = make_double2(0.0, 0.0);
#pragma unroll
          for (int mx = 0; mx < M; ++mx) {
            const double2 cw = w[mx], v = row[-mx];
            ac.x = fma(cw.x, v.x, ac.x);
            ac.y = fma(cw.x, v.y, ac.y);
            db.x = fma(cw.y, v.x, db.x);
            db.y = fma(cw.y, v.y, db.y);
          }
          const int c0 = G::base(bg) + K;
          rs[(c0 + bkx) * TW + bx] = make_double2(ac.x - db.y, ac.y + db.x);
          if (bkx > 0) rs[(c0 - bkx) * TW + bx] = make_double2(ac.x + db.y, ac.y - db.x);
        }
        return;
      } else {                            // FP32: this warp's kx chunk (compile-time weights)
        const float2* row = twr + bg * G::SW + bx + 2 * K;
        switch (bch) {
          case 0: xdft_chunk<M, MZ, 0>(row, rs, bg, bx); break;
          case 1: xdft_chunk<M, MZ, 1>(row, rs, bg, bx); break;
          case 2: xdft_chunk<M, MZ, 2>(row, rs, bg, bx); break;
          case 3: xdft_chunk<M, MZ, 3>(row, rs, bg, bx); break;
          case 4: xdft_chunk<M, MZ, 4>(row, rs, bg, bx); break;
          case 5: xdft_chunk<M, MZ, 5>(row, rs, bg, bx); break;
          case 6: xdft_chunk<M, MZ, 6>(row, rs, bg, bx); break;
          default: xdft_chunk<M, MZ, 7>(row, rs, bg, bx); break;
        }
      }
    };
    auto doC = [&](int i) {               // y-SDFT, Hann(ky), high-pass, power of row i
      if (!cthr) return;
      const int yo = y0 + i - 2 * K;
      if constexpr (F64) {                // Y_k <- w_k Y_k + c_k d in double, Hann, correction, power
        const double2 xn = ring[(i % (M + 1)) * RING_SLOT + tid];
        double2 d = xn;
        if (i >= M) d = csub(xn, ring[((i + 1) % (M + 1)) * RING_SLOT + tid]);
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const double2 w = c_dw[MI][k], c = c_dc[MI][k], y = Yd[k];
          const double cr = fma(c.x, d.x, -c.y * d.y), ci = fma(c.x, d.y, c.y * d.x);
          Yd[k] = make_double2(fma(w.x, y.x, fma(-w.y, y.y, cr)), fma(w.x, y.y, fma(w.y, y.x, ci)));
        }
        if (!(i >= 2 * K && yo < y1)) return;
        const double2 D = dbuf[(i & 1) * DC_SLOT + plc * TW + xy];
        float* pb = pbuf + xy * PS + cy * M;
#pragma unroll
        for (int k = 0; k < M; ++k) {
          const double2 yp = Yd[(k + 1) % M], ym = Yd[(k + M - 1) % M];
          double zx = fma(2.0, Yd[k].x, yp.x + ym.x), zy = fma(2.0, Yd[k].y, yp.y + ym.y);
          const double f = k == K ? 2.0 * wxh : ((k == K - 1 || k == K + 1) ? double(wxh) : 0.0);
          zx -= D.x * f;
          zy -= D.y * f;
          const double pw = fma(zx, zx, zy * zy);
          pb[k] = float(pw);
          if (DUMP && x0 + xy < W) {
            const SpecTables& tb = *a.tables;
            const size_t pix = size_t(yo) * W + x0 + xy;
            const int izp = plc + J, izm = ((-plc) + J + MZ) % MZ;
            const double sc = 0.25 * double(MZ) / sqrt(double(M * M * MZ)) / sigd;
            const float2 u = cmul(tb.uncenter[kxc + K], tb.uncenter[k]);
            const float2 sv = make_float2(float((double(u.x) * zx - double(u.y) * zy) * sc),
                                          float((double(u.x) * zy + double(u.y) * zx) * sc));
            const size_t op = ((pix * MZ + izp) * M + k) * M + (kxc + K);
            const size_t om = ((pix * MZ + izm) * M + (M - 1 - k)) * M + (K - kxc);
            a.dump_win[op] = sv;
            a.dump_win[om] = conjf2(sv);
            if (a.dump_pow) { a.dump_pow[op] = float(pw); a.dump_pow[om] = float(pw); }
          }
        }
      } else {
      const float2 xn = ring[(i % (M + 1)) * RING_SLOT + tid];
      float2 d = xn;
      if (i >= M) d = csub(xn, ring[((i + 1) % (M + 1)) * RING_SLOT + tid]);
      // Y_k <- w_k Y_k + c_k d for the bin pairs (packed), and the centre bin
      // (w = c = 1); per component the same fmaf sequence as the complex form
      const float2 dx2 = make_float2(d.x, d.x), dy2 = make_float2(d.y, d.y);
#pragma unroll
      for (int p = 0; p < K; ++p) {
        const float2 tr = __ffma2_rn(c_rcx[MI][p], dx2, __fmul2_rn(c_rncy[MI][p], dy2));
        const float2 ti = __ffma2_rn(c_rcx[MI][p], dy2, __fmul2_rn(c_rcy[MI][p], dx2));
        const float2 r = YR[p];
        YR[p] = __ffma2_rn(c_rwx[MI][p], r, __ffma2_rn(c_rnwy[MI][p], YI[p], tr));
        YI[p] = __ffma2_rn(c_rwx[MI][p], YI[p], __ffma2_rn(c_rwy[MI][p], r, ti));
      }
      Yc = cadd(Yc, d);
      if (!(i >= 2 * K && yo < y1)) return;
      // 4 x [Hann along ky (taps 1/4, 1/2, 1/4 in the centred basis), minus
      // Hann_x Hann_y of the removed (0,0) bin]; the 1/16 is in sig^2
      const float2 D = dbuf[(i & 1) * DC_SLOT + plc * TW + xy];
      float* pb = pbuf + xy * PS + cy * M;
      const float2 two2 = make_float2(2.f, 2.f);
      float2 psum = make_float2(0.f, 0.f);   // features: this channel's power summed over ky
      auto dump = [&](int k, float zx, float zy, float pw) {
        // uncentred S'' = e^{+j2pi (kx+ky)K/M} Z, and its conjugate partner at -k
        if (!(DUMP && x0 + xy < W)) return;
        const SpecTables& tb = *a.tables;
        const size_t pix = size_t(yo) * W + x0 + xy;
        const int izp = plc + J, izm = ((-plc) + J + MZ) % MZ;
        const float2 sv = cscale(cmul(cmul(tb.uncenter[kxc + K], tb.uncenter[k]), make_float2(zx, zy)),
                                 0.25f * float(MZ) / sqrtf(float(M * M * MZ)) / sig);
        const size_t op = ((pix * MZ + izp) * M + k) * M + (kxc + K);
        const size_t om = ((pix * MZ + izm) * M + (M - 1 - k)) * M + (K - kxc);
        a.dump_win[op] = sv;
        a.dump_win[om] = conjf2(sv);
        if (a.dump_pow) { a.dump_pow[op] = pw; a.dump_pow[om] = pw; }
      };
#pragma unroll
      for (int p = 0; p < K; ++p) {
        // neighbours k+1 and k-1 of the pair's bins (k = p, p+K+1), cyclic in k
        float2 nr, ni, mr, mi;
        if (p + 1 < K) { nr = YR[p + 1]; ni = YI[p + 1]; }
        else { nr = make_float2(Yc.x, YR[0].x); ni = make_float2(Yc.y, YI[0].x); }
        if (p > 0) { mr = YR[p - 1]; mi = YI[p - 1]; }
        else { mr = make_float2(YR[K - 1].y, Yc.x); mi = make_float2(YI[K - 1].y, Yc.y); }
        float2 zr = __ffma2_rn(two2, YR[p], __fadd2_rn(nr, mr));
        float2 zi = __ffma2_rn(two2, YI[p], __fadd2_rn(ni, mi));
        if (p == K - 1) { zr.x -= D.x * wxh; zi.x -= D.y * wxh; }   // bin K-1
        if (p == 0) { zr.y -= D.x * wxh; zi.y -= D.y * wxh; }       // bin K+1
        const float2 pw = __ffma2_rn(zr, zr, __fmul2_rn(zi, zi));
        pb[p] = pw.x;
        pb[p + K + 1] = pw.y;
        if constexpr (MODE != 0) psum = __fadd2_rn(psum, pw);
        dump(p, zr.x, zi.x, pw.x);
        dump(p + K + 1, zr.y, zi.y, pw.y);
      }
      // centre bin K
      float zcx = fmaf(2.f, Yc.x, YR[0].y + YR[K - 1].x), zcy = fmaf(2.f, Yc.y, YI[0].y + YI[K - 1].x);
      zcx -= D.x * (wxh * 2.f);
      zcy -= D.y * (wxh * 2.f);
      const float pwc = fmaf(zcx, zcx, zcy * zcy);
      pb[K] = pwc;
      dump(K, zcx, zcy, pwc);
      if (feat) {
        // every bin of a complex plane, and of a real plane's kx > 0 channel,
        // stands for itself and its mirror -k (not stored); a real plane's
        // kx = 0 channel holds both ky and -ky
        const bool self_mirror = (plc == 0 || (EVEN && plc == NPL - 1)) && kxc == 0;
        const float sc = psum.x + psum.y + pwc;
        fch[xy * NCHY + cy] = self_mirror ? sc : 2.f * sc;
      }
      }
    };
    auto doD = [&](int i) {               // reduce over kz, smooth (in place in the row ring)
      const int yo = y0 + i - 2 * K, r = i - 2 * K;
      if (!(i >= 2 * K && yo < y1) || !dthr) return;
      const int b = row_slot(r);
      if (!tc::mbar_wait(&mbar[b], uint32_t(((gbase + r) / 3) & 1), 1000000000ull)) timed_out = true;
      float* st = srow + b * G::SROW;
      auto one = [&](uint32_t t) {
        const int x = int(t & 0xffu), hi = int(t >> 8);
        if (x >= ncols) return;
        // P(h, kz) for the slots kz = 0, +j, -j (= P(-h, +j)), Mz/2 of this h:
        // offsets x*PS + (c*M + ky + K) with c the channel of (plane, +-hx)
        const int op = x * PS + hi + K, om = x * PS - hi + K;
        const float p0 = pbuf[op];
        float Ac = p0, As = 0.f;
#pragma unroll
        for (int j = 1; j <= J; ++j) {
          const float pp = pbuf[op + (G::base(j) + K) * M], pm = pbuf[om + (G::base(j) + K) * M];
          Ac = fmaf(pp + pm, c_cz[ZI][j], Ac);
          As = fmaf(pp - pm, c_sz[ZI][j], As);
        }
        if (EVEN) {
          const float pn = pbuf[op + G::base(NPL - 1) * M];
          Ac -= pn;
        }
        float* sp = st + x * KPAD + hi;
        sp[0] = fmaf(oma, Ac, alpha * sp[0]);
        if (hi > 0) sp[NH] = fmaf(oma, As, alpha * sp[NH]);
      };
      if (bown) {
#pragma unroll
        for (int q = 0; q < RB; ++q) one(dtask[q]);
      } else {
#pragma unroll
        for (int q = 0; q < RD; ++q) one(dtask[q]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the bulk store
      // learned-estimator features of this output row, (log2(P / sum P + 1e-6) + 10) / 10
      // of every requested bin, BF16.  Lanes take consecutive bin pairs (one
      // 4-byte store each, 128 contiguous bytes per warp; gathers from the power
      // block at most 2-way bank-conflicted), and a thread's two gather offsets
      // serve all TW pixels of the row.
      if (feat) {
        // the observer warp's 1 / sum P of the row's pixels (doT)
        asm volatile("bar.sync 1, %0;" ::"r"(NTHR) : "memory");
        const int np = a.feat_ld / 2, nfeat = a.feat_n;
        const int nx = W - x0 < TW ? W - x0 : TW;
        __nv_bfloat162* frow = reinterpret_cast<__nv_bfloat162*>(a.feat) + (size_t(yo) * W + x0) * np;
        float2 iv2[TW];
#pragma unroll
        for (int x = 0; x < TW; ++x) iv2[x] = make_float2(ftot[x], ftot[x]);
        for (int j = tid; j < np; j += NTW) {
          const int b0 = 2 * j;
          __nv_bfloat162* fp = frow + j;
          if (b0 + 1 < nfeat) {
            const int g0 = fgs[b0], g1 = fgs[b0 + 1];
            // every shared-memory read of the TW pixels first: the global stores
            // would otherwise order the next pixel's reads behind them
            float2 v[TW];
#pragma unroll
            for (int x = 0; x < TW; ++x) v[x] = make_float2(pbuf[x * PS + g0], pbuf[x * PS + g1]);
#pragma unroll
            for (int x = 0; x < TW; ++x) {
              if (x >= nx) break;
              // P / sum P + 1e-6 >= 1e-6: a normal number, so log2 with flush-to-zero is exact
              // to the same approximation; (log2 y + 10) / 10 as one FMA
              const float2 y = __ffma2_rn(v[x], iv2[x], make_float2(1e-6f, 1e-6f));
              float l0, l1;
              asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l0) : "f"(y.x));
              asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l1) : "f"(y.y));
              const float2 f = __ffma2_rn(make_float2(l0, l1), make_float2(0.1f, 0.1f), make_float2(1.f, 1.f));
              *fp = __floats2bfloat162_rn(f.x, f.y);
              fp += np;
            }
          } else {
            // the odd last feature and the row padding
            const int g0 = b0 < nfeat ? fgs[b0] : -1;
#pragma unroll
            for (int x = 0; x < TW; ++x) {
              if (x >= nx) break;
              const float f0 = g0 >= 0 ? 0.1f * (__log2f(fmaf(pbuf[x * PS + g0], iv2[x].x, 1e-6f)) + 10.f) : 0.f;
              *fp = __floats2bfloat162_rn(f0, 0.f);
              fp += np;
            }
          }
        }
      }
    };

    // observer warp, learned-estimator features only: 1 / (sum of P over all M^2 Mz
    // bins) of every pixel of output row i from the y-SDFT threads' channel sums
    // (fixed order), released to the feature threads by a named barrier that
    // they wait on after their reduction tasks (both sides take it once per
    // output row under the same condition)
    auto doT = [&](int i) {
      if constexpr (MODE != 0 && !F64) {
        const int yo = y0 + i - 2 * K;
        if (!(feat && i >= 2 * K && yo < y1)) return;
        // LP lanes per pixel (a power of two), each summing every LP-th channel
        constexpr int LP = 32 / TW >= 16 ? 16 : (32 / TW >= 8 ? 8 : (32 / TW >= 4 ? 4 : (32 / TW >= 2 ? 2 : 1)));
        constexpr int PPASS = 32 / LP;
#pragma unroll
        for (int x0p = 0; x0p < TW; x0p += PPASS) {
          const int x = x0p + lane / LP, q = lane % LP;
          float t = 0.f;
          if (x < TW) {
#pragma unroll
            for (int c = q; c < NCHY; c += LP) t += fch[x * NCHY + c];
          }
#pragma unroll
          for (int off = 1; off < LP; off <<= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
          if (x < TW && q == 0) ftot[x] = t > 0.f ? 1.f / t : 0.f;
        }
        __syncwarp();
        asm volatile("bar.arrive 1, %0;" ::"r"(NTHR) : "memory");
      }
    };

    // ---- prologue: offsets, observer of row 0, x-DFT of row 0 ----------------
    // Per-plane offset removed from every Tw of this segment before the spatial
    // sums.  The high-passed, Hann-windowed spectrum is exactly invariant to a
    // spatially constant offset per temporal plane (it only feeds the removed
    // kx = ky = 0 bin and the correction that cancels its window leakage), so
    // subtracting one constant per segment leaves the result unchanged while
    // keeping the FP32 sums at the scale of the texture instead of the DC level.
    // The constant is the mean of Tw over the segment's first window rows (min(M,
    // rows) input rows of the TW + 2K columns), so the residual DC that the sums
    // and the leakage correction carry is the variation of the local mean, not
    // the full texture amplitude at one pixel.  It is formed as the first
    // pixel's Tw plus the mean difference from it, which is exactly that pixel's
    // value when the block is constant (a constant input then leaves exact
    // zeros in every spatial sum, as the oracle's high-pass does).
    {
      // all threads: one pixel (row i, column u) of the block each (at most two)
      constexpr int NW = NTHR / 32;
      const int nr0 = min(M, nrows), ntask = nr0 * RW;
      float2 tw[2][NPL];
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const int t = tid + r * NTHR;
#pragma unroll
        for (int p = 0; p < NPL; ++p) tw[r][p] = make_float2(0.f, 0.f);
        if (t < ntask) {
          const int i = t / RW, u = t - i * RW;
          const int rs = clampi(y0 - K + i, H), xs = clampi(x0 - K + u, W);
          const size_t o = size_t(rs) * W + xs, plane = size_t(H) * W;
          float pa[MZ + 1];
          pa[0] = a.frame[o];
#pragma unroll
          for (int f = 0; f < MZ; ++f) pa[1 + f] = a.obs_old[f * plane + o];
          float2 Tn[NPL];
          observer_hann<M, MZ>(pa, Tn, tw[r]);
        }
      }
      if (tid == 0) {
#pragma unroll
        for (int p = 0; p < NPL; ++p) offs[p] = tw[0][p];      // the reference: row 0, column 0
      }
      __syncthreads();
      float2* red = reinterpret_cast<float2*>(pbuf);           // [NW][NPL] scratch (pbuf is free here)
#pragma unroll
      for (int p = 0; p < NPL; ++p) {
        float2 v = make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 2; ++r)
          if (tid + r * NTHR < ntask) v = cadd(v, csub(tw[r][p], offs[p]));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          v.x += __shfl_xor_sync(0xffffffffu, v.x, off);
          v.y += __shfl_xor_sync(0xffffffffu, v.y, off);
        }
        if (lane == 0) red[(tid >> 5) * NPL + p] = v;
      }
      __syncthreads();
      if (tid == 0) {
        const float inv = 1.0f / float(ntask);
#pragma unroll
        for (int p = 0; p < NPL; ++p) {
          float2 v = make_float2(0.f, 0.f);
          for (int w = 0; w < NW; ++w) v = cadd(v, red[w * NPL + p]);   // fixed order
          offs[p] = cadd(offs[p], cscale(v, inv));
        }
      }
    }
    if (owarp) loadA(0);
    if (tid == 0) {
      load_row(0);
      if (TH > 1) load_row(1);
    }
    __syncthreads();
    cp_async_wait0();
    if (owarp) {
      doA(0);
      if (nrows > 1) loadA(1);
    }
    __syncthreads();
    doB(0);
    if (owarp) doA2(0);
    __syncthreads();

    // ---- pipelined rows: {y-SDFT(i), observer(i+1)},
    //      {reduce(i), x-DFT(i+1), box sums(i+1)}
    for (int i = 0; i < nrows; ++i) {
      if (tid == 0 && i > 2 * K && i - 1 - 2 * K < TH) {
        // the previous iteration finished output row rp: store it, then reuse
        // the slot of row rp - 1 (its store has read it) for row rp + 2
        const int rp = i - 1 - 2 * K;
        store_row(rp);
        asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
        if (rp + 2 < TH) load_row(rp + 2);
      }
      doC(i);
      if (owarp && i + 1 < nrows) {
        cp_async_wait0();
        doA(i + 1);
        if (i + 2 < nrows) loadA(i + 2);
      }
      __syncthreads();
      if (owarp) doT(i);
      doD(i);
      if (i + 1 < nrows) {
        doB(i + 1);
        if (owarp) doA2(i + 1);
      }
      __syncthreads();
    }
    if (tid == 0) {
      store_row(TH - 1);
      asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
    gbase += TH;
    cp_async_wait0();
    __syncthreads();   // before the next segment rewrites offs and the row ring
  }
  if (timed_out && a.err) atomicExch(a.err, 1);
}

template <int M, int MZ>
cudaError_t launch_spec_t(const SpecArgs& a, cudaStream_t st) {
  using G = SG<M, MZ>;
  using G64 = SG<M, MZ, true>;
  if (a.tw != G::TW || a.kpad != G::KPAD) return cudaErrorInvalidValue;
  if (a.f64 && a.feat) return cudaErrorInvalidValue;     // no features in the precision form
  auto kern = a.f64 ? (a.dump_win ? spectrum_kernel<M, MZ, 1, true> : spectrum_kernel<M, MZ, 0, true>)
                    : (a.dump_win ? spectrum_kernel<M, MZ, 1>
                                  : (a.feat ? spectrum_kernel<M, MZ, 2> : spectrum_kernel<M, MZ, 0>));
  const size_t smem = a.f64 ? G64::SMEM : G::SMEM;
  ResidentShape rs{};
  cudaError_t e = resident_shape(kern, G::NTHR, smem, &rs);
  if (e != cudaSuccess) return e;
  const int nsm = rs.nsm, per_sm = rs.per_sm;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // one wave of CTAs, each with an equal share of the (strip, row) units
  const long long units = (long long)((a.W + G::TW - 1) / G::TW) * a.H;
  long long grid = (long long)nsm * per_sm;
  if (grid > units) grid = units;
  kern<<<unsigned(grid), G::NTHR, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

#define WH_SPEC_CASES(X) \
  X(5, 3) X(5, 4) X(5, 5) X(5, 6) \
  X(7, 3) X(7, 4) X(7, 5) X(7, 6) \
  X(9, 3) X(9, 4) X(9, 5) X(9, 6) \
  X(15, 4) X(15, 5) X(15, 6)

// Upload the constant tables (all window sizes and temporal orders, per device).
cudaError_t spectrum_init_constants() {
  static std::atomic<bool> done[64];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && done[dev].load()) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);      // one upload per device even with concurrent creators
  if (dev < 64 && done[dev].load()) return cudaSuccess;
  const double pi = 3.14159265358979323846;
  float2 w[7][kMaxM], c[7][kMaxM];
  for (int mi = 0; mi < 7; ++mi) {
    const int M = 2 * mi + 3, K = (M - 1) / 2;
    for (int i = 0; i < kMaxM; ++i) {
      const int k = i - K;
      w[mi][i] = make_float2(float(std::cos(2 * pi * k / M)), float(std::sin(2 * pi * k / M)));
      c[mi][i] = make_float2(float(std::cos(-2 * pi * k * K / M)), float(std::sin(-2 * pi * k * K / M)));
    }
  }
  float2 lam[kZN][kMaxPlanes] = {}, hz[kZN] = {};
  float cz[kZN][kMaxPlanes] = {}, sz[kZN][kMaxPlanes] = {};
  for (int zi = 0; zi < kZN; ++zi) {
    const int Mz = zi + 3;
    for (int p = 0; p <= Mz / 2 && p < kMaxPlanes; ++p) {
      // the Nyquist plane p = Mz/2 rotates by e^{j pi} = -1
      lam[zi][p] = make_float2(float(std::cos(2 * pi * p / Mz)), float(std::sin(2 * pi * p / Mz)));
      cz[zi][p] = float(std::cos(2 * pi * p / Mz));
      sz[zi][p] = float(std::sin(2 * pi * p / Mz));
    }
    const double ph = -2 * pi * ((Mz - 1) / 2.0) / Mz;
    hz[zi] = make_float2(float(std::cos(ph)), float(std::sin(ph)));
  }
  float2 rwx[7][kMaxK] = {}, rwy[7][kMaxK] = {}, rnwy[7][kMaxK] = {};
  float2 rcx[7][kMaxK] = {}, rcy[7][kMaxK] = {}, rncy[7][kMaxK] = {};
  for (int mi = 0; mi < 7; ++mi) {
    const int K = mi + 1;
    for (int p = 0; p < K; ++p) {
      const int q = p + K + 1;
      rwx[mi][p] = make_float2(w[mi][p].x, w[mi][q].x);
      rwy[mi][p] = make_float2(w[mi][p].y, w[mi][q].y);
      rnwy[mi][p] = make_float2(-w[mi][p].y, -w[mi][q].y);
      rcx[mi][p] = make_float2(c[mi][p].x, c[mi][q].x);
      rcy[mi][p] = make_float2(c[mi][p].y, c[mi][q].y);
      rncy[mi][p] = make_float2(-c[mi][p].y, -c[mi][q].y);
    }
  }
  // x-DFT weights, the centred Hann-windowed DFT of Eq. (6)-(7) along x:
  // Hann(mx) = 1/2 + 1/2 cos(2pi (mx-K)/M), phase 2pi kx (mx-K)/M
  static float2 xrr[7][kMaxK + 1][kMaxM], xii[7][kMaxK + 1][kMaxM];
  for (int mi = 0; mi < 7; ++mi) {
    const int M = 2 * mi + 3, K = (M - 1) / 2;
    for (int kx = 0; kx <= K; ++kx)
      for (int mx = 0; mx < M; ++mx) {
        const double hann = 0.5 + 0.5 * std::cos(2.0 * pi * (mx - K) / M);
        const double ph = 2.0 * pi * kx * (mx - K) / M;
        const float wr = float(hann * std::cos(ph)), wi = float(hann * std::sin(ph));
        xrr[mi][kx][mx] = make_float2(wr, wr);
        xii[mi][kx][mx] = make_float2(wi, wi);
      }
  }
  double2 dw[7][kMaxM] = {}, dc[7][kMaxM] = {};
  for (int mi = 0; mi < 7; ++mi) {
    const int M = 2 * mi + 3, K = (M - 1) / 2;
    for (int i = 0; i < M; ++i) {
      const int k = i - K;
      dw[mi][i] = make_double2(std::cos(2 * pi * k / M), std::sin(2 * pi * k / M));
      dc[mi][i] = make_double2(std::cos(-2 * pi * k * K / M), std::sin(-2 * pi * k * K / M));
    }
  }
  cudaError_t e = cudaMemcpyToSymbol(c_rwx, rwx, sizeof(rwx));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dw, dw, sizeof(dw));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_dc, dc, sizeof(dc));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rwy, rwy, sizeof(rwy));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rnwy, rnwy, sizeof(rnwy));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rcx, rcx, sizeof(rcx));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rcy, rcy, sizeof(rcy));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_rncy, rncy, sizeof(rncy));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_lam, lam, sizeof(lam));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_hz, hz, sizeof(hz));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_cz, cz, sizeof(cz));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_sz, sz, sizeof(sz));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_xrr, xrr, sizeof(xrr));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_xii, xii, sizeof(xii));
  if (e == cudaSuccess && dev < 64) done[dev].store(true);
  return e;
}

bool spectrum_supported(int M, int Mz) {
#define X(m, z) if (M == m && Mz == z) return true;
  WH_SPEC_CASES(X)
#undef X
  return false;
}

int spectrum_threads(int M, int Mz) {
#define X(m, z) if (M == m && Mz == z) return SG<m, z>::NTHR;
  WH_SPEC_CASES(X)
#undef X
  return 0;
}

size_t spectrum_smem(int M, int Mz, bool f64) {
#define X(m, z) if (M == m && Mz == z) return f64 ? SG<m, z, true>::SMEM : SG<m, z>::SMEM;
  WH_SPEC_CASES(X)
#undef X
  return 0;
}

cudaError_t launch_spectrum(const SpecArgs& a, cudaStream_t st) {
#define X(m, z) if (a.M == m && a.Mz == z) return launch_spec_t<m, z>(a, st);
  WH_SPEC_CASES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace wh
