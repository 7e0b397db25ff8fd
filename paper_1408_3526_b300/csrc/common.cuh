// Device-side definitions shared by the whitening kernels (sm_103a).
//
// Data layout in HBM (one stream, frame H x W, window M = 2K+1, Mz bins):
//   obs[2]  [Mz][H][W] f32   observer a-posteriori state T_t(kz), Hermitian
//                            packed: f=0 Re T(0); f=2j-1,2j Re/Im T(j),
//                            j=1..J; f=Mz-1 Re T(Mz/2) if Mz even.  Ping-pong:
//                            the spectrum kernel reads one, writes the other.
//   Astate  [H*W][kpad] f32  smoothed autocorrelation basis A'(h): index 0 =
//                            A_c(0,0); 1..nh = A_c(h); nh+1..2nh = A_s(h),
//                            h over the half plane (kx=0, ky=1..K; then kx=1..K,
//                            ky=-K..K).  R(l) is a fixed linear map of it.
//   whitened, vx, vy [H][W] f32; vidx [H][W] i32.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace wh {

constexpr int kMaxM = 15;
constexpr int kMaxMz = 8;
constexpr int kMaxL = 31;
constexpr int kMaxPlanes = kMaxMz / 2 + 1;
constexpr int kMaxChan = 2 * (kMaxM) + (kMaxPlanes) * kMaxM + kMaxPlanes;

// Tables of the spectrum kernel, built on the host in double precision.
struct SpecTables {
  int nch;                      // channels incl. the per-plane box-sum (DC) channels
  int nchy;                     // channels that run the y-SDFT (first nchy)
  int nplanes;                  // stored temporal planes p = 0..nplanes-1
  int nh;                       // (M*M-1)/2
  int nslot;                    // P-gather slots per h: 1 + 2J + even
  int ch_plane[kMaxChan];
  int ch_kx[kMaxChan];          // kx of the channel (0 for DC channels)
  float2 xcoef[kMaxChan][kMaxM];  // x-DFT weights: Hann(mx) e^{j2pi kx (mx-K)/M}; DC: 1
  float2 wres[kMaxM];           // resonator twiddle e^{+j2pi ky/M}, index ky+K
  float2 cphase[kMaxM];         // centring phase e^{-j2pi ky K/M}
  float2 lam[kMaxPlanes];       // observer rotation e^{+j2pi p/Mz}
  float2 hann_z;                // e^{-j2pi Dz/Mz}
  float cz[kMaxPlanes], sz[kMaxPlanes];   // cos/sin(2pi p/Mz)
  float2 uncenter[kMaxM];       // e^{+j2pi k K/M} (debug dump only)
};

struct SpecArgs {
  int H, W;
  int M, Mz;
  int tw, th;                   // output tile
  int kpad;
  float alpha;
  const float* frame;
  const float* obs_old;
  float* obs_new;
  float* Astate;                // smoothed state of the previous frame (read)
  float* Astate_out;            // where the updated state goes; nullptr: in place
  const SpecTables* tables;     // device copy
  const int* hgather;           // [nh+1][nslot] offsets (c*M + iy) into a pixel's P block
  float2* dump_win;             // optional [H*W][Mz][M][M]
  float* dump_pow;              // optional [H*W][Mz][M][M]
  // learned-estimator features (optional): per pixel, (log2(P(k)/sum P + 1e-6) + 10)/10 of
  // the bins in the order [kz][ky][kx] (kz = -J.., ky, kx = -K..) -- all M*M*Mz of them,
  // or only those whose mirror -b does not come earlier (P(-b) = P(b)) -- BF16, row
  // stride feat_ld; feat_gather[i] = offset (c*M + iy) of feature i's bin (or of its
  // mirror) in a pixel's power block.
  void* feat;
  int feat_ld;
  int feat_n;                   // features per pixel (<= M*M*Mz): all bins, or one per mirror pair
  const int* feat_gather;
  int* err;                     // device status word: set nonzero if a bounded wait gives up
  int f64;                      // 1: the precision form (spatial sums in double)
};

struct AutocorrArgs {
  int H, W, M, L, kpad;
  float vmax, vstep;
  const float* Astate;
  int* vidx;
  float* vx;
  float* vy;
  float* rs_out;                // optional [H*W][L*L]
  const int* pix_list;          // optional: evaluate only these pixels ...
  const int* n_list;            // ... (count on the device)
  const float2* tab_y;          // e^{j2pi ky ly/M}: [L][M]   (index ky+K)
  const float2* tab_x;          // e^{j2pi kx lx/M}: [L][K+1]
};

struct AutocorrTcArgs {
  int H, W, M, L, kpad;
  int kg;                       // leading dimension of a16 and the table (M^2 rounded up to 8)
  int ntile;                    // 128-column tiles of the grid
  int ncand;                    // shortlist entries per pixel (cand_* row stride)
  int ovf_group;                // entries per shortlist group (last of a group inside the window -> incomplete)
  int mode;                     // 0: exact FP32 re-rank of the shortlist; 1: tensor-core value decides
  int bf16;
  float vmax, vstep;
  const float* Astate;
  void* a16;                    // [H*W][kg] F16 or BF16
  float* l1;                    // [H*W] sum |a16|
  float* cand_val;              // [H*W][ncand]
  int* cand_idx;
  int* vidx;
  float* vx;
  float* vy;
  const float2* tab_x;          // e^{j2pi kx lx/M}: [L][K+1]
  int* n_fallback;              // optional counter of pixels evaluated on the whole grid
};

// Autocorrelation search with the separable stage on tensor cores
// (k_autocorr_tcsep.cu); bop: the stage-1 operand [64][32] TF32 values in the
// 128-byte-swizzled K-major layout (row n = 2 gy + re/im, column k = 4 (ky-1) +
// {sr, dr, si, di}, k = 28/29: Qr/Qi(kx, 0)).
struct TcSepArgs {
  int npix, M, L, kpad;
  float vmax, vstep;
  float wcoef;                  // bound widening per unit of sum |Q sums| (TF32 error)
  const float* Astate;
  int* vidx;
  float* vx;
  float* vy;
  const float* bop;
  const float2* tab_x;          // e^{j2pi kx lx/M}: [L][K+1]
  int* err;
};

// Autocorrelation search with the whole contraction on tensor cores
// (k_autocorr_tcd.cu): per pixel the F16 product decides alone where one grid
// point lies within the rigorous error window of the maximum; the others are
// listed (ccount > 0 points in cand, or -1: the whole grid) and evaluated
// exactly in FP32 by the same kernel.
struct TcDenseArgs {
  int npix, M, L, kpad;
  float vmax, vstep;
  const float* Astate;
  int* vidx;
  float* vx;
  float* vy;
  const float2* tab_x;          // e^{j2pi kx lx/M}: [L][K+1]
  int* ccount;                  // [npix] scratch
  int* cand;                    // [npix][8] scratch
  unsigned long long* counts;   // optional: [0] pixels with listed points, [1] whole-grid pixels
  int* err;
};

struct PefArgs {
  int H, W, M, Mz, L, mpz;
  const float* obs;             // T_t, just written
  const int* vidx;
  // separable FIR weights h(d; v, mz) of Eq. (2), incl. scale, in one buffer
  // (layout: pef_hw2_offset / pef_hwp_offset):
  //   float  [L][Mz][M]            h
  //   float2 [L][Mz][M]            (h, h)              at pef_hw2_offset floats
  //   float2 [L][Mz][(M-1)/2]      (h(2i), h(2i+1))    at pef_hwp_offset floats
  const float* hw;
  float* whitened;
};
__host__ __device__ inline size_t pef_hw2_offset(int L, int Mz, int M) {
  return (size_t(L) * Mz * M + 3) & ~size_t(3);
}
__host__ __device__ inline size_t pef_hwp_offset(int L, int Mz, int M) {
  return pef_hw2_offset(L, Mz, M) + 2 * size_t(L) * Mz * M;
}
__host__ __device__ inline size_t pef_table_floats(int L, int Mz, int M) {
  return pef_hwp_offset(L, Mz, M) + 2 * size_t(L) * Mz * ((M - 1) / 2);
}

struct RawSpecArgs {
  int H, W, M, Mz;
  const float* obs;
  float2* out;                  // [H*W][Mz][M][M]
};

// complex helpers
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ inline float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Output-tile width of the spectrum kernel for window M and temporal order Mz:
// the largest TW with TW + 2K <= 32 (one observer lane per input pixel of the
// row segment) and TW * (y-SDFT channels), rounded to warps, plus the observer
// warp within 384 threads (two CTAs per SM).
__host__ __device__ constexpr int spec_tile_w(int M, int Mz) {
  const int K = (M - 1) / 2, J = (Mz - 1) / 2;
  const int nchy = ((Mz % 2) == 0 ? 2 : 1) * (K + 1) + J * M;
  int tw = 32 - 2 * K;
  while (tw > 1 && ((tw * nchy + 31) / 32) * 32 + 32 > 384) --tw;
  return tw;
}

// Resident blocks per SM (and the SM count) of a kernel at a block size and
// dynamic shared-memory size, with that shared-memory size allowed on the
// kernel; the result is cached per (kernel, device, threads, smem), so the
// attribute call and the occupancy query run once rather than every frame.
struct ResidentShape { int nsm, per_sm; };
// carveout >= 0: also set the kernel's preferred shared-memory carveout (percent
// of the unified L1/shared storage), once per kernel and device.
cudaError_t resident_shape_of(const void* kernel, int threads, size_t smem, ResidentShape* out,
                              int carveout = -1);
template <typename F>
inline cudaError_t resident_shape(F* kernel, int threads, size_t smem, ResidentShape* out,
                                  int carveout = -1) {
  return resident_shape_of(reinterpret_cast<const void*>(kernel), threads, smem, out, carveout);
}

// launchers (return cudaError_t of the launch)
cudaError_t launch_spectrum(const SpecArgs& a, cudaStream_t st);
cudaError_t launch_autocorr(const AutocorrArgs& a, cudaStream_t st);
cudaError_t launch_pef(const PefArgs& a, cudaStream_t st);
cudaError_t pef_init_constants();          // once per device (also done by the first launch)
cudaError_t launch_raw_spectrum(const RawSpecArgs& a, cudaStream_t st);
bool spectrum_supported(int M, int Mz);
cudaError_t spectrum_init_constants();
int spectrum_threads(int M, int Mz);      // block size of the spectrum kernel
size_t spectrum_smem(int M, int Mz, bool f64 = false);   // its dynamic shared memory (bytes)
bool autocorr_tc_supported(int M);
cudaError_t launch_autocorr_convert(const AutocorrTcArgs& a, cudaStream_t st);
cudaError_t launch_autocorr_rerank(const AutocorrTcArgs& a, cudaStream_t st);
bool autocorr_tcsep_supported(int M, int L);
cudaError_t launch_autocorr_tcsep(const TcSepArgs& a, cudaStream_t st);
bool autocorr_tcd_supported(int M, int L);
// table: the constant F16 operand, tcd_table_rows(L) rows of tcd_table_ld(M) values
cudaError_t launch_autocorr_tcd(const TcDenseArgs& a, const void* table, cudaStream_t st);
int tcd_table_rows(int L);
int tcd_table_ld(int M);
void build_tcd_table(int M, int L, double vmax, double vstep, uint16_t* out);
// Stage-1 operand of the tensor-core separable search (2048 floats, see TcSepArgs)
void build_tcsep_operand(int M, int L, double vstep, float* out);

}  // namespace wh
