// Host runtime of the whitening stream and the C ABI declared in whiten.h.
//
// Owns the per-stream device state (observer bank, smoothed autocorrelation
// basis, outputs), builds the tables in double precision on the host, and
// enqueues the three kernels of one frame on the stream's CUDA stream:
//   spectrum (observer + SDFT + high-pass + Hann + power + A reduction + smoothing)
//   autocorrelation on the velocity grid + argmax
//   prediction-error filter + subtraction.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/whiten.h"
#include "common.cuh"
#include "stream_internal.h"
#include "tc_gemm.cuh"

namespace wh {
}  // namespace wh

using namespace wh;

static std::atomic<long long> g_launches{0};
static thread_local char g_err[512] = "";

static int set_cuda_err(cudaError_t e, const char* what) {
  std::snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return WH_ECUDA;
}
#define WH_CU(call)                                   \
  do {                                                \
    cudaError_t e__ = (call);                         \
    if (e__ != cudaSuccess) return set_cuda_err(e__, #call); \
  } while (0)

static const double kPi = 3.14159265358979323846;
// Row-bound widening of the tensor-core separable search per unit of a pixel's
// sum |Q sums|: TF32 operands (10 explicit mantissa bits, |B| <= 1) bound
// |T~ - T| by sqrt(2) 1.53 2^-10 per kx row, 4.23e-3 after the sum over kx.
static const float kTcSepWiden = 4.5e-3f;

char* wh_error_buffer() { return g_err; }
int wh_cuda_fail(cudaError_t e, const char* what) { return set_cuda_err(e, what); }
void wh_count_launches(long long n) { g_launches.fetch_add(n); }


// ---------------------------------------------------------------------------
static double dirichlet(int Wd, double w) {   // Eq. (3), limit value at integers
  double j = std::nearbyint(w), d = w - j;
  long long ji = (long long)j;
  double sgn = ((ji * (Wd - 1)) % 2 == 0) ? 1.0 : -1.0;
  if (std::fabs(d) < 1e-12) return sgn;
  return sgn * std::sin(kPi * Wd * d) / (Wd * std::sin(kPi * d));
}

static float2 cexpf2(double ph) { return make_float2(float(std::cos(ph)), float(std::sin(ph))); }

static void build_spec_tables(const wh_stream* s, SpecTables& tb, std::vector<int>& hg) {
  std::memset(&tb, 0, sizeof(tb));
  const int M = s->M, K = s->K, Mz = s->Mz;
  const int J = (Mz - 1) / 2;
  const bool even = (Mz % 2) == 0;
  const int npl = J + 1 + (even ? 1 : 0);
  tb.nplanes = npl;
  tb.nh = (M * M - 1) / 2;
  tb.nslot = 1 + 2 * J + (even ? 1 : 0);
  std::vector<int> base(npl);
  int c = 0;
  auto hann = [&](int m) { return 0.5 + 0.5 * std::cos(2.0 * kPi * (m - K) / M); };
  for (int p = 0; p < npl; ++p) {
    const bool real = (p == 0) || (even && p == npl - 1);
    base[p] = c;
    const int klo = real ? 0 : -K;
    for (int kx = klo; kx <= K; ++kx, ++c) {
      tb.ch_plane[c] = p;
      tb.ch_kx[c] = kx;
      for (int mx = 0; mx < M; ++mx) {
        // centred, Hann-windowed x-DFT weight
        const double ph = 2.0 * kPi * kx * (mx - K) / M;
        tb.xcoef[c][mx] = make_float2(float(hann(mx) * std::cos(ph)), float(hann(mx) * std::sin(ph)));
      }
    }
  }
  tb.nchy = c;
  for (int p = 0; p < npl; ++p, ++c) {   // box-sum channels for the high-pass correction
    tb.ch_plane[c] = p;
    tb.ch_kx[c] = 0;
    for (int mx = 0; mx < M; ++mx) tb.xcoef[c][mx] = make_float2(1.f, 0.f);
  }
  tb.nch = c;
  for (int i = 0; i < M; ++i) {
    const int k = i - K;
    tb.wres[i] = cexpf2(2.0 * kPi * k / M);
    tb.cphase[i] = cexpf2(-2.0 * kPi * k * K / M);
    tb.uncenter[i] = cexpf2(2.0 * kPi * k * K / M);
  }
  for (int p = 0; p < npl; ++p) {
    const int kz = p;   // the Nyquist plane p = Mz/2 rotates by e^{j pi} = -1
    tb.lam[p] = cexpf2(2.0 * kPi * kz / Mz);
    tb.cz[p] = float(std::cos(2.0 * kPi * kz / Mz));
    tb.sz[p] = float(std::sin(2.0 * kPi * kz / Mz));
  }
  tb.hann_z = cexpf2(-2.0 * kPi * ((Mz - 1) / 2.0) / Mz);
  // gather offsets (c*M + iy) of P for every h in {0} + half plane
  auto chan = [&](int p, int kx) {
    const bool real = (p == 0) || (even && p == npl - 1);
    return base[p] + (real ? kx : kx + K);
  };
  const int nslot = tb.nslot;
  hg.assign(size_t(tb.nh + 1) * nslot, 0);
  auto fill = [&](int hi, int hx, int hy) {
    int* g = &hg[size_t(hi) * nslot];
    g[0] = chan(0, hx) * M + (hy + K);
    for (int j = 1; j <= J; ++j) {
      g[j] = chan(j, hx) * M + (hy + K);
      g[J + j] = chan(j, -hx) * M + (-hy + K);
    }
    if (even) g[2 * J + 1] = chan(npl - 1, hx) * M + (hy + K);
  };
  fill(0, 0, 0);
  int hi = 1;
  for (int ky = 1; ky <= K; ++ky) fill(hi++, 0, ky);
  for (int kx = 1; kx <= K; ++kx)
    for (int ky = -K; ky <= K; ++ky) fill(hi++, kx, ky);
}

// Learned mode: MLP velocity where its confidence passes the threshold (rounded
// to the grid), the exact autocorrelation search for every other pixel.
// y: the network's output rows (vx, vy, confidence logit) with row pitch ldy.
__global__ void learned_select_kernel(const float* y, int ldy, int npix, float thr, float vmax, float vstep,
                                      int L, int* vidx, float* vx, float* vy, int* list, int* nlist) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const float* yp = y + size_t(p) * ldy;
    const float c = yp[2];
    const float conf = 1.f / (1.f + __expf(-c));
    if (conf >= thr) {
      int ix = __float2int_rn((yp[0] + vmax) / vstep), iy = __float2int_rn((yp[1] + vmax) / vstep);
      ix = ix < 0 ? 0 : (ix >= L ? L - 1 : ix);
      iy = iy < 0 ? 0 : (iy >= L ? L - 1 : iy);
      vidx[p] = iy * L + ix;
      vx[p] = -vmax + ix * vstep;
      vy[p] = -vmax + iy * vstep;
    } else {
      list[atomicAdd(nlist, 1)] = p;
    }
  }
}

__global__ void accumulate_count_kernel(const int* n, long long* total) { *total += *n; }

namespace wh {
int mlp_forward_on(wh_mlp* m, const void* x, int ldx, int n, float* y, int ldy, cudaStream_t st);
int mlp_n_in(const wh_mlp* m);
const float* mlp_output(const wh_mlp* m, int* ld);
}

static int learned_search(wh_stream* s) {
  const int npix = s->H * s->W;
  // on the search's stream: the network reads the features this frame's
  // spectrum kernel wrote and the selection below reads its output
  // (read in place from the network's padded output rows, no copy)
  int rc = wh::mlp_forward_on(s->mlp, s->d_feat, s->feat_ld, npix, nullptr, 0, s->st);
  if (rc != WH_OK) return rc;
  int ldy = 0;
  const float* y = wh::mlp_output(s->mlp, &ldy);
  WH_CU(cudaMemsetAsync(s->d_nlist, 0, sizeof(int), s->st));
  learned_select_kernel<<<148 * 8, 256, 0, s->st>>>(y, ldy, npix, s->conf_thr, float(s->vmax),
                                                    float(s->vstep), s->L, s->vidx, s->vx, s->vy,
                                                    s->d_list, s->d_nlist);
  WH_CU(cudaGetLastError());
  AutocorrArgs aa{};
  aa.H = s->H; aa.W = s->W; aa.M = s->M; aa.L = s->L; aa.kpad = s->kpad;
  aa.vmax = float(s->vmax); aa.vstep = float(s->vstep); aa.Astate = s->Astate;
  aa.vidx = s->vidx; aa.vx = s->vx; aa.vy = s->vy; aa.rs_out = nullptr;
  aa.tab_y = s->d_taby; aa.tab_x = s->d_tabx; aa.pix_list = s->d_list; aa.n_list = s->d_nlist;
  cudaError_t e = launch_autocorr(aa, s->st);
  if (e != cudaSuccess) return set_cuda_err(e, "autocorrelation kernel (fallback pixels)");
  accumulate_count_kernel<<<1, 1, 0, s->st>>>(s->d_nlist, s->d_nfb_total);
  WH_CU(cudaGetLastError());
  s->mlp_frames += 1;
  return WH_OK;
}

static void fill_tc_args(const wh_stream* s, AutocorrTcArgs& ta) {
  ta.H = s->H; ta.W = s->W; ta.M = s->M; ta.L = s->L; ta.kpad = s->kpad; ta.kg = s->kg;
  ta.ntile = s->ntile; ta.ncand = 8; ta.ovf_group = 8; ta.mode = s->tc_mode; ta.bf16 = s->tc_bf16;
  ta.vmax = float(s->vmax); ta.vstep = float(s->vstep); ta.Astate = s->Astate;
  ta.a16 = s->d_a16; ta.l1 = s->d_l1; ta.cand_val = s->d_cval; ta.cand_idx = s->d_cidx;
  ta.vidx = s->vidx; ta.vx = s->vx; ta.vy = s->vy; ta.tab_x = s->d_tabx; ta.n_fallback = s->d_nfb;
}

static void free_async(wh_stream* s) {
  wh_stream::Async* a = s->as;
  if (!a) return;
  if (a->in) cudaStreamSynchronize(a->in);
  if (a->out) cudaStreamSynchronize(a->out);
  // set 0 is the stream's own buffers (freed with the stream), set 1 was added
  s->frame = a->frame[0]; s->whitened = a->w[0]; s->vx = a->vx[0]; s->vy = a->vy[0];
  for (void* p : {(void*)a->frame[1], (void*)a->w[1], (void*)a->vx[1], (void*)a->vy[1]})
    if (p) cudaFree(p);
  for (int b = 0; b < 2; ++b)
    for (cudaEvent_t e : {a->ev_in[b], a->ev_comp[b], a->ev_out[b]})
      if (e) cudaEventDestroy(e);
  if (a->in) cudaStreamDestroy(a->in);
  if (a->out) cudaStreamDestroy(a->out);
  delete a;
  s->as = nullptr;
}

static void free_pipeline(wh_stream* s) {
  if (!s->pipeline) return;
  if (s->st_s) cudaStreamSynchronize(s->st_s);
  if (s->st_p) cudaStreamSynchronize(s->st_p);
  for (cudaEvent_t e : {s->ev_user, s->ev_spec, s->ev_join, s->ev_pef[0], s->ev_pef[1], s->ev_feat})
    if (e) cudaEventDestroy(e);
  if (s->st_s) cudaStreamDestroy(s->st_s);
  if (s->st_p) cudaStreamDestroy(s->st_p);
  if (s->Astate_alt) cudaFree(s->Astate_alt);
  s->st_s = s->st_p = nullptr;
  s->Astate_alt = nullptr;
}

static void free_stream(wh_stream* s) {
  if (!s) return;
  free_async(s);
  free_pipeline(s);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  void* ptrs[] = {s->obs[0], s->obs[1], s->Astate, s->frame, s->whitened, s->vx, s->vy, s->vidx,
                  s->d_spec, s->d_hgather, s->d_taby, s->d_tabx, s->d_hw, s->d_dump_win,
                  s->d_dump_pow, s->d_raw, s->d_rs, s->d_a16, s->d_l1, s->d_cval, s->d_cidx,
                  s->d_table, s->d_err, s->d_nfb, s->d_feat, s->d_fgather,
                  s->d_list, s->d_nlist, s->d_nfb_total, s->d_det, s->d_det_list, s->d_bop,
                  s->d_tcd_table, s->d_ccount, s->d_cand, s->d_tcd_counts};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete s;
}

// ---------------------------------------------------------------------------
extern "C" {

int wh_default_params(int window, int temporal_order, wh_params* p) {
  if (!p || window < 3 || (window % 2) == 0 || temporal_order < 2) return WH_EINVAL;
  p->band = int(std::lround(window / 3.0));
  if (p->band < 1) p->band = 1;
  p->delay_z = (temporal_order - 1) / 2;
  p->alpha = std::exp(-0.1);
  p->precision = WH_PREC_FP32;
  p->debug_dump = 0;
  p->pipeline = 0;
  return WH_OK;
}

// h * w limit (far beyond what fits in device memory with the per-pixel state)
constexpr long long kMaxPixels = 1LL << 30;

int wh_create_stream(int H, int W, int M, int Mz, wh_vgrid grid, const wh_params* opt,
                     void* cuda_stream, wh_stream** out) {
  if (!out) return WH_EINVAL;
  *out = nullptr;
  if (H < 1 || W < 1 || M < 3 || (M % 2) == 0 || M > kMaxM || Mz < 2 || Mz > kMaxMz) return WH_EINVAL;
  if ((long long)H * W > kMaxPixels) return WH_EINVAL;   // pixel counts stay 32-bit in the kernels
  if (!(grid.step > 0.f) || !(grid.vmax >= 0.f)) return WH_EINVAL;
  const double Ld = 2.0 * grid.vmax / grid.step + 1.0;
  const int L = int(std::lround(Ld));
  if (std::fabs(Ld - L) > 1e-4 || L < 1 || L > kMaxL) return WH_EINVAL;
  wh_params p;
  wh_default_params(M, Mz, &p);
  if (opt) {
    if (opt->band > 0) p.band = opt->band;
    if (opt->delay_z >= 0) p.delay_z = opt->delay_z;
    if (opt->alpha >= 0) p.alpha = opt->alpha;
    p.precision = opt->precision;
    p.debug_dump = opt->debug_dump;
    p.pipeline = opt->pipeline;
  }
  const int K = (M - 1) / 2;
  if (p.band > K || p.delay_z >= Mz || p.alpha >= 1.0) return WH_EINVAL;
  if (!spectrum_supported(M, Mz)) return WH_EUNSUP;
  const int pmode = p.precision & 3;
  if (p.precision &
      ~(3 | WH_PREC_CUDA_CORES | WH_PREC_TC_SHORTLIST | WH_PREC_TC_SEPARABLE | WH_PREC_SPEC_F64 | WH_PREC_TC_DENSE))
    return WH_EUNSUP;
  if (pmode == 3) return WH_EINVAL;
  if (pmode != 0 && !autocorr_tc_supported(M)) return WH_EUNSUP;

  wh_stream* s = new (std::nothrow) wh_stream();
  if (!s) return WH_ENOMEM;
  s->obs[0] = s->obs[1] = nullptr;
  s->Astate = s->frame = s->whitened = s->vx = s->vy = nullptr;
  s->vidx = nullptr; s->d_spec = nullptr; s->d_hgather = nullptr; s->d_taby = nullptr;
  s->d_tabx = nullptr; s->d_hw = nullptr; s->d_dump_win = nullptr; s->d_dump_pow = nullptr;
  s->d_raw = nullptr; s->d_rs = nullptr; s->prof = 0; s->ev_used = 0; s->t = 0; s->cur = 0;
  s->d_a16 = nullptr; s->d_l1 = nullptr; s->d_cval = nullptr; s->d_cidx = nullptr;
  s->d_table = nullptr; s->d_err = nullptr; s->d_nfb = nullptr;
  s->d_feat = nullptr; s->feat_ld = 0; s->feat_n = 0; s->feat_mode = 0; s->d_fgather = nullptr; s->mlp = nullptr;
  s->conf_thr = 0.8f;
  s->d_list = nullptr; s->d_nlist = nullptr; s->d_nfb_total = nullptr;
  s->mlp_frames = 0;
  s->as = nullptr;
  s->d_det = nullptr; s->det_bytes = 0; s->d_det_list = nullptr; s->det_list_cap = 0;
  s->d_bop = nullptr;
  s->d_tcd_table = nullptr; s->d_ccount = nullptr; s->d_cand = nullptr; s->d_tcd_counts = nullptr;
  s->spec_f64 = (p.precision & WH_PREC_SPEC_F64) ? 1 : 0;
  s->use_tcd = pmode == 0 && (p.precision & WH_PREC_TC_DENSE) &&
               !(p.precision & (WH_PREC_TC_SHORTLIST | WH_PREC_CUDA_CORES | WH_PREC_TC_SEPARABLE)) &&
               autocorr_tcd_supported(M, L);
  s->use_tcsep = pmode == 0 && !(p.precision & (WH_PREC_TC_SHORTLIST | WH_PREC_CUDA_CORES)) &&
                 (p.precision & WH_PREC_TC_SEPARABLE) && autocorr_tcsep_supported(M, L);
  s->tc_mode = pmode == 0 ? 0 : 1;
  s->tc_bf16 = pmode == 2 ? 1 : 0;
  s->use_tc = (pmode != 0) || ((p.precision & WH_PREC_TC_SHORTLIST) && autocorr_tc_supported(M));
  s->kg = ((M * M) + 7) & ~7;
  s->ntile = (L * L + 127) / 128;
  s->H = H; s->W = W; s->M = M; s->K = K; s->Mz = Mz; s->B = p.band; s->mpz = p.delay_z;
  s->L = L; s->precision = p.precision; s->debug = p.debug_dump;
  s->alpha = p.alpha; s->vmax = grid.vmax; s->vstep = grid.step;
  s->st = (cudaStream_t)cuda_stream;
  s->tw = spec_tile_w(M, Mz);
  s->th = 64;
  s->kpad = ((M * M) + 3) & ~3;
  cudaGetDevice(&s->device);

  const size_t npix = size_t(H) * W;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(ptr, bytes);
  };
  alloc((void**)&s->obs[0], sizeof(float) * npix * Mz);
  alloc((void**)&s->obs[1], sizeof(float) * npix * Mz);
  alloc((void**)&s->Astate, sizeof(float) * npix * s->kpad);
  s->pipeline = p.pipeline ? 1 : 0;
  if (s->pipeline) {
    alloc((void**)&s->Astate_alt, sizeof(float) * npix * s->kpad);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st_s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st_p, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&s->ev_user, &s->ev_spec, &s->ev_join, &s->ev_pef[0], &s->ev_pef[1], &s->ev_feat})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  }
  alloc((void**)&s->frame, sizeof(float) * npix);
  alloc((void**)&s->whitened, sizeof(float) * npix);
  alloc((void**)&s->vx, sizeof(float) * npix);
  alloc((void**)&s->vy, sizeof(float) * npix);
  alloc((void**)&s->vidx, sizeof(int) * npix);
  alloc((void**)&s->d_spec, sizeof(SpecTables));
  alloc((void**)&s->d_err, sizeof(int));
  if (s->debug) {
    alloc((void**)&s->d_dump_win, sizeof(float2) * npix * M * M * Mz);
    alloc((void**)&s->d_dump_pow, sizeof(float) * npix * M * M * Mz);
  }
  if (e != cudaSuccess) {
    int rc = (e == cudaErrorMemoryAllocation) ? WH_ENOMEM : set_cuda_err(e, "cudaMalloc");
    free_stream(s);
    return rc;
  }
  e = spectrum_init_constants();
  if (e == cudaSuccess) e = pef_init_constants();
  if (e != cudaSuccess) {
    int rc = set_cuda_err(e, "cudaMemcpyToSymbol");
    free_stream(s);
    return rc;
  }
  // tables
  SpecTables tb;
  std::vector<int> hg;
  build_spec_tables(s, tb, hg);
  std::vector<float2> taby(size_t(L) * M), tabx(size_t(L) * (K + 1));
  for (int g = 0; g < L; ++g) {
    const double l = -s->vmax + g * s->vstep;
    for (int iy = 0; iy < M; ++iy) taby[size_t(g) * M + iy] = cexpf2(2.0 * kPi * (iy - K) * l / M);
    for (int kx = 0; kx <= K; ++kx) tabx[size_t(g) * (K + 1) + kx] = cexpf2(2.0 * kPi * kx * l / M);
  }
  const int Wb = 2 * s->B + 1;
  const double hscale = std::sqrt(double(Wb) * Wb / (double(M) * M * Mz));
  std::vector<float> hw(pef_table_floats(L, Mz, M), 0.f);
  float* hw2 = hw.data() + pef_hw2_offset(L, Mz, M);
  float* hwp = hw.data() + pef_hwp_offset(L, Mz, M);
  for (int g = 0; g < L; ++g) {
    const double v = -s->vmax + g * s->vstep;
    for (int m = 0; m < Mz; ++m) {
      const size_t r = size_t(g) * Mz + m;
      for (int j = 0; j < M; ++j) {
        const int d = j - K;
        const float h = float(hscale * dirichlet(Wb, (d + v * (m - s->mpz)) / M));
        hw[r * M + j] = h;
        hw2[2 * (r * M + j)] = h;
        hw2[2 * (r * M + j) + 1] = h;
      }
      for (int i = 0; i < K; ++i) {
        hwp[2 * (r * K + i)] = hw[r * M + 2 * i];
        hwp[2 * (r * K + i) + 1] = hw[r * M + 2 * i + 1];
      }
    }
  }
  alloc((void**)&s->d_hgather, sizeof(int) * hg.size());
  alloc((void**)&s->d_taby, sizeof(float2) * taby.size());
  alloc((void**)&s->d_tabx, sizeof(float2) * tabx.size());
  alloc((void**)&s->d_hw, sizeof(float) * hw.size());
  if (e != cudaSuccess) {
    int rc = (e == cudaErrorMemoryAllocation) ? WH_ENOMEM : set_cuda_err(e, "cudaMalloc");
    free_stream(s);
    return rc;
  }
  cudaError_t c1 = cudaMemcpy(s->d_spec, &tb, sizeof(tb), cudaMemcpyHostToDevice);
  if (c1 == cudaSuccess) c1 = cudaMemset(s->d_err, 0, sizeof(int));
  cudaError_t c2 = cudaMemcpy(s->d_hgather, hg.data(), sizeof(int) * hg.size(), cudaMemcpyHostToDevice);
  cudaError_t c3 = cudaMemcpy(s->d_taby, taby.data(), sizeof(float2) * taby.size(), cudaMemcpyHostToDevice);
  cudaError_t c4 = cudaMemcpy(s->d_tabx, tabx.data(), sizeof(float2) * tabx.size(), cudaMemcpyHostToDevice);
  cudaError_t c5 = cudaMemcpy(s->d_hw, hw.data(), sizeof(float) * hw.size(), cudaMemcpyHostToDevice);
  for (cudaError_t c : {c1, c2, c3, c4, c5})
    if (c != cudaSuccess) {
      int rc = set_cuda_err(c, "cudaMemcpy(tables)");
      free_stream(s);
      return rc;
    }
  if (s->use_tcd) {
    const size_t nt = size_t(tcd_table_rows(L)) * tcd_table_ld(M);
    std::vector<uint16_t> tab(nt);
    build_tcd_table(M, L, s->vmax, s->vstep, tab.data());
    alloc((void**)&s->d_tcd_table, sizeof(uint16_t) * nt);
    alloc((void**)&s->d_ccount, sizeof(int) * npix);
    alloc((void**)&s->d_cand, sizeof(int) * 8 * npix);
    alloc((void**)&s->d_tcd_counts, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(s->d_tcd_table, tab.data(), sizeof(uint16_t) * nt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->d_tcd_counts, 0, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
      int rc = (e == cudaErrorMemoryAllocation) ? WH_ENOMEM : set_cuda_err(e, "tensor-core search operand");
      free_stream(s);
      return rc;
    }
  }
  if (s->use_tcsep) {
    std::vector<float> bop(2048);
    build_tcsep_operand(M, L, s->vstep, bop.data());
    alloc((void**)&s->d_bop, sizeof(float) * bop.size());
    if (e == cudaSuccess) e = cudaMemcpy(s->d_bop, bop.data(), sizeof(float) * bop.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      int rc = (e == cudaErrorMemoryAllocation) ? WH_ENOMEM : set_cuda_err(e, "tensor-core search operand");
      free_stream(s);
      return rc;
    }
  }
  if (s->use_tc) {
    alloc((void**)&s->d_a16, 2 * npix * s->kg);
    alloc((void**)&s->d_l1, sizeof(float) * npix);
    const size_t nc = size_t(s->ntile * 4 > 8 ? s->ntile * 4 : 8);
    alloc((void**)&s->d_cval, sizeof(float) * npix * nc);
    alloc((void**)&s->d_cidx, sizeof(int) * npix * nc);
    alloc((void**)&s->d_table, 2 * size_t(s->ntile) * 128 * s->kg);
    alloc((void**)&s->d_nfb, sizeof(int));
    if (e != cudaSuccess) {
      int rc = (e == cudaErrorMemoryAllocation) ? WH_ENOMEM : set_cuda_err(e, "cudaMalloc");
      free_stream(s);
      return rc;
    }
    // B(l, k) in the state's basis: [1, 2 cos a_h(l), -2 sin a_h(l)], a_h(l) =
    // 2pi (hx lx + hy ly)/M; rows l >= L^2 are zero.
    const int nh = (M * M - 1) / 2, Np = s->ntile * 128;
    std::vector<float> tb32(size_t(Np) * s->kg, 0.f);
    std::vector<int> hx(nh + 1), hyv(nh + 1);
    int hi = 1;
    for (int ky = 1; ky <= K; ++ky) { hx[hi] = 0; hyv[hi] = ky; ++hi; }
    for (int kx = 1; kx <= K; ++kx)
      for (int ky = -K; ky <= K; ++ky) { hx[hi] = kx; hyv[hi] = ky; ++hi; }
    for (int g = 0; g < L * L; ++g) {
      const double lx = -s->vmax + (g % L) * s->vstep, ly = -s->vmax + (g / L) * s->vstep;
      float* row = &tb32[size_t(g) * s->kg];
      row[0] = 1.f;
      for (int h = 1; h <= nh; ++h) {
        const double ph = 2.0 * kPi * (hx[h] * lx + hyv[h] * ly) / M;
        row[h] = float(2.0 * std::cos(ph));
        row[nh + h] = float(-2.0 * std::sin(ph));
      }
    }
    std::vector<uint16_t> tb16(tb32.size());
    for (size_t i = 0; i < tb32.size(); ++i) {
      if (s->tc_bf16) {
        __nv_bfloat16 b = __float2bfloat16(tb32[i]);
        std::memcpy(&tb16[i], &b, 2);
      } else {
        __half h = __float2half(tb32[i]);
        std::memcpy(&tb16[i], &h, 2);
      }
    }
    cudaError_t c6 = cudaMemcpy(s->d_table, tb16.data(), 2 * tb16.size(), cudaMemcpyHostToDevice);
    cudaError_t c7 = cudaSuccess;
    cudaError_t c8 = cudaMemset(s->d_nfb, 0, sizeof(int));
    cudaError_t c9 = cudaMemset(s->d_a16, 0, 2 * npix * s->kg);
    for (cudaError_t c : {c6, c7, c8, c9})
      if (c != cudaSuccess) {
        int rc = set_cuda_err(c, "tensor-core tables");
        free_stream(s);
        return rc;
      }
  }
  // the spectrum kernel's shared memory must fit one CTA
  if (spectrum_threads(M, Mz) <= 0 || spectrum_smem(M, Mz, s->spec_f64 != 0) > 227 * 1024) {
    free_stream(s);
    return WH_EUNSUP;
  }
  int rc = wh_reset_stream(s);
  if (rc != WH_OK) {
    free_stream(s);
    return rc;
  }
  *out = s;
  return WH_OK;
}

}  // extern "C"

// Order the caller's stream after every frame-pipeline kernel enqueued so far.
static int join_pipeline(wh_stream* s) { return wh_join_pipeline(s); }
int wh_join_pipeline(wh_stream* s) {
  if (!s->pipeline || !s->pipe_work) return WH_OK;
  WH_CU(cudaEventRecord(s->ev_join, s->st_s));
  WH_CU(cudaStreamWaitEvent(s->st, s->ev_join, 0));
  WH_CU(cudaEventRecord(s->ev_join, s->st_p));
  WH_CU(cudaStreamWaitEvent(s->st, s->ev_join, 0));
  return WH_OK;
}

extern "C" {

int wh_reset_stream(wh_stream* s) {
  if (!s) return WH_EINVAL;
  const size_t npix = size_t(s->H) * s->W;
  if (s->as) {                // asynchronous copies may still read the buffers reset below
    if (s->as->in) WH_CU(cudaStreamSynchronize(s->as->in));
    if (s->as->out) WH_CU(cudaStreamSynchronize(s->as->out));
  }
  if (s->pipeline) {
    WH_CU(cudaStreamSynchronize(s->st_s));
    WH_CU(cudaStreamSynchronize(s->st_p));
    WH_CU(cudaMemsetAsync(s->Astate_alt, 0, sizeof(float) * npix * s->kpad, s->st));
    s->pef_used[0] = s->pef_used[1] = 0;
    s->pipe_work = 0;
    s->user_sync = 1;         // the next push orders the internal streams after these memsets
  }
  WH_CU(cudaMemsetAsync(s->obs[0], 0, sizeof(float) * npix * s->Mz, s->st));
  WH_CU(cudaMemsetAsync(s->obs[1], 0, sizeof(float) * npix * s->Mz, s->st));
  WH_CU(cudaMemsetAsync(s->Astate, 0, sizeof(float) * npix * s->kpad, s->st));
  WH_CU(cudaMemsetAsync(s->whitened, 0, sizeof(float) * npix, s->st));
  WH_CU(cudaMemsetAsync(s->vidx, 0, sizeof(int) * npix, s->st));
  s->t = 0;
  s->cur = 0;
  return WH_OK;
}

static int check_device_status(wh_stream* s);

// The three kernels of one frame, reading the device frame src and writing
// s->whitened / s->vx / s->vy / s->vidx.  Without the frame pipeline all run on
// s->st; with it the spectrum kernel runs on st_s (after the PEF of frame t-2,
// whose observer and smoothed-state buffers it reuses) and the search and PEF
// on st_p (after this frame's spectrum).  wait_spec / wait_search: optional
// events the spectrum / the search must follow.
static int push_kernels(wh_stream* s, const float* src, cudaEvent_t wait_spec = nullptr,
                        cudaEvent_t wait_search = nullptr) {
  const cudaStream_t user = s->st;
  const cudaStream_t ss = s->pipeline ? s->st_s : s->st;
  const cudaStream_t sp = s->pipeline ? s->st_p : s->st;
  const int k = int(s->t & 1);
  if (s->pipeline && s->user_sync) {
    // the state was reset on the caller's stream: the internal streams start after it
    WH_CU(cudaEventRecord(s->ev_user, user));
    WH_CU(cudaStreamWaitEvent(ss, s->ev_user, 0));
    WH_CU(cudaStreamWaitEvent(sp, s->ev_user, 0));
    s->user_sync = 0;
  }
  if (s->pipeline && s->pef_used[k]) WH_CU(cudaStreamWaitEvent(ss, s->ev_pef[k], 0));
  // one feature buffer: with features on, the spectrum of this frame waits
  // until the previous frame's learned search has read it (no overlap there)
  if (s->pipeline && s->d_feat) WH_CU(cudaStreamWaitEvent(ss, s->ev_feat, 0));
  if (wait_spec) WH_CU(cudaStreamWaitEvent(ss, wait_spec, 0));
  cudaEvent_t* ev = nullptr;
  if (s->prof && s->ev_used + 4 <= 4 * 65536) {
    while (s->ev.size() < s->ev_used + 4) {
      cudaEvent_t e;
      WH_CU(cudaEventCreate(&e));
      s->ev.push_back(e);
    }
    ev = &s->ev[s->ev_used];
    s->ev_used += 4;
  }
  if (ev) WH_CU(cudaEventRecord(ev[0], ss));
  SpecArgs sa{};
  sa.H = s->H; sa.W = s->W; sa.M = s->M; sa.Mz = s->Mz; sa.tw = s->tw; sa.th = s->th;
  sa.kpad = s->kpad; sa.alpha = float(s->alpha); sa.frame = src;
  sa.obs_old = s->obs[s->cur]; sa.obs_new = s->obs[1 - s->cur]; sa.Astate = s->Astate;
  sa.Astate_out = s->pipeline ? s->Astate_alt : nullptr;
  sa.tables = s->d_spec; sa.hgather = s->d_hgather;
  sa.dump_win = s->d_dump_win; sa.dump_pow = s->d_dump_pow;
  sa.feat = s->d_feat; sa.feat_ld = s->feat_ld; sa.feat_n = s->feat_n; sa.feat_gather = s->d_fgather;
  sa.err = s->d_err;
  sa.f64 = s->spec_f64;
  cudaError_t e = launch_spectrum(sa, ss);
  if (e != cudaSuccess) return set_cuda_err(e, "spectrum kernel");
  if (ev) WH_CU(cudaEventRecord(ev[1], ss));
  if (s->pipeline) {
    std::swap(s->Astate, s->Astate_alt);      // the frame's smoothed state
    WH_CU(cudaEventRecord(s->ev_spec, ss));
    WH_CU(cudaStreamWaitEvent(sp, s->ev_spec, 0));
  }
  if (wait_search) WH_CU(cudaStreamWaitEvent(sp, wait_search, 0));
  s->st = sp;                                 // the search helpers enqueue on s->st
  int nlaunch = 3;
  int rc = WH_OK;
  if (s->mlp) {
    rc = learned_search(s);
    nlaunch = 4;
  } else if (s->use_tc) {
    AutocorrTcArgs ta{};
    fill_tc_args(s, ta);
    e = launch_autocorr_convert(ta, sp);
    if (e != cudaSuccess) rc = set_cuda_err(e, "autocorrelation convert kernel");
    if (rc == WH_OK) {
      e = tc_autocorr_shortlist(s->d_a16, s->kg, s->d_table, s->kg, s->H * s->W, s->M * s->M, s->ntile,
                                s->L * s->L, s->tc_bf16 != 0, s->tc_mode == 0 ? s->d_l1 : nullptr,
                                s->d_cval, s->d_cidx, s->d_err, sp);
      if (e != cudaSuccess) rc = set_cuda_err(e, "tensor-core autocorrelation");
    }
    if (rc == WH_OK && (e = launch_autocorr_rerank(ta, sp)) != cudaSuccess)
      rc = set_cuda_err(e, "autocorrelation re-rank kernel");
    nlaunch = 5;
  } else if (s->use_tcd) {
    TcDenseArgs ta{};
    ta.npix = s->H * s->W; ta.M = s->M; ta.L = s->L; ta.kpad = s->kpad;
    ta.vmax = float(s->vmax); ta.vstep = float(s->vstep);
    ta.Astate = s->Astate; ta.vidx = s->vidx; ta.vx = s->vx; ta.vy = s->vy;
    ta.tab_x = s->d_tabx; ta.ccount = s->d_ccount; ta.cand = s->d_cand; ta.counts = s->d_tcd_counts;
    ta.err = s->d_err;
    if ((e = launch_autocorr_tcd(ta, s->d_tcd_table, sp)) != cudaSuccess)
      rc = set_cuda_err(e, "tensor-core search kernel");
  } else if (s->use_tcsep) {
    TcSepArgs ta{};
    ta.npix = s->H * s->W; ta.M = s->M; ta.L = s->L; ta.kpad = s->kpad;
    ta.vmax = float(s->vmax); ta.vstep = float(s->vstep); ta.wcoef = kTcSepWiden;
    ta.Astate = s->Astate; ta.vidx = s->vidx; ta.vx = s->vx; ta.vy = s->vy;
    ta.bop = s->d_bop; ta.tab_x = s->d_tabx; ta.err = s->d_err;
    if ((e = launch_autocorr_tcsep(ta, sp)) != cudaSuccess) rc = set_cuda_err(e, "tensor-core search kernel");
  } else {
    AutocorrArgs aa{};
    aa.H = s->H; aa.W = s->W; aa.M = s->M; aa.L = s->L; aa.kpad = s->kpad;
    aa.vmax = float(s->vmax); aa.vstep = float(s->vstep); aa.Astate = s->Astate;
    aa.vidx = s->vidx; aa.vx = s->vx; aa.vy = s->vy; aa.rs_out = nullptr;
    aa.tab_y = s->d_taby; aa.tab_x = s->d_tabx; aa.pix_list = nullptr; aa.n_list = nullptr;
    if ((e = launch_autocorr(aa, sp)) != cudaSuccess) rc = set_cuda_err(e, "autocorrelation kernel");
  }
  if (rc == WH_OK && s->pipeline && s->d_feat && (e = cudaEventRecord(s->ev_feat, sp)) != cudaSuccess)
    rc = set_cuda_err(e, "cudaEventRecord");
  if (rc == WH_OK && ev && (e = cudaEventRecord(ev[2], sp)) != cudaSuccess) rc = set_cuda_err(e, "cudaEventRecord");
  if (rc == WH_OK) {
    PefArgs pa{};
    pa.H = s->H; pa.W = s->W; pa.M = s->M; pa.Mz = s->Mz; pa.L = s->L; pa.mpz = s->mpz;
    pa.obs = s->obs[1 - s->cur]; pa.vidx = s->vidx; pa.hw = s->d_hw; pa.whitened = s->whitened;
    if ((e = launch_pef(pa, sp)) != cudaSuccess) rc = set_cuda_err(e, "PEF kernel");
  }
  if (rc == WH_OK && ev && (e = cudaEventRecord(ev[3], sp)) != cudaSuccess) rc = set_cuda_err(e, "cudaEventRecord");
  if (rc == WH_OK && s->pipeline) {
    if ((e = cudaEventRecord(s->ev_pef[k], sp)) != cudaSuccess) rc = set_cuda_err(e, "cudaEventRecord");
    s->pef_used[k] = 1;
    s->pipe_work = 1;
  }
  s->st = user;
  if (rc != WH_OK) return rc;
  g_launches.fetch_add(nlaunch);
  s->cur = 1 - s->cur;
  s->t += 1;
  return WH_OK;
}

int wh_push_frame(wh_stream* s, const float* frame, int is_device) {
  if (!s || !frame) return WH_EINVAL;
  const size_t npix = size_t(s->H) * s->W;
  const float* src = frame;
  const cudaStream_t ss = s->pipeline ? s->st_s : s->st;
  const cudaStream_t sp = s->pipeline ? s->st_p : s->st;
  if (s->as) {   // the buffers in use may still be read by an asynchronous output copy
    for (int b = 0; b < 2; ++b)
      if (s->as->used[b]) {
        WH_CU(cudaStreamWaitEvent(ss, s->as->ev_out[b], 0));
        WH_CU(cudaStreamWaitEvent(sp, s->as->ev_out[b], 0));
      }
  }
  cudaEvent_t wait_spec = nullptr;
  if (!is_device) {
    WH_CU(cudaMemcpyAsync(s->frame, frame, sizeof(float) * npix, cudaMemcpyHostToDevice, ss));
    src = s->frame;
  } else if (s->pipeline) {      // a device frame is ready in the caller's stream order
    WH_CU(cudaEventRecord(s->ev_user, s->st));
    wait_spec = s->ev_user;
  }
  return push_kernels(s, src, wait_spec);
}

static int init_async(wh_stream* s) {
  if (s->as) return WH_OK;
  wh_stream::Async* a = new wh_stream::Async{};
  s->as = a;
  const size_t bytes = sizeof(float) * size_t(s->H) * s->W;
  a->frame[0] = s->frame; a->w[0] = s->whitened; a->vx[0] = s->vx; a->vy[0] = s->vy;
  cudaError_t e = cudaSuccess;
  for (float** p : {&a->frame[1], &a->w[1], &a->vx[1], &a->vy[1]})
    if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(a->w[1], 0, bytes, s->st);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a->in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a->out, cudaStreamNonBlocking);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    for (cudaEvent_t* ev : {&a->ev_in[b], &a->ev_comp[b], &a->ev_out[b]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    free_async(s);
    return e == cudaErrorMemoryAllocation ? WH_ENOMEM : wh_cuda_fail(e, "asynchronous push set-up");
  }
  return WH_OK;
}

int wh_push_frame_async(wh_stream* s, const float* frame_host, float* whitened_host, float* vx_host,
                        float* vy_host, long long* frame_index) {
  if (!s || !frame_host) return WH_EINVAL;
  int rc = init_async(s);
  if (rc != WH_OK) return rc;
  wh_stream::Async* a = s->as;
  const int b = a->par;
  const size_t bytes = sizeof(float) * size_t(s->H) * s->W;
  // input copy: the set's frame buffer was last read by the kernels of the
  // push before the previous one
  if (a->used[b]) WH_CU(cudaStreamWaitEvent(a->in, a->ev_comp[b], 0));
  WH_CU(cudaMemcpyAsync(a->frame[b], frame_host, bytes, cudaMemcpyHostToDevice, a->in));
  WH_CU(cudaEventRecord(a->ev_in[b], a->in));
  // kernels: after the input copy, and after the set's previous outputs were copied out
  s->frame = a->frame[b]; s->whitened = a->w[b]; s->vx = a->vx[b]; s->vy = a->vy[b];
  rc = push_kernels(s, a->frame[b], a->ev_in[b], a->used[b] ? a->ev_out[b] : nullptr);
  if (rc != WH_OK) return rc;
  WH_CU(cudaEventRecord(a->ev_comp[b], s->pipeline ? s->st_p : s->st));
  // output copies
  WH_CU(cudaStreamWaitEvent(a->out, a->ev_comp[b], 0));
  if (whitened_host) WH_CU(cudaMemcpyAsync(whitened_host, a->w[b], bytes, cudaMemcpyDeviceToHost, a->out));
  if (vx_host) WH_CU(cudaMemcpyAsync(vx_host, a->vx[b], bytes, cudaMemcpyDeviceToHost, a->out));
  if (vy_host) WH_CU(cudaMemcpyAsync(vy_host, a->vy[b], bytes, cudaMemcpyDeviceToHost, a->out));
  WH_CU(cudaEventRecord(a->ev_out[b], a->out));
  a->used[b] = 1;
  a->frame_of[b] = s->t - 1;
  a->par = 1 - b;
  if (frame_index) *frame_index = s->t - 1;
  return WH_OK;
}

int wh_stream_selftest_status(wh_stream* s, int code) {
  if (!s || code < 0) return WH_EINVAL;
  WH_CU(cudaMemcpyAsync(s->d_err, &code, sizeof(int), cudaMemcpyHostToDevice, s->st));
  WH_CU(cudaStreamSynchronize(s->st));
  return WH_OK;
}

int wh_stream_join(wh_stream* s) {
  if (!s) return WH_EINVAL;
  return join_pipeline(s);
}

int wh_stream_sync(wh_stream* s) {
  if (!s) return WH_EINVAL;
  if (s->pipeline) {
    WH_CU(cudaStreamSynchronize(s->st_s));
    WH_CU(cudaStreamSynchronize(s->st_p));
  }
  WH_CU(cudaStreamSynchronize(s->st));
  if (s->as) {
    WH_CU(cudaStreamSynchronize(s->as->in));
    WH_CU(cudaStreamSynchronize(s->as->out));
  }
  return check_device_status(s);
}

int wh_stream_query_frame(wh_stream* s, long long frame_index, int wait) {
  if (!s || frame_index < 0 || frame_index >= s->t) return WH_EINVAL;
  wh_stream::Async* a = s->as;
  if (!a) return WH_OK;                       // no asynchronous push made
  // output copies run in order on one stream: the oldest tracked push at or
  // after frame_index completes after it
  cudaEvent_t ev = nullptr;
  long long best = 0;
  for (int b = 0; b < 2; ++b)
    if (a->used[b] && a->frame_of[b] >= frame_index && (ev == nullptr || a->frame_of[b] < best)) {
      best = a->frame_of[b];
      ev = a->ev_out[b];
    }
  if (!ev) return WH_OK;                      // pushed synchronously
  if (wait) {
    WH_CU(cudaEventSynchronize(ev));
    return check_device_status(s);
  }
  const cudaError_t q = cudaEventQuery(ev);
  if (q == cudaErrorNotReady) return WH_ENOTREADY;
  if (q != cudaSuccess) return wh_cuda_fail(q, "cudaEventQuery");
  return WH_OK;
}

// After a synchronisation: the device status word is nonzero if a bounded
// wait inside one of this stream's kernels gave up (the results of that frame
// are not valid); reported once as WH_ETIMEOUT.
static int check_device_status(wh_stream* s) {
  int h = 0;
  WH_CU(cudaMemcpy(&h, s->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h != 0) {
    cudaMemset(s->d_err, 0, sizeof(int));
    std::snprintf(wh_error_buffer(), 512, "a bounded device-side wait gave up (code %d)", h);
    return WH_ETIMEOUT;
  }
  return WH_OK;
}

static int copy_out(wh_stream* s, void* dst, const void* src, size_t bytes, int is_device) {
  if (is_device) {
    WH_CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, s->st));
  } else {
    WH_CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->st));
    WH_CU(cudaStreamSynchronize(s->st));
    return check_device_status(s);
  }
  return WH_OK;
}

int wh_read_whitened(wh_stream* s, float* out, int is_device, long long* frame_index) {
  if (!s || !out) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  if (s->t < s->mpz + 1) return WH_ENOTREADY;
  if (frame_index) *frame_index = s->t - 1 - s->mpz;
  return copy_out(s, out, s->whitened, sizeof(float) * size_t(s->H) * s->W, is_device);
}

int wh_read_velocity(wh_stream* s, float* vx, float* vy, int* vidx, int is_device,
                     long long* frame_index) {
  if (!s) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  if (s->t < 1) return WH_ENOTREADY;
  if (frame_index) *frame_index = s->t - 1;
  const size_t n = size_t(s->H) * s->W;
  int rc = WH_OK;
  if (vx && (rc = copy_out(s, vx, s->vx, sizeof(float) * n, is_device)) != WH_OK) return rc;
  if (vy && (rc = copy_out(s, vy, s->vy, sizeof(float) * n, is_device)) != WH_OK) return rc;
  if (vidx && (rc = copy_out(s, vidx, s->vidx, sizeof(int) * n, is_device)) != WH_OK) return rc;
  return WH_OK;
}

int wh_read_spectrum(wh_stream* s, int kind, void* out, int is_device) {
  if (!s || !out) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  if (s->t < 1) return WH_ENOTREADY;
  const size_t nb = size_t(s->H) * s->W * s->M * s->M * s->Mz;
  if (kind == WH_SPEC_RAW) {
    if (!s->d_raw) WH_CU(cudaMalloc((void**)&s->d_raw, sizeof(float2) * nb));
    RawSpecArgs ra{};
    ra.H = s->H; ra.W = s->W; ra.M = s->M; ra.Mz = s->Mz; ra.obs = s->obs[s->cur]; ra.out = s->d_raw;
    cudaError_t e = launch_raw_spectrum(ra, s->st);
    if (e != cudaSuccess) return set_cuda_err(e, "raw spectrum kernel");
    g_launches.fetch_add(1);
    return copy_out(s, out, s->d_raw, sizeof(float2) * nb, is_device);
  }
  if (!s->debug) return WH_EINVAL;
  if (kind == WH_SPEC_WINDOWED) return copy_out(s, out, s->d_dump_win, sizeof(float2) * nb, is_device);
  if (kind == WH_SPEC_POWER) return copy_out(s, out, s->d_dump_pow, sizeof(float) * nb, is_device);
  return WH_EINVAL;
}

int wh_read_autocorr(wh_stream* s, float* out, int is_device) {
  if (!s || !out) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  if (s->t < 1) return WH_ENOTREADY;
  const size_t n = size_t(s->H) * s->W * s->L * s->L;
  if (!s->d_rs) {
    const cudaError_t me = cudaMalloc((void**)&s->d_rs, sizeof(float) * n);
    if (me != cudaSuccess) {
      s->d_rs = nullptr;
      return me == cudaErrorMemoryAllocation ? WH_ENOMEM : set_cuda_err(me, "cudaMalloc");
    }
  }
  AutocorrArgs aa{};
  aa.H = s->H; aa.W = s->W; aa.M = s->M; aa.L = s->L; aa.kpad = s->kpad;
  aa.vmax = float(s->vmax); aa.vstep = float(s->vstep); aa.Astate = s->Astate;
  aa.vidx = s->vidx; aa.vx = s->vx; aa.vy = s->vy; aa.rs_out = s->d_rs;
  aa.tab_y = s->d_taby; aa.tab_x = s->d_tabx; aa.pix_list = nullptr; aa.n_list = nullptr;
  cudaError_t e = launch_autocorr(aa, s->st);
  if (e != cudaSuccess) return set_cuda_err(e, "autocorrelation kernel");
  g_launches.fetch_add(1);
  return copy_out(s, out, s->d_rs, sizeof(float) * n, is_device);
}

int wh_stream_info(const wh_stream* s, int* grid_len, int* delay_z, int* band,
                   long long* frames_pushed) {
  if (!s) return WH_EINVAL;
  if (grid_len) *grid_len = s->L;
  if (delay_z) *delay_z = s->mpz;
  if (band) *band = s->B;
  if (frames_pushed) *frames_pushed = s->t;
  return WH_OK;
}

int wh_stream_stats(wh_stream* s, long long* fallback_pixels) {
  if (!s) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  int h = 0;
  WH_CU(cudaStreamSynchronize(s->st));
  if (s->d_nfb) WH_CU(cudaMemcpy(&h, s->d_nfb, sizeof(int), cudaMemcpyDeviceToHost));
  if (fallback_pixels) *fallback_pixels = h;
  return check_device_status(s);
}

int wh_stream_search_counts(wh_stream* s, long long* listed_pixels, long long* whole_grid_pixels) {
  if (!s) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  unsigned long long h[2] = {0ull, 0ull};
  WH_CU(cudaStreamSynchronize(s->st));
  if (s->d_tcd_counts) WH_CU(cudaMemcpy(h, s->d_tcd_counts, sizeof(h), cudaMemcpyDeviceToHost));
  if (listed_pixels) *listed_pixels = (long long)h[0];
  if (whole_grid_pixels) *whole_grid_pixels = (long long)h[1];
  return check_device_status(s);
}

int wh_stream_set_features(wh_stream* s, int enable) {
  if (!s || enable < 0 || enable > 2) return WH_EINVAL;
  if (s->d_feat && enable == s->feat_mode) return WH_OK;
  if (s->d_feat || !enable) {
    if (s->mlp) return WH_EINVAL;          // the learned mode reads the current layout
    if (s->d_feat) cudaFree(s->d_feat);
    if (s->d_fgather) cudaFree(s->d_fgather);
    s->d_feat = nullptr; s->d_fgather = nullptr; s->feat_ld = 0; s->feat_n = 0; s->feat_mode = 0;
    if (!enable) return WH_OK;
  }
  if (s->spec_f64) return WH_EUNSUP;     // the precision form writes no features
  const int M = s->M, K = s->K, Mz = s->Mz, J = (Mz - 1) / 2;
  const bool even = (Mz % 2) == 0;
  const int npl = J + 1 + (even ? 1 : 0), nb = M * M * Mz;
  std::vector<int> base(npl);
  int c = 0;
  for (int p = 0; p < npl; ++p) {
    const bool real = (p == 0) || (even && p == npl - 1);
    base[p] = c;
    c += real ? K + 1 : M;
  }
  auto chan = [&](int p, int kx) {
    const bool real = (p == 0) || (even && p == npl - 1);
    return base[p] + (real ? kx : kx + K);
  };
  // bin order [kz][ky][kx]: the bin itself if its plane/channel is stored, else its mirror
  std::vector<int> fg(nb);
  for (int iz = 0; iz < Mz; ++iz)
    for (int iy = 0; iy < M; ++iy)
      for (int ix = 0; ix < M; ++ix) {
        int kz = iz - J, ky = iy - K, kx = ix - K;
        const bool nyq = even && kz == Mz / 2;
        bool stored = kz >= 0 && kz <= (even ? Mz / 2 : J);
        const bool real = kz == 0 || nyq;
        if (stored && real && kx < 0) stored = false;
        if (!stored) {
          kx = -kx; ky = -ky;
          if (!nyq) kz = -kz;
        }
        fg[(iz * M + iy) * M + ix] = chan(kz, kx) * M + (ky + K);
      }
  if (enable == 2) {   // one feature per mirror pair (P(-k) = P(k)): bins not after their mirror
    std::vector<int> uniq;
    for (int iz = 0; iz < Mz; ++iz)
      for (int iy = 0; iy < M; ++iy)
        for (int ix = 0; ix < M; ++ix) {
          int kzm = -(iz - J);
          if (kzm < -J) kzm += Mz;
          const int b = (iz * M + iy) * M + ix, bm = ((kzm + J) * M + (2 * K - iy)) * M + (2 * K - ix);
          if (b <= bm) uniq.push_back(fg[b]);
        }
    fg.swap(uniq);
  }
  const int nf = int(fg.size());
  s->feat_n = nf;
  s->feat_mode = enable;
  s->feat_ld = (nf + 7) / 8 * 8;
  cudaError_t e = cudaMalloc(&s->d_feat, 2 * size_t(s->H) * s->W * s->feat_ld);
  if (e == cudaSuccess) e = cudaMalloc((void**)&s->d_fgather, sizeof(int) * nf);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_fgather, fg.data(), sizeof(int) * nf, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->d_feat, 0, 2 * size_t(s->H) * s->W * s->feat_ld);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? WH_ENOMEM : set_cuda_err(e, "features");
  return WH_OK;
}

int wh_read_features(wh_stream* s, void* out, int is_device, int* ld) {
  if (!s || !s->d_feat) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  if (ld) *ld = s->feat_ld;
  if (!out) return WH_OK;
  return copy_out(s, out, s->d_feat, 2 * size_t(s->H) * s->W * s->feat_ld, is_device);
}

int wh_stream_set_learned(wh_stream* s, wh_mlp* mlp, float conf_threshold) {
  if (!s) return WH_EINVAL;
  if (!mlp) {
    s->mlp = nullptr;
    return WH_OK;
  }
  // the feature layout the network takes: every bin, or one per mirror pair
  const int n_in = wh::mlp_n_in(mlp), nb = s->M * s->M * s->Mz;
  int mode = 0;
  if (n_in == nb) mode = 1;
  else if (n_in == (nb + 2 - (s->Mz % 2)) / 2) mode = 2;
  if (!mode) return WH_EINVAL;
  s->mlp = nullptr;
  int rc = wh_stream_set_features(s, mode);
  if (rc != WH_OK) return rc;
  const size_t npix = size_t(s->H) * s->W;
  cudaError_t e = cudaSuccess;
  if (!s->d_list) e = cudaMalloc((void**)&s->d_list, sizeof(int) * npix);
  if (e == cudaSuccess && !s->d_nlist) e = cudaMalloc((void**)&s->d_nlist, sizeof(int));
  if (e == cudaSuccess && !s->d_nfb_total) {
    e = cudaMalloc((void**)&s->d_nfb_total, sizeof(long long));
    if (e == cudaSuccess) e = cudaMemset(s->d_nfb_total, 0, sizeof(long long));
  }
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? WH_ENOMEM : set_cuda_err(e, "learned mode");
  s->mlp = mlp;
  s->conf_thr = conf_threshold;
  return WH_OK;
}

int wh_stream_learned_stats(wh_stream* s, long long* frames, long long* fallback_pixels) {
  if (!s) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  long long h = 0;
  if (s->d_nfb_total) {
    WH_CU(cudaMemcpyAsync(&h, s->d_nfb_total, sizeof(long long), cudaMemcpyDeviceToHost, s->st));
    WH_CU(cudaStreamSynchronize(s->st));
  }
  if (frames) *frames = s->mlp_frames;
  if (fallback_pixels) *fallback_pixels = h;
  return WH_OK;
}

int wh_output_pointers(wh_stream* s, float** whitened, float** vx, float** vy, int** vidx) {
  if (!s) return WH_EINVAL;
  { const int jr = join_pipeline(s); if (jr != WH_OK) return jr; }
  if (whitened) *whitened = s->whitened;
  if (vx) *vx = s->vx;
  if (vy) *vy = s->vy;
  if (vidx) *vidx = s->vidx;
  return WH_OK;
}

int wh_profile_enable(wh_stream* s, int on) {
  if (!s) return WH_EINVAL;
  s->prof = on ? 1 : 0;
  return WH_OK;
}

int wh_profile_read(wh_stream* s, double* ms, long long* n, int reset) {
  if (!s) return WH_EINVAL;
  WH_CU(cudaStreamSynchronize(s->st));
  double acc[3] = {0, 0, 0};
  for (size_t f = 0; f + 4 <= s->ev_used; f += 4)
    for (int k = 0; k < 3; ++k) {
      float t = 0.f;
      WH_CU(cudaEventElapsedTime(&t, s->ev[f + k], s->ev[f + k + 1]));
      acc[k] += t;
    }
  for (int k = 0; k < 3; ++k) {
    if (ms) ms[k] = acc[k];
    if (n) n[k] = (long long)(s->ev_used / 4);
  }
  if (reset) s->ev_used = 0;
  return WH_OK;
}

int wh_destroy_stream(wh_stream* s) {
  if (!s) return WH_OK;
  cudaStreamSynchronize(s->st);
  free_stream(s);
  return WH_OK;
}

const char* wh_status_string(int st) {
  switch (st) {
    case WH_OK: return "ok";
    case WH_EINVAL: return "invalid argument";
    case WH_ENOMEM: return "out of memory";
    case WH_EADMIT: return "over the memory budget (not admitted)";
    case WH_ENOTREADY: return "output not ready (too few frames pushed)";
    case WH_ECUDA: return "CUDA error";
    case WH_ETIMEOUT: return "device wait timed out";
    case WH_EUNSUP: return "unsupported parameter combination";
    default: return "unknown status";
  }
}

const char* wh_last_error(void) { return g_err; }

long long wh_kernel_launch_count(void) { return g_launches.load(); }

}  // extern "C"
