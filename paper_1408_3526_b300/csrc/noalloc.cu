// wh_push_frame_noalloc: a frame push that allocates no device memory.
//
// Some callers cannot call cudaMalloc at frame time: real-time loops whose
// memory is fixed at start-up, code running under an allocation-free policy
// (e.g. after a pool has been frozen), or hosts that forbid driver
// allocations once streaming begins.  This entry point runs the same per-pixel
// path as wh_push_frame on an existing stream, but its autocorrelation search
// always uses the tensor-core shortlist with exact FP32 re-evaluation, and all
// scratch of that search (the F16 copy of the smoothed state, per-pixel norms,
// the shortlist, the grid table) lives in one file-scope __device__ array
// instead of memory allocated by the library.  A bounded device wait that gives
// up reports through the stream's own status word (allocated with the stream),
// so the next synchronising read returns WH_ETIMEOUT as after wh_push_frame.
//
// Limits: window M <= 15, grid length L <= 25 (L^2 <= 640 table rows).  Frames
// of any size are processed in chunks of kChunk pixels.  The array (about
// 10.2 MB) is part of the module: every GPU that loads the library holds it
// until the process exits.
//
// Sharing: every call, from every stream on a device, uses the same array and
// leaves the last call's contents there.  Calls that overlap on the GPU (on
// different CUDA streams, or from several host threads) race on it; callers
// must serialise them (one CUDA stream, or events).  Nothing in the array needs
// to start at zero: every value a call reads was written earlier in that call.
//
// Set-up: the first call on a device looks up the array's device address
// (cudaGetSymbolAddress) with that device current and caches it; make that
// first call before any stream capture.
#include <cuda_fp16.h>

#include <cstdint>
#include <cstdio>

#include "../../include/whiten.h"
#include "common.cuh"
#include "stream_internal.h"
#include "tc_gemm.cuh"

using namespace wh;

namespace {

constexpr int kChunk = 16384;     // pixels per pass
constexpr int kKg = 232;          // M^2 (<= 225) rounded up to 8
constexpr int kRows = 640;        // table rows: L^2 <= 640
constexpr int kTiles = kRows / 128;

struct NoAllocScratch {
  uint16_t a16[kChunk * kKg];     // F16 copy of the smoothed state (chunk)
  uint16_t table[kRows * kKg];    // F16 [1, 2cos, -2sin] grid table
  float l1[kChunk];
  float cval[kChunk * kTiles * 4];
  int cidx[kChunk * kTiles * 4];
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of the array on the current device (looked up once per device).
cudaError_t scratch_ptr(NoAllocScratch** out) {
  static NoAllocScratch* cache[64] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!cache[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    cache[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = cache[dev];
  return cudaSuccess;
}

// B(l, k) = [1, 2 cos a_h(l), -2 sin a_h(l)] in F16, a_h(l) = 2pi (hx lx + hy ly)/M,
// rows l >= L^2 zero (same basis as the stream state).
__global__ void noalloc_table_kernel(uint16_t* table, int M, int L, float vmax, float vstep) {
  const int K = (M - 1) / 2, nh = (M * M - 1) / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kRows * kKg; i += gridDim.x * blockDim.x) {
    const int g = i / kKg, k = i % kKg;
    float v = 0.f;
    if (g < L * L && k <= 2 * nh) {
      if (k == 0) v = 1.f;
      else {
        const int h = k <= nh ? k : k - nh;
        int hx, hy;
        if (h <= K) { hx = 0; hy = h; }
        else { const int r = h - K - 1; hx = r / M + 1; hy = r % M - K; }
        const float lx = -vmax + (g % L) * vstep, ly = -vmax + (g / L) * vstep;
        float s, c;
        sincospif(2.f * (hx * lx + hy * ly) / float(M), &s, &c);
        v = k <= nh ? 2.f * c : -2.f * s;
      }
    }
    const __half hv = __float2half_rn(v);
    table[i] = *reinterpret_cast<const uint16_t*>(&hv);
  }
}

}  // namespace

extern "C" int wh_push_frame_noalloc(wh_stream* s, const float* frame, int is_device) {
  if (!s || !frame) return WH_EINVAL;
  if (s->pipeline) return WH_EUNSUP;          // runs on the caller's stream only
  if (s->M > 15 || s->L * s->L > kRows || !autocorr_tc_supported(s->M)) {
    std::snprintf(wh_error_buffer(), 512,
                  "wh_push_frame_noalloc: window %d / grid %dx%d beyond its limits (M <= 15, L <= 25)",
                  s->M, s->L, s->L);
    return WH_EUNSUP;
  }
  NoAllocScratch* sc = nullptr;
  cudaError_t e = scratch_ptr(&sc);
  if (e != cudaSuccess) return wh_cuda_fail(e, "cudaGetSymbolAddress");
  const size_t npix = size_t(s->H) * s->W;
  const float* src = frame;
  if (s->as) {   // after wh_push_frame_async, an output copy may still read the buffers below
    for (int b = 0; b < 2; ++b)
      if (s->as->used[b]) {
        e = cudaStreamWaitEvent(s->st, s->as->ev_out[b], 0);
        if (e != cudaSuccess) return wh_cuda_fail(e, "cudaStreamWaitEvent");
      }
  }
  if (!is_device) {
    e = cudaMemcpyAsync(s->frame, frame, sizeof(float) * npix, cudaMemcpyHostToDevice, s->st);
    if (e != cudaSuccess) return wh_cuda_fail(e, "cudaMemcpyAsync");
    src = s->frame;
  }
  // 1. spectrum, observer and smoothing (same kernel as wh_push_frame)
  SpecArgs sa{};
  sa.H = s->H; sa.W = s->W; sa.M = s->M; sa.Mz = s->Mz; sa.tw = s->tw; sa.th = s->th;
  sa.kpad = s->kpad; sa.alpha = float(s->alpha); sa.frame = src;
  sa.obs_old = s->obs[s->cur]; sa.obs_new = s->obs[1 - s->cur]; sa.Astate = s->Astate;
  sa.tables = s->d_spec; sa.hgather = s->d_hgather;
  sa.dump_win = s->d_dump_win; sa.dump_pow = s->d_dump_pow;
  sa.feat = s->d_feat; sa.feat_ld = s->feat_ld; sa.feat_n = s->feat_n; sa.feat_gather = s->d_fgather;
  sa.err = s->d_err;
  sa.f64 = s->spec_f64;
  e = launch_spectrum(sa, s->st);
  if (e != cudaSuccess) return wh_cuda_fail(e, "spectrum kernel");
  // 2. autocorrelation search with all scratch in the static array
  noalloc_table_kernel<<<148, 256, 0, s->st>>>(sc->table, s->M, s->L, float(s->vmax), float(s->vstep));
  if ((e = cudaGetLastError()) != cudaSuccess) return wh_cuda_fail(e, "table kernel");
  long long launches = 2;
  for (size_t p0 = 0; p0 < npix; p0 += kChunk) {
    const int n = int(npix - p0 < size_t(kChunk) ? npix - p0 : size_t(kChunk));
    AutocorrTcArgs ta{};
    ta.H = 1; ta.W = n; ta.M = s->M; ta.L = s->L; ta.kpad = s->kpad; ta.kg = kKg;
    ta.ntile = (s->L * s->L + 127) / 128; ta.ncand = ta.ntile * 4; ta.ovf_group = 4; ta.mode = 0; ta.bf16 = 0;
    ta.vmax = float(s->vmax); ta.vstep = float(s->vstep);
    ta.Astate = s->Astate + p0 * s->kpad;
    ta.a16 = sc->a16; ta.l1 = sc->l1; ta.cand_val = sc->cval; ta.cand_idx = sc->cidx;
    ta.vidx = s->vidx + p0; ta.vx = s->vx + p0; ta.vy = s->vy + p0;
    ta.tab_x = s->d_tabx; ta.n_fallback = nullptr;
    if ((e = launch_autocorr_convert(ta, s->st)) != cudaSuccess) return wh_cuda_fail(e, "convert kernel");
    GemmArgs g{};
    g.M = n; g.N = ta.ntile * 128; g.K = s->M * s->M; g.bf16 = 0; g.epi = EPI_TOPK;
    g.cand_val = sc->cval; g.cand_idx = sc->cidx; g.n_valid = s->L * s->L; g.err = s->d_err;
    if ((e = tc_gemm(g, sc->a16, kKg, sc->table, kKg, 128, s->st)) != cudaSuccess)
      return wh_cuda_fail(e, "tensor-core autocorrelation");
    if ((e = launch_autocorr_rerank(ta, s->st)) != cudaSuccess) return wh_cuda_fail(e, "re-rank kernel");
    launches += 3;
  }
  // 3. prediction-error filter (same kernel as wh_push_frame)
  PefArgs pa{};
  pa.H = s->H; pa.W = s->W; pa.M = s->M; pa.Mz = s->Mz; pa.L = s->L; pa.mpz = s->mpz;
  pa.obs = s->obs[1 - s->cur]; pa.vidx = s->vidx; pa.hw = s->d_hw; pa.whitened = s->whitened;
  e = launch_pef(pa, s->st);
  if (e != cudaSuccess) return wh_cuda_fail(e, "PEF kernel");
  wh_count_launches(launches + 1);
  s->cur = 1 - s->cur;
  s->t += 1;
  return WH_OK;
}
