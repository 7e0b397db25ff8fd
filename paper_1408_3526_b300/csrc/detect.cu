// Downstream threshold detector (the detection step the whitening feeds,
// Sec. 1): pixels of the latest whitened frame E with E >= k * sigma, sigma =
// RMS of E over the frame, listed in raster order with the velocity that tuned
// the frame's prediction-error filter at that pixel.  Deterministic: the
// sum of squares is reduced in a fixed order and detections are placed by a
// per-row count and an exclusive scan.
#include <cstdio>

#include "../../include/whiten.h"
#include "common.cuh"
#include "stream_internal.h"

namespace wh {
namespace {

constexpr int kRB = 256;      // threads of the reduction / row blocks

__global__ void sumsq_partial_kernel(const float* e, long long n, double* partial) {
  __shared__ double sh[kRB / 32];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * kRB + threadIdx.x; i < n; i += (long long)gridDim.x * kRB) {
    const double v = e[i];
    acc = fma(v, v, acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kRB / 32; ++w) t += sh[w];
    partial[blockIdx.x] = t;
  }
}

// one thread: sigma and the threshold from the partial sums (fixed order)
__global__ void threshold_kernel(const double* partial, int nb, long long n, float k, float* sig_thr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int b = 0; b < nb; ++b) t += partial[b];
  const float sigma = float(sqrt(t / double(n)));
  sig_thr[0] = sigma;
  sig_thr[1] = k * sigma;
}

__global__ void row_count_kernel(const float* e, int H, int W, const float* sig_thr, int* counts) {
  __shared__ int sh[kRB / 32];
  const int y = blockIdx.x;
  if (y >= H) return;
  const float thr = sig_thr[1];
  int c = 0;
  for (int x = threadIdx.x; x < W; x += kRB) c += e[size_t(y) * W + x] >= thr;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < kRB / 32; ++w) t += sh[w];
    counts[y] = t;
  }
}

// one block: exclusive scan of the row counts (serial over chunks of 1024)
__global__ void row_scan_kernel(const int* counts, int H, int* offsets, int* total) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < H; b += 1024) {
    const int i = b + threadIdx.x;
    const int v = i < H ? counts[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {      // Hillis-Steele inclusive scan
      const int add = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
      __syncthreads();
      sh[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < H) offsets[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void emit_kernel(const float* e, const float* vx, const float* vy, int H, int W,
                            const float* sig_thr, const int* offsets, int max_det, wh_detection* out) {
  const int y = blockIdx.x;
  if (y >= H || threadIdx.x >= 32) return;       // one warp per row keeps raster order simply
  const float thr = sig_thr[1];
  const int lane = threadIdx.x;
  int pos = offsets[y];
  for (int x0 = 0; x0 < W; x0 += 32) {
    const int x = x0 + lane;
    const size_t i = size_t(y) * W + x;
    const bool hit = x < W && e[i] >= thr;
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    const int p = pos + __popc(m & ((1u << lane) - 1u));
    if (hit && p < max_det) {
      wh_detection d;
      d.y = y; d.x = x; d.value = e[i]; d.vx = vx[i]; d.vy = vy[i];
      out[p] = d;
    }
    pos += __popc(m);
  }
}

}  // namespace
}  // namespace wh

using namespace wh;

extern "C" int wh_detect(wh_stream* s, float k_sigma, int max_det, wh_detection* out, int* n_out,
                         float* sigma_out, int is_device, long long* frame_index) {
  if (!s || max_det < 0 || (max_det > 0 && !out) || !n_out || !(k_sigma > 0.f)) return WH_EINVAL;
  if (s->t < s->mpz + 1) return WH_ENOTREADY;
  { const int jr = wh_join_pipeline(s); if (jr != WH_OK) return jr; }
  const long long n = (long long)s->H * s->W;
  constexpr int kNB = 296;
  // scratch: partial sums, sigma/threshold, row counts and offsets, total, and
  // a device list when the caller's buffer is on the host
  const size_t need = sizeof(double) * kNB + 16 + sizeof(int) * (2 * size_t(s->H) + 1);
  if (!s->d_det || s->det_bytes < need) {
    if (s->d_det) cudaFree(s->d_det);
    s->d_det = nullptr;
    s->det_bytes = 0;
    cudaError_t e = cudaMalloc(&s->d_det, need);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? WH_ENOMEM : wh_cuda_fail(e, "cudaMalloc");
    s->det_bytes = need;
  }
  char* base = static_cast<char*>(s->d_det);
  double* partial = reinterpret_cast<double*>(base);
  float* sig_thr = reinterpret_cast<float*>(base + sizeof(double) * kNB);
  int* counts = reinterpret_cast<int*>(base + sizeof(double) * kNB + 16);
  int* offsets = counts + s->H;
  int* total = offsets + s->H;
  wh_detection* dlist = out;
  if (!is_device && max_det > 0) {
    if (s->det_list_cap < max_det) {
      if (s->d_det_list) cudaFree(s->d_det_list);
      s->d_det_list = nullptr;
      s->det_list_cap = 0;
      cudaError_t e = cudaMalloc((void**)&s->d_det_list, sizeof(wh_detection) * size_t(max_det));
      if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? WH_ENOMEM : wh_cuda_fail(e, "cudaMalloc");
      s->det_list_cap = max_det;
    }
    dlist = s->d_det_list;
  }
  sumsq_partial_kernel<<<kNB, kRB, 0, s->st>>>(s->whitened, n, partial);
  threshold_kernel<<<1, 32, 0, s->st>>>(partial, kNB, n, k_sigma, sig_thr);
  row_count_kernel<<<s->H, kRB, 0, s->st>>>(s->whitened, s->H, s->W, sig_thr, counts);
  row_scan_kernel<<<1, 1024, 0, s->st>>>(counts, s->H, offsets, total);
  if (max_det > 0)
    emit_kernel<<<s->H, 32, 0, s->st>>>(s->whitened, s->vx, s->vy, s->H, s->W, sig_thr, offsets, max_det, dlist);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return wh_cuda_fail(e, "detector kernels");
  wh_count_launches(max_det > 0 ? 5 : 4);
  int tot = 0;
  float st[2] = {0.f, 0.f};
  if ((e = cudaMemcpyAsync(&tot, total, sizeof(int), cudaMemcpyDeviceToHost, s->st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(st, sig_thr, sizeof(st), cudaMemcpyDeviceToHost, s->st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s->st)) != cudaSuccess)
    return wh_cuda_fail(e, "detector read-back");
  const int nw = tot < max_det ? tot : max_det;
  if (!is_device && nw > 0) {
    if ((e = cudaMemcpy(out, dlist, sizeof(wh_detection) * size_t(nw), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return wh_cuda_fail(e, "detector list copy");
  }
  *n_out = tot;
  if (sigma_out) *sigma_out = st[0];
  if (frame_index) *frame_index = s->t - 1 - s->mpz;
  return WH_OK;
}
