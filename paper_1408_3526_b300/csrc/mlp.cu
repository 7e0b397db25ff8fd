// Learned velocity estimator: an MLP n_in -> h1 -> h2 -> n_out (GELU, tanh
// form) on the per-pixel log-power spectrum, BF16 weights and activations,
// FP32 accumulation on tcgen05 tensor cores, FP32 master weights and AdamW.
//
// Forward (x: [n][ldx] BF16):
//   Z1 = x W1^T + b1, H1 = GELU(Z1)    GEMM, fused bias + GELU epilogue (BF16 out)
//   Z2 = H1 W2^T + b2, H2 = GELU(Z2)   GEMM, fused epilogue
//   Y  = H2 W3^T + b3                  GEMM, F32 out; Y = (vx, vy, confidence logit)
// Loss (per sample, averaged): (vx - tx)^2 + (vy - ty)^2 + BCE(sigmoid(c), tc),
// tc = 1 when max(|vx - tx|, |vy - ty|) <= one grid step (the network's own
// velocity is within one step of the label), else 0.
// Backward: dY -> dW3 = dY^T H2, dH2 = dY W3, dZ2 = dH2 * GELU'(Z2), dW2 = dZ2^T H1,
// dH1 = dZ2 W2, dZ1 = dH1 * GELU'(Z1), dW1 = dZ1^T x, bias gradients by column
// sums; every product is a tcgen05 GEMM with both operands K-major (explicit
// BF16 transposes of the [n][.] activations).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/whiten.h"
#include "common.cuh"
#include "stream_internal.h"
#include "tc_gemm.cuh"

using namespace wh;
typedef __nv_bfloat16 bf16;

struct wh_mlp {
  int n_in, ld_in, h1, h2, n_out, o_pad;
  cudaStream_t st;
  // FP32 master parameters, gradients, Adam moments: one flat buffer each
  float *p, *g, *m, *v;
  size_t np;                       // total parameter floats (padded layout)
  size_t oW1, ob1, oW2, ob2, oW3, ob3;
  bf16 *W1h, *W2h, *W3h, *W2T, *W3T;   // BF16 copies (and transposes for backward)
  long long step;
  int* err;
  float* d_loss;                   // [4]: loss sum, mse sum, bce sum, within-step count
  // activation buffers (capacity cap rows)
  long long cap;
  bf16 *H1, *H2, *dY, *dZ1, *dZ2, *T1, *T2;
  float *Z1, *Z2, *Y, *dH;
};

namespace {

__device__ __forceinline__ float gelu_t(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  return 0.5f * x * (1.f + tanhf(k0 * (x + k1 * x * x * x)));
}
__device__ __forceinline__ float gelu_t_grad(float x) {
  const float k0 = 0.7978845608028654f, k1 = 0.044715f;
  const float t = tanhf(k0 * (x + k1 * x * x * x));
  return 0.5f * (1.f + t) + 0.5f * x * (1.f - t * t) * k0 * (1.f + 3.f * k1 * x * x);
}

__global__ void to_bf16_kernel(const float* src, bf16* dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

// dst[c][r] = src[r][c]   (src [rows][lds], dst [cols][ldd]); 32x32 tiles
__global__ void transpose_bf16_kernel(const bf16* src, int lds, bf16* dst, int ldd, int rows, int cols) {
  __shared__ bf16 tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < rows && c < cols) ? src[size_t(r) * lds + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (c < cols && r < rows) dst[size_t(c) * ldd + r] = tile[threadIdx.x][j];
  }
}

// loss, dY (BF16 [n][o_pad]) and statistics
__global__ void loss_grad_kernel(const float* Y, int ldy, const float* tgt, int n, float vstep, bf16* dY,
                                 int o_pad, float* stats) {
  float l = 0.f, mse = 0.f, bce = 0.f, within = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float vx = Y[size_t(i) * ldy], vy = Y[size_t(i) * ldy + 1], c = Y[size_t(i) * ldy + 2];
    const float tx = tgt[2 * i], ty = tgt[2 * i + 1];
    const float ex = vx - tx, ey = vy - ty;
    const float tc = (fmaxf(fabsf(ex), fabsf(ey)) <= vstep) ? 1.f : 0.f;
    const float sg = 1.f / (1.f + __expf(-c));
    const float b = fmaxf(c, 0.f) - c * tc + log1pf(__expf(-fabsf(c)));
    mse += ex * ex + ey * ey;
    bce += b;
    l += ex * ex + ey * ey + b;
    within += tc;
    const float inv = 1.f / float(n);
    bf16* d = dY + size_t(i) * o_pad;
    d[0] = __float2bfloat16(2.f * ex * inv);
    d[1] = __float2bfloat16(2.f * ey * inv);
    d[2] = __float2bfloat16((sg - tc) * inv);
    for (int j = 3; j < o_pad; ++j) d[j] = __float2bfloat16(0.f);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    l += __shfl_xor_sync(0xffffffffu, l, off);
    mse += __shfl_xor_sync(0xffffffffu, mse, off);
    bce += __shfl_xor_sync(0xffffffffu, bce, off);
    within += __shfl_xor_sync(0xffffffffu, within, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats + 0, l);
    atomicAdd(stats + 1, mse);
    atomicAdd(stats + 2, bce);
    atomicAdd(stats + 3, within);
  }
}

// dZ = dH * GELU'(Z)  -> BF16
__global__ void gelu_bwd_kernel(const float* dH, const float* Z, bf16* dZ, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dZ[i] = __float2bfloat16(dH[i] * gelu_t_grad(Z[i]));
}

// g[c] = sum_r d[r][c] (BF16 in, F32 out); one block per column block
__global__ void colsum_kernel(const bf16* d, int ld, int rows, int cols, float* g) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  float acc = 0.f;
  if (c < cols)
    for (int r = threadIdx.x >> 5; r < rows; r += blockDim.x >> 5) acc += __bfloat162float(d[size_t(r) * ld + c]);
  __shared__ float part[32][33];
  part[threadIdx.x >> 5][threadIdx.x & 31] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    float s = 0.f;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) s += part[w][threadIdx.x];
    if (c < cols) g[c] = s;
  }
}

__global__ void adamw_kernel(float* p, const float* g, float* m, float* v, long long n, float lr, float b1,
                             float b2, float eps, float wd, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * ((mi * c1) / (sqrtf(vi * c2) + eps) + wd * p[i]);
  }
}

unsigned blocks_for(long long n, int t = 256) {
  long long b = (n + t - 1) / t;
  if (b > 148LL * 32) b = 148LL * 32;
  if (b < 1) b = 1;
  return unsigned(b);
}

uint64_t splitmix(uint64_t& x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int refresh_bf16(wh_mlp* m) {
  to_bf16_kernel<<<blocks_for(size_t(m->h1) * m->ld_in), 256, 0, m->st>>>(m->p + m->oW1, m->W1h, size_t(m->h1) * m->ld_in);
  to_bf16_kernel<<<blocks_for(size_t(m->h2) * m->h1), 256, 0, m->st>>>(m->p + m->oW2, m->W2h, size_t(m->h2) * m->h1);
  to_bf16_kernel<<<blocks_for(size_t(m->o_pad) * m->h2), 256, 0, m->st>>>(m->p + m->oW3, m->W3h, size_t(m->o_pad) * m->h2);
  dim3 tb(32, 8);
  transpose_bf16_kernel<<<dim3((m->h1 + 31) / 32, (m->h2 + 31) / 32), tb, 0, m->st>>>(m->W2h, m->h1, m->W2T, m->h2, m->h2, m->h1);
  transpose_bf16_kernel<<<dim3((m->h2 + 31) / 32, (m->o_pad + 31) / 32), tb, 0, m->st>>>(m->W3h, m->h2, m->W3T, m->o_pad, m->o_pad, m->h2);
  wh_count_launches(5);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? WH_OK : wh_cuda_fail(e, "mlp weight refresh");
}

void free_mlp(wh_mlp* m) {
  if (!m) return;
  void* ptrs[] = {m->p, m->g, m->m, m->v, m->W1h, m->W2h, m->W3h, m->W2T, m->W3T, m->err, m->d_loss,
                  m->H1, m->H2, m->dY, m->dZ1, m->dZ2, m->T1, m->T2, m->Z1, m->Z2, m->Y, m->dH};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete m;
}

int ensure_cap(wh_mlp* m, long long n, bool train) {
  if (n <= m->cap && (!train || m->dY)) return WH_OK;
  void** bufs[] = {(void**)&m->H1, (void**)&m->H2, (void**)&m->dY, (void**)&m->dZ1, (void**)&m->dZ2,
                   (void**)&m->T1, (void**)&m->T2, (void**)&m->Z1, (void**)&m->Z2, (void**)&m->Y,
                   (void**)&m->dH};
  for (void** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  const long long c = (n + 7) / 8 * 8;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
  al((void**)&m->H1, sizeof(bf16) * c * m->h1);
  al((void**)&m->H2, sizeof(bf16) * c * m->h2);
  al((void**)&m->Y, sizeof(float) * c * m->o_pad);
  if (train) {
    al((void**)&m->Z1, sizeof(float) * c * m->h1);
    al((void**)&m->Z2, sizeof(float) * c * m->h2);
    al((void**)&m->dY, sizeof(bf16) * c * m->o_pad);
    al((void**)&m->dZ1, sizeof(bf16) * c * m->h1);
    al((void**)&m->dZ2, sizeof(bf16) * c * m->h2);
    al((void**)&m->dH, sizeof(float) * c * m->h1);
    const size_t tmax = size_t(m->ld_in > m->h1 ? m->ld_in : m->h1);
    al((void**)&m->T1, sizeof(bf16) * c * tmax);
    al((void**)&m->T2, sizeof(bf16) * c * m->h1);
  }
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? WH_ENOMEM : wh_cuda_fail(e, "mlp buffers");
  m->cap = c;
  return WH_OK;
}

int gemm(wh_mlp* m, const void* A, int lda, const void* B, int ldb, void* C, int ldc, int M, int N, int K,
         int epi, const float* bias, int act, float* preact, int ldp) {
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K; g.bf16 = 1; g.epi = epi; g.act = act; g.bias = bias;
  g.C = C; g.ldc = ldc; g.preact = preact; g.ldp = ldp; g.err = m->err;
  const int bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
  const cudaError_t e = tc_gemm(g, A, lda, B, ldb, bn, m->st);
  wh_count_launches(1);
  return e == cudaSuccess ? WH_OK : wh_cuda_fail(e, "mlp gemm");
}

int forward_impl(wh_mlp* m, const void* x, int ldx, int n, bool train) {
  int rc;
  if ((rc = gemm(m, x, ldx, m->W1h, m->ld_in, m->H1, m->h1, n, m->h1, m->n_in, EPI_BF16, m->p + m->ob1, 1,
                 train ? m->Z1 : nullptr, m->h1)) != WH_OK) return rc;
  if ((rc = gemm(m, m->H1, m->h1, m->W2h, m->h1, m->H2, m->h2, n, m->h2, m->h1, EPI_BF16, m->p + m->ob2, 1,
                 train ? m->Z2 : nullptr, m->h2)) != WH_OK) return rc;
  return gemm(m, m->H2, m->h2, m->W3h, m->h2, m->Y, m->o_pad, n, m->o_pad, m->h2, EPI_F32, m->p + m->ob3, 0,
              nullptr, 0);
}

}  // namespace

// ---------------------------------------------------------------------------
namespace wh {
int mlp_n_in(const wh_mlp* m) { return m ? m->n_in : 0; }

// The last forward pass's outputs in the network's own buffer: [n][ld] FP32,
// columns 0..n_out-1 used; valid until the next pass on this network.
const float* mlp_output(const wh_mlp* m, int* ld) {
  if (ld) *ld = m ? m->o_pad : 0;
  return m ? m->Y : nullptr;
}

// Forward pass enqueued on `st` (the caller's stream) instead of the network's
// own: the whitening stream's learned search runs it between its spectrum and
// selection kernels, which must see its input and output in stream order.
// The network's buffers are shared, so one network serves one caller at a time.

int mlp_forward_on(wh_mlp* m, const void* x, int ldx, int n, float* y, int ldy, cudaStream_t st) {
  if (!m || !x || n < 1 || ldx < m->n_in || (ldx % 8)) return WH_EINVAL;
  const cudaStream_t own = m->st;
  m->st = st;
  int rc = ensure_cap(m, n, false);
  if (rc == WH_OK) rc = forward_impl(m, x, ldx, n, false);
  if (rc == WH_OK && y) {
    const cudaError_t e = cudaMemcpy2DAsync(y, sizeof(float) * ldy, m->Y, sizeof(float) * m->o_pad,
                                            sizeof(float) * m->n_out, n, cudaMemcpyDeviceToDevice, m->st);
    if (e != cudaSuccess) rc = wh_cuda_fail(e, "mlp output copy");
  }
  m->st = own;
  return rc;
}
}  // namespace wh

extern "C" {

int wh_mlp_create(int n_in, int h1, int h2, int n_out, unsigned long long seed, void* cuda_stream, wh_mlp** out) {
  if (!out || n_in < 1 || h1 < 16 || h2 < 16 || n_out < 1 || n_out > 16 || (h1 % 8) || (h2 % 8)) return WH_EINVAL;
  *out = nullptr;
  wh_mlp* m = new (std::nothrow) wh_mlp();
  if (!m) return WH_ENOMEM;
  m->n_in = n_in; m->ld_in = (n_in + 7) / 8 * 8; m->h1 = h1; m->h2 = h2; m->n_out = n_out; m->o_pad = 16;
  m->st = (cudaStream_t)cuda_stream;
  m->oW1 = 0; m->ob1 = m->oW1 + size_t(h1) * m->ld_in;
  m->oW2 = m->ob1 + h1; m->ob2 = m->oW2 + size_t(h2) * h1;
  m->oW3 = m->ob2 + h2; m->ob3 = m->oW3 + size_t(m->o_pad) * h2;
  m->np = m->ob3 + m->o_pad;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
  al((void**)&m->p, sizeof(float) * m->np);
  al((void**)&m->g, sizeof(float) * m->np);
  al((void**)&m->m, sizeof(float) * m->np);
  al((void**)&m->v, sizeof(float) * m->np);
  al((void**)&m->W1h, sizeof(bf16) * size_t(h1) * m->ld_in);
  al((void**)&m->W2h, sizeof(bf16) * size_t(h2) * h1);
  al((void**)&m->W3h, sizeof(bf16) * size_t(m->o_pad) * h2);
  al((void**)&m->W2T, sizeof(bf16) * size_t(h1) * h2);
  al((void**)&m->W3T, sizeof(bf16) * size_t(h2) * m->o_pad);
  al((void**)&m->err, sizeof(int));
  al((void**)&m->d_loss, sizeof(float) * 4);
  if (e != cudaSuccess) {
    free_mlp(m);
    return e == cudaErrorMemoryAllocation ? WH_ENOMEM : wh_cuda_fail(e, "mlp create");
  }
  // U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases; padded entries 0
  std::vector<float> hp(m->np, 0.f);
  uint64_t st = seed ? seed : 1;
  auto uni = [&](float bound) { return bound * (2.f * float(splitmix(st) >> 40) / float(1ull << 24) - 1.f); };
  const float bd1 = 1.f / std::sqrt(float(n_in)), bd2 = 1.f / std::sqrt(float(h1)), bd3 = 1.f / std::sqrt(float(h2));
  for (int r = 0; r < h1; ++r)
    for (int c = 0; c < n_in; ++c) hp[m->oW1 + size_t(r) * m->ld_in + c] = uni(bd1);
  for (int r = 0; r < h1; ++r) hp[m->ob1 + r] = uni(bd1);
  for (int r = 0; r < h2; ++r)
    for (int c = 0; c < h1; ++c) hp[m->oW2 + size_t(r) * h1 + c] = uni(bd2);
  for (int r = 0; r < h2; ++r) hp[m->ob2 + r] = uni(bd2);
  for (int r = 0; r < n_out; ++r)
    for (int c = 0; c < h2; ++c) hp[m->oW3 + size_t(r) * h2 + c] = uni(bd3);
  for (int r = 0; r < n_out; ++r) hp[m->ob3 + r] = uni(bd3);
  e = cudaMemcpy(m->p, hp.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, sizeof(float) * m->np);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, sizeof(float) * m->np);
  if (e == cudaSuccess) e = cudaMemset(m->g, 0, sizeof(float) * m->np);
  if (e == cudaSuccess) e = cudaMemset(m->err, 0, sizeof(int));
  if (e != cudaSuccess) {
    free_mlp(m);
    return wh_cuda_fail(e, "mlp init");
  }
  int rc = refresh_bf16(m);
  if (rc != WH_OK) {
    free_mlp(m);
    return rc;
  }
  *out = m;
  return WH_OK;
}

int wh_mlp_destroy(wh_mlp* m) {
  if (!m) return WH_OK;
  cudaStreamSynchronize(m->st);
  free_mlp(m);
  return WH_OK;
}

long long wh_mlp_num_params(const wh_mlp* m) {
  if (!m) return 0;
  return (long long)m->h1 * m->n_in + m->h1 + (long long)m->h2 * m->h1 + m->h2 + (long long)m->n_out * m->h2 +
         m->n_out;
}

// Copy logical parameters (W1 [h1][n_in], b1, W2 [h2][h1], b2, W3 [n_out][h2], b3)
// or the gradients of the last training step between host and device.
static int params_io(wh_mlp* m, float* host, long long n, bool to_host, bool grads) {
  if (!m || !host || n != wh_mlp_num_params(m)) return WH_EINVAL;
  float* dev = grads ? m->g : m->p;
  std::vector<float> buf(m->np);
  cudaError_t e = cudaMemcpyAsync(buf.data(), dev, sizeof(float) * m->np, cudaMemcpyDeviceToHost, m->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
  if (e != cudaSuccess) return wh_cuda_fail(e, "mlp params");
  size_t o = 0;
  auto blk = [&](size_t off, int rows, int cols, int ld) {
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c, ++o) {
        if (to_host) host[o] = buf[off + size_t(r) * ld + c];
        else buf[off + size_t(r) * ld + c] = host[o];
      }
  };
  blk(m->oW1, m->h1, m->n_in, m->ld_in);
  blk(m->ob1, 1, m->h1, m->h1);
  blk(m->oW2, m->h2, m->h1, m->h1);
  blk(m->ob2, 1, m->h2, m->h2);
  blk(m->oW3, m->n_out, m->h2, m->h2);
  blk(m->ob3, 1, m->n_out, m->n_out);
  if (!to_host) {
    e = cudaMemcpyAsync(dev, buf.data(), sizeof(float) * m->np, cudaMemcpyHostToDevice, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) return wh_cuda_fail(e, "mlp params");
    if (!grads) return refresh_bf16(m);
  }
  return WH_OK;
}

int wh_mlp_get_params(wh_mlp* m, float* host, long long n) { return params_io(m, host, n, true, false); }
int wh_mlp_set_params(wh_mlp* m, const float* host, long long n) {
  return params_io(m, const_cast<float*>(host), n, false, false);
}
int wh_mlp_get_grads(wh_mlp* m, float* host, long long n) { return params_io(m, host, n, true, true); }

int wh_mlp_forward(wh_mlp* m, const void* x, int ldx, int n, float* y, int ldy) {
  if (!m) return WH_EINVAL;
  return wh::mlp_forward_on(m, x, ldx, n, y, ldy, m->st);
}

int wh_mlp_train_step(wh_mlp* m, const void* x, int ldx, int n, const float* target, float vstep, float lr,
                      float weight_decay, int apply, float* stats_out) {
  if (!m || !x || !target || n < 8 || (n % 8) || ldx < m->n_in || (ldx % 8) || m->n_out != 3) return WH_EINVAL;
  int rc = ensure_cap(m, n, true);
  if (rc != WH_OK) return rc;
  cudaError_t e = cudaMemsetAsync(m->d_loss, 0, sizeof(float) * 4, m->st);
  if (e != cudaSuccess) return wh_cuda_fail(e, "mlp");
  if ((rc = forward_impl(m, x, ldx, n, true)) != WH_OK) return rc;
  loss_grad_kernel<<<blocks_for(n), 256, 0, m->st>>>(m->Y, m->o_pad, target, n, vstep, m->dY, m->o_pad, m->d_loss);
  const dim3 tb(32, 8);
  auto transpose = [&](const bf16* src, int lds, bf16* dst, int rows, int cols) {
    transpose_bf16_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32), tb, 0, m->st>>>(src, lds, dst, rows, rows, cols);
  };
  float* g = m->g;
  // layer 3
  transpose(m->dY, m->o_pad, m->T1, n, m->o_pad);          // dY^T [o_pad][n]
  transpose(m->H2, m->h2, m->T2, n, m->h2);                // H2^T [h2][n]
  if ((rc = gemm(m, m->T1, n, m->T2, n, g + m->oW3, m->h2, m->o_pad, m->h2, n, EPI_F32, nullptr, 0, nullptr, 0)) != WH_OK) return rc;
  colsum_kernel<<<(m->o_pad + 31) / 32, 256, 0, m->st>>>(m->dY, m->o_pad, n, m->o_pad, g + m->ob3);
  if ((rc = gemm(m, m->dY, m->o_pad, m->W3T, m->o_pad, m->dH, m->h2, n, m->h2, m->o_pad, EPI_F32, nullptr, 0, nullptr, 0)) != WH_OK) return rc;
  gelu_bwd_kernel<<<blocks_for((long long)n * m->h2), 256, 0, m->st>>>(m->dH, m->Z2, m->dZ2, (long long)n * m->h2);
  // layer 2
  colsum_kernel<<<(m->h2 + 31) / 32, 256, 0, m->st>>>(m->dZ2, m->h2, n, m->h2, g + m->ob2);
  transpose(m->dZ2, m->h2, m->T1, n, m->h2);               // dZ2^T [h2][n]
  transpose(m->H1, m->h1, m->T2, n, m->h1);                // H1^T [h1][n]
  if ((rc = gemm(m, m->T1, n, m->T2, n, g + m->oW2, m->h1, m->h2, m->h1, n, EPI_F32, nullptr, 0, nullptr, 0)) != WH_OK) return rc;
  if ((rc = gemm(m, m->dZ2, m->h2, m->W2T, m->h2, m->dH, m->h1, n, m->h1, m->h2, EPI_F32, nullptr, 0, nullptr, 0)) != WH_OK) return rc;
  gelu_bwd_kernel<<<blocks_for((long long)n * m->h1), 256, 0, m->st>>>(m->dH, m->Z1, m->dZ1, (long long)n * m->h1);
  // layer 1
  colsum_kernel<<<(m->h1 + 31) / 32, 256, 0, m->st>>>(m->dZ1, m->h1, n, m->h1, g + m->ob1);
  transpose(m->dZ1, m->h1, m->T2, n, m->h1);               // dZ1^T [h1][n]
  transpose(reinterpret_cast<const bf16*>(x), ldx, m->T1, n, m->ld_in);   // x^T [ld_in][n]
  if ((rc = gemm(m, m->T2, n, m->T1, n, g + m->oW1, m->ld_in, m->h1, m->ld_in, n, EPI_F32, nullptr, 0, nullptr, 0)) != WH_OK) return rc;
  wh_count_launches(11);
  if (apply) {
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, float(m->step))), c2 = 1.f / (1.f - std::pow(b2, float(m->step)));
    adamw_kernel<<<blocks_for(m->np), 256, 0, m->st>>>(m->p, m->g, m->m, m->v, m->np, lr, b1, b2, 1e-8f,
                                                      weight_decay, c1, c2);
    wh_count_launches(1);
    if ((rc = refresh_bf16(m)) != WH_OK) return rc;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return wh_cuda_fail(e, "mlp train step");
  if (stats_out) {
    float h[4];
    e = cudaMemcpyAsync(h, m->d_loss, sizeof(h), cudaMemcpyDeviceToHost, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) return wh_cuda_fail(e, "mlp loss");
    for (int i = 0; i < 4; ++i) stats_out[i] = h[i] / float(n);
    int herr = 0;
    cudaMemcpy(&herr, m->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (herr) {
      cudaMemset(m->err, 0, sizeof(int));
      return WH_ETIMEOUT;
    }
  }
  return WH_OK;
}

}  // extern "C"
