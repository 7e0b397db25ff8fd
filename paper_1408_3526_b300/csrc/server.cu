// Multi-stream serving runtime: many sensor streams of different sizes and
// parameters, recursive state resident on the device, admission against a
// device-memory budget, continuous submission with overlap on the GPU.
//
// Model:
//   - open: a stream is admitted if its device footprint fits in the budget
//     left; otherwise WH_EADMIT (the caller retries once others close).
//   - submit: a frame (host memory, with its arrival time) joins its stream's
//     queue; a full queue (queue_limit frames waiting) rejects it with
//     WH_EADMIT (back-pressure, counted as shed load).
//   - a dispatcher thread keeps up to max_inflight frames on the GPU: it takes
//     the oldest waiting frame of any stream whose previous frame has been
//     dispatched, copies it into a pinned slot, and enqueues upload + the
//     stream's per-pixel path + download of the whitened frame on the CUDA
//     stream assigned to that sensor stream.  Streams are spread over a pool
//     of CUDA streams, so frames of different streams run concurrently;
//     frames of one stream stay in order on its CUDA stream.
//   - completion is signalled by a host callback on the CUDA stream; latency
//     = completion time - arrival time (queueing included).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/whiten.h"
#include "stream_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  long long id;
  int stream;
  double arrival;          // seconds on the server clock
  int slot = -1;
  double done = -1.0;
  bool finished = false;
  std::vector<float> result;   // whitened frame (host copy, if kept)
};

struct SStream {
  wh_stream* s = nullptr;
  int h = 0, w = 0;
  size_t bytes = 0;
  int cuda_idx = 0;
  std::deque<long long> queue;            // waiting request ids
  std::vector<float*> pinned_in;          // one per slot use (ring)
  float* pinned_out = nullptr;
  int ring = 0;
  bool busy = false;                      // a frame of this stream is on the GPU (or its result
                                          // is still in pinned_out)
  bool closing = false;
  long long harvest = -1;                 // request whose result waits in pinned_out
};

}  // namespace

struct wh_server {
  size_t budget = 0, used = 0;
  int max_inflight = 8, queue_limit = 4, keep_results = 1;
  std::vector<cudaStream_t> cuda;
  std::map<int, SStream> streams;
  std::map<long long, Request> reqs;
  int next_stream = 0;
  long long next_req = 0;
  int inflight = 0;
  long long shed = 0, served = 0, submitted = 0;
  long long pixels_served = 0;
  std::vector<double> latencies;
  double first_arrival = -1, last_done = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::thread dispatcher;
  Clock::time_point t0 = Clock::now();
  int error = WH_OK;
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

struct DoneCtx {
  wh_server* srv;
  long long req;
};

// Host callback at the end of a frame's work on its CUDA stream: timestamps
// the completion.  It copies nothing: with kept results the whitened frame
// waits in the stream's pinned buffer and the dispatcher thread moves it to
// the request (outside the lock) before the stream's next frame may reuse it.
void CUDART_CB on_done(void* p) {
  DoneCtx* c = static_cast<DoneCtx*>(p);
  wh_server* srv = c->srv;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    Request& r = srv->reqs[c->req];
    r.done = srv->now();
    SStream& st = srv->streams[r.stream];
    srv->served += 1;
    srv->pixels_served += (long long)st.h * st.w;
    srv->latencies.push_back(r.done - r.arrival);
    srv->last_done = std::max(srv->last_done, r.done);
    if (srv->keep_results && st.pinned_out) {
      st.harvest = c->req;
    } else {
      r.finished = true;
      st.busy = false;
      srv->inflight -= 1;
    }
  }
  srv->cv_work.notify_all();
  srv->cv_done.notify_all();
  delete c;
}

// Move one finished frame's result from its stream's pinned buffer to the
// request (called by the dispatcher with the lock held; copies unlocked).
bool harvest_one(wh_server* srv, std::unique_lock<std::mutex>& lk) {
  for (auto& kv : srv->streams) {
    SStream& st = kv.second;
    if (st.harvest < 0) continue;
    const long long rid = st.harvest;
    const float* src = st.pinned_out;
    const size_t n = size_t(st.h) * st.w;
    lk.unlock();
    std::vector<float> res(src, src + n);      // the stream stays busy: nothing rewrites src
    lk.lock();
    Request& r = srv->reqs[rid];
    r.result = std::move(res);
    r.finished = true;
    SStream& st2 = srv->streams[r.stream];
    st2.harvest = -1;
    st2.busy = false;
    srv->inflight -= 1;
    srv->cv_done.notify_all();
    return true;
  }
  return false;
}

// Oldest waiting frame of a stream that is not on the GPU (FIFO across streams).
long long pick(wh_server* srv, int* sid) {
  long long best = -1;
  double t = 1e300;
  for (auto& kv : srv->streams) {
    SStream& st = kv.second;
    if (st.busy || st.queue.empty()) continue;
    const Request& r = srv->reqs[st.queue.front()];
    if (r.arrival < t) { t = r.arrival; best = r.id; *sid = kv.first; }
  }
  return best;
}

void dispatch_loop(wh_server* srv) {
  std::unique_lock<std::mutex> lk(srv->mu);
  while (!srv->stop) {
    if (harvest_one(srv, lk)) continue;
    int sid = -1;
    long long rid = -1;
    if (srv->inflight < srv->max_inflight) rid = pick(srv, &sid);
    if (rid < 0) {
      srv->cv_work.wait(lk);
      continue;
    }
    SStream& st = srv->streams[sid];
    st.queue.pop_front();
    st.busy = true;
    srv->inflight += 1;
    Request& r = srv->reqs[rid];
    float* in = st.pinned_in[r.slot];
    cudaStream_t cs = srv->cuda[st.cuda_idx];
    wh_stream* s = st.s;
    const size_t bytes = sizeof(float) * size_t(st.h) * st.w;
    float* out = st.pinned_out;
    lk.unlock();
    // the stream object belongs to this sensor stream; its CUDA stream is cs
    s->st = cs;
    int rc = wh_push_frame(s, in, 0);
    float* dw = nullptr;
    if (rc == WH_OK) rc = wh_output_pointers(s, &dw, nullptr, nullptr, nullptr);
    if (rc == WH_OK && out) {
      if (cudaMemcpyAsync(out, dw, bytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess) rc = WH_ECUDA;
    }
    DoneCtx* ctx = new (std::nothrow) DoneCtx{srv, rid};
    if (rc == WH_OK && ctx && cudaLaunchHostFunc(cs, on_done, ctx) != cudaSuccess) rc = WH_ECUDA;
    lk.lock();
    if (rc != WH_OK) {
      srv->error = rc;
      delete ctx;
      st.busy = false;
      srv->inflight -= 1;
      r.finished = true;
      srv->cv_done.notify_all();
    }
  }
}

}  // namespace

extern "C" {

long long wh_stream_device_bytes_opt(int h, int w, int window, int temporal_order, wh_vgrid grid,
                                     const wh_params* opt) {
  if (h < 1 || w < 1 || window < 3 || temporal_order < 2 || !(grid.step > 0.f)) return -1;
  const long long npix = (long long)h * w;
  const long long kpad = ((long long)window * window + 3) & ~3LL;
  const long long L = (long long)(2.0 * grid.vmax / grid.step + 1.5);
  // observer ping-pong, smoothed state, frame, whitened/vx/vy/vidx, tables
  long long b = npix * (2LL * temporal_order * 4 + kpad * 4 + 4 + 16) + L * 64 * 1024 + (1 << 20);
  const int prec0 = opt ? opt->precision : 0;
  if ((prec0 & 3) == 0 && (prec0 & WH_PREC_TC_DENSE) &&
      !(prec0 & (WH_PREC_CUDA_CORES | WH_PREC_TC_SHORTLIST | WH_PREC_TC_SEPARABLE))) {
    // whole contraction on tensor cores: per-pixel listed points and the operand
    const long long nhg = (L * L + 1) / 2, nch = (nhg + 127) / 128;
    b += npix * 4 * 9 + 2 * nch * 128 * 128 * 2;
  }
  if (opt) {
    if (opt->pipeline) b += npix * kpad * 4;                       // second smoothed-state buffer
    const int prec = opt->precision;
    if ((prec & 3) || (prec & WH_PREC_TC_SHORTLIST)) {             // tensor-core shortlist scratch
      const long long kg = ((long long)window * window + 7) & ~7LL;
      const long long ntile = (L * L + 127) / 128;
      const long long nc = ntile * 4 > 8 ? ntile * 4 : 8;
      b += npix * (2 * kg + 4 + 8 * nc) + 2 * ntile * 128 * kg + 4;
    }
    if (prec & WH_PREC_TC_SEPARABLE) b += 8192;                    // stage-1 operand
    if (opt->debug_dump) b += npix * (long long)window * window * temporal_order * 12;
  }
  return b;
}

long long wh_stream_device_bytes(int h, int w, int window, int temporal_order, wh_vgrid grid) {
  return wh_stream_device_bytes_opt(h, w, window, temporal_order, grid, nullptr);
}

int wh_server_create(double hbm_budget_bytes, int max_inflight, int queue_limit, int n_cuda_streams,
                     int keep_results, wh_server** out) {
  if (!out || hbm_budget_bytes <= 0 || max_inflight < 1 || queue_limit < 1 || n_cuda_streams < 1)
    return WH_EINVAL;
  wh_server* srv = new (std::nothrow) wh_server();
  if (!srv) return WH_ENOMEM;
  srv->budget = size_t(hbm_budget_bytes);
  srv->max_inflight = max_inflight;
  srv->queue_limit = queue_limit;
  srv->keep_results = keep_results;
  for (int i = 0; i < n_cuda_streams; ++i) {
    cudaStream_t c;
    if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : srv->cuda) cudaStreamDestroy(x);
      delete srv;
      return WH_ECUDA;
    }
    srv->cuda.push_back(c);
  }
  srv->dispatcher = std::thread(dispatch_loop, srv);
  *out = srv;
  return WH_OK;
}

int wh_server_open(wh_server* srv, int h, int w, int window, int temporal_order, wh_vgrid grid,
                   const wh_params* opt, int* stream_id) {
  if (!srv || !stream_id) return WH_EINVAL;
  const long long need = wh_stream_device_bytes_opt(h, w, window, temporal_order, grid, opt);
  if (need < 0) return WH_EINVAL;
  int id;
  int cuda_idx;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->used + size_t(need) > srv->budget) return WH_EADMIT;
    srv->used += size_t(need);
    id = srv->next_stream++;
    cuda_idx = id % int(srv->cuda.size());
  }
  wh_stream* s = nullptr;
  int rc = wh_create_stream(h, w, window, temporal_order, grid, opt, srv->cuda[cuda_idx], &s);
  SStream st;
  if (rc == WH_OK) {
    st.s = s; st.h = h; st.w = w; st.bytes = size_t(need); st.cuda_idx = cuda_idx;
    const size_t fb = sizeof(float) * size_t(h) * w;
    st.pinned_in.resize(srv->queue_limit + 1, nullptr);
    for (auto& p : st.pinned_in)
      if (cudaMallocHost((void**)&p, fb) != cudaSuccess) rc = WH_ENOMEM;
    if (rc == WH_OK && srv->keep_results && cudaMallocHost((void**)&st.pinned_out, fb) != cudaSuccess)
      rc = WH_ENOMEM;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  if (rc != WH_OK) {
    srv->used -= size_t(need);
    for (float* p : st.pinned_in)
      if (p) cudaFreeHost(p);
    if (st.pinned_out) cudaFreeHost(st.pinned_out);
    if (s) wh_destroy_stream(s);
    return rc;
  }
  srv->streams[id] = std::move(st);
  *stream_id = id;
  return WH_OK;
}

int wh_server_submit(wh_server* srv, int stream_id, const float* frame, double arrival_s, long long* request_id) {
  if (!srv || !frame) return WH_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->streams.find(stream_id);
  if (it == srv->streams.end() || it->second.closing) return WH_EINVAL;
  SStream& st = it->second;
  srv->submitted += 1;
  if (srv->first_arrival < 0) srv->first_arrival = arrival_s;
  if (int(st.queue.size()) >= srv->queue_limit) {
    srv->shed += 1;
    return WH_EADMIT;
  }
  Request r;
  r.id = srv->next_req++;
  r.stream = stream_id;
  r.arrival = arrival_s;
  r.slot = st.ring;
  st.ring = (st.ring + 1) % int(st.pinned_in.size());
  std::memcpy(st.pinned_in[r.slot], frame, sizeof(float) * size_t(st.h) * st.w);
  st.queue.push_back(r.id);
  if (request_id) *request_id = r.id;
  srv->reqs[r.id] = std::move(r);
  lk.unlock();
  srv->cv_work.notify_all();
  return WH_OK;
}

double wh_server_now(wh_server* srv) { return srv ? srv->now() : 0.0; }

int wh_server_wait(wh_server* srv, long long request_id, float* whitened, double* latency_s) {
  if (!srv) return WH_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(request_id);
  if (it == srv->reqs.end()) return WH_EINVAL;
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::seconds(60), [&] { return it->second.finished; });
  if (!ok) return WH_ETIMEOUT;
  if (srv->error) return srv->error;
  Request& r = it->second;
  if (latency_s) *latency_s = r.done - r.arrival;
  if (whitened && !r.result.empty()) std::memcpy(whitened, r.result.data(), sizeof(float) * r.result.size());
  srv->reqs.erase(it);              // a request is returned once; the table stays bounded
  return WH_OK;
}

int wh_server_drain(wh_server* srv) {
  if (!srv) return WH_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::seconds(600), [&] {
    if (srv->error) return true;
    if (srv->inflight) return false;
    for (auto& kv : srv->streams)
      if (!kv.second.queue.empty()) return false;
    return true;
  });
  if (!ok) return WH_ETIMEOUT;
  return srv->error;
}

int wh_server_stats(wh_server* srv, double* p50_ms, double* p99_ms, double* mpix_per_s, long long* served,
                    long long* shed, long long* submitted) {
  if (!srv) return WH_EINVAL;
  std::lock_guard<std::mutex> lk(srv->mu);
  std::vector<double> l = srv->latencies;
  std::sort(l.begin(), l.end());
  auto q = [&](double f) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, size_t(f * (l.size() - 1) + 0.5))]; };
  if (p50_ms) *p50_ms = 1e3 * q(0.50);
  if (p99_ms) *p99_ms = 1e3 * q(0.99);
  const double span = srv->last_done - (srv->first_arrival < 0 ? 0 : srv->first_arrival);
  if (mpix_per_s) *mpix_per_s = span > 0 ? srv->pixels_served / span / 1e6 : 0.0;
  if (served) *served = srv->served;
  if (shed) *shed = srv->shed;
  if (submitted) *submitted = srv->submitted;
  return WH_OK;
}

int wh_server_close(wh_server* srv, int stream_id) {
  if (!srv) return WH_EINVAL;
  SStream st;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->streams.find(stream_id);
    if (it == srv->streams.end()) return WH_EINVAL;
    it->second.closing = true;
    srv->cv_done.wait_for(lk, std::chrono::seconds(60),
                          [&] { return !it->second.busy && it->second.queue.empty(); });
    st = std::move(it->second);
    srv->streams.erase(it);
    srv->used -= st.bytes;
  }
  if (st.s) wh_destroy_stream(st.s);
  for (float* p : st.pinned_in)
    if (p) cudaFreeHost(p);
  if (st.pinned_out) cudaFreeHost(st.pinned_out);
  return WH_OK;
}

int wh_server_destroy(wh_server* srv) {
  if (!srv) return WH_OK;
  wh_server_drain(srv);
  std::vector<int> ids;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    for (auto& kv : srv->streams) ids.push_back(kv.first);
  }
  for (int id : ids) wh_server_close(srv, id);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  if (srv->dispatcher.joinable()) srv->dispatcher.join();
  for (cudaStream_t c : srv->cuda) cudaStreamDestroy(c);
  delete srv;
  return WH_OK;
}

}  // extern "C"
