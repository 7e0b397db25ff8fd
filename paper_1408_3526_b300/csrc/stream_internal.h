// Internal definition of the stream object shared by the library's host
// files (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/whiten.h"
#include "common.cuh"

struct wh_stream {
  int H, W, M, K, Mz, B, mpz, L, precision, debug;
  double alpha, vmax, vstep;
  int tw, th, kpad;
  int device;
  cudaStream_t st;
  long long t;          // frames pushed
  int cur;              // observer buffer holding T_{t-1}
  float* obs[2];
  float* Astate;
  float* frame;
  float* whitened;
  float* vx;
  float* vy;
  int* vidx;
  wh::SpecTables* d_spec;
  int* d_hgather;
  float2* d_taby;
  float2* d_tabx;
  float* d_hw;
  float2* d_dump_win;
  float* d_dump_pow;
  float2* d_raw;
  float* d_rs;
  // tensor-core autocorrelation
  int use_tc, tc_mode, tc_bf16, kg, ntile;
  void* d_a16;
  float* d_l1;
  float* d_cval;
  int* d_cidx;
  void* d_table;
  int* d_err;
  int* d_nfb;
  // autocorrelation search with the whole contraction on tensor cores (default)
  int use_tcd;
  void* d_tcd_table;     // constant F16 operand
  int* d_ccount;         // [H*W] per-pixel code of listed grid points
  int* d_cand;           // [H*W][8] listed grid points
  unsigned long long* d_tcd_counts;   // [2] pixel-frames with listed points / whole grid
  // autocorrelation search with the separable stage on tensor cores
  int use_tcsep;
  int spec_f64;          // the precision form of the spectrum kernel (spatial sums in double)
  float* d_bop;          // its stage-1 operand (2048 floats)
  // learned-estimator features and learned velocity mode
  void* d_feat;          // BF16 [H*W][feat_ld]
  int feat_ld;
  int feat_n;            // features per pixel: M*M*Mz (mode 1) or one per mirror pair (mode 2)
  int feat_mode;
  int* d_fgather;        // [feat_n]
  struct wh_mlp* mlp;    // not owned
  float conf_thr;
  int* d_list;           // [H*W] pixels sent to the exact search
  int* d_nlist;          // [1]
  long long* d_nfb_total;// fallback pixels accumulated
  long long mlp_frames;
  // asynchronous pipelined push (wh_push_frame_async): two sets of frame and
  // output buffers (set 0 is the stream's own), copy streams and events
  struct Async {
    float* frame[2];
    float* w[2];
    float* vx[2];
    float* vy[2];
    cudaStream_t in, out;
    cudaEvent_t ev_in[2], ev_comp[2], ev_out[2];
    int used[2];               // the set's events have been recorded
    long long frame_of[2];     // frame index last pushed with the set
    int par;                   // set of the next push
  };
  Async* as;
  // frame pipeline (wh_params.pipeline): spectrum kernels on st_s, search and
  // PEF on st_p; the smoothed state alternates between Astate and Astate_alt
  int pipeline;
  cudaStream_t st_s, st_p;
  cudaEvent_t ev_user, ev_spec, ev_join, ev_pef[2];
  cudaEvent_t ev_feat;       // the search of the last frame has read the feature buffer
  int pef_used[2];
  int pipe_work;              // kernels were enqueued since the last join
  int user_sync;              // the state was (re)initialised on the caller's stream
  float* Astate_alt;
  // threshold detector scratch (wh_detect)
  void* d_det;
  size_t det_bytes;
  wh_detection* d_det_list;
  int det_list_cap;
  // per-kernel timing (wh_profile_enable)
  int prof;
  std::vector<cudaEvent_t> ev;   // 4 per timed frame
  size_t ev_used;
};

// error text of the calling thread (512 bytes), CUDA failure -> WH_ECUDA, launch counter
char* wh_error_buffer();
int wh_cuda_fail(cudaError_t e, const char* what);
// order the stream's own CUDA stream after its frame-pipeline work (no-op without the pipeline)
int wh_join_pipeline(wh_stream* s);
void wh_count_launches(long long n);
