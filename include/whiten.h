/*
 * whiten.h -- C ABI of the B300 clutter-whitening preprocessor.
 *
 * Method: H. L. Kennedy, "Parallel software implementation of recursive
 * multidimensional digital filters for point-target detection in cluttered
 * infrared scenes" (arXiv:1408.3526).  For every pixel of a frame stream the
 * library
 *   (a) updates a local 3-D spectrum recursively: a deadbeat observer bank
 *       over time and a sliding DFT (comb + resonator) over the M x M spatial
 *       window (Sec. 1; Eq. (6)-(7));
 *   (b) forms the high-passed, Hann-windowed power spectrum, its 3-D
 *       autocorrelation on the lz = 1 slice, smooths it over time and takes
 *       the background velocity as its peak (Sec. 2; Eq. (9)-(10));
 *   (c) applies the velocity-tuned frequency-sampling prediction-error
 *       filter and subtracts the predicted background (Eq. (1)-(5), (8)).
 *
 * Conventions (all calls):
 *   - Frames are float32 intensities, row-major [frame_h][frame_w]; x is the
 *     column (fast) axis, y the row axis.  A positive velocity moves content
 *     toward +x / +y by that many pixels per frame.
 *   - Reads outside the frame clamp to the edge pixel, so every pixel has an
 *     output; history before the first frame is zero.
 *   - The caller owns every buffer passed in; the library owns the device
 *     state and tables it allocates in wh_create_stream and frees in
 *     wh_destroy_stream.  Nothing is retained after a call returns except
 *     through the stream object.
 *   - Every call returns 0 (WH_OK) or a negative WH_E* status; nothing
 *     aborts and no C++ exception crosses this boundary.
 *   - Work is enqueued on the CUDA stream given at creation (NULL = the
 *     legacy default stream).  wh_push_frame is asynchronous; the wh_read_*
 *     calls with a host destination synchronise that stream before returning,
 *     with a device destination they only enqueue a device-to-device copy.
 *   - Pointers flagged is_device = 1 must be device pointers on the stream's
 *     device; is_device = 0 means pageable or pinned host memory.
 *   - A stream object must not be used from two threads at once.
 */
#ifndef WHITEN_H
#define WHITEN_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define WH_OK         0
#define WH_EINVAL    -1   /* bad argument: even or < 3 window, Mz < 2, grid step <= 0, h or w < 1,
                             h * w > 2^30, NULL */
#define WH_ENOMEM    -2   /* device or host allocation failed */
#define WH_EADMIT    -3   /* request exceeds the memory budget (serving admission) */
#define WH_ENOTREADY -4   /* output not available yet (fewer than m'_z + 1 frames pushed) */
#define WH_ECUDA     -5   /* a CUDA runtime call failed; the message is in wh_last_error() */
#define WH_ETIMEOUT  -6   /* a bounded device-side wait ran out (error flag set, no hang) */
#define WH_EUNSUP    -7   /* parameter combination not built into this library */

/* ---- precision / engine of the autocorrelation search ------------------- */
/* WH_PREC_FP32: FP32 recursion and the exact FP32 argmax of Eq. (10), by the
 *   separable evaluation on CUDA cores (default), or with WH_PREC_TC_SHORTLIST
 *   by a tcgen05 F16 contraction that shortlists peaks followed by an FP32
 *   re-evaluation of every shortlisted grid point within the rigorous F16
 *   error window (whole grid when the shortlist could be incomplete).
 * WH_PREC_TC_FP16 / WH_PREC_TC_BF16: precision study, the tensor-core F16 or
 *   BF16 contraction (F32 accumulation) decides alone.
 * WH_PREC_TC_SEPARABLE: the exact FP32 argmax by the separable evaluation
 *   with its first stage (T for every grid row, a [pixels x 32] x [32 x 2L]
 *   contraction) on tcgen05 tensor cores in TF32: the row upper bounds come
 *   from the tensor-core T widened by the TF32 error, and only the rows whose
 *   bound reaches the best row's exact value are evaluated in FP32 on CUDA
 *   cores, so the velocity is identical to the CUDA-core search's.  Windows
 *   5..15, grids up to 31 x 31.
 * WH_PREC_TC_DENSE: the exact FP32 argmax with the whole contraction of
 *   Eq. (10) on tcgen05 tensor cores: per pixel the state is scaled by a power
 *   of two and rounded to F16, C(l) and S(l) (R(l) = C + S, R(-l) = C - S) come
 *   from one F16 product with F32 accumulation over the half grid, and a grid
 *   point is decided by the tensor cores alone when it is the only one within
 *   the rigorous error window of the maximum; otherwise the (at most 8) points
 *   within it, or the whole grid, are evaluated exactly in FP32 with the
 *   CUDA-core search's operation sequence, so the velocity is identical to that
 *   search's.  Windows 5..15, grids up to 31 x 31; wh_stream_search_counts
 *   reports how many pixel-frames needed the exact evaluation.
 * WH_PREC_CUDA_CORES: the separable evaluation on CUDA cores only.
 * WH_PREC_SPEC_F64 (combinable with the search flags): the precision form of the
 *   recursive spectrum: the spatial sums (x-direction DFT, comb differences and
 *   y-direction resonator running sums, the box sums of the high-pass, the
 *   Hann convolution and the power) in double precision with double
 *   twiddles, the rounding that the comb/resonator pole-zero cancellation on
 *   the unit circle would otherwise accumulate (Sec. 1); the observer, the
 *   smoothed state and the search stay FP32.  Several times slower (one CTA
 *   per SM, the GPU's reduced FP64 rate); no learned-estimator features. */
#define WH_PREC_FP32          0
#define WH_PREC_TC_FP16       1
#define WH_PREC_TC_BF16       2
#define WH_PREC_CUDA_CORES    8
#define WH_PREC_TC_SHORTLIST 16
#define WH_PREC_TC_SEPARABLE 32
#define WH_PREC_SPEC_F64     64
#define WH_PREC_TC_DENSE    128

/* Velocity grid: {-vmax, -vmax + step, ..., +vmax} on both axes
 * (Sec. 3: l_x = l_y = [-8 .. 8]/4, a 17 x 17 grid at vmax = 2, step 1/4).
 * vmax must be an integer multiple of step; L = 2 vmax/step + 1 <= 31. */
typedef struct {
    float vmax;
    float step;
} wh_vgrid;

/* Optional parameters; a field left at its "default" value takes the
 * default shown.  Pass NULL to take every default. */
typedef struct {
    int    band;        /* B, PEF spatial half-bandwidth (Eq. (2), W = 2B+1); <= 0: round(M/3) */
    int    delay_z;     /* m'_z, output delay in frames; < 0: floor((Mz-1)/2) */
    double alpha;       /* smoother pole (Sec. 2 after Eq. (10)); < 0: exp(-1/10) */
    int    precision;   /* WH_PREC_* flags */
    int    debug_dump;  /* 1: keep the windowed spectrum and power of the last frame for
                           wh_read_spectrum (slow; tests only) */
    int    pipeline;    /* 1: overlap consecutive frames: the spectrum kernel of frame t+1
                           runs on an internal CUDA stream while the search and PEF of frame
                           t run on a second one (the smoothed state is double-buffered,
                           +kpad*4 bytes per pixel); results are identical to pipeline = 0.
                           With the learned estimator's features on, the spectrum of frame
                           t+1 also waits for the search of frame t (one feature buffer).
                           The work no longer runs on the caller's CUDA stream: the wh_read_*
                           calls and wh_detect order themselves after it, and raw pointers
                           from wh_output_pointers are valid after wh_stream_sync.
                           Default 0. */
} wh_params;

typedef struct wh_stream wh_stream;   /* opaque */

/* Fill *p with the defaults for a window M and order Mz. */
int wh_default_params(int window, int temporal_order, wh_params *p);

/*
 * Create a stream: allocate its device state (observer bank, smoothed
 * autocorrelation basis, outputs) and build its tables (SDFT twiddles, Hann
 * taps, Eq. (8)/(2) filter weights per grid velocity, Eq. (10) basis).
 *   frame_h, frame_w   frame size (>= 1 each, frame_h * frame_w <= 2^30)
 *   window             spatial window M = 2K+1 (odd, 3..15)
 *   temporal_order     Mz, temporal bins / observer states (2..8)
 *   velocity_grid      search grid for the autocorrelation peak (at most 31 points
 *                      per axis).  R(l) is periodic in l with period M, so a grid
 *                      with 2*vmax >= M holds exact duplicates of its maximum
 *                      (velocities equal modulo M), decided by rounding; keep
 *                      vmax <= (M-1)/2 for an unambiguous velocity.
 *   opt                NULL or optional parameters
 *   cuda_stream        a cudaStream_t (NULL = default stream); not owned
 *   out                receives the stream handle
 * Errors: WH_EINVAL, WH_EUNSUP, WH_ENOMEM, WH_ECUDA.
 */
int wh_create_stream(int frame_h, int frame_w, int window, int temporal_order,
                     wh_vgrid velocity_grid, const wh_params *opt, void *cuda_stream,
                     wh_stream **out);

/*
 * Push one frame (float32 [h][w]); runs the whole per-pixel path for it:
 * observer + spatial SDFT + high-pass + Hann + power + smoothing (Sec. 1-2,
 * Eq. (6)-(7) and (9)), the autocorrelation search (Eq. (10) on the lz = 1
 * slice, smoothed as described after Eq. (10)), and the prediction-error
 * filter (Eq. (1)-(2), equal to Eq. (4) with the coefficients of Eq. (8)).
 * Asynchronous on
 * the stream's CUDA stream; a host frame is copied first (the copy is done
 * before the call returns only if the memory is pageable).
 * Errors: WH_EINVAL (NULL), WH_ECUDA.
 */
int wh_push_frame(wh_stream *s, const float *frame, int is_device);

/*
 * Pipelined push for streaming from host memory: enqueues the copy of the
 * host frame to the device, the whole per-pixel path of wh_push_frame for it,
 * and the copies of its whitened pixel and velocity back to the host, then
 * returns without waiting.  The copies run on two internal CUDA streams and
 * the stream keeps two sets of device frame/output buffers, so the copies of
 * one frame overlap the kernels of the next (ordering by CUDA events).
 *   frame_host         float32 [h][w], page-locked host memory; must stay
 *                      unchanged until the frame has been consumed (after the
 *                      next call returns, or after wh_stream_sync)
 *   whitened_host      NULL or float32 [h][w] page-locked: the whitened pixel
 *                      of frame *frame_index - delay_z (zeros while fewer
 *                      than delay_z + 1 frames were pushed)
 *   vx_host, vy_host   NULL or float32 [h][w] page-locked: the velocity of
 *                      frame *frame_index
 *   frame_index        NULL or receives the index of the frame just pushed
 * The host outputs are complete once wh_stream_query_frame(s, index, 1) or
 * wh_stream_sync(s) returns WH_OK.  After asynchronous pushes, call
 * wh_stream_sync before wh_read_* with host destinations if their results
 * are needed in program order.  The paper has no counterpart (it is I/O
 * plumbing around Sec. 1-2's per-frame path).
 * Errors: WH_EINVAL (NULL), WH_ENOMEM (first call allocates the second
 * buffer set, 4 * h * w floats), WH_ECUDA.
 */
int wh_push_frame_async(wh_stream *s, const float *frame_host, float *whitened_host, float *vx_host,
                        float *vy_host, long long *frame_index);

/*
 * Wait until every kernel and copy enqueued on the stream (including
 * asynchronous pushes) has finished.  Returns WH_ETIMEOUT if a bounded
 * device-side wait gave up since the last check (the frame's results are then
 * not valid); the synchronising wh_read_* calls report it the same way.
 * Errors: WH_EINVAL (NULL), WH_ETIMEOUT, WH_ECUDA.
 */
int wh_stream_sync(wh_stream *s);

/*
 * Make the stream's CUDA stream (the one given at creation) wait, on the
 * device, for every kernel enqueued so far: with wh_params.pipeline = 1 the
 * kernels run on internal streams, and work the caller enqueues on its own
 * stream after this call (events, copies, kernels) sees all of them.  No
 * host synchronisation; a no-op without the pipeline.
 * Errors: WH_EINVAL (NULL), WH_ECUDA.
 */
int wh_stream_join(wh_stream *s);

/*
 * Whether the host outputs of frame frame_index (from wh_push_frame_async)
 * are complete: wait = 1 blocks until they are and returns WH_OK; wait = 0
 * returns WH_OK or WH_ENOTREADY.  Frames pushed with wh_push_frame report
 * WH_OK.
 * Errors: WH_EINVAL (NULL, or an index never pushed), WH_ECUDA.
 */
int wh_stream_query_frame(wh_stream *s, long long frame_index, int wait);

/* One detection of the threshold detector. */
typedef struct {
  int y, x;      /* pixel: row, column */
  float value;   /* whitened value E at the pixel */
  float vx, vy;  /* velocity (pixels/frame) that tuned the prediction-error filter there */
} wh_detection;

/*
 * Threshold detector on the latest whitened frame (the point-target detection
 * that the whitening prepares, Sec. 1; the paper's detector and tracker are
 * not specified further, the tracker is not part of this library): every
 * pixel with E >= k_sigma * sigma, sigma = RMS of E over the frame, in raster
 * order (row, then column), with the velocity of the same push (the one
 * used by the PEF that produced E).
 *   k_sigma     threshold in units of sigma (> 0)
 *   max_det     capacity of out; at most max_det entries are written
 *   out         wh_detection[max_det], device (is_device = 1) or host memory
 *   n_out       receives the number of pixels above the threshold (may exceed max_det)
 *   sigma_out   NULL or receives sigma
 *   frame_index NULL or receives the index of the whitened frame (t - delay_z)
 * Synchronises the stream.  Deterministic (fixed-order reductions).
 * Errors: WH_EINVAL, WH_ENOTREADY (fewer than delay_z + 1 frames), WH_ENOMEM, WH_ECUDA.
 */
int wh_detect(wh_stream *s, float k_sigma, int max_det, wh_detection *out, int *n_out,
              float *sigma_out, int is_device, long long *frame_index);

/*
 * Self-tests of the failure path (no fault, no hang).
 * wh_selftest_wait_timeout: runs one kernel whose bounded device-side wait
 * (the helper every waiting kernel of this library uses) waits for an
 * mbarrier phase that never completes; it gives up after limit_us
 * microseconds (1..1000000), records it in a device flag and returns.
 * Returns WH_ETIMEOUT when the timeout was detected (the expected result);
 * the CUDA context stays usable.
 * wh_stream_selftest_status: writes code into the stream's device status word
 * as a kernel whose wait gave up would; the next synchronising call reports
 * WH_ETIMEOUT once (code 0 clears it).
 * Errors: WH_EINVAL, WH_ENOMEM, WH_ECUDA.
 */
int wh_selftest_wait_timeout(int limit_us, void *cuda_stream);
int wh_stream_selftest_status(wh_stream *s, int code);

/*
 * Allocation-free variant of wh_push_frame.  The paper has no counterpart; it
 * exists for callers that cannot allocate device memory once streaming has
 * started (fixed-memory real-time loops, allocation-free pools, hosts that
 * forbid driver allocations after start-up).  Same arguments, same outputs
 * (read with wh_read_whitened / wh_read_velocity) and the same FP32-exact
 * velocity as wh_push_frame; its autocorrelation search always uses the
 * tensor-core shortlist with exact FP32 re-evaluation, and that search's
 * scratch lives in one statically sized device array of the library (about
 * 10.2 MB, held by every GPU that loads the library until the process exits)
 * instead of memory allocated per call or per stream.  Nothing is allocated.
 *   Limits: window <= 15 and grid length L <= 25 (WH_EUNSUP otherwise, with a
 *   message in wh_last_error); frames of any size (processed in chunks); not
 *   with the frame pipeline (WH_EUNSUP).  A stream in learned mode still gets
 *   the exact search here (the network is not run).
 *   Sharing: all calls on a device share the array and leave their contents
 *   in it; calls that overlap on the GPU (different CUDA streams or host
 *   threads) race, so serialise them.  No part of the array needs to start at
 *   zero (each call writes everything it reads).
 *   Errors on the device: a bounded wait that gives up sets the stream's own
 *   status word, so the next synchronising call (wh_read_*, wh_stream_sync)
 *   returns WH_ETIMEOUT, as after wh_push_frame.  After wh_push_frame_async on
 *   the same stream the call first waits (on the device) for its output copies.
 *   Frames pushed here are not timed by wh_profile_* and not counted by
 *   wh_stream_learned_stats.
 *   Set-up: the first call on a device looks up the array's device address;
 *   make that first call before any stream capture.
 * Errors: WH_EINVAL, WH_EUNSUP, WH_ECUDA.
 */
int wh_push_frame_noalloc(wh_stream *s, const float *frame, int is_device);

/*
 * Whitened (prediction-error) frame E for frame index t - m'_z, where t is
 * the index of the last frame pushed (first frame = 0), written to
 * out[h][w]: E = I(n - m') - I^(n - m') with the prediction of Eq. (1)/(4),
 * delayed by the temporal part m'_z of the filter delay m' (Sec. 2, Eq. (2);
 * Sec. 3 uses m' = K).  *frame_index (may be NULL) receives t - m'_z.
 * Errors: WH_ENOTREADY before m'_z + 1 frames, WH_EINVAL, WH_ECUDA.
 */
int wh_read_whitened(wh_stream *s, float *out, int is_device, long long *frame_index);

/*
 * Background velocity estimate of the last frame pushed, in pixels/frame:
 * vx[h][w], vy[h][w] (either may be NULL): v^ = l^/lz with l^ the grid point
 * of the largest smoothed autocorrelation on the lz = 1 slice (Sec. 2,
 * Eq. (10) and the text after it).  vidx (may be NULL) receives the
 * flat grid index iy*L + ix (int32 [h][w]) with vx = -vmax + ix*step.
 * *frame_index receives t.  Errors: WH_ENOTREADY before the first frame.
 */
int wh_read_velocity(wh_stream *s, float *vx, float *vy, int *vidx, int is_device,
                     long long *frame_index);

/* Spectrum kinds for wh_read_spectrum. */
#define WH_SPEC_RAW       0  /* S(k; n) of Eq. (6)-(7), from the observer state */
#define WH_SPEC_WINDOWED  1  /* high-passed, Hann-windowed spectrum (needs debug_dump) */
#define WH_SPEC_POWER     2  /* P(k; n) of Eq. (9) (needs debug_dump; real, float32) */

/*
 * Per-pixel spectrum of the last frame pushed, layout [h][w][Mz][M][M] with
 * bins kz = -((Mz-1)/2) .. Mz/2, ky, kx = -K .. K (slowest to fastest);
 * complex64 interleaved (re, im) for RAW and WINDOWED, float32 for POWER.
 * Errors: WH_ENOTREADY, WH_EINVAL (kind needs debug_dump), WH_ECUDA.
 */
int wh_read_spectrum(wh_stream *s, int kind, void *out, int is_device);

/*
 * Smoothed autocorrelation R'(l; n) of the last frame on the velocity grid,
 * float32 [h][w][L][L] (ly slowest), recomputed from the stream's smoothed
 * spectral state (Sec. 2: R is linear in P).  For tests and diagnostics.
 * The recomputation evaluates every grid value (the per-frame search skips
 * rows that provably hold no maximum) and rewrites the velocity field of the
 * last frame from it; the values are identical, so wh_read_velocity before
 * and after compares the two searches.  The library allocates the H*W*L*L
 * float buffer on first use and keeps it until the stream is destroyed.
 * Errors: WH_ENOTREADY (no frame pushed), WH_EINVAL, WH_ENOMEM, WH_ECUDA.
 */
int wh_read_autocorr(wh_stream *s, float *out, int is_device);

/*
 * The constant stage-1 operand of the tensor-core separable search
 * (WH_PREC_TC_SEPARABLE), for inspection and tests; host only, no GPU needed.
 * Writes 64 x 32 floats: row n = 2 gy + c holds the coefficients of Re T (c = 0)
 * or Im T (c = 1) of grid row gy (l = -vmax + gy * step) in T(kx, l) =
 * sum_ky Q(kx, ky) e^{j2pi ky l/M} (the separable form of Eq. (10)), as
 * functions of a pixel's Q sums: column 4 (ky - 1) + {0, 1, 2, 3} for
 * Q(kx, ky) +- Q(kx, -ky) (real sum, real difference, imaginary sum,
 * imaginary difference), ky = 1..K, column 28 / 29 for Re / Im Q(kx, 0);
 * values rounded to TF32 and stored in the tensor cores' 128-byte-swizzled
 * K-major layout (element (n, k) at n * 32 + ((k / 4) ^ (n % 8)) * 4 + k % 4).
 *   window      M (odd, 5..15); grid_len L (odd, <= 31); step the grid step
 * Returns 0, or -1 (WH_EINVAL) for arguments out of range.
 */
int wh_tcsep_operand(int window, int grid_len, double step, float *out);

/* Grid length L and the output delay m'_z of a stream. */
int wh_stream_info(const wh_stream *s, int *grid_len, int *delay_z, int *band,
                   long long *frames_pushed);

/* Counters: pixel-frames whose tensor-core shortlist could be incomplete and
 * were evaluated on the whole grid (WH_PREC_TC_SHORTLIST only; else 0). */
int wh_stream_stats(wh_stream *s, long long *fallback_pixels);

/* Counters of the default search engine (the whole contraction of Eq. (10)
 * on tensor cores; zero for the other engines), accumulated since the stream
 * was created: pixel-frames whose F16 tensor-core values left 2..8 grid
 * points within the rigorous error window of the maximum (those points were
 * evaluated exactly in FP32), and pixel-frames evaluated exactly on the whole
 * grid (more points, or a non-finite or subnormal-range state).  Every other
 * pixel-frame was decided by the tensor-core product alone. */
int wh_stream_search_counts(wh_stream *s, long long *listed_pixels, long long *whole_grid_pixels);

/* Device pointers of the stream's output buffers (valid until destroy):
 * whitened[h][w], vx[h][w], vy[h][w] (float32), vidx[h][w] (int32).
 * Any argument may be NULL.  Lets a device consumer read outputs in place. */
int wh_output_pointers(wh_stream *s, float **whitened, float **vx, float **vy, int **vidx);

/*
 * Per-kernel timing for measurement: when enabled, wh_push_frame records CUDA
 * events on the stream around each of its kernels (spectrum, autocorrelation
 * search, prediction-error filter).  wh_profile_read synchronises the stream
 * and returns, per kernel, the summed device time in ms (ms[3]) and the number
 * of timed launches (n[3]); reset = 1 clears the accumulators.  At most 65536
 * frames are kept between reads; later frames are not timed.
 */
int wh_profile_enable(wh_stream *s, int on);
int wh_profile_read(wh_stream *s, double *ms, long long *n, int reset);

/*
 * Tensor-core GEMM (tcgen05, F32 accumulation in tensor memory):
 *   C[M][N] = A[M][K] * B[N][K]^T (+ bias[N]) (then GELU if gelu = 1),
 * A and B row-major with K contiguous (leading dimensions lda, ldb >= K,
 * rows 16-byte aligned), both F16 (bf16 = 0) or both BF16 (bf16 = 1).  C is
 * float32 (out_bf16 = 0) or BF16 (out_bf16 = 1) with leading dimension ldc.
 * All pointers are device pointers; the call runs on cuda_stream and
 * synchronises it to read the kernel's error flag.  This is the contraction
 * engine of the learned velocity estimator and of the tensor-core
 * autocorrelation (Eq. (10) as [pixels x bins] x [bins x grid]).
 * Errors: WH_EINVAL (shapes, alignment), WH_ETIMEOUT (a bounded device wait ran
 * out), WH_ECUDA.
 */
int wh_tc_gemm(const void *A, int lda, const void *B, int ldb, void *C, int ldc, int M, int N, int K,
               int bf16, int out_bf16, const float *bias, int gelu, void *cuda_stream);

/*
 * Same contraction with a row-wise selection epilogue: for every row of C and
 * every 128-column tile, the 4 largest values among the first n_valid columns
 * (ties to the lowest column), written to cand_val/cand_idx[M][ceil(N/128)][4]
 * (device pointers).  Used to shortlist autocorrelation peaks.
 */
int wh_tc_gemm_topk(const void *A, int lda, const void *B, int ldb, int M, int N, int K, int bf16,
                    int n_valid, float *cand_val, int *cand_idx, void *cuda_stream);

/* ---- learned velocity estimator --------------------------------------------
 * An MLP n_in -> h1 -> h2 -> n_out (GELU) on each pixel's log-power spectrum
 * predicts (vx, vy, confidence logit); it is trained on velocities produced by
 * the plain search and, in a stream's learned mode, replaces the search for
 * pixels whose confidence reaches a threshold (the rest still run the exact
 * search).  The paper's method is the plain search (Sec. 2, Eq. (10)); the
 * network is an addition of this library.  BF16 weights and activations,
 * FP32 accumulation on tensor cores, FP32 master weights, AdamW.
 */
typedef struct wh_mlp wh_mlp;

/* Create with weights drawn U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from 'seed'.
 * h1, h2 multiples of 8, n_out <= 16 (3 for the velocity head). */
int wh_mlp_create(int n_in, int h1, int h2, int n_out, unsigned long long seed, void *cuda_stream,
                  wh_mlp **out);
int wh_mlp_destroy(wh_mlp *m);
/* Number of parameters: W1 [h1][n_in], b1, W2 [h2][h1], b2, W3 [n_out][h2], b3. */
long long wh_mlp_num_params(const wh_mlp *m);
/* Copy all parameters (in the order above, row-major, float32) to / from a
 * host buffer of wh_mlp_num_params floats; get_grads copies the gradients of
 * the last wh_mlp_train_step in the same layout. */
int wh_mlp_get_params(wh_mlp *m, float *host, long long n);
int wh_mlp_set_params(wh_mlp *m, const float *host, long long n);
int wh_mlp_get_grads(wh_mlp *m, float *host, long long n);
/* Inference: x BF16 [n][ldx] (device, ldx % 8 == 0, columns >= n_in ignored),
 * y float32 [n][ldy] (device; first n_out columns written; may be NULL). */
int wh_mlp_forward(wh_mlp *m, const void *x, int ldx, int n, float *y, int ldy);
/* One training step on n samples (n % 8 == 0): x BF16 [n][ldx], target float
 * [n][2] velocity labels (device).  Loss = |v - t|^2 + BCE(sigmoid(c), tc) with
 * tc = 1 when max(|vx-tx|, |vy-ty|) <= vstep.  apply = 0 computes gradients
 * only; stats (host, 4 floats, may be NULL: then the call does not
 * synchronise) receives mean loss, mean squared velocity error, mean BCE and
 * the fraction within one step. */
int wh_mlp_train_step(wh_mlp *m, const void *x, int ldx, int n, const float *target, float vstep,
                      float lr, float weight_decay, int apply, float *stats);

/* Per-pixel features for the network: (log2(P(k)/sum_k P(k) + 1e-6) + 10)/10 of the
 * high-passed, Hann-windowed power, sum over all M*M*Mz bins, order [kz][ky][kx]
 * as in wh_read_spectrum, BF16 rows of stride *ld (padding zero).
 * set_features(1): all M*M*Mz bins.  set_features(2): one feature per mirror
 * pair, since P(-k) = P(k) for a real input (Eq. (9)): the bins k whose flat
 * index is not larger than that of -k (kz -> -kz mod Mz, ky -> -ky, kx -> -kx),
 * in increasing order: (M*M*Mz + 2 - Mz % 2) / 2 features (676 at 15 x 15 x 6);
 * a network on them equals one on all bins whose first-layer columns of k and
 * -k are summed.  0 turns features off.  Every push then writes them; read
 * copies the last frame's.  In learned mode the layout follows the network's
 * input width. */
int wh_stream_set_features(wh_stream *s, int enable);
int wh_read_features(wh_stream *s, void *out, int is_device, int *ld);
/* Learned velocity mode: per frame the network (not owned; must outlive its
 * use) runs on every pixel; a pixel whose confidence sigmoid(c) >= threshold
 * takes the network's velocity rounded to the grid, every other pixel runs
 * the exact autocorrelation search.  mlp = NULL returns to the plain mode.
 * The network's forward runs on the stream's own CUDA stream (its search
 * stream with the frame pipeline).  Its activation and output buffers are
 * shared (the selection reads the output rows in place), so one network
 * serves one stream at a time: streams pushing concurrently from different
 * CUDA streams need a network each. */
int wh_stream_set_learned(wh_stream *s, wh_mlp *mlp, float conf_threshold);
/* Frames processed in learned mode and pixel-frames sent to the search. */
int wh_stream_learned_stats(wh_stream *s, long long *frames, long long *fallback_pixels);

/* ---- multi-stream serving --------------------------------------------------
 * Many sensor streams of different sizes and parameters share one GPU; each
 * stream's recursive state stays resident on the device.  The paper processes
 * one stream; this runtime is an addition of the library.
 *   open    admits a stream if its device footprint (wh_stream_device_bytes)
 *           fits in what is left of the budget, else WH_EADMIT.
 *   submit  queues one frame (host memory, copied into a pinned slot) with its
 *           arrival time on the server clock (wh_server_now); a stream with
 *           queue_limit frames already waiting rejects it with WH_EADMIT
 *           (back-pressure; counted as shed).
 *   A dispatcher thread keeps up to max_inflight frames on the GPU, oldest
 *   arrival first among streams whose previous frame has left the queue; each
 *   stream runs on one of n_cuda_streams CUDA streams, so different streams'
 *   frames overlap on the device while one stream's frames stay in order.
 *   wait    blocks until a request completes; returns its whitened frame
 *           (if keep_results) and its latency = completion - arrival.  Each
 *           request is returned once and then forgotten (a second wait on
 *           the same id returns WH_EINVAL).  The result is copied off the
 *           stream's pinned buffer by the dispatcher thread, not inside the
 *           CUDA host callback.
 *   stats   p50/p99 latency of served frames, served Mpixel/s between the
 *           first arrival and the last completion, served/shed/submitted.
 */
typedef struct wh_server wh_server;
long long wh_stream_device_bytes(int h, int w, int window, int temporal_order, wh_vgrid grid);
/* The same with the stream's optional parameters (NULL = defaults): adds the
 * frame pipeline's second smoothed-state buffer, the tensor-core shortlist's
 * scratch, the separable search's operand and the debug dump.  wh_server_open
 * admits a stream against this figure. */
long long wh_stream_device_bytes_opt(int h, int w, int window, int temporal_order, wh_vgrid grid,
                                     const wh_params *opt);
int wh_server_create(double hbm_budget_bytes, int max_inflight, int queue_limit, int n_cuda_streams,
                     int keep_results, wh_server **out);
int wh_server_open(wh_server *srv, int h, int w, int window, int temporal_order, wh_vgrid grid,
                   const wh_params *opt, int *stream_id);
int wh_server_submit(wh_server *srv, int stream_id, const float *frame, double arrival_s,
                     long long *request_id);
double wh_server_now(wh_server *srv);
int wh_server_wait(wh_server *srv, long long request_id, float *whitened, double *latency_s);
int wh_server_drain(wh_server *srv);
int wh_server_stats(wh_server *srv, double *p50_ms, double *p99_ms, double *mpix_per_s,
                    long long *served, long long *shed, long long *submitted);
int wh_server_close(wh_server *srv, int stream_id);
int wh_server_destroy(wh_server *srv);

/* Reset the recursive state to zero (as if no frame had been pushed). */
int wh_reset_stream(wh_stream *s);

/* Free everything the stream owns.  NULL is accepted (no-op). */
int wh_destroy_stream(wh_stream *s);

/* Human-readable text of a status code (static storage). */
const char *wh_status_string(int status);

/* Text of the last CUDA error seen on this thread (static per thread). */
const char *wh_last_error(void);

/* Number of this library's kernels launched since load (all streams). */
long long wh_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* WHITEN_H */
