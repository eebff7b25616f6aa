/*
 * crb.h -- C ABI of the GB300 (sm_103a) L.A.Cosmic cosmic-ray cleaner.
 *
 * The operation is the L.A.Cosmic work function that CRBLASTER runs on each
 * sub-image (Mighell, PASP 2010, Sec. 5; the algorithm is van Dokkum 2001),
 * one iteration repeated niter times ("typically 4 iterations", Sec. 5):
 *   (a) L+  : 2x block replication, 3x3 Laplacian [[0,-1,0],[-1,4,-1],[0,-1,0]],
 *             negatives set to 0, 2x2 average;
 *   (b) N   = sqrt(gain*med5(I) + readnoise^2)/gain,  S = L+/(2N),
 *       S'  = S - med5(S);
 *   (c) F   = med3(I) - med7(med3(I));
 *   (d) candidates where S' > sigclip and S'/max(F/N, 0.01) > objlim, grown over
 *       3x3 neighbours with S' > sigclip, then over 3x3 neighbours with
 *       S' > sigfrac*sigclip;
 *   (e) flagged pixels replaced by the lower median of the unflagged pixels of
 *       their 5x5 window (the 5x5 median of the frame when none is unflagged).
 * Flags accumulate over iterations. Every filter clamps its coordinates into
 * the frame (replicate edge); the paper leaves the outer pixels undefined
 * (Sec. 6.1). The method's arithmetic is IEEE float32 with no contraction.
 * The library also provides the paper's POISSON work function (Sec. 6.3.2;
 * crb_poisson), the probe the paper uses to measure its framework's overhead.
 *
 * Conventions for every call:
 *   - Images are float32 DN, row-major, contiguous (row pitch = w), DEVICE
 *     pointers. Masks are uint8 (0/1), same layout. The caller owns all buffers.
 *   - Sizes: 1 <= w, h; w*h < 2^31. Input must be finite (a NaN gives undefined
 *     output, never a fault).
 *   - Calls are asynchronous on `stream`: they validate, enqueue and return.
 *     Validation errors are returned synchronously. Device-side errors are
 *     latched in the context and reported by crb_sync_status().
 *   - A context is not thread-safe: use one per host thread (or lock).
 *   - Return value: CRB_OK or one of the error codes below.
 */
#ifndef CRB_H_
#define CRB_H_

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum crb_status {
  CRB_OK = 0,
  CRB_EINVAL = 1,   /* invalid argument (sizes, null pointers, parameters)        */
  CRB_ENOMEM = 2,   /* device memory could not be allocated                        */
  CRB_ECUDA = 3,    /* a CUDA runtime call failed (message in crb_last_error)      */
  CRB_ETIMEOUT = 4, /* a bounded device-side wait gave up                          */
  CRB_EBUSY = 5,    /* serving: admission refused (over budget or queue full)      */
  CRB_EALIAS = 6,   /* an output overlaps an input                                 */
  CRB_EDEVICE = 7   /* a device-side check failed (recorded, no access was made)   */
};

typedef struct crb_ctx crb_ctx;

/* Options of crb_create_ex. Zero-initialise, then set what differs. */
typedef struct {
  /* objlim statistic: 0 = S'/max(F/N, 0.01) (script form, default);
   *                   1 = 2S/max(F/N, 0.01), i.e. L+/F with F floored at 0.01 N (article form). */
  int objlim_form;
  /* 1: stop iterating once an iteration adds no flag and leaves no flagged pixel
   * without an unflagged neighbour; the result is then a fixed point, so the
   * output is identical to running all niter iterations. Default 0.            */
  int early_exit;
  /* Tile shape of the detection kernel (index of crb_tile_shape; default 0).
   * 0 takes 64 x 32 tiles, or the 64 x 28 tiles of index 5 (one image buffer,
   * three blocks per SM) when all of a call's tiles then fit in one round of
   * resident blocks and the 64 x 32 tiles do not (one 800 x 800 frame).
   * -1 = autotune: the first call with a new signature (the list of frame
   * sizes and niter) runs the clean once per compiled shape, timing each on
   * the stream (that call synchronises the stream), and keeps the fastest for
   * later calls with the same signature. */
  int tile_shape;
  /* 1: capture the work of a call (the memsets and the niter loop of launches)
   * in a CUDA graph once per launch signature and replay it afterwards; the
   * per-frame descriptors are uploaded before each replay. Ignored while
   * profiling. */
  int use_graphs;
  /* 1: bracket every kernel launch with CUDA events on the launching stream;
   * read the accumulated device times with crb_profile_read. Default 0.       */
  int profile;
  /* 1: run each iteration as two launches (detection, replacement) instead of
   * fusing the replacement of iteration k-1 into the detection of iteration k
   * (niter + 1 launches). Same results; for comparison. Default 0.            */
  int no_fusion;
  /* Detection pipeline. 2: queue pipeline -- a dense bound pass writes bit
   * planes, and the medians run in separate kernels over global work queues
   * of the positions that can change a flag; iterations after the first
   * recompute only near the pixels the previous replacement changed, and the
   * replacement runs in place in out_clean. 1: tile pipeline -- one kernel per
   * iteration does all stages of a tile in shared memory (the form used by
   * crb_iterate's map export and by crb_clean_noalloc). 0 (default): per
   * call, the queue pipeline from 6,000,000 pixels on (all frames of the call
   * together), the tile pipeline below: the queue pipeline's ~60 dependent
   * launches cost about 0.5 ms per call, the tile pipeline's cost is about 4.5
   * times more per pixel. All give identical results. */
  int pipeline;
  /* 1: autotune the queue pipeline. The first call with a new signature (the
   * list of frame sizes and niter) times trial cleans of its own frames on the
   * stream (that call synchronises the stream; about 15 cleans): four
   * occupancy levels (all, 3/4, 1/2 and 1/4 of each queue-pipeline kernel's
   * largest blocks per SM), each kernel keeping the level at which its own
   * launches took least device time; then the first iteration from which the
   * bit-plane kernels walk listed segments (2, 3, 4 or none); then, for calls
   * under 2^25 pixels with pipeline 0, the tile pipeline against the result.
   * Later calls with the same signature reuse the choice (crb_tuned_config
   * reports it). The launch configuration changes no result. Default 0. */
  int autotune;
  /* 1: in the tile pipeline, iterations 2 and 3 run as one launch (temporal
   * fusion): each 64 x 16 tile first runs iteration 2 over itself widened by
   * 32 columns and 8 rows each way (the halo iteration 3 needs: 6 for the
   * flags, 2 for the replacement), keeping that result in shared memory, then
   * iteration 3 on itself. One launch less, at the cost of recomputing the
   * widened ring; the other launches of such a call use 64 x 16 tiles too.
   * Needs niter >= 3 and fusion; otherwise ignored. Same results. The work
   * counters then leave out iteration 2's detection. Default 0. */
  int fuse2;
} crb_options;

/* Creates a context with the cleaning parameters (Sec. 5 lists gain, readn,
 * sigfrac, objlim; sigclip and niter as in lacos_im.cl). Returns NULL when
 * gain <= 0, readnoise < 0, sigclip <= 0, sigfrac <= 0, objlim <= 0 or
 * niter < 0 (see crb_last_error). niter == 0 copies the input and clears the
 * mask. The context owns its device workspace, graphs and tuning cache. */
crb_ctx* crb_create(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter);
crb_ctx* crb_create_ex(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter,
                       const crb_options* opts);
/* Waits for the context's last call, then frees its workspace, graphs, streams
 * and events. No counterpart in the paper (its actors hold no state between
 * images). NULL is ignored. */
void crb_destroy(crb_ctx* ctx);

/* Cleans one frame: img (device, w*h floats) -> out_clean (device, w*h floats,
 * must not overlap img: CRB_EALIAS) and out_mask (device, w*h bytes, 0/1, the
 * cumulative flags of all iterations). Enqueued on `stream`. The context's
 * workspace grows on demand (about 37 bytes per pixel with the default queue
 * pipeline). */
int crb_clean(crb_ctx* ctx, const float* img, int w, int h, float* out_clean, uint8_t* out_mask,
              cudaStream_t stream);

/* Cleans n frames of different sizes in one launch per stage and iteration
 * (a persistent tile loop over all frames). The paper's director hands every
 * actor a sub-image and gathers the results with no barrier between them
 * (Sec. 6.2); here the frames of one call are that set of work items, each
 * cleaned as by crb_clean. Arrays of length n in HOST memory:
 * imgs[i] (device, ws[i]*hs[i] floats), out_cleans[i], out_masks[i] (device).
 * gains / readnoises may be NULL (use the context's values) or give per-frame
 * values (> 0 and >= 0). The result of each frame equals crb_clean's. */
int crb_clean_batch(crb_ctx* ctx, int n, const float* const* imgs, const int* ws, const int* hs,
                    const float* gains, const float* readnoises, float* const* out_cleans,
                    uint8_t* const* out_masks, cudaStream_t stream);

/* crb_clean_batch for frames in HOST memory: imgs[i] (ws[i]*hs[i] floats) in,
 * out_cleans[i] and out_masks[i] out, all host pointers (page-locked memory,
 * e.g. cudaHostAlloc, lets the copies overlap the work). The frames are cut
 * into chunks of consecutive frames of about 1/8 of the pixels each; chunk k+1
 * is copied to the device while chunk k is cleaned and chunk k-1 is copied
 * back, on the context's own streams with four device staging slots, and
 * consecutive chunks are cleaned by the context and a second one it creates
 * (own workspace and stream), so that their kernels overlap (all allocated on
 * the first call and reused). Starts after the work already enqueued
 * on `stream`; `stream` waits for the last copy-out, so a synchronisation of
 * `stream` makes the host outputs valid. The results equal crb_clean_batch's on
 * the same frames; crb_last_counts / crb_last_work of this context then
 * describe its last chunk. CRB_ENOMEM when the staging buffers or the second
 * context cannot be created. */
int crb_clean_batch_host(crb_ctx* ctx, int n, const float* const* imgs, const int* ws, const int* hs,
                         const float* gains, const float* readnoises, float* const* out_cleans,
                         uint8_t* const* out_masks, cudaStream_t stream);

/* Allocation-free clean of one frame. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while they
 * run -- onboard or embedded pipelines that fix their memory plan at start-up,
 * latency-bound loops in which cudaMalloc/cudaFree would synchronise the
 * device, and processes whose device memory is owned by another allocator.
 * It takes the parameters of crb_create directly (no context) and computes
 * the same result as crb_clean with objlim_form 0 and the default tile shape.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * (one image buffer, the flag bits, the counters and the descriptor, about
 * 17 MB) is a fixed device array in the library, held by every GPU that loads
 * the library until the process exits.
 * Limits: w, h <= 16384, w*h <= 4194304 (4 Mpix, e.g. 2048x2048), niter <= 64;
 * larger frames return CRB_EINVAL with a message (use crb_clean).
 * The first call on a device, with that device current, loads the library's
 * device code there if that has not happened yet (CUDA loads modules lazily by
 * default), which commits the scratch array's memory on that device, looks up
 * the array's device address and sets the kernels' launch attributes. That
 * first call can therefore fail with CRB_ECUDA when the device has no room for
 * the scratch, and it may synchronise the device: make it once at start-up,
 * before any stream capture (a call with niter = 0 on a 1x1 frame does the
 * set-up and nothing else of note). Every call on a device uses the same
 * scratch, which keeps the previous call's contents (each call clears what
 * must start at zero): calls that overlap on the GPU -- on unordered streams
 * or from several host threads -- race and corrupt each other's results;
 * order them on one stream or with events. Calls on different devices are
 * independent. */
int crb_clean_noalloc(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter,
                      const float* img, int w, int h, float* out_clean, uint8_t* out_mask, cudaStream_t stream);

/* ---- The paper's 2-D image segmentation (Sec. 6.2, Sec. 6.3.1) --------------
 * CRBLASTER cuts a frame into N rectangular sub-images of nearly equal area and
 * widens each by BORDER pixels beyond every edge it shares with another, so
 * that its actors clean them with no communication. A rectangle here is its
 * interior (x0, y0, w, h) and its context region (cx0, cy0, cw, ch): the
 * interior widened by `context` pixels on each side, clipped to the frame. A
 * context of 8 * niter pixels makes the cleaned interior identical to that of
 * the whole-frame clean (every iteration's result depends on its input within
 * 8 pixels: 6 for the flags, 2 more for the replacement). */
typedef struct {
  int x0, y0, w, h;      /* interior */
  int cx0, cy0, cw, ch;  /* context region (contains the interior) */
} crb_rect;

/* The segmentation of a w x h frame into nparts = cols x rows rectangles, row
 * by row (rects[r * cols + c]); the first w % cols columns (h % rows rows) are
 * one pixel wider (taller). cols = 0 takes the factorisation whose sub-images
 * are closest to square (|log(aspect)| smallest, ties to fewer columns), the
 * paper's 2-D algorithm: a prime nparts gives 1 x nparts horizontal slices,
 * its 1-D scheme, which cols = 1 forces. Writes *out_cols, *out_rows (if not
 * NULL) and, when max_rects >= nparts, the rectangles; returns nparts, or
 * -CRB_EINVAL (sizes < 1, context < 0, cols not dividing nparts, or no cut that
 * fits the frame). Host only: needs no GPU. */
int crb_partition(int w, int h, int nparts, int cols, int context, crb_rect* rects, int max_rects, int* out_cols,
                  int* out_rows);

/* Cleans n rectangles of one frame img (device, w*h floats) as independent
 * frames, each its context region, and writes each rectangle's interior, only,
 * into out_clean and out_mask (device, w*h): the work of the paper's actors
 * and the director's assembly (Sec. 6.2) on one GPU. Rectangles whose
 * interiors tile the frame fill the outputs; with context >= 8 * niter (as
 * crb_partition gives) the result equals crb_clean's. The context region of
 * every rectangle must contain its interior and lie in the frame
 * (CRB_EINVAL); outputs must not overlap img (CRB_EALIAS). The crops go
 * through the context's own staging buffers (grown on demand) and one
 * crb_clean_batch. Asynchronous on `stream`. */
int crb_clean_rects(crb_ctx* ctx, const float* img, int w, int h, int n, const crb_rect* rects, float* out_clean,
                    uint8_t* out_mask, cudaStream_t stream);

/* Synchronises `stream` and returns the latched device status of the context
 * (CRB_OK, CRB_ETIMEOUT, CRB_EDEVICE or CRB_ECUDA), then clears it. No
 * counterpart in the paper (its MPI calls block until they complete). */
int crb_sync_status(crb_ctx* ctx, cudaStream_t stream);

/* After crb_sync_status: per-iteration counters of the last crb_clean /
 * crb_clean_batch / crb_iterate, summed over its frames: out[2k] = pixels newly
 * flagged in iteration k+1, out[2k+1] = flagged pixels with no unflagged 5x5
 * neighbour. Returns the number of iterations written (<= max_iter), or -1. */
int crb_last_counts(crb_ctx* ctx, long long* out, int max_iter);

/* After crb_sync_status: the work the detection kernels did in each iteration
 * of the last call, summed over its frames: out[6k..6k+5] = positions at which
 * they evaluated S (5x5 median of J), S' (5x5 median of S), med3, the
 * candidate test, the full 7x7 median of med3 for that test (the tests that
 * bounds of the median leave open; every test in the tile pipeline), and the
 * upper-bound test. The stages are evaluated only where they can change a
 * flag, so these counts are the method's work on this input. Returns the
 * number of iterations, or -1. */
int crb_last_work(crb_ctx* ctx, long long* out, int max_iter);

/* Kernel launches the last crb_clean / crb_clean_batch / crb_iterate enqueued
 * (memsets and copies not counted; a graph replay counts its kernels). The
 * queue pipeline launches 1 descriptor upload, 12 kernels in iteration 1, 14
 * in each later one (15 with the segment list, from the iteration the autotuner
 * or the default of 3 picks) and the mask kernel; the fused tile pipeline 1
 * upload and niter + 1 kernels.
 * -1 for a NULL context. */
int crb_last_launches(const crb_ctx* ctx);

/* One iteration from an explicit state, for stage-by-stage checks:
 * J (device, w*h floats) = I_{k-1}, Mprev (device, w*h bytes, may be NULL for
 * no flags) -> out_J = I_k, out_M = M_k (device). If maps is not NULL it
 * receives 11 float maps of w*h (device): floored m5, L+, N, S, S', m3, F, R,
 * cand, g1, g2 (F and R are computed only where S' > sigclip; NaN elsewhere). */
int crb_iterate(crb_ctx* ctx, const float* J, const uint8_t* Mprev, int w, int h, float* out_J,
                uint8_t* out_M, float* maps, cudaStream_t stream);

/* Profiling (crb_options.profile = 1): after the stream has been synchronised,
 * writes the total device time in milliseconds and the number of timed
 * brackets of the detection kernels (stages a-d) and of the replacement kernels
 * (stage e) since the last reset, then resets if reset != 0 (all kinds of
 * crb_profile_kernels). Returns CRB_OK or CRB_EINVAL (profiling off). */
int crb_profile_read(crb_ctx* ctx, double* detect_ms, int* detect_launches, double* replace_ms,
                     int* replace_launches, int reset);

/* Measures the FP32 min/max issue rate of the device (the ALU roofline of the
 * selection networks): a grid of independent fminf/fmaxf chains timed with
 * CUDA events on `stream` (synchronous). Writes min/max operations per second
 * for 2-input (ops2) and 3-input (ops3, counting each as one operation) forms.
 * Returns CRB_OK or CRB_ECUDA. A measurement aid for the roofline, not a
 * step of the method. */
int crb_alu_peak(double* ops2_per_s, double* ops3_per_s, cudaStream_t stream);

/* Measures the FP32 add issue rate the same way (independent add chains).
 * Writes adds per second. Returns CRB_OK or CRB_ECUDA. A measurement aid. */
int crb_fadd_peak(double* ops_per_s, cudaStream_t stream);

/* Profiling by kernel kind (crb_options.profile = 1): after the stream has been
 * synchronised, writes for up to max kinds the total device time in ms and the
 * number of timed brackets since the last reset (then resets if reset != 0).
 * Kinds, in order: 0 bound pass (iteration 1: the dense pass; later: the
 * segment list, the dilation of the changed pixels and the re-test), 1 need,
 * 2 S, 3 S', 4 m3need, 5 med3, 6 candidate tests, 7 growth, 8 reserved (no
 * kernel is timed under it), 9 tile-pipeline detection, 10 replacement,
 * 11 u8 mask, 12 tile-pipeline replacement, 13 work counters.
 * Returns the number of kinds written, or CRB_EINVAL. */
int crb_profile_kernels(crb_ctx* ctx, double* ms, int* brackets, int max, int reset);

/* Test aid for the device-side bounded waits (no counterpart in the paper):
 * enqueues on `stream` a kernel that waits, polls times at most (1 <= polls <=
 * 2^22), on a barrier that nothing completes -- as the tile kernels wait for
 * their TMA loads -- and records the timeout in the context's device status,
 * so that the next crb_sync_status returns CRB_ETIMEOUT. The context stays
 * usable. Returns CRB_OK or CRB_EINVAL. */
int crb_selftest_wait_timeout(crb_ctx* ctx, unsigned polls, cudaStream_t stream);

/* The launch configuration of the context's last call: blocks per SM of the
 * queue-pipeline kernels, in the order bound (dense), need, S, S', m3need,
 * med3, candidate test, replacement, bound re-test, replacement queue,
 * replacement write, changed-pixel dilation, full candidate test, growth,
 * flag queue and u8 mask, segment list, segment-form dilation, need and
 * m3need, m3need of iteration 1 (up to max of them); the first iteration of
 * the segment-list forms; the pipeline (1 tile, 2 queue). Returns the number of
 * kernels written, or CRB_EINVAL. A measurement aid, not a step of the method
 * (the paper has no counterpart). */
int crb_tuned_config(const crb_ctx* ctx, int* blocks_per_sm, int max, int* seg_from, int* pipeline);

/* Number of compiled tile shapes and their sizes (output tile of the detection kernel). */
int crb_num_tile_shapes(void);
int crb_tile_shape(int index, int* tile_w, int* tile_h);

/* ---- Serving: continuous batching of frames that arrive over time ----------
 * The paper's director collects each actor's result as soon as it is ready,
 * without a barrier (Sec. 6.2, 6.3.3). The server does the same on one GPU:
 * submitted frames are queued; a worker thread packs everything queued into
 * the next wave (one crb_clean_batch call, at most max_batch frames) whenever
 * one of max_inflight wave slots is free. Each slot has its own stream and
 * context, so waves overlap on the GPU. Frames and outputs are device buffers
 * owned by the caller, which keeps them resident until the frame is reported
 * done. Results are bit-identical to crb_clean on the same frame. */
typedef struct crb_server crb_server;

/* Creates a server with the cleaning parameters of crb_create_ex (opts may be
 * NULL). budget_bytes caps the device memory of the admitted, not yet done
 * frames, each counted as crb_server_frame_bytes(w, h) (input, output, mask
 * and workspace). 1 <= max_inflight <= 16, max_batch >= 1. NULL on error. */
crb_server* crb_server_create(float gain, float readnoise, float sigclip, float sigfrac, float objlim, int niter,
                              const crb_options* opts, size_t budget_bytes, int max_inflight, int max_batch);

/* Queues one frame (device pointers, as crb_clean) with its own gain and read
 * noise under an opaque tag. Returns CRB_OK; CRB_EBUSY when admitting it now
 * would exceed the budget (poll, then submit again); CRB_EINVAL for invalid
 * arguments and for a frame whose crb_server_frame_bytes alone exceed the
 * whole budget (it could never be admitted). An earlier device failure of the
 * server is returned as its status. Thread-safe. */
int crb_server_submit(crb_server* srv, const float* img, int w, int h, float gain, float readnoise,
                      float* out_clean, uint8_t* out_mask, uint64_t tag);

/* Moves up to max finished frames out of the server: their tags, and (if not
 * NULL) the seconds from submission to completion and their status. Waits up
 * to block_ms for at least one if none is finished. Returns the count, or -1. */
int crb_server_poll(crb_server* srv, uint64_t* done_tags, double* latency_s, int* status, int max, int block_ms);

/* Device bytes a w x h frame counts against the server budget: 9 per pixel of
 * the caller's buffers, 36 per pixel of workspace (4 float maps, 5 queue
 * entries), 14 bit planes, 8 bytes per cell of 32 x 8 pixels and 12 per
 * segment of 32 x 16 pixels (0 for invalid sizes). */
size_t crb_server_frame_bytes(int w, int h);

/* Counters: submitted, done, waves launched, largest wave, rejected submissions,
 * resident bytes, peak resident bytes, queued frames, the longest host time
 * spent enqueueing one wave (microseconds; the worker does not hold the
 * server's lock meanwhile) and the longest time a crb_server_submit waited for
 * that lock (microseconds). Returns the count written (at most 10). */
int crb_server_stats(crb_server* srv, long long* out, int max);

/* Stops the worker after the waves in flight complete and frees the server. */
void crb_server_destroy(crb_server* srv);

/* ---- The POISSON work function (Sec. 6.3.2) ---------------------------------
 * The paper measures the cost of its framework by swapping L.A.Cosmic for a
 * work function with a known, nearly equal load per pixel and no overlap
 * regions: each output pixel is a Poisson deviate whose mean is the input
 * pixel, drawn with Knuth's multiplicative method (Algorithm Q): uniforms are
 * multiplied until the product falls below e^-mu; the number of factors taken
 * before that is the deviate, so the cost per pixel grows linearly with mu.
 *
 * img, out: device, w*h floats, row-major; out receives the deviates (integer
 * values). out may equal img (each output depends only on its own input) but
 * must not overlap it otherwise. The uniforms come from SplitMix64 (golden
 * gamma 0x9e3779b97f4a7c15, Stafford's Mix13 finaliser) used as a
 * counter-based generator, value(s, j) = mix(s + (j+1)*gamma): pixel p
 * (row-major index in its frame) draws from the stream keyed by value(seed, p),
 * its j-th uniform being the top 53 bits of value(key, j) times 2^-53. e^-mu is
 * formed in double by fixed steps: -mu = n ln2 + r (ln2 rounded to double and
 * split at its low 20 significand bits), the Taylor polynomial of e^r to degree
 * 13 by Horner's rule with coefficients 1/i! by repeated division, times 2^n.
 * mu <= 0 or NaN gives 0; mu above 700 is taken as 700; at most 4096 factors
 * are drawn. Asynchronous on `stream`; no allocation. CRB_EINVAL for null
 * pointers or sizes outside 1 <= w, h and w*h < 2^31, CRB_ECUDA if the launch
 * fails. */
int crb_poisson(const float* img, int w, int h, uint64_t seed, float* out, cudaStream_t stream);

/* The POISSON work function on n frames in one launch per 256 frames: frame i
 * (imgs[i], ws[i] x hs[i], device) with seed seeds[i] into outs[i]; arrays in
 * host memory. Each frame's result equals crb_poisson's with the same seed. */
int crb_poisson_batch(int n, const float* const* imgs, const int* ws, const int* hs, const uint64_t* seeds,
                      float* const* outs, cudaStream_t stream);

/* Message of the last error on this host thread ("" if none). */
const char* crb_last_error(void);
const char* crb_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* CRB_H_ */
