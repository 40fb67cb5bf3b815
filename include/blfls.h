/*
 * blfls.h -- C ABI of the GB300 (sm_103a) BLF-LS edge-preserving smoother.
 *
 * BLF-LS ("Embedding Bilateral Filter in Least Squares for Efficient Edge-preserving Image
 * Smoothing", Section III-A) smooths an image f in two steps:
 *   (1) the bilateral filter of Eq. 1 is run on the periodic forward-difference gradients
 *       g_x = D_x f and g_y = D_y f (Section II-B operators), giving v_x, v_y;
 *   (2) the least-squares problem of Eq. 7,
 *           min_u  sum_s (u_s - f_s)^2 + lambda * sum_{*=x,y} (D_* u - v_*)_s^2,
 *       is solved in closed form in the Fourier domain (Eq. 8) under periodic boundaries.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Images are planar FP32, C channels of H x W, row-major, contiguous: element (c, y, x) is at
 * img[(c * H + y) * W + x]; x runs along W.  Channels are smoothed independently.
 * The bilateral window is the square of radius `radius` ((2r+1)^2 taps, centre included) with
 * periodic wrap; spatial weight exp(-(dx^2+dy^2) / (2 sigma_s^2)), range weight
 * exp(-(g_s - g_t)^2 / (2 sigma_r^2)) on the scalar field value (Eq. 1).  sigma_r = +INFINITY
 * drops the range weight (a truncated Gaussian blur of the gradients).
 * `iters` applies the whole smoother repeatedly: u_0 = img, u_k = BLFLS(u_{k-1}); iters = 0
 * copies img to out.
 *
 * Argument rules (checked on the host; a violation returns BLFLS_EINVAL and launches nothing):
 *   1 <= H, W <= BLFLS_MAX_DIM;  1 <= C <= BLFLS_MAX_CHANNELS;  radius >= 0 and
 *   2*radius + 1 <= min(H, W);  sigma_s > 0;  sigma_r > 0 (may be +INFINITY);
 *   lambda >= 0 and finite;  0 <= iters <= BLFLS_MAX_ITERS;  pointers non-NULL.
 *
 * Memory and streams: unless stated otherwise, image pointers are DEVICE pointers on the
 * handle's device, owned by the caller, and work is enqueued asynchronously on `stream`
 * (a cudaStream_t passed as void*; NULL is the legacy default stream).  The handle owns all
 * scratch memory (FFT twiddle/permutation tables, the per-channel gradient residuals and
 * spectrum) and grows it on demand, never beyond the budget given to blfls_create.
 * out may equal img (in-place).  A handle must not be used from two threads at once, and two
 * calls on the same handle must not run concurrently on different streams, because they share
 * the handle's scratch memory (enqueue them on one stream).
 *
 * Errors: every call returns a blfls_status; nothing aborts or traps.  blfls_last_error()
 * returns a human-readable message for the last failing call on the calling thread.
 */
#ifndef BLFLS_H
#define BLFLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLFLS_MAX_DIM 8192
#define BLFLS_MAX_CHANNELS 4
#define BLFLS_MAX_ITERS 64

typedef struct blfls_handle blfls_handle;

typedef enum {
    BLFLS_OK = 0,
    BLFLS_EINVAL = -1,   /* an argument broke the rules above */
    BLFLS_ENOMEM = -2,   /* the scratch memory would exceed the budget, or cudaMalloc failed */
    BLFLS_ECUDA = -3,    /* a CUDA runtime call or a kernel launch failed */
    BLFLS_ETIMEOUT = -4, /* a bounded device-side wait gave up (persistent work queue) */
    BLFLS_EBUSY = -5     /* the serving queue is full */
} blfls_status;

/* Arithmetic of the bilateral window (step 1).  The Fourier solve is FP32 in every mode.
 * FP16W/BF16W accept radius <= BLFLS_MAX_HALF_RADIUS (BLFLS_EINVAL above). */
typedef enum {
    BLFLS_FP32 = 0,  /* exponent, weights, products and sums in FP32 */
    BLFLS_FP16W = 1, /* gradient values, exponent, weights exp(.) and products w*g in FP16
                        (half2); each window column's sums in FP16, accumulated across columns
                        in FP32 */
    BLFLS_BF16W = 2  /* exponent in FP32; weights exp(.) computed and rounded in BF16
                        (bfloat162); products and sums in FP32 */
} blfls_precision;
#define BLFLS_MAX_HALF_RADIUS 16

/* Create a handle on CUDA device `device`.  mem_budget_bytes caps the scratch memory the
 * handle may allocate (0 = no cap).  tune_table_path names a tile-shape table written by the
 * autotuner (blfls_autotune); NULL or a missing file selects the built-in defaults.
 * On success *out receives the handle.  Errors: BLFLS_EINVAL (out NULL, bad device),
 * BLFLS_ECUDA. */
int blfls_create(blfls_handle **out, int device, size_t mem_budget_bytes,
                 const char *tune_table_path);

/* Free everything the handle owns, after waiting for its outstanding work.  NULL-safe. */
void blfls_destroy(blfls_handle *h);

/* Message of the last failing call on this thread ("" if none).  h may be NULL. */
const char *blfls_last_error(blfls_handle *h);

/* BLF-LS (Section III-A, Eqs. 1, 7, 8): out = BLFLS^iters(img).  Device pointers, async on
 * `stream`.  `prec` is a blfls_precision. */
int blfls_smooth(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                 float lambda, float sigma_s, float sigma_r, int radius, int iters, int prec,
                 void *stream);

/* The same smoother on HOST buffers: copies img to the device, smooths, copies the result to
 * out and waits for the stream.  img/out are host pointers; with pinned memory the uploads run
 * one channel at a time on the handle's own copy stream, each channel starts as soon as its
 * data has landed, the channels run side by side on streams of graded priority (so they finish
 * one after another), and each result is copied back on its channel's stream as soon as it is
 * done, under the remaining channels' work (when the budget has no room for per-channel
 * scratch, the channels run one after another on `stream`).  out may equal img.  The device
 * copies live in the handle's scratch memory. */
int blfls_smooth_host(blfls_handle *h, const float *img_host, float *out_host, int H, int W,
                      int C, float lambda, float sigma_s, float sigma_r, int radius, int iters,
                      int prec, void *stream);

/* ---- The LS model and the base/detail applications ------------------------------------ */

/* The LS model (Section II-B, Eqs. 5-6): u = F^-1[F(f) / (1 + lam (4 sin^2(pi kx / W) +
 * 4 sin^2(pi ky / H)))], the un-weighted quadratic smoother (BLF-LS with the guidance
 * gradients set to zero), applied `iters` times (0 copies).  Device pointers [C][H][W], async on
 * `stream`; out may equal img.  Errors: BLFLS_EINVAL (as blfls_smooth), BLFLS_ENOMEM,
 * BLFLS_ECUDA. */
int blfls_smooth_ls(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                    float lambda, int iters, void *stream);

typedef enum { BLFLS_DETAIL_ENHANCE = 0, BLFLS_LOG_TONE = 1 } blfls_layer_mode;
#define BLFLS_LOG_FLOOR 1e-6f

/* The base/detail applications of Section IV on top of the smoother (u = BLFLS^iters):
 *   BLFLS_DETAIL_ENHANCE: u = BLFLS^iters(f); out = f + strength (f - u): the detail layer
 *     f - u magnified by strength >= 0 and added back to the input;
 *   BLFLS_LOG_TONE: l = ln(max(f, BLFLS_LOG_FLOOR)); b = BLFLS^iters(l);
 *     out = exp(strength b + (l - b)): the base layer of the logarithmic image compressed by
 *     strength in [0, 1], the detail layer kept (the caller rescales the result for display).
 * Other arguments as blfls_smooth (iters >= 1); out may equal img; the handle keeps one
 * [C][H][W] scratch image.  Errors: BLFLS_EINVAL (unknown mode, strength out of range or not
 * finite, other arguments as blfls_smooth), BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_layers(blfls_handle *h, const float *img, float *out, int H, int W, int C, int mode,
                 float strength, float lambda, float sigma_s, float sigma_r, int radius,
                 int iters, int prec, void *stream);

/* ---- Joint (guided) BLF-LS and rolling guidance (Section III-D) -------------------------- */

#define BLFLS_MAX_GAUSS_SIGMA 32.0f

/* Joint BLF-LS: as blfls_smooth, but the range weights of the bilateral filter on each gradient
 * field compare that field of the guidance image's gradients (guide: device [Cg][H][W],
 * Cg = C, or Cg = 1 shared by every channel); the values averaged are the input's gradients,
 * as in a joint bilateral filter.  Pass k > 1 smooths the previous output with the same
 * guidance.  With sigma_r = +inf the guidance has no effect.  Radii up to
 * BLFLS_MAX_HALF_RADIUS run the tiled kernels in every precision; larger radii (FP32 only) a
 * per-pixel kernel.  out may equal img but not guide.  Errors: BLFLS_EINVAL (guide NULL, Cg
 * not 1 or C, out == guide, other arguments as blfls_smooth), BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_smooth_guided(blfls_handle *h, const float *img, const float *guide, float *out, int H,
                        int W, int C, int Cg, float lambda, float sigma_s, float sigma_r,
                        int radius, int iters, int prec, void *stream);

/* Rolling guidance: the first guidance is the input smoothed by the periodic Gaussian of
 * standard deviation sigma_g (blfls_gaussian); pass k is joint BLF-LS of the INPUT guided by
 * guidance k, and its output is guidance k + 1; out receives pass `iters` (iters = 0 copies).
 * out must not equal img (every pass reads the input).  Errors: BLFLS_EINVAL (out == img,
 * sigma_g outside (0, BLFLS_MAX_GAUSS_SIGMA], other arguments as blfls_smooth), BLFLS_ENOMEM,
 * BLFLS_ECUDA. */
int blfls_smooth_rolling(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                         float lambda, float sigma_s, float sigma_r, int radius, int iters,
                         float sigma_g, int prec, void *stream);

/* Periodic Gaussian blur, rows then columns, taps exp(-x^2 / (2 sigma^2)) for
 * |x| <= ceil(3 sigma) normalised to sum 1 (computed in FP64 on the host, stored FP32); device
 * [C][H][W] buffers, async; out may equal img.  Errors: BLFLS_EINVAL (sigma outside
 * (0, BLFLS_MAX_GAUSS_SIGMA], image arguments), BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_gaussian(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                   float sigma, void *stream);

/* ---- BLF-LS on normalised gradients (the paper's Section IV setting) -------------------- */

/* BLF-LS (Eqs. 7-8) with every gradient field normalised to [0, 1] before the bilateral filter
 * and restored after it, per channel and per field, in every pass (Section IV normalises images
 * and gradients to [0, 1]).  The filter of Eq. 1 is exact under an affine map of its field (the
 * weights sum to 1 and the range kernel sees only differences), so normalising a field of range
 * R = max - min and restoring it is the filter with sigma_r R on the raw field: this is what the
 * call computes, with R from the FP32 gradients (a constant field, R = 0, keeps sigma_r).  The
 * result does not change when the image is scaled by any factor (scaled by it).  Arguments,
 * precisions, radii and errors as blfls_smooth; device pointers [C][H][W], out may equal img.
 * The fields' ranges and the range constants derived from them are computed on the device, so
 * the call is asynchronous on `stream` like blfls_smooth (no host synchronisation); the channels
 * run one after another on `stream`. */
int blfls_smooth_normalized(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                            float lambda, float sigma_s, float sigma_r, int radius, int iters,
                            int prec, void *stream);

/* ---- BLF-LS with the bilateral-grid filter (the fast approximation the paper uses) -------- */

#define BLFLS_GRID_MAX_BYTES (8ull << 30)
#define BLFLS_GRID_MAX_RANGE_CELLS 65536

/* BLF-LS (Eqs. 7-8) with each gradient field filtered by the bilateral-grid approximation of
 * Eq. 1 (Paris and Durand's fast bilateral filter, which the paper's experiments use,
 * Sections III-A and IV): sampling steps sigma_s in space and sigma_r in range, a 2-cell zero
 * padding, splat to the nearest cell, 3-tap Gaussian blur of one cell along each grid axis,
 * trilinear slice; open image borders in the grid (the solve stays periodic).  FP32; a pixel's
 * cell is floor(t + 1/2) of the real value t of its coordinates for its FP32 gradient (taken in
 * FP64 where the FP32 value is near a rounding boundary).  Device pointers [C][H][W]; out may
 * equal img; asynchronous on `stream` (the fields' ranges, which fix the number of range cells,
 * stay on the device: the grid buffers hold a chunk of range levels sized from sigma_r for
 * fields of range up to 2, and a wider field is filtered chunk by chunk with the same result).
 * A field whose range spans more than BLFLS_GRID_MAX_RANGE_CELLS cells of sigma_r, or holds a
 * NaN, cannot be gridded: its channel's output is NaN.  sigma_s must be finite and >= 0.5;
 * sigma_r may be +inf (one range cell).  Errors: BLFLS_EINVAL (arguments as blfls_smooth
 * without radius and precision, sigma_s out of range, grid buffers above
 * BLFLS_GRID_MAX_BYTES), BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_smooth_grid(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                      float lambda, float sigma_s, float sigma_r, int iters, void *stream);

/* ---- NC-LS (Section III-D) -------------------------------------------------------------- */

#define BLFLS_MAX_NC_ITERS 8
#define BLFLS_MAX_NC_SIGMA_S 256.0f

/* NC-LS: BLF-LS with the bilateral filter on each gradient field replaced by the normalised
 * convolution of the domain transform (Section III-D): per field g, the transform
 * ct = running sum of 1 + (sigma_s / sigma_r) |g[j] - g[j-1]| along each row and each column
 * (periodic lines; computed once per pass from the unfiltered field), then nc_iters box
 * iterations of radius r_k = sigma_s sqrt(3) 2^(nc_iters-k) / sqrt(4^nc_iters - 1) sqrt(3) in the
 * transformed domain, rows then columns; then the Fourier solve of Eq. 8.  FP32 values.  Each
 * step of the transform is formed from the exact difference of the FP32 image's gradient samples
 * as a double-float (a = sigma_s / sigma_r in FP64) and held as an integer number of units of
 * 2^-q, rounded down, q the largest integer <= 30 with floor(r_1 2^q) + 1 < 2^32; sums of steps
 * are exact, so the samples in a box do not depend on the order of any sum, and they are exactly
 * those within r_k of its centre in the real-valued transform except where a distance lies
 * within (its number of steps) x 2^-q of r_k.  Device
 * pointers [C][H][W], async; out may equal img.  sigma_s in (0, BLFLS_MAX_NC_SIGMA_S]; sigma_r
 * > 0 (+inf: plain box iterations); nc_iters in [1, BLFLS_MAX_NC_ITERS] (3 is the usual choice).
 * Errors: BLFLS_EINVAL, BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_smooth_nc(blfls_handle *h, const float *img, float *out, int H, int W, int C,
                    float lambda, float sigma_s, float sigma_r, int iters, int nc_iters,
                    void *stream);

/* Step 1 alone (Eq. 1 on the gradients of Section II-B): for every channel,
 *   ex = f_BLF(D_x img) - D_x img,   ey = f_BLF(D_y img) - D_y img,
 * i.e. how far the bilateral filter moves each gradient field.  ex, ey: device [C][H][W]. */
int blfls_blf_residual(blfls_handle *h, const float *img, float *ex, float *ey, int H, int W,
                       int C, float sigma_s, float sigma_r, int radius, int prec, void *stream);

/* Step 2 alone (Eq. 8 in residual form): given guidance residuals e_* = v_* - D_* img,
 *   out = img + (I + lambda L)^-1 lambda (D_x^T ex + D_y^T ey),   L = D_x^T D_x + D_y^T D_y,
 * which equals Eq. 8 with v_* = D_* img + e_* (by linearity).  D^T are the backward
 * differences of Section II-B.  All pointers device [C][H][W]; out may equal img. */
int blfls_solve_residual(blfls_handle *h, const float *img, const float *ex, const float *ey,
                         float *out, int H, int W, int C, float lambda, void *stream);

/* One smoothing job of the batched and served forms. */
typedef struct {
    const float *img; /* device [C][H][W] */
    float *out;       /* device [C][H][W]; may equal img */
    int H, W, C;
    float lambda, sigma_s, sigma_r;
    int radius, iters;
    int prec; /* blfls_precision */
} blfls_job;

/* Batched form: smooth n independent jobs of uneven sizes and parameters with one launch per
 * pipeline phase (persistent kernels over a device work list).  Jobs are validated first; one
 * bad job fails the call with BLFLS_EINVAL before anything is enqueued.  Results equal those
 * of blfls_smooth on each job alone (same kernels, same arithmetic). */
int blfls_smooth_batch(blfls_handle *h, const blfls_job *jobs, int n, void *stream);

/* Served form on device buffers (the request loop around Eq. 7's solver): queue one job and
 * return at once with a ticket.  The job's img and out are DEVICE pointers owned by the caller:
 * img must already hold its data when blfls_submit is called (work that fills it must have
 * completed, e.g. its stream synchronised), and neither buffer may be touched or freed until
 * blfls_poll has reported the job done.  Jobs queued on a handle run in batches on the handle's
 * own queue -- continuous batching: whenever one of its two streams is free, every queued job
 * that fits (up to 64, within the queue's scratch budget) joins the next blfls_smooth_batch call,
 * so jobs submitted while others run are admitted as those finish and batches overlap on the
 * device.  The first call creates the queue: two internal handles with the calling handle's
 * launch shapes, and scratch reserved up front (the calling handle's budget, or 8 GiB when it has
 * none; a job that could never fit returns BLFLS_ENOMEM).  A job's result equals blfls_smooth on
 * it alone.  Arguments are validated here (BLFLS_EINVAL, as blfls_smooth).  blfls_destroy
 * cancels jobs not yet started and waits for running ones.  The queue is thread-safe: submit and
 * poll may be called from any thread, unlike the handle's other calls. */
int blfls_submit(blfls_handle *h, const blfls_job *job, uint64_t *ticket);
/* *done = 0 while the job is queued or running, 1 once it has finished and out holds the result.
 * The call that reports done also forgets the ticket (a later poll of it returns BLFLS_EINVAL);
 * if the job failed, that call returns the job's error (BLFLS_ECUDA, ...) with *done = 1.
 * Errors: BLFLS_EINVAL (NULL arguments, unknown ticket). */
int blfls_poll(blfls_handle *h, uint64_t ticket, int *done);

/* ---- Served form (no counterpart in the paper): continuous batching on one GPU ------------
 *
 * A server owns one device arena (a fixed share of mem_budget_bytes, allocated at creation) from
 * which every request's input and output buffers are carved, `slots` concurrent streams each
 * with its own resident handle (FFT plans and scratch, capped by the slot's share of the budget),
 * and a scheduler thread.  Requests carry HOST buffers.  Whenever a slot is free the scheduler
 * takes queued requests in arrival order, first fit -- a request joins the batch if its buffers
 * fit in the arena and the batch's scratch fits the slot -- up to max_batch of them, copies them
 * in, smooths them with one blfls_smooth_batch call and copies the results out, all on the
 * slot's stream, so batches on different slots overlap on the device.  A request's result is the
 * same as blfls_smooth on it alone.  Budget split: 60% arena, 35% slot scratch, 5% plans and
 * tables.  Latency is measured from submit to the result being in host memory. */
typedef struct blfls_server blfls_server;

typedef struct {
    const float *img_host; /* host [C][H][W]: read until the request completes */
    float *out_host;       /* host [C][H][W]: written when the request completes */
    int H, W, C;
    float lambda, sigma_s, sigma_r;
    int radius, iters;
    int prec; /* blfls_precision */
} blfls_request;

typedef struct {
    uint64_t submitted, completed, failed, cancelled, rejected;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> result in host memory */
    double megapixels;                      /* sum of H*W over completed requests */
    double busy_s;                          /* first submit -> last completion */
    double mp_per_s;                        /* megapixels / busy_s */
    size_t device_bytes_peak;               /* arena peak + handles' scratch and plans */
    size_t device_bytes_budget;
    int max_batch_seen;
} blfls_server_stats;

/* Create a server on `device` with 1..16 slots and batches of at most max_batch (1..1024)
 * requests; mem_budget_bytes >= 64 MiB.  Errors: BLFLS_EINVAL, BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_server_create(blfls_server **out, int device, size_t mem_budget_bytes, int slots,
                        int max_batch, const char *tune_table_path);
/* Cancel queued requests, finish running ones, free everything.  NULL-safe. */
void blfls_server_destroy(blfls_server *s);
/* Queue a request; returns at once with a ticket.  Arguments are validated here (BLFLS_EINVAL);
 * a request that could never fit the budget is rejected with BLFLS_ENOMEM.  The caller keeps
 * img_host and out_host alive until the request has finished or been cancelled. */
int blfls_server_submit(blfls_server *s, const blfls_request *r, uint64_t *ticket);
/* *state: 0 queued or running, 1 done, 2 cancelled, < 0 the error code it failed with. */
int blfls_server_poll(blfls_server *s, uint64_t ticket, int *state);
/* Wait up to timeout_ms for the request: BLFLS_OK when done, BLFLS_ETIMEOUT, or its error. */
int blfls_server_wait(blfls_server *s, uint64_t ticket, int timeout_ms);
/* Cancel a request that has not been admitted yet (BLFLS_EBUSY once it is running or done). */
int blfls_server_cancel(blfls_server *s, uint64_t ticket);
/* Forget a finished or cancelled request's record (BLFLS_EBUSY while queued or running). */
int blfls_server_release(blfls_server *s, uint64_t ticket);
int blfls_server_get_stats(blfls_server *s, blfls_server_stats *out);

/* Kernel timing (no counterpart in the paper; measurement support for the benchmark).
 * blfls_profile_begin pre-creates `max_events` CUDA events and starts recording an event pair
 * around every kernel launch the handle makes, on the launch's own stream.  Stages:
 * 0 = K1 bilateral residuals, 1 = K2 row FFTs, 2 = K3 column FFT / divide / inverse,
 * 3 = K4 row inverse FFTs.  blfls_profile_end waits for the recorded events and writes, per
 * stage, the summed device time in milliseconds (ms[4]) and the number of launches
 * (launches[4]); either pointer may be NULL.  Events beyond max_events are not recorded and
 * make blfls_profile_end return BLFLS_EINVAL. */
int blfls_profile_begin(blfls_handle *h, int max_events);
int blfls_profile_end(blfls_handle *h, double *ms, int *launches);

/* Autotuner (no counterpart in the paper; launch shapes only, results never change).  Times the
 * candidate K1 tile heights for (radius, prec) and the candidate K3 column blocks for columns of
 * length H on a synthetic H x W x C image generated on the device, keeps the fastest in the
 * handle (used by every later call on it), and, if table_path is not NULL, writes the handle's
 * whole table there as JSON (readable by blfls_create).  Synchronous; allocates temporary device
 * buffers of 3*H*W*C floats plus one spectrum (outside the handle's budget).
 * Errors: BLFLS_EINVAL (bad sizes, or an unwritable table_path), BLFLS_ENOMEM, BLFLS_ECUDA. */
int blfls_autotune(blfls_handle *h, int H, int W, int C, int radius, int prec,
                   const char *table_path);

/* Measured throughput of the arithmetic pipes the bilateral kernels use (no counterpart in the
 * paper; measurement support for the roofline).  On `device`, writes up to n of: rates[0] FP32
 * FFMA results, [1] packed fma.f32x2 FP32 results, [2] MUFU ex2.f32 results, [3] ex2.f16x2 FP16
 * results, [4] ex2.bf16x2 BF16 results, [5] packed fma.f16x2 FP16 results, [6] multiply-adds
 * of mma.sync m16n8k16 (FP16 inputs, FP32 accumulators) -- each per clock per SM, from clock64
 * cycle counts of one fully occupied block per SM.  Synchronous; allocates (and frees) a few bytes of device
 * memory.  Returns BLFLS_EINVAL for a bad device or rates == NULL. */
int blfls_pipe_rates(int device, double *rates, int n);

/* Device-side range checks (no counterpart in the paper; a stand-in for a memory checker).  A
 * library compiled with -DBLFLS_DEVICE_CHECKS (paper_1812_07122_gb300/build.py, debug=True)
 * checks the index arithmetic of its kernels at run time -- image tile loads and window reads
 * of the bilateral kernels, every FFT butterfly's buffer offsets, the solve drivers' global
 * indices, grid cells, NC tile indices -- and, instead of performing an access that would leave
 * its buffer, sets one bit per kind of check in a device word and skips it (no trap, no assert,
 * no wait).  This call waits for `device` to finish its work, then writes the OR of those words
 * since the last call to *word (bits: 0 tile load, 1 window read, 2 residual store, 3 FFT
 * stage, 4 solve global index, 5 grid cell, 6 NC tile) and clears them.  In a release build the
 * checks compile away and *word is always 0.  Errors: BLFLS_EINVAL (word NULL, bad device),
 * BLFLS_ECUDA. */
int blfls_device_checks(int device, unsigned int *word);

/* Step 2 without any device allocation (the paper has no counterpart; this is a deployment
 * variant of blfls_solve_residual).
 *
 * For callers that cannot call cudaMalloc/cudaFree: a plug-in whose host application owns all
 * device memory through its own arena, or a real-time video path that cannot afford an
 * allocation's possible device-wide synchronisation.  It computes exactly what
 * blfls_solve_residual computes, on the calling thread's current device and without a handle.
 * The caller passes inputs and outputs as usual (device pointers, [C][H][W] FP32); the scratch
 * (the half spectrum and the FFT tables) lives in one static device array of
 * BLFLS_NOALLOC_SPECTRUM_BYTES + BLFLS_NOALLOC_TABLE_BYTES bytes that every GPU loading this
 * library keeps until the process exits.
 *
 * Limits: 1 <= H, W <= BLFLS_NOALLOC_MAX_DIM and H * (W/2 + 1) * 8 <= BLFLS_NOALLOC_SPECTRUM_BYTES
 * (1024 x 1024 fits); larger sizes return BLFLS_EINVAL with a message and launch nothing.
 * No cudaMalloc, cudaFree or allocating library call is made.
 *
 * The first call on a device sets up that device (looks up the static array's device address,
 * the SM count and the kernels' shared-memory limits); make that first call before any stream
 * capture begins on the device.  The array holds the FFT tables of one size pair at a time: a
 * call whose size differs from the previous call's copies new tables into it from host memory,
 * ordered on `stream`, replacing the old ones for every later kernel that reads them; such a call
 * returns BLFLS_EINVAL and enqueues nothing while `stream` is capturing.
 * Every call shares the one array, which keeps the previous call's contents; each call
 * overwrites all of the scratch it reads.  Calls that overlap on the GPU (for example on two
 * streams of one device) race on the array: issue them on one stream, one after another.  The
 * host-side bookkeeping is protected by a lock, so calling from several threads is safe as long
 * as the GPU work itself does not overlap. */
#define BLFLS_NOALLOC_SPECTRUM_BYTES 4456448u /* 4.25 MiB: H * (W/2+1) <= 557056 */
#define BLFLS_NOALLOC_TABLE_BYTES 1048576u    /* 1 MiB of FFT tables */
#define BLFLS_NOALLOC_MAX_DIM 4096
int blfls_solve_residual_noalloc(const float *img, const float *ex, const float *ey, float *out,
                                 int H, int W, int C, float lambda, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BLFLS_H */
