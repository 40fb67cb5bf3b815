// C ABI of the BLF-LS smoother (declarations and contracts in include/blfls.h).
//
// A handle owns the FFT plans (per transform length), the per-channel scratch (the two gradient
// residual planes of step 1 and the half spectrum of step 2) and, for the host-buffer entry
// point, device copies of the image.  Calls validate on the host, grow scratch when needed
// (within the byte budget), then enqueue for every iteration and channel:
//   K1 (bilateral residuals) -> K2 (row FFTs) -> K3 (column FFTs, divide, inverse) -> K4 (row
//   inverse FFTs, u = f + correction).
#include "blfls.h"
#include "handle.h"
#include "nvtx_range.h"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>

using namespace blfls;


namespace {
thread_local std::string g_last_error;
}  // namespace

int blfls::fail(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int blfls::cuda_fail(cudaError_t e, const char* where)
{
    return fail(BLFLS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool blfls::budget_allows(blfls_handle* h, size_t extra)
{
    return h->budget == 0 || h->used + extra <= h->budget;
}

int blfls::grow_bytes(blfls_handle* h, void** ptr, size_t* cap_bytes, size_t need, const char* what)
{
    if (need <= *cap_bytes) return BLFLS_OK;
    const size_t old_bytes = *cap_bytes, new_bytes = need;
    if (!budget_allows(h, new_bytes - old_bytes))
        return fail(BLFLS_ENOMEM, std::string("scratch for ") + what + " exceeds the memory budget");
    if (*ptr) {
        cudaFree(*ptr);  // waits for work still using it
        h->used -= old_bytes;
        *ptr = nullptr;
        *cap_bytes = 0;
    }
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, new_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BLFLS_ENOMEM, std::string("cudaMalloc for ") + what + ": " + cudaGetErrorString(e));
    }
    *ptr = p;
    *cap_bytes = need;
    h->used += new_bytes;
    h->generation++;
    return BLFLS_OK;
}

namespace {
template <typename T>
int grow(blfls_handle* h, T*& ptr, size_t& cap, size_t need, const char* what)
{
    void* p = ptr;
    size_t bytes = cap * sizeof(T);
    const int rc = blfls::grow_bytes(h, &p, &bytes, need * sizeof(T), what);
    ptr = static_cast<T*>(p);
    cap = bytes / sizeof(T);
    return rc;
}
}  // namespace

int blfls::get_plan(blfls_handle* h, int N, const FftPlanDev** out)
{
    auto it = h->plans.find(N);
    if (it == h->plans.end()) {
        FftPlanHost p;
        const cudaError_t e = build_fft_plan(N, p);
        if (e != cudaSuccess) return cuda_fail(e, "FFT plan");
        if (!budget_allows(h, p.bytes)) {
            free_fft_plan(p);
            return fail(BLFLS_ENOMEM, "FFT plan exceeds the memory budget");
        }
        h->used += p.bytes;
        it = h->plans.emplace(N, p).first;
    }
    *out = &it->second.dev;
    return BLFLS_OK;
}

int blfls::check_image_args(const void* a, const void* b, int H, int W, int C)
{
    if (!a || !b) return fail(BLFLS_EINVAL, "image pointer is NULL");
    if (H < 1 || W < 1 || H > BLFLS_MAX_DIM || W > BLFLS_MAX_DIM)
        return fail(BLFLS_EINVAL, "H and W must lie in [1, BLFLS_MAX_DIM]");
    if (C < 1 || C > BLFLS_MAX_CHANNELS) return fail(BLFLS_EINVAL, "C must lie in [1, BLFLS_MAX_CHANNELS]");
    return BLFLS_OK;
}

int blfls::check_blf_args(int H, int W, float sigma_s, float sigma_r, int radius, int prec)
{
    if (radius < 0 || 2LL * radius + 1 > (long long)std::min(H, W))
        return fail(BLFLS_EINVAL, "radius must satisfy 0 <= radius and 2*radius+1 <= min(H, W)");
    if (!(sigma_s > 0.f)) return fail(BLFLS_EINVAL, "sigma_s must be > 0");
    if (!(sigma_r > 0.f)) return fail(BLFLS_EINVAL, "sigma_r must be > 0");
    if (prec < BLFLS_FP32 || prec > BLFLS_BF16W) return fail(BLFLS_EINVAL, "unknown precision");
    if (prec != BLFLS_FP32 && radius > BLFLS_MAX_HALF_RADIUS)
        return fail(BLFLS_EINVAL, "the FP16W/BF16W forms support radius <= BLFLS_MAX_HALF_RADIUS");
    return BLFLS_OK;
}

int blfls::check_lambda(float lambda)
{
    if (!(lambda >= 0.f) || !std::isfinite(lambda)) return fail(BLFLS_EINVAL, "lambda must be finite and >= 0");
    return BLFLS_OK;
}

void blfls::set_last_error(const std::string& msg) { g_last_error = msg; }

// The residual planes ex/ey share one capacity; keep them in lock-step.
static int ensure_residual_planes(blfls_handle* h, size_t plane)
{
    if (plane <= h->e_cap && h->ex && h->ey) return BLFLS_OK;
    const size_t old_bytes = 2 * h->e_cap * sizeof(float), new_bytes = 2 * plane * sizeof(float);
    if (!budget_allows(h, new_bytes - std::min(old_bytes, new_bytes)))
        return fail(BLFLS_ENOMEM, "scratch for gradient residuals exceeds the memory budget");
    if (h->ex) cudaFree(h->ex);
    h->used -= old_bytes;
    h->ex = h->ey = nullptr;
    h->e_cap = 0;
    void* p = nullptr;
    const cudaError_t e = cudaMalloc(&p, new_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BLFLS_ENOMEM, std::string("cudaMalloc for gradient residuals: ") + cudaGetErrorString(e));
    }
    h->ex = static_cast<float*>(p);
    h->ey = h->ex + plane;
    h->e_cap = plane;
    h->used += new_bytes;
    h->generation++;
    return BLFLS_OK;
}

static int prepare(blfls_handle* h, int H, int W, int radius, bool need_blf, bool need_solve,
                   const FftPlanDev** rp, const FftPlanDev** cp)
{
    int rc;
    const size_t plane = (size_t)H * W;
    if ((rc = ensure_residual_planes(h, plane)) != BLFLS_OK) return rc;
    if (need_blf && radius > blf_tiled_max_radius())
        if ((rc = grow(h, h->gscratch, h->g_cap, 2 * plane, "gradients")) != BLFLS_OK) return rc;
    if (need_solve) {
        if ((rc = grow(h, h->spec, h->spec_cap, (size_t)H * (W / 2 + 1), "spectrum")) != BLFLS_OK) return rc;
        if ((rc = get_plan(h, W, rp)) != BLFLS_OK) return rc;
        if ((rc = get_plan(h, H, cp)) != BLFLS_OK) return rc;
    }
    return BLFLS_OK;
}

// Take the next pre-created profiling event and record it on s; -1 when profiling is off or the
// pool is exhausted.
static int prof_mark(blfls_handle* h, cudaStream_t s)
{
    if (!h->prof_on) return -1;
    if (h->prof_next >= h->prof_pool.size()) {
        h->prof_overflow = true;
        return -1;
    }
    const int i = int(h->prof_next++);
    cudaEventRecord(h->prof_pool[i], s);
    return i;
}

static void prof_span(blfls_handle* h, int stage, int a, int b)
{
    if (a >= 0 && b >= 0) h->prof_spans.push_back({stage, {a, b}});
}

// K1 on `C` channels with optional timing.
static cudaError_t blf_launch(blfls_handle* h, const float* img, float* ex, float* ey, int C,
                              const BlfParams& bp, cudaStream_t s)
{
    const int a = prof_mark(h, s);
    const cudaError_t e = launch_blf_residual(img, ex, ey, C, bp, h->gscratch, s);
    prof_span(h, 0, a, prof_mark(h, s));
    return e;
}

// K2-K4 on one channel with optional timing.
static cudaError_t solve_launch(blfls_handle* h, const float* f, const float* ex, const float* ey,
                                float* out, const FftPlanDev& rp, const FftPlanDev& cp,
                                const SolveParams& sp, cudaStream_t s, float2* spec = nullptr)
{
    const int a = prof_mark(h, s);
    cudaEvent_t marks[2];
    int mi[2] = {-1, -1};
    const bool timed = a >= 0 && h->prof_next + 3 <= h->prof_pool.size();
    if (timed) {
        mi[0] = int(h->prof_next++);
        mi[1] = int(h->prof_next++);
        marks[0] = h->prof_pool[mi[0]];
        marks[1] = h->prof_pool[mi[1]];
    }
    const cudaError_t e = launch_solve_residual(f, ex, ey, out, spec ? spec : h->spec, rp, cp, rp.lap, cp.lap, sp,
                                                s, h->num_sms, timed ? marks : nullptr);
    const int b = timed ? prof_mark(h, s) : -1;
    if (timed) {
        prof_span(h, 1, a, mi[0]);
        prof_span(h, 2, mi[0], mi[1]);
        prof_span(h, 3, mi[1], b);
    } else if (h->prof_on) {
        h->prof_overflow = true;
    }
    return e;
}

// The passes of one channel (the channels of an image are filtered and solved independently),
// with the given residual planes and spectrum.
static int run_channel(blfls_handle* h, const float* img, float* out, const BlfParams& bp,
                       const SolveParams& sp, const FftPlanDev& rp, const FftPlanDev& cp,
                       int iters, cudaStream_t s, float* ex = nullptr, float* ey = nullptr,
                       float2* spec = nullptr)
{
    if (!ex) {
        ex = h->ex;
        ey = h->ey;
    }
    for (int it = 0; it < iters; ++it) {
        const float* src = (it == 0) ? img : out;
        const NvtxRange range("pass");
        cudaError_t e = blf_launch(h, src, ex, ey, 1, bp, s);
        if (e != cudaSuccess) return cuda_fail(e, "bilateral kernel launch");
        e = solve_launch(h, src, ex, ey, out, rp, cp, sp, s, spec);
        if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
    }
    return BLFLS_OK;
}

// Scratch and streams for running the channels of an image side by side: channels 1..C-1 get
// their own residual planes and spectrum (channel 0 uses the handle's), every channel its own
// stream.  Returns false (and the caller runs the channels one after another on its stream)
// when the memory budget has no room or a stream or event cannot be made.
static bool ensure_channel_slots(blfls_handle* h, int C, size_t plane, size_t spec_elems)
{
    const size_t per = 2 * plane + 2 * spec_elems;   // ex, ey, then the spectrum as floats
    const size_t need = per * (size_t)(C - 1);
    if (need > h->chan_cap) {
        const size_t old_bytes = h->chan_cap * sizeof(float), new_bytes = need * sizeof(float);
        if (!budget_allows(h, new_bytes - std::min(old_bytes, new_bytes))) return false;
        if (h->chan_scratch) cudaFree(h->chan_scratch);
        h->used -= old_bytes;
        h->chan_scratch = nullptr;
        h->chan_cap = 0;
        void* p = nullptr;
        if (cudaMalloc(&p, new_bytes) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        h->chan_scratch = static_cast<float*>(p);
        h->chan_cap = need;
        h->used += new_bytes;
    }
    while ((int)h->chan_streams.size() < C) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return false;
        h->chan_streams.push_back(st);
    }
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    while ((int)h->chan_streams_graded.size() < C) {
        const int c = (int)h->chan_streams_graded.size();
        const int prio = std::min(least, greatest + c);   // lower number = higher priority
        cudaStream_t st;
        if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess) return false;
        h->chan_streams_graded.push_back(st);
    }
    while ((int)h->chan_done.size() < C) {
        cudaEvent_t ev;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return false;
        h->chan_done.push_back(ev);
    }
    if (!h->chan_fork && cudaEventCreateWithFlags(&h->chan_fork, cudaEventDisableTiming) != cudaSuccess)
        return false;
    return true;
}

// The passes of every channel side by side, each channel on its own stream (one channel's
// latency-bound solve overlaps another channel's bilateral kernel); ordered after the work
// queued on `s` before the call, and `s` waits for all of it.  `in_ready[c]`, when given, is an
// event the channel's first kernel waits for; `done[c]` receives each channel's end.
static int run_channels_concurrent(blfls_handle* h, const float* img, float* out, int C,
                                   size_t plane, size_t spec_elems, const BlfParams& bp,
                                   const SolveParams& sp, const FftPlanDev& rp,
                                   const FftPlanDev& cp, int iters, cudaStream_t s,
                                   const cudaEvent_t* in_ready, const cudaEvent_t* done,
                                   const std::vector<cudaStream_t>& streams)
{
    cudaEventRecord(h->chan_fork, s);
    for (int c = 0; c < C; ++c) {
        cudaStream_t sc = streams[c];
        cudaStreamWaitEvent(sc, h->chan_fork, 0);
        if (in_ready) cudaStreamWaitEvent(sc, in_ready[c], 0);
        float *ex = nullptr, *ey = nullptr;
        float2* spec = nullptr;
        if (c > 0) {
            float* base = h->chan_scratch + (size_t)(c - 1) * (2 * plane + 2 * spec_elems);
            ex = base;
            ey = base + plane;
            spec = reinterpret_cast<float2*>(base + 2 * plane);
        }
        const int rc = run_channel(h, img + c * plane, out + c * plane, bp, sp, rp, cp, iters, sc,
                                   ex, ey, spec);
        if (rc != BLFLS_OK) return rc;
        cudaEventRecord(h->chan_done[c], sc);
        if (done) cudaEventRecord(done[c], sc);
        cudaStreamWaitEvent(s, h->chan_done[c], 0);
    }
    return BLFLS_OK;
}

int blfls::run_smooth(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                      float lambda, float sigma_s, float sigma_r, int radius, int iters, int prec,
                      cudaStream_t s)
{
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        if (out != img) {
            const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                                  cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "copy for iters = 0");
        }
        return BLFLS_OK;
    }
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    int rc = prepare(h, H, W, radius, true, true, &rp, &cp);
    if (rc != BLFLS_OK) return rc;
    const BlfParams bp{H, W, radius, sigma_s, sigma_r, prec, tuned_tile_h(h, radius, prec)};
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    const size_t spec_elems = (size_t)H * (W / 2 + 1);
    // Channels side by side: one channel's latency-bound solve overlaps another channel's
    // bilateral kernel.  Radii that use the shared gradient scratch run in order, and so does a
    // profiled call (its per-kernel spans must not overlap).
    if (C > 1 && !h->prof_on && radius <= blf_tiled_max_radius() &&
        ensure_channel_slots(h, C, plane, spec_elems))
        return run_channels_concurrent(h, img, out, C, plane, spec_elems, bp, sp, *rp, *cp, iters,
                                       s, nullptr, nullptr, h->chan_streams);
    for (int c = 0; c < C; ++c)
        if ((rc = run_channel(h, img + c * plane, out + c * plane, bp, sp, *rp, *cp, iters, s)) != BLFLS_OK)
            return rc;
    return BLFLS_OK;
}

// blfls_smooth_host: channel c is computed on the caller's stream while the copy stream uploads
// the channels after it and downloads the channels before it.
static int smooth_host_pipelined(blfls_handle* h, const float* img_host, float* out_host, int H,
                                 int W, int C, float lambda, float sigma_s, float sigma_r,
                                 int radius, int iters, int prec, cudaStream_t s)
{
    const size_t plane = (size_t)H * W;
    const size_t n = plane * C;
    int rc;
    if ((rc = grow(h, h->io, h->io_cap, 2 * n, "host-buffer staging")) != BLFLS_OK) return rc;
    float* dimg = h->io;
    float* dout = h->io + n;
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare(h, H, W, radius, true, true, &rp, &cp)) != BLFLS_OK) return rc;
    const BlfParams bp{H, W, radius, sigma_s, sigma_r, prec, tuned_tile_h(h, radius, prec)};
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    cudaError_t e = cudaSuccess;
    if (!h->copy_stream) {
        e = cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            h->copy_stream = nullptr;
            return cuda_fail(e, "copy stream");
        }
    }
    while ((int)h->io_events.size() < 2 * C + 1) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "copy events");
        h->io_events.push_back(ev);
    }
    cudaStream_t cs = h->copy_stream;
    cudaEvent_t* ev_in = h->io_events.data();
    cudaEvent_t* ev_done = ev_in + C;
    cudaEvent_t ev_fin = ev_in[2 * C];
    // The copy stream starts after whatever the caller queued on s before this call.
    if ((e = cudaEventRecord(ev_fin, s)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, ev_fin, 0)) != cudaSuccess)
        return cuda_fail(e, "stream ordering");
    for (int c = 0; c < C; ++c) {
        e = cudaMemcpyAsync(dimg + c * plane, img_host + c * plane, plane * sizeof(float),
                            cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
        if ((e = cudaEventRecord(ev_in[c], cs)) != cudaSuccess) return cuda_fail(e, "event record");
    }
    // Channels side by side (as in run_smooth) when the scratch fits and no profile runs.
    const size_t spec_elems = (size_t)H * (W / 2 + 1);
    const bool par = C > 1 && !h->prof_on && radius <= blf_tiled_max_radius() &&
                     ensure_channel_slots(h, C, plane, spec_elems);
    if (par) {
        // Graded priorities make the channels finish one after another, and each channel's
        // result goes back on the channel's own stream as soon as it is done, so all but the
        // last copy run under the remaining channels' compute.
        if ((rc = run_channels_concurrent(h, dimg, dout, C, plane, spec_elems, bp, sp, *rp, *cp,
                                          iters, s, ev_in, ev_done, h->chan_streams_graded)) != BLFLS_OK)
            return rc;
        for (int c = 0; c < C; ++c) {
            cudaStream_t sc = h->chan_streams_graded[c];
            e = cudaMemcpyAsync(out_host + c * plane, dout + c * plane, plane * sizeof(float),
                                cudaMemcpyDeviceToHost, sc);
            if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
            if ((e = cudaEventRecord(h->chan_done[c], sc)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(s, h->chan_done[c], 0)) != cudaSuccess)
                return cuda_fail(e, "stream ordering");
        }
    } else {
        for (int c = 0; c < C; ++c) {
            if ((e = cudaStreamWaitEvent(s, ev_in[c], 0)) != cudaSuccess) return cuda_fail(e, "stream wait");
            if ((rc = run_channel(h, dimg + c * plane, dout + c * plane, bp, sp, *rp, *cp, iters, s)) != BLFLS_OK)
                return rc;
            if ((e = cudaEventRecord(ev_done[c], s)) != cudaSuccess) return cuda_fail(e, "event record");
            if ((e = cudaStreamWaitEvent(cs, ev_done[c], 0)) != cudaSuccess) return cuda_fail(e, "stream wait");
            e = cudaMemcpyAsync(out_host + c * plane, dout + c * plane, plane * sizeof(float),
                                cudaMemcpyDeviceToHost, cs);
            if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
        }
    }
    if ((e = cudaEventRecord(ev_fin, cs)) != cudaSuccess || (e = cudaStreamWaitEvent(s, ev_fin, 0)) != cudaSuccess)
        return cuda_fail(e, "stream ordering");
    return BLFLS_OK;
}

// The queue behind blfls_submit: two slots (batches on two streams overlap), batches of up to
// 64 jobs, scratch from the handle's budget or 8 GiB when the handle has none.
constexpr size_t kSubmitDefaultBudget = (size_t)8 << 30;
constexpr int kSubmitSlots = 2;
constexpr int kSubmitMaxBatch = 64;

namespace blfls {
// The check words of the translation units with device range checks (dcheck.cuh).
unsigned int dcheck_fetch_blf_f32();
unsigned int dcheck_fetch_blf_f16();
unsigned int dcheck_fetch_blf_bf16();
unsigned int dcheck_fetch_blf_kernels();
unsigned int dcheck_fetch_solve_kernels();
unsigned int dcheck_fetch_grid();
unsigned int dcheck_fetch_nc();
}  // namespace blfls

extern "C" {

int blfls_device_checks(int device, unsigned int* word)
{
    if (!word) return fail(BLFLS_EINVAL, "word is NULL");
    *word = 0;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(BLFLS_EINVAL, "no such CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize");
    *word = dcheck_fetch_blf_f32() | dcheck_fetch_blf_f16() | dcheck_fetch_blf_bf16() |
            dcheck_fetch_blf_kernels() | dcheck_fetch_solve_kernels() | dcheck_fetch_grid() |
            dcheck_fetch_nc();
    return BLFLS_OK;
}

int blfls_create(blfls_handle** out, int device, size_t mem_budget_bytes,
                 const char* tune_table_path)
{
    if (!out) return fail(BLFLS_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(BLFLS_EINVAL, "no such CUDA device");
    DeviceGuard g(device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    blfls_handle* h = new blfls_handle();
    h->device = device;
    h->budget = mem_budget_bytes;
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    init_blf_kernel_attributes();
    init_solve_kernel_attributes();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "kernel attributes");
    }
    load_tune_table(h, tune_table_path);
    *out = h;
    return BLFLS_OK;
}

void blfls_destroy(blfls_handle* h)
{
    if (!h) return;
    blfls_server_destroy(h->submit_srv);   // cancels queued jobs, finishes running ones
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    for (cudaEvent_t ev : h->prof_pool) cudaEventDestroy(ev);
    for (cudaEvent_t ev : h->io_events) cudaEventDestroy(ev);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    destroy_batch_state(h->batch);
    for (auto& kv : h->plans) free_fft_plan(kv.second);
    if (h->ex) cudaFree(h->ex);
    if (h->spec) cudaFree(h->spec);
    if (h->gscratch) cudaFree(h->gscratch);
    if (h->io) cudaFree(h->io);
    if (h->layer) cudaFree(h->layer);
    if (h->gtmp) cudaFree(h->gtmp);
    if (h->grid_a) cudaFree(h->grid_a);
    if (h->grid_keys) cudaFree(h->grid_keys);
    if (h->kap_dev) cudaFree(h->kap_dev);
    if (h->nc_scratch) cudaFree(h->nc_scratch);
    if (h->chan_scratch) cudaFree(h->chan_scratch);
    for (cudaStream_t st : h->chan_streams) cudaStreamDestroy(st);
    for (cudaStream_t st : h->chan_streams_graded) cudaStreamDestroy(st);
    for (cudaEvent_t ev : h->chan_done) cudaEventDestroy(ev);
    if (h->chan_fork) cudaEventDestroy(h->chan_fork);
    delete h;
}

const char* blfls_last_error(blfls_handle* h)
{
    (void)h;
    return g_last_error.c_str();
}

int blfls_smooth(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                 float lambda, float sigma_s, float sigma_r, int radius, int iters, int prec,
                 void* stream)
{
    const NvtxRange range("blfls_smooth");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    return run_smooth(h, img, out, H, W, C, lambda, sigma_s, sigma_r, radius, iters, prec,
                      static_cast<cudaStream_t>(stream));
}

int blfls_smooth_host(blfls_handle* h, const float* img_host, float* out_host, int H, int W,
                      int C, float lambda, float sigma_s, float sigma_r, int radius, int iters,
                      int prec, void* stream)
{
    const NvtxRange range("blfls_smooth_host");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img_host, out_host, H, W, C)) != BLFLS_OK) return rc;
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (iters > 0) {
        rc = smooth_host_pipelined(h, img_host, out_host, H, W, C, lambda, sigma_s, sigma_r, radius,
                                   iters, prec, s);
        if (rc != BLFLS_OK) return rc;
    } else if (out_host != img_host) {
        const size_t n = (size_t)H * W * C;
        const cudaError_t e = cudaMemcpyAsync(out_host, img_host, n * sizeof(float),
                                              cudaMemcpyHostToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "copy for iters = 0");
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return BLFLS_OK;
}

int blfls_smooth_ls(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                    float lambda, int iters, void* stream)
{
    const NvtxRange range("blfls_smooth_ls");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        if (out == img) return BLFLS_OK;
        const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "copy for iters = 0");
    }
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare(h, H, W, 0, false, true, &rp, &cp)) != BLFLS_OK) return rc;
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int c = 0; c < C; ++c)
        for (int it = 0; it < iters; ++it) {
            const float* src = (it == 0 ? img : out) + c * plane;
            cudaError_t e = launch_ls_residuals(src, h->ex, h->ey, H, W, s, h->num_sms);
            if (e != cudaSuccess) return cuda_fail(e, "LS residual kernel launch");
            e = solve_launch(h, src, h->ex, h->ey, out + c * plane, *rp, *cp, sp, s);
            if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
        }
    return BLFLS_OK;
}

int blfls_layers(blfls_handle* h, const float* img, float* out, int H, int W, int C, int mode,
                 float strength, float lambda, float sigma_s, float sigma_r, int radius,
                 int iters, int prec, void* stream)
{
    const NvtxRange range("blfls_layers");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 1 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [1, BLFLS_MAX_ITERS]");
    if (mode != BLFLS_DETAIL_ENHANCE && mode != BLFLS_LOG_TONE) return fail(BLFLS_EINVAL, "unknown layer mode");
    if (!std::isfinite(strength) || strength < 0.f || (mode == BLFLS_LOG_TONE && strength > 1.f))
        return fail(BLFLS_EINVAL, "strength must be finite, >= 0, and <= 1 for BLFLS_LOG_TONE");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t n = (size_t)H * W * C;
    if ((rc = grow(h, h->layer, h->layer_cap, n, "layer image")) != BLFLS_OK) return rc;
    cudaError_t e;
    if (mode == BLFLS_DETAIL_ENHANCE) {
        // u into the scratch image, then out = f + m (f - u)
        if ((rc = run_smooth(h, img, h->layer, H, W, C, lambda, sigma_s, sigma_r, radius, iters,
                             prec, s)) != BLFLS_OK)
            return rc;
        e = launch_layer_epilogue(0, img, h->layer, out, n, strength, s, h->num_sms);
    } else {
        // l into the scratch image, b = BLFLS(l) into out, then out = exp(c b + (l - b))
        e = launch_log_image(img, h->layer, n, BLFLS_LOG_FLOOR, s, h->num_sms);
        if (e != cudaSuccess) return cuda_fail(e, "log kernel launch");
        if ((rc = run_smooth(h, h->layer, out, H, W, C, lambda, sigma_s, sigma_r, radius, iters,
                             prec, s)) != BLFLS_OK)
            return rc;
        e = launch_layer_epilogue(1, h->layer, out, out, n, strength, s, h->num_sms);
    }
    return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "layer epilogue launch");
}

// Joint filter: channel c of a pass, with an optional guidance plane (nullptr = plain filter).
static int joint_pass(blfls_handle* h, const float* src, const float* guide, float* dst,
                      BlfParams bp, const SolveParams& sp, const FftPlanDev& rp,
                      const FftPlanDev& cp, cudaStream_t s)
{
    bp.guide = guide;
    bp.guide_stride = 0;
    cudaError_t e = blf_launch(h, src, h->ex, h->ey, 1, bp, s);
    if (e != cudaSuccess) return cuda_fail(e, "bilateral kernel launch");
    e = solve_launch(h, src, h->ex, h->ey, dst, rp, cp, sp, s);
    if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
    return BLFLS_OK;
}

// Scratch of the joint filter: per-pixel kernel radii need the guidance's gradients too.
static int prepare_joint(blfls_handle* h, int H, int W, int radius, const FftPlanDev** rp,
                         const FftPlanDev** cp)
{
    int rc = prepare(h, H, W, radius, true, true, rp, cp);
    if (rc != BLFLS_OK) return rc;
    if (radius > blf_joint_tiled_max_radius())
        rc = grow(h, h->gscratch, h->g_cap, 4 * (size_t)H * W, "gradients");
    return rc;
}

static int check_sigma_g(float sigma)
{
    if (!(sigma > 0.f) || !(sigma <= BLFLS_MAX_GAUSS_SIGMA))
        return fail(BLFLS_EINVAL, "sigma must lie in (0, BLFLS_MAX_GAUSS_SIGMA]");
    return BLFLS_OK;
}

// Periodic Gaussian of C planes (in may equal out); the taps in FP64, stored FP32.
static int gaussian_planes(blfls_handle* h, const float* in, float* out, int H, int W, int C,
                           float sigma, cudaStream_t s)
{
    int rc;
    const size_t plane = (size_t)H * W;
    if ((rc = grow(h, h->gtmp, h->gtmp_cap, plane, "Gaussian scratch")) != BLFLS_OK) return rc;
    const int R = (int)std::ceil(3.0 * (double)sigma);
    std::vector<double> wd(2 * R + 1);
    double sum = 0.0;
    for (int k = -R; k <= R; ++k) sum += (wd[k + R] = std::exp(-(double)k * k / (2.0 * (double)sigma * sigma)));
    std::vector<float> w(2 * R + 1);
    for (int k = 0; k <= 2 * R; ++k) w[k] = (float)(wd[k] / sum);
    for (int c = 0; c < C; ++c) {
        const cudaError_t e = launch_gaussian(in + c * plane, h->gtmp, out + c * plane, H, W,
                                              w.data(), R, s, h->num_sms);
        if (e != cudaSuccess) return cuda_fail(e, "Gaussian kernel launch");
    }
    return BLFLS_OK;
}

int blfls_gaussian(blfls_handle* h, const float* img, float* out, int H, int W, int C, float sigma,
                   void* stream)
{
    const NvtxRange range("blfls_gaussian");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if ((rc = check_sigma_g(sigma)) != BLFLS_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    return gaussian_planes(h, img, out, H, W, C, sigma, static_cast<cudaStream_t>(stream));
}

int blfls_smooth_guided(blfls_handle* h, const float* img, const float* guide, float* out, int H,
                        int W, int C, int Cg, float lambda, float sigma_s, float sigma_r,
                        int radius, int iters, int prec, void* stream)
{
    const NvtxRange range("blfls_smooth_guided");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if (!guide) return fail(BLFLS_EINVAL, "guide is NULL");
    if (Cg != 1 && Cg != C) return fail(BLFLS_EINVAL, "Cg must be 1 or C");
    if (out == guide) return fail(BLFLS_EINVAL, "out must not alias guide");
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        if (out == img) return BLFLS_OK;
        const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "copy for iters = 0");
    }
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare_joint(h, H, W, radius, &rp, &cp)) != BLFLS_OK) return rc;
    const BlfParams bp{H, W, radius, sigma_s, sigma_r, prec, tuned_tile_h(h, radius, prec)};
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int c = 0; c < C; ++c) {
        const float* gc = guide + (Cg == 1 ? 0 : c * plane);
        for (int it = 0; it < iters; ++it) {
            const float* src = (it == 0 ? img : out) + c * plane;
            if ((rc = joint_pass(h, src, gc, out + c * plane, bp, sp, *rp, *cp, s)) != BLFLS_OK) return rc;
        }
    }
    return BLFLS_OK;
}

int blfls_smooth_rolling(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                         float lambda, float sigma_s, float sigma_r, int radius, int iters,
                         float sigma_g, int prec, void* stream)
{
    const NvtxRange range("blfls_smooth_rolling");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if (out == img) return fail(BLFLS_EINVAL, "out must not alias img (every pass reads the input)");
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if ((rc = check_sigma_g(sigma_g)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "copy for iters = 0");
    }
    if ((rc = grow(h, h->layer, h->layer_cap, plane * C, "rolling guidance")) != BLFLS_OK) return rc;
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare_joint(h, H, W, radius, &rp, &cp)) != BLFLS_OK) return rc;
    if ((rc = gaussian_planes(h, img, h->layer, H, W, C, sigma_g, s)) != BLFLS_OK) return rc;
    const BlfParams bp{H, W, radius, sigma_s, sigma_r, prec, tuned_tile_h(h, radius, prec)};
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int c = 0; c < C; ++c)
        for (int it = 0; it < iters; ++it) {
            // the bilateral kernel reads the whole guidance plane before K4 overwrites it
            const float* gc = (it == 0 ? h->layer : out) + c * plane;
            if ((rc = joint_pass(h, img + c * plane, gc, out + c * plane, bp, sp, *rp, *cp, s)) != BLFLS_OK)
                return rc;
        }
    return BLFLS_OK;
}

// Both grid buffers in one allocation of 2 * cells float2.
static int ensure_grid(blfls_handle* h, size_t cells)
{
    if (cells <= h->grid_cap && h->grid_a) return BLFLS_OK;
    float2* p = h->grid_a;
    size_t cap2 = 2 * h->grid_cap;
    const int rc = grow(h, p, cap2, 2 * cells, "bilateral grid");
    if (rc != BLFLS_OK) return rc;
    h->grid_a = p;
    h->grid_b = p + cells;
    h->grid_cap = cells;
    return BLFLS_OK;
}

int blfls_smooth_grid(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                      float lambda, float sigma_s, float sigma_r, int iters, void* stream)
{
    const NvtxRange range("blfls_smooth_grid");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if (!(sigma_s >= 0.5f) || !std::isfinite(sigma_s)) return fail(BLFLS_EINVAL, "sigma_s must be finite and >= 0.5");
    if (!(sigma_r > 0.f)) return fail(BLFLS_EINVAL, "sigma_r must be > 0");
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        if (out == img) return BLFLS_OK;
        const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "copy for iters = 0");
    }
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare(h, H, W, 0, false, true, &rp, &cp)) != BLFLS_OK) return rc;
    // range keys (4 ints per channel), then the levels of every field (one int4 each)
    if ((rc = grow(h, h->grid_keys, h->grid_keys_cap, 12 * (size_t)BLFLS_MAX_CHANNELS, "grid keys")) != BLFLS_OK)
        return rc;
    int4* lev = reinterpret_cast<int4*>(h->grid_keys + 4 * BLFLS_MAX_CHANNELS);
    // the buffers hold one chunk of range levels; a wider range takes more chunks on the device
    int gx = 0, gy = 0;
    grid_spatial_dims(H, W, sigma_s, &gx, &gy);
    const int zc = grid_chunk_levels(sigma_r, gx, gy);
    const size_t cells = (size_t)gx * gy * (size_t)(zc + 2);
    if (2 * cells * sizeof(float2) > BLFLS_GRID_MAX_BYTES)
        return fail(BLFLS_EINVAL, "bilateral grid above BLFLS_GRID_MAX_BYTES: raise sigma_s or sigma_r");
    if ((rc = ensure_grid(h, cells)) != BLFLS_OK) return rc;
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int it = 0; it < iters; ++it) {
        const float* src = (it == 0) ? img : out;
        cudaError_t e = launch_grid_minmax(src, H, W, C, h->grid_keys, s, h->num_sms);
        if (e == cudaSuccess) e = launch_grid_levels(h->grid_keys, C, sigma_r, zc, lev, s);
        if (e != cudaSuccess) return cuda_fail(e, "grid range kernel launch");
        for (int c = 0; c < C; ++c) {
            const float* fc = src + c * plane;
            for (int field = 0; field < 2; ++field) {
                e = launch_grid_field(fc, field == 0 ? h->ex : h->ey, field, H, W, sigma_s,
                                      sigma_r, lev + 2 * c + field, gx, gy, zc,
                                      h->grid_a, h->grid_b, s, h->num_sms);
                if (e != cudaSuccess) return cuda_fail(e, "grid kernel launch");
            }
            e = solve_launch(h, fc, h->ex, h->ey, out + c * plane, *rp, *cp, sp, s);
            if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
        }
    }
    return BLFLS_OK;
}

// Device room for the range keys and range constants of both fields of every channel.
static int ensure_range_keys(blfls_handle* h)
{
    int rc = grow(h, h->grid_keys, h->grid_keys_cap, 4 * (size_t)BLFLS_MAX_CHANNELS, "range keys");
    if (rc != BLFLS_OK) return rc;
    return grow(h, h->kap_dev, h->kap_cap, (size_t)BLFLS_MAX_CHANNELS, "range constants");
}

int blfls_smooth_normalized(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                            float lambda, float sigma_s, float sigma_r, int radius, int iters,
                            int prec, void* stream)
{
    const NvtxRange range("blfls_smooth_normalized");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        if (out == img) return BLFLS_OK;
        const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "copy for iters = 0");
    }
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare(h, H, W, radius, true, true, &rp, &cp)) != BLFLS_OK) return rc;
    if ((rc = ensure_range_keys(h)) != BLFLS_OK) return rc;
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int it = 0; it < iters; ++it) {
        const float* src = (it == 0) ? img : out;
        // the ranges of both fields of every channel of this pass's input, and from them the
        // range constants K1 reads, all on the device (no read-back)
        cudaError_t e = launch_grid_minmax(src, H, W, C, h->grid_keys, s, h->num_sms);
        if (e == cudaSuccess) e = launch_range_kappa(h->grid_keys, C, sigma_r, h->kap_dev, s);
        if (e != cudaSuccess) return cuda_fail(e, "range kernel launch");
        for (int c = 0; c < C; ++c) {
            BlfParams bp{H, W, radius, sigma_s, sigma_r, prec, tuned_tile_h(h, radius, prec)};
            bp.kap_dev = h->kap_dev + c;
            const float* fc = src + c * plane;
            e = blf_launch(h, fc, h->ex, h->ey, 1, bp, s);
            if (e != cudaSuccess) return cuda_fail(e, "bilateral kernel launch");
            e = solve_launch(h, fc, h->ex, h->ey, out + c * plane, *rp, *cp, sp, s);
            if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
        }
    }
    return BLFLS_OK;
}

int blfls_smooth_nc(blfls_handle* h, const float* img, float* out, int H, int W, int C,
                    float lambda, float sigma_s, float sigma_r, int iters, int nc_iters,
                    void* stream)
{
    const NvtxRange range("blfls_smooth_nc");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if (!(sigma_s > 0.f) || !(sigma_s <= BLFLS_MAX_NC_SIGMA_S))
        return fail(BLFLS_EINVAL, "sigma_s must lie in (0, BLFLS_MAX_NC_SIGMA_S]");
    if (!(sigma_r > 0.f)) return fail(BLFLS_EINVAL, "sigma_r must be > 0");
    if (nc_iters < 1 || nc_iters > BLFLS_MAX_NC_ITERS) return fail(BLFLS_EINVAL, "nc_iters must lie in [1, BLFLS_MAX_NC_ITERS]");
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    if (iters < 0 || iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters must lie in [0, BLFLS_MAX_ITERS]");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t plane = (size_t)H * W;
    if (iters == 0) {
        if (out == img) return BLFLS_OK;
        const cudaError_t e = cudaMemcpyAsync(out, img, plane * C * sizeof(float),
                                              cudaMemcpyDeviceToDevice, s);
        return e == cudaSuccess ? BLFLS_OK : cuda_fail(e, "copy for iters = 0");
    }
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = prepare(h, H, W, 0, false, true, &rp, &cp)) != BLFLS_OK) return rc;
    if ((rc = grow(h, h->nc_scratch, h->nc_cap, nc_scratch_floats(H, W), "NC scratch")) != BLFLS_OK)
        return rc;
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int c = 0; c < C; ++c)
        for (int it = 0; it < iters; ++it) {
            const float* src = (it == 0 ? img : out) + c * plane;
            cudaError_t e = launch_nc_residuals(src, h->ex, h->ey, H, W, sigma_s, sigma_r,
                                                nc_iters, h->nc_scratch, s, h->num_sms);
            if (e != cudaSuccess) return cuda_fail(e, "NC kernel launch");
            e = solve_launch(h, src, h->ex, h->ey, out + c * plane, *rp, *cp, sp, s);
            if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
        }
    return BLFLS_OK;
}

int blfls_blf_residual(blfls_handle* h, const float* img, float* ex, float* ey, int H, int W,
                       int C, float sigma_s, float sigma_r, int radius, int prec, void* stream)
{
    const NvtxRange range("blfls_blf_residual");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, ex, H, W, C)) != BLFLS_OK) return rc;
    if (!ey) return fail(BLFLS_EINVAL, "ey is NULL");
    if ((rc = check_blf_args(H, W, sigma_s, sigma_r, radius, prec)) != BLFLS_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    if (radius > blf_tiled_max_radius())
        if ((rc = grow(h, h->gscratch, h->g_cap, 2 * (size_t)H * W, "gradients")) != BLFLS_OK) return rc;
    const BlfParams bp{H, W, radius, sigma_s, sigma_r, prec, tuned_tile_h(h, radius, prec)};
    const cudaError_t e = blf_launch(h, img, ex, ey, C, bp, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "bilateral kernel launch");
    return BLFLS_OK;
}

int blfls_solve_residual(blfls_handle* h, const float* img, const float* ex, const float* ey,
                         float* out, int H, int W, int C, float lambda, void* stream)
{
    const NvtxRange range("blfls_solve_residual");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if ((rc = check_image_args(img, out, H, W, C)) != BLFLS_OK) return rc;
    if (!ex || !ey) return fail(BLFLS_EINVAL, "residual pointer is NULL");
    if ((rc = check_lambda(lambda)) != BLFLS_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = grow(h, h->spec, h->spec_cap, (size_t)H * (W / 2 + 1), "spectrum")) != BLFLS_OK) return rc;
    if ((rc = get_plan(h, W, &rp)) != BLFLS_OK) return rc;
    if ((rc = get_plan(h, H, &cp)) != BLFLS_OK) return rc;
    const size_t plane = (size_t)H * W;
    const SolveParams sp{H, W, lambda, tuned_col_block(h, cp->L)};
    for (int c = 0; c < C; ++c) {
        const cudaError_t e = solve_launch(h, img + c * plane, ex + c * plane, ey + c * plane,
                                           out + c * plane, *rp, *cp, sp,
                                           static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
    }
    return BLFLS_OK;
}

int blfls_smooth_batch(blfls_handle* h, const blfls_job* jobs, int n, void* stream)
{
    const NvtxRange range("blfls_smooth_batch");
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    if (n < 0 || (n > 0 && !jobs)) return fail(BLFLS_EINVAL, "bad job list");
    for (int i = 0; i < n; ++i) {
        const blfls_job& j = jobs[i];
        int rc;
        if ((rc = check_image_args(j.img, j.out, j.H, j.W, j.C)) != BLFLS_OK) return rc;
        if ((rc = check_blf_args(j.H, j.W, j.sigma_s, j.sigma_r, j.radius, j.prec)) != BLFLS_OK) return rc;
        if ((rc = check_lambda(j.lambda)) != BLFLS_OK) return rc;
        if (j.iters < 0 || j.iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters out of range");
    }
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    return run_batch(h, jobs, n, static_cast<cudaStream_t>(stream));
}

int blfls_submit(blfls_handle* h, const blfls_job* job, uint64_t* ticket)
{
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    const NvtxRange range("blfls_submit");
    blfls_server* srv;
    {
        std::lock_guard<std::mutex> lock(h->submit_mu);
        if (!h->submit_srv) {
            const size_t budget = h->budget ? h->budget : kSubmitDefaultBudget;
            const int rc = create_job_server(&h->submit_srv, h, budget, kSubmitSlots, kSubmitMaxBatch);
            if (rc != BLFLS_OK) return rc;
        }
        srv = h->submit_srv;
    }
    return server_submit_job(srv, job, ticket);
}

int blfls_poll(blfls_handle* h, uint64_t ticket, int* done)
{
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    blfls_server* srv;
    {
        std::lock_guard<std::mutex> lock(h->submit_mu);
        srv = h->submit_srv;
    }
    if (!srv) return fail(BLFLS_EINVAL, "unknown ticket (nothing was submitted)");
    return server_poll_job(srv, ticket, done);
}

int blfls_profile_begin(blfls_handle* h, int max_events)
{
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    if (max_events < 0) return fail(BLFLS_EINVAL, "max_events must be >= 0");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    while (h->prof_pool.size() < (size_t)max_events) {
        cudaEvent_t ev;
        const cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
        h->prof_pool.push_back(ev);
    }
    h->prof_on = true;
    h->prof_overflow = false;
    h->prof_next = 0;
    h->prof_spans.clear();
    return BLFLS_OK;
}

int blfls_profile_end(blfls_handle* h, double* ms, int* launches)
{
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    h->prof_on = false;
    double tot[4] = {0, 0, 0, 0};
    int cnt[4] = {0, 0, 0, 0};
    for (const auto& sp : h->prof_spans) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(h->prof_pool[sp.second.second]);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&t, h->prof_pool[sp.second.first], h->prof_pool[sp.second.second]);
        if (e != cudaSuccess) return cuda_fail(e, "profiling events");
        tot[sp.first] += t;
        cnt[sp.first] += 1;
    }
    for (int i = 0; i < 4; ++i) {
        if (ms) ms[i] = tot[i];
        if (launches) launches[i] = cnt[i];
    }
    if (h->prof_overflow) return fail(BLFLS_EINVAL, "more launches than profiling events");
    return BLFLS_OK;
}

}  // extern "C"
