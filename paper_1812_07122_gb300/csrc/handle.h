// The handle behind the C ABI, and host helpers shared by the API files (not part of the ABI).
#pragma once

#include "blfls.h"
#include "internal.h"

#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

namespace blfls {
struct BatchState;   // batched executor state (batch.cu)
void destroy_batch_state(BatchState* b);
}

struct blfls_handle {
    int device = 0;
    int num_sms = 0;
    size_t budget = 0;  // 0 = unlimited
    size_t used = 0;
    int col_block = 4;   // K3 column block of the batched executor when none is tuned
    std::map<int, blfls::FftPlanHost> plans;
    // scratch (device)
    float* ex = nullptr;
    float* ey = nullptr;
    size_t e_cap = 0;  // floats per plane
    float2* spec = nullptr;
    size_t spec_cap = 0;  // complex values
    float* gscratch = nullptr;
    size_t g_cap = 0;
    float* io = nullptr;  // device copies for blfls_smooth_host: img then out
    size_t io_cap = 0;
    float* layer = nullptr;  // blfls_layers: the smoothed (or logarithmic) image; rolling: guide
    size_t layer_cap = 0;
    float* gtmp = nullptr;   // blfls_gaussian: one plane after the row pass
    size_t gtmp_cap = 0;
    // blfls_smooth_grid: the two grid buffers (one chunk of range levels each) and the range keys
    float2* grid_a = nullptr;
    float2* grid_b = nullptr;
    size_t grid_cap = 0;     // cells per buffer
    int* grid_keys = nullptr;
    size_t grid_keys_cap = 0;
    float4* kap_dev = nullptr;       // blfls_smooth_normalized: range constants per channel
    size_t kap_cap = 0;
    float* nc_scratch = nullptr;     // blfls_smooth_nc: gradients, transforms, two buffers
    size_t nc_cap = 0;
    // blfls_smooth: channels 1..C-1 run on their own streams with their own residual planes and
    // spectrum (channel 0 uses ex/ey/spec and the caller's stream)
    float* chan_scratch = nullptr;
    size_t chan_cap = 0;             // floats
    std::vector<cudaStream_t> chan_streams;   // one per channel
    // one per channel with graded priorities (channel 0 highest): the host-buffer path, where
    // channels that finish one after another let each result's copy run under the others' work
    std::vector<cudaStream_t> chan_streams_graded;
    std::vector<cudaEvent_t> chan_done;       // one per channel
    cudaEvent_t chan_fork = nullptr;
    // blfls_smooth_host: copy stream (non-blocking) and per-channel events
    cudaStream_t copy_stream = nullptr;
    std::vector<cudaEvent_t> io_events;
    // kernel timing (blfls_profile_begin / _end)
    bool prof_on = false;
    bool prof_overflow = false;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_next = 0;
    std::vector<std::pair<int, std::pair<int, int>>> prof_spans;  // stage, (start, end) event
    unsigned long long generation = 0;  // bumped whenever a scratch buffer is reallocated
    // autotuned launch shapes (tune.cu): K1 tile height per (radius, precision), K3 column
    // block per ceil(log2) of the column-transform length
    std::map<std::pair<int, int>, int> tune_tile_h;
    std::map<int, int> tune_col_block;
    blfls::BatchState* batch = nullptr;
    // blfls_submit / blfls_poll: a continuous-batching queue of device-pointer jobs with its own
    // slot handles and streams, created by the first blfls_submit
    blfls_server* submit_srv = nullptr;
    std::mutex submit_mu;   // guards the queue's creation
};

namespace blfls {

// Make the handle's device current for the duration of a call and restore the caller's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* where);
bool budget_allows(blfls_handle* h, size_t extra);
// Grow a device buffer to `need` bytes within the handle's budget (contents are not kept).
int grow_bytes(blfls_handle* h, void** ptr, size_t* cap_bytes, size_t need, const char* what);
int get_plan(blfls_handle* h, int N, const FftPlanDev** out);
int check_image_args(const void* a, const void* b, int H, int W, int C);
int check_blf_args(int H, int W, float sigma_s, float sigma_r, int radius, int prec);
int check_lambda(float lambda);
int run_smooth(blfls_handle* h, const float* img, float* out, int H, int W, int C, float lambda,
               float sigma_s, float sigma_r, int radius, int iters, int prec, cudaStream_t s);
int run_batch(blfls_handle* h, const blfls_job* jobs, int n, cudaStream_t s);
// Size the handle's batched-executor scratch arena up front (no reallocation later).
int reserve_batch_scratch(blfls_handle* h, size_t bytes);
int tuned_tile_h(const blfls_handle* h, int radius, int prec);
// The tuned K3 column block for column length L, or 0 (none: the column driver's own choice).
int tuned_col_block(const blfls_handle* h, int L);
int load_tune_table(blfls_handle* h, const char* path);
// The queue behind blfls_submit / blfls_poll (serve.cu): a server without a host-buffer arena
// whose `slots` slot handles share `budget` bytes of scratch and take h's launch shapes.
int create_job_server(blfls_server** out, const blfls_handle* h, size_t budget, int slots,
                      int max_batch);
int server_submit_job(blfls_server* S, const blfls_job* j, uint64_t* ticket);
// *done = 1 once the job has finished (the record is then forgotten; its error, if it failed,
// is returned), 0 while it is queued or running.
int server_poll_job(blfls_server* S, uint64_t ticket, int* done);
int save_tune_table(const blfls_handle* h, const char* path);

}  // namespace blfls
