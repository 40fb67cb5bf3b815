// Served form of BLF-LS: a continuous-batching request loop on one GPU (no counterpart in the
// paper).
//
// Requests arrive with host buffers (blfls_server_submit returns a ticket at once), or -- for the
// handle-level blfls_submit / blfls_poll -- as jobs on device buffers the caller owns, which
// skip the arena and the copies.  A scheduler thread keeps
//   * an arena: one device allocation made at creation, from which every request's input and
//     output buffers are carved (first fit, coalescing on release) -- resident memory, so the
//     steady state makes no cudaMalloc or cudaFree;
//   * `slots`: concurrent streams, each with its own handle (resident FFT plans and scratch,
//     capped by the slot's share of the budget);
//   * the pending queue, in arrival order.
// Whenever a slot is free it forms the next batch from the pending queue, first fit: a request
// joins if its buffers fit in the arena and the batch's scratch estimate fits the slot's share.
// The batch is copied in, smoothed by one blfls_smooth_batch call and copied out on the slot's
// stream; a host callback on that stream stamps the completion time of each request.  Requests
// that arrive while other batches run are admitted as soon as a slot and memory free up, so
// copies and kernels of different batches overlap on the device.  Latency = submit -> result in
// host memory.  Nothing here waits without a bound: the scheduler sleeps on a condition variable
// with a timeout, and blfls_server_wait takes a timeout.
#include "handle.h"
#include "nvtx_range.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace blfls;

namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// First-fit sub-allocator over the device arena (host-side bookkeeping only).
class Arena {
public:
    void init(unsigned char* base, size_t bytes)
    {
        base_ = base;
        total_ = bytes;
        free_.clear();
        if (bytes) free_[0] = bytes;
        used_ = peak_ = 0;
    }
    // Returns an offset or SIZE_MAX.
    size_t alloc(size_t bytes)
    {
        bytes = align_up(std::max<size_t>(bytes, 1), 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_ += bytes;
                peak_ = std::max(peak_, used_);
                sizes_[off] = bytes;
                return off;
            }
        }
        return SIZE_MAX;
    }
    void release(size_t off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t start = off, len = s->second;
        sizes_.erase(s);
        used_ -= len;
        auto next = free_.lower_bound(start);
        if (next != free_.end() && start + len == next->first) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }
    unsigned char* at(size_t off) const { return base_ + off; }
    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto& kv : free_) m = std::max(m, kv.second);
        return m;
    }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }
    size_t total() const { return total_; }

private:
    size_t total_ = 0;
    unsigned char* base_ = nullptr;
    std::map<size_t, size_t> free_;   // offset -> length
    std::map<size_t, size_t> sizes_;  // live allocations
    size_t used_ = 0, peak_ = 0;
};

struct Request {
    uint64_t id = 0;
    blfls_request r{};   // parameters (and host buffers unless device_io)
    bool device_io = false;
    blfls_job job{};     // device buffers of a device-pointer job
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::atomic<int> status{0};    // 0 queued, 3 running, 1 done, 2 cancelled, < 0 error
    size_t off_in = SIZE_MAX, off_out = SIZE_MAX;
    size_t scratch = 0;
};

struct Slot {
    blfls_handle* h = nullptr;
    cudaStream_t s = nullptr;
    std::vector<Request*> reqs;
    std::atomic<bool> busy{false};
    std::atomic<bool> finished{false};
    double t_finish = 0;
    struct blfls_server* srv = nullptr;
};

size_t io_bytes(const blfls_request& r) { return sizeof(float) * (size_t)r.C * r.H * r.W; }

// Scratch the batched executor needs for one request: residual planes, spectra, table slack.
size_t scratch_bytes(const blfls_request& r)
{
    const size_t planes = (size_t)r.C * r.H * r.W;
    return align_up(2 * sizeof(float) * planes, 256) +
           align_up(sizeof(float2) * (size_t)r.C * r.H * (r.W / 2 + 1), 256) + 4096;
}

}  // namespace

struct blfls_server {
    int device = 0;
    size_t budget = 0;
    int max_batch = 8;
    size_t slot_scratch = 0;
    void* arena_mem = nullptr;
    Arena arena;
    std::vector<Slot*> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> incoming;
    std::vector<Request*> pending;
    std::unordered_map<uint64_t, Request*> all;
    uint64_t next_id = 1;
    std::thread thread;
    bool stop = false;
    // statistics
    std::vector<double> lat_ms;
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, rejected = 0;
    double first_submit = -1, last_done = 0, megapixels = 0;
    int max_batch_seen = 0;
    int last_error = 0;
};

namespace {

void CUDART_CB on_slot_done(void* arg)
{
    Slot* slot = static_cast<Slot*>(arg);
    slot->t_finish = now_s();
    slot->finished.store(true);
    slot->srv->cv.notify_all();
}

// Retire finished slots (scheduler thread, lock held).
void retire(blfls_server* S)
{
    for (Slot* slot : S->slots) {
        if (!slot->busy.load() || !slot->finished.load()) continue;
        const cudaError_t e = cudaStreamQuery(slot->s);   // the callback ran; the stream is idle
        for (Request* q : slot->reqs) {
            S->arena.release(q->off_in);
            S->arena.release(q->off_out);
            q->t_done = slot->t_finish;
            if (e != cudaSuccess && e != cudaErrorNotReady) {
                q->status.store(BLFLS_ECUDA);
                S->failed++;
            } else {
                q->status.store(1);
                S->completed++;
                S->lat_ms.push_back((q->t_done - q->t_submit) * 1e3);
                S->megapixels += (double)q->r.H * q->r.W / 1e6;
                S->last_done = std::max(S->last_done, q->t_done);
            }
        }
        slot->reqs.clear();
        slot->finished.store(false);
        slot->busy.store(false);
    }
}

// Pick the next batch for a free slot from the pending queue, first fit (scheduler thread,
// lock held).  Buffers are carved from the arena here.
std::vector<Request*> select_batch(blfls_server* S)
{
    std::vector<Request*> batch;
    size_t scratch = 0;
    for (auto it = S->pending.begin(); it != S->pending.end() && (int)batch.size() < S->max_batch;) {
        Request* q = *it;
        if (q->status.load() == 2) {   // cancelled while queued
            it = S->pending.erase(it);
            continue;
        }
        if (scratch + q->scratch > S->slot_scratch) {
            ++it;
            continue;
        }
        if (q->device_io) {   // the caller's device buffers: nothing to carve
            int expected = 0;
            if (!q->status.compare_exchange_strong(expected, 3)) {
                it = S->pending.erase(it);
                continue;
            }
            scratch += q->scratch;
            batch.push_back(q);
            it = S->pending.erase(it);
            continue;
        }
        const size_t in = S->arena.alloc(io_bytes(q->r));
        if (in == SIZE_MAX) {
            ++it;
            continue;
        }
        const size_t out = S->arena.alloc(io_bytes(q->r));
        if (out == SIZE_MAX) {
            S->arena.release(in);
            ++it;
            continue;
        }
        int expected = 0;
        if (!q->status.compare_exchange_strong(expected, 3)) {   // cancelled just now
            S->arena.release(in);
            S->arena.release(out);
            it = S->pending.erase(it);
            continue;
        }
        q->off_in = in;
        q->off_out = out;
        scratch += q->scratch;
        batch.push_back(q);
        it = S->pending.erase(it);
    }
    return batch;
}

// Copy in, smooth, copy out, and stamp completion, on the slot's stream (scheduler thread,
// lock NOT held: only this thread touches slots and the arena's device memory).
void launch_batch(blfls_server* S, Slot* slot, const std::vector<Request*>& batch)
{
    const NvtxRange range("server batch");
    const double t = now_s();
    std::vector<blfls_job> jobs;
    jobs.reserve(batch.size());
    int rc = BLFLS_OK;
    for (Request* q : batch) {
        q->t_admit = t;
        if (q->device_io) {
            jobs.push_back(q->job);
            continue;
        }
        float* din = reinterpret_cast<float*>(S->arena.at(q->off_in));
        float* dout = reinterpret_cast<float*>(S->arena.at(q->off_out));
        if (cudaMemcpyAsync(din, q->r.img_host, io_bytes(q->r), cudaMemcpyHostToDevice, slot->s) != cudaSuccess)
            rc = BLFLS_ECUDA;
        jobs.push_back(blfls_job{din, dout, q->r.H, q->r.W, q->r.C, q->r.lambda, q->r.sigma_s,
                                 q->r.sigma_r, q->r.radius, q->r.iters, q->r.prec});
    }
    if (rc == BLFLS_OK) rc = blfls_smooth_batch(slot->h, jobs.data(), (int)jobs.size(), slot->s);
    if (rc == BLFLS_OK) {
        for (Request* q : batch) {
            if (q->device_io) continue;
            if (cudaMemcpyAsync(q->r.out_host, S->arena.at(q->off_out), io_bytes(q->r),
                                cudaMemcpyDeviceToHost, slot->s) != cudaSuccess)
                rc = BLFLS_ECUDA;
        }
    }
    if (rc == BLFLS_OK && cudaLaunchHostFunc(slot->s, on_slot_done, slot) == cudaSuccess) return;
    cudaStreamSynchronize(slot->s);
    std::lock_guard<std::mutex> lock(S->mu);
    for (Request* q : batch) {
        S->arena.release(q->off_in);
        S->arena.release(q->off_out);
        q->status.store(rc != BLFLS_OK ? rc : BLFLS_ECUDA);
        S->failed++;
    }
    S->last_error = rc;
    slot->reqs.clear();
    slot->busy.store(false);
}

void scheduler(blfls_server* S)
{
    cudaSetDevice(S->device);
    while (true) {
        std::vector<std::pair<Slot*, std::vector<Request*>>> work;
        {
            std::unique_lock<std::mutex> lock(S->mu);
            while (!S->incoming.empty()) {
                S->pending.push_back(S->incoming.front());
                S->incoming.pop_front();
            }
            retire(S);
            for (Slot* slot : S->slots) {
                if (slot->busy.load() || S->pending.empty()) continue;
                std::vector<Request*> batch = select_batch(S);
                if (batch.empty()) continue;
                slot->reqs = batch;
                slot->finished.store(false);
                slot->busy.store(true);
                S->max_batch_seen = std::max(S->max_batch_seen, (int)batch.size());
                work.emplace_back(slot, std::move(batch));
            }
            bool any_busy = false;
            for (Slot* slot : S->slots) any_busy |= slot->busy.load();
            if (S->stop && S->pending.empty() && S->incoming.empty() && !any_busy) break;
            if (work.empty()) {
                S->cv.wait_for(lock, std::chrono::microseconds(200));
                continue;
            }
        }
        for (auto& w : work) launch_batch(S, w.first, w.second);
    }
}

}  // namespace

namespace {

// Server with `arena_pct` percent of the budget for request buffers (0: device-pointer jobs
// only), the rest split 7:1 between the slots' batch scratch and their plans and tables; the
// slot handles take their launch shapes from `tune_from` when given.
int create_server(blfls_server** out, int device, size_t mem_budget_bytes, int slots,
                  int max_batch, const char* tune_table_path, int arena_pct,
                  const blfls_handle* tune_from)
{
    if (!out) return fail(BLFLS_EINVAL, "out is NULL");
    *out = nullptr;
    if (slots < 1 || slots > 16 || max_batch < 1 || max_batch > 1024)
        return fail(BLFLS_EINVAL, "slots must lie in [1, 16] and max_batch in [1, 1024]");
    if (mem_budget_bytes < ((size_t)64 << 20)) return fail(BLFLS_EINVAL, "budget below 64 MiB");
    DeviceGuard g(device);
    if (!g.ok) return fail(BLFLS_EINVAL, "no such CUDA device");
    blfls_server* S = new blfls_server();
    S->device = device;
    S->budget = mem_budget_bytes;
    S->max_batch = max_batch;
    // budget split: arena_pct% I/O arena, the rest 7:1 between the slots' batch scratch and their
    // plans and tables (60 / 35 / 5 for host-buffer requests)
    const size_t arena_bytes = align_up(mem_budget_bytes / 100 * arena_pct, 256);
    const size_t rest = mem_budget_bytes / 100 * (100 - arena_pct);
    S->slot_scratch = rest / 8 * 7 / slots;
    const size_t slot_extra = rest / 8 / slots;
    if (arena_bytes) {
        cudaError_t e = cudaMalloc(&S->arena_mem, arena_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return fail(BLFLS_ENOMEM, std::string("server arena: ") + cudaGetErrorString(e));
        }
    }
    S->arena.init(static_cast<unsigned char*>(S->arena_mem), arena_bytes);
    for (int i = 0; i < slots; ++i) {
        Slot* slot = new Slot();
        slot->srv = S;
        int rc = blfls_create(&slot->h, device, S->slot_scratch + slot_extra, tune_table_path);
        if (rc == BLFLS_OK && tune_from) {
            slot->h->tune_tile_h = tune_from->tune_tile_h;
            slot->h->tune_col_block = tune_from->tune_col_block;
            slot->h->col_block = tune_from->col_block;
        }
        if (rc == BLFLS_OK) rc = reserve_batch_scratch(slot->h, S->slot_scratch);
        if (rc == BLFLS_OK && cudaStreamCreateWithFlags(&slot->s, cudaStreamNonBlocking) != cudaSuccess)
            rc = BLFLS_ECUDA;
        S->slots.push_back(slot);
        if (rc != BLFLS_OK) {
            for (Slot* sl : S->slots) {
                if (sl->s) cudaStreamDestroy(sl->s);
                if (sl->h) blfls_destroy(sl->h);
                delete sl;
            }
            if (S->arena_mem) cudaFree(S->arena_mem);
            delete S;
            return rc;
        }
    }
    S->thread = std::thread(scheduler, S);
    *out = S;
    return BLFLS_OK;
}

}  // namespace

namespace blfls {

int create_job_server(blfls_server** out, const blfls_handle* h, size_t budget, int slots,
                      int max_batch)
{
    return create_server(out, h->device, budget, slots, max_batch, nullptr, 0, h);
}

int server_submit_job(blfls_server* S, const blfls_job* j, uint64_t* ticket)
{
    if (!S || !j || !ticket) return fail(BLFLS_EINVAL, "NULL argument");
    int rc;
    if ((rc = check_image_args(j->img, j->out, j->H, j->W, j->C)) != BLFLS_OK) return rc;
    if ((rc = check_blf_args(j->H, j->W, j->sigma_s, j->sigma_r, j->radius, j->prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(j->lambda)) != BLFLS_OK) return rc;
    if (j->iters < 0 || j->iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters out of range");
    Request* q = new Request();
    q->device_io = true;
    q->job = *j;
    q->r = blfls_request{nullptr, nullptr, j->H, j->W, j->C, j->lambda, j->sigma_s, j->sigma_r,
                         j->radius, j->iters, j->prec};
    q->scratch = scratch_bytes(q->r);
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (q->scratch > S->slot_scratch) {
            S->rejected++;
            delete q;
            return fail(BLFLS_ENOMEM, "job larger than the submit queue's scratch budget allows");
        }
        q->id = S->next_id++;
        if (S->first_submit < 0) S->first_submit = q->t_submit;
        S->all[q->id] = q;
        S->incoming.push_back(q);
        S->submitted++;
        *ticket = q->id;
    }
    S->cv.notify_all();
    return BLFLS_OK;
}

int server_poll_job(blfls_server* S, uint64_t ticket, int* done)
{
    if (!S || !done) return fail(BLFLS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(BLFLS_EINVAL, "unknown ticket");
    const int st = it->second->status.load();
    if (st == 0 || st == 3) {
        *done = 0;
        return BLFLS_OK;
    }
    *done = 1;
    delete it->second;   // reported once: the record is forgotten
    S->all.erase(it);
    if (st < 0) return fail(st, "job failed");
    return BLFLS_OK;
}

}  // namespace blfls

extern "C" {

int blfls_server_create(blfls_server** out, int device, size_t mem_budget_bytes, int slots,
                        int max_batch, const char* tune_table_path)
{
    return create_server(out, device, mem_budget_bytes, slots, max_batch, tune_table_path, 60,
                         nullptr);
}

void blfls_server_destroy(blfls_server* S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        for (Request* q : S->pending) {
            q->status.store(2);
            S->cancelled++;
        }
        S->pending.clear();
        for (Request* q : S->incoming) {
            q->status.store(2);
            S->cancelled++;
        }
        S->incoming.clear();
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->thread.joinable()) S->thread.join();
    DeviceGuard g(S->device);
    for (Slot* slot : S->slots) {
        if (slot->s) {
            cudaStreamSynchronize(slot->s);
            cudaStreamDestroy(slot->s);
        }
        blfls_destroy(slot->h);
        delete slot;
    }
    if (S->arena_mem) cudaFree(S->arena_mem);
    for (auto& kv : S->all) delete kv.second;
    delete S;
}

int blfls_server_submit(blfls_server* S, const blfls_request* r, uint64_t* ticket)
{
    if (!S || !r || !ticket) return fail(BLFLS_EINVAL, "NULL argument");
    int rc;
    if ((rc = check_image_args(r->img_host, r->out_host, r->H, r->W, r->C)) != BLFLS_OK) return rc;
    if ((rc = check_blf_args(r->H, r->W, r->sigma_s, r->sigma_r, r->radius, r->prec)) != BLFLS_OK) return rc;
    if ((rc = check_lambda(r->lambda)) != BLFLS_OK) return rc;
    if (r->iters < 0 || r->iters > BLFLS_MAX_ITERS) return fail(BLFLS_EINVAL, "iters out of range");
    Request* q = new Request();
    q->r = *r;
    q->scratch = scratch_bytes(*r);
    q->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (q->scratch > S->slot_scratch || 2 * align_up(io_bytes(*r), 256) > S->arena.total()) {
            S->rejected++;
            delete q;
            return fail(BLFLS_ENOMEM, "request larger than the server's memory budget allows");
        }
        q->id = S->next_id++;
        if (S->first_submit < 0) S->first_submit = q->t_submit;
        S->all[q->id] = q;
        S->incoming.push_back(q);
        S->submitted++;
        *ticket = q->id;
    }
    S->cv.notify_all();
    return BLFLS_OK;
}

int blfls_server_poll(blfls_server* S, uint64_t ticket, int* state)
{
    if (!S || !state) return fail(BLFLS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(BLFLS_EINVAL, "unknown ticket");
    const int st = it->second->status.load();
    *state = st == 3 ? 0 : st;
    return BLFLS_OK;
}

int blfls_server_wait(blfls_server* S, uint64_t ticket, int timeout_ms)
{
    if (!S) return fail(BLFLS_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(BLFLS_EINVAL, "unknown ticket");
    Request* q = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(timeout_ms, 0));
    while (true) {
        const int st = q->status.load();
        if (st == 1) return BLFLS_OK;
        if (st == 2) return fail(BLFLS_EINVAL, "request was cancelled");
        if (st < 0) return fail(st, "request failed");
        if (Clock::now() >= deadline) return fail(BLFLS_ETIMEOUT, "timed out waiting for the request");
        S->cv.wait_until(lock, std::min(deadline, Clock::now() + std::chrono::milliseconds(1)));
    }
}

int blfls_server_cancel(blfls_server* S, uint64_t ticket)
{
    if (!S) return fail(BLFLS_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(BLFLS_EINVAL, "unknown ticket");
    int expected = 0;
    if (it->second->status.compare_exchange_strong(expected, 2)) {
        S->cancelled++;
        return BLFLS_OK;
    }
    return fail(BLFLS_EBUSY, "request already admitted or finished");
}

int blfls_server_release(blfls_server* S, uint64_t ticket)
{
    if (!S) return fail(BLFLS_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lock(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return fail(BLFLS_EINVAL, "unknown ticket");
    const int st = it->second->status.load();
    if (st == 0 || st == 3) return fail(BLFLS_EBUSY, "request still queued or running");
    delete it->second;
    S->all.erase(it);
    return BLFLS_OK;
}

int blfls_server_get_stats(blfls_server* S, blfls_server_stats* out)
{
    if (!S || !out) return fail(BLFLS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(S->mu);
    blfls_server_stats st{};
    st.submitted = S->submitted;
    st.completed = S->completed;
    st.failed = S->failed;
    st.cancelled = S->cancelled;
    st.rejected = S->rejected;
    std::vector<double> lat = S->lat_ms;
    if (!lat.empty()) {
        std::sort(lat.begin(), lat.end());
        auto pct = [&](double p) {
            const double idx = p * (lat.size() - 1);
            const size_t lo = (size_t)idx, hi = std::min(lo + 1, lat.size() - 1);
            return lat[lo] + (lat[hi] - lat[lo]) * (idx - lo);
        };
        st.p50_ms = pct(0.50);
        st.p99_ms = pct(0.99);
        double sum = 0;
        for (double v : lat) sum += v;
        st.mean_ms = sum / lat.size();
        st.max_ms = lat.back();
    }
    st.megapixels = S->megapixels;
    st.busy_s = (S->first_submit >= 0 && S->last_done > S->first_submit) ? S->last_done - S->first_submit : 0;
    st.mp_per_s = st.busy_s > 0 ? st.megapixels / st.busy_s : 0;
    size_t handles = 0;
    for (Slot* slot : S->slots) handles += slot->h->used;
    st.device_bytes_peak = S->arena.peak() + handles;
    st.device_bytes_budget = S->budget;
    st.max_batch_seen = S->max_batch_seen;
    *out = st;
    return BLFLS_OK;
}

}  // extern "C"
