// Batched form of BLF-LS (blfls_smooth_batch): many independent jobs of uneven sizes, channel
// counts and parameters run as a handful of persistent launches per pass.
//
// For every pass the host builds a device job table (one BatchJob per job still iterating) and
// item lists: the K1 items (32x32 tiles of every channel) grouped by the kernel template they
// need -- (radius, range kernel on/off, precision) -- and the row-pair and column-block items of
// the solve phases.  A pass is then
//     K1 group 0 | K1 group 1 | ...   (concurrent, one persistent launch per group)
//     -> K2 (all jobs) -> K3 (all jobs) -> K4 (all jobs)
// on handle-owned streams ordered after the caller's stream.  Tables travel in one pinned-host
// to device copy per call.  The launch sequence depends only on the batch's shape, so a call whose
// shape repeats the previous call's is captured into a CUDA graph, and later calls of that shape
// replay the graph (the tables it reads are refreshed by the copy before each replay).
// Jobs use the same device functions as blfls_smooth, so their results are identical to running
// each job alone.  Jobs whose radius exceeds the batched kernels' limit run through the single-
// image path inside the same call.
#include "handle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

namespace blfls {

// Shared-memory cap of one column block in the batched column kernel (see run_batch).
constexpr size_t kBatchColBytes = 32 * 1024;

struct BatchState {
    void* arena = nullptr;   // residuals and spectra of all batched jobs (device)
    size_t arena_cap = 0;
    void* table = nullptr;   // job tables and item groups of all passes (device)
    size_t table_cap = 0;
    void* host = nullptr;    // pinned staging for the tables
    size_t host_cap = 0;
    cudaEvent_t host_free = nullptr;  // the upload that last read `host`
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    std::vector<long long> last_sig;
    std::map<std::vector<long long>, cudaGraphExec_t> graphs;
};

void destroy_batch_state(BatchState* b)
{
    if (!b) return;
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (cudaStream_t s : b->aux) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    if (b->main) cudaStreamDestroy(b->main);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->host_free) cudaEventDestroy(b->host_free);
    if (b->host) cudaFreeHost(b->host);
    if (b->arena) cudaFree(b->arena);
    if (b->table) cudaFree(b->table);
    delete b;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Group {  // one K1 launch: jobs sharing a kernel template and tile height
    int radius, range, prec, tile_h;
    std::vector<int2> items;  // (table entry, first item)
    int total = 0;
};

struct Pass {
    std::vector<BatchJob> table;
    std::vector<Group> groups;
    std::vector<int2> rows, cols;
    int total_rows = 0, total_cols = 0;
    size_t smem_rows = 0, smem_cols = 0;
    int max_w = 0;   // widest row of the pass (sizes the staged row drivers)
    // byte offsets inside the uploaded blob
    size_t o_table = 0, o_rows = 0, o_cols = 0;
    std::vector<size_t> o_groups;
};

int ensure_state(blfls_handle* h, int ngroups)
{
    if (!h->batch) h->batch = new BatchState();
    BatchState* b = h->batch;
    cudaError_t e = cudaSuccess;
    if (!b->main) {
        if ((e = cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "batch stream");
        if ((e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "batch event");
        if ((e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "batch event");
        if ((e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "batch event");
        if ((e = cudaEventCreateWithFlags(&b->host_free, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "batch event");
    }
    while ((int)b->aux.size() < ngroups - 1) {
        cudaStream_t s;
        cudaEvent_t ev;
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "batch stream");
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "batch event");
        b->aux.push_back(s);
        b->ev_join.push_back(ev);
    }
    return BLFLS_OK;
}

// Enqueue every pass on b->main (and the aux streams for concurrent K1 groups).
cudaError_t enqueue(blfls_handle* h, const std::vector<Pass>& passes)
{
    BatchState* b = h->batch;
    unsigned char* dev = static_cast<unsigned char*>(b->table);
    cudaError_t e = cudaSuccess;
    for (const Pass& p : passes) {
        const BatchJob* tab = reinterpret_cast<const BatchJob*>(dev + p.o_table);
        const int ng = (int)p.groups.size();
        if (ng > 1) {
            cudaEventRecord(b->ev_fork, b->main);
            for (int g = 1; g < ng; ++g) cudaStreamWaitEvent(b->aux[g - 1], b->ev_fork, 0);
        }
        for (int g = 0; g < ng; ++g) {
            const Group& G = p.groups[g];
            cudaStream_t s = g == 0 ? b->main : b->aux[g - 1];
            e = launch_blf_batch(tab, reinterpret_cast<const int2*>(dev + p.o_groups[g]),
                                 (int)G.items.size(), G.total, G.radius, G.range != 0, G.prec,
                                 G.tile_h, h->num_sms, s);
            if (e != cudaSuccess) return e;
            if (g > 0) cudaEventRecord(b->ev_join[g - 1], s);
        }
        for (int g = 1; g < ng; ++g) cudaStreamWaitEvent(b->main, b->ev_join[g - 1], 0);
        e = launch_solve_batch(tab, (int)p.table.size(), reinterpret_cast<const int2*>(dev + p.o_rows),
                               p.total_rows, reinterpret_cast<const int2*>(dev + p.o_cols),
                               p.total_cols, p.smem_rows, p.smem_cols, p.max_w, h->num_sms, b->main);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace

int reserve_batch_scratch(blfls_handle* h, size_t bytes)
{
    DeviceGuard g(h->device);
    int rc = ensure_state(h, 1);
    if (rc != BLFLS_OK) return rc;
    return grow_bytes(h, &h->batch->arena, &h->batch->arena_cap, bytes, "batch scratch");
}

int run_batch(blfls_handle* h, const blfls_job* jobs, int n, cudaStream_t user)
{
    int rc;
    // --- jobs with nothing to iterate, and jobs the batched kernels do not cover --------------
    std::vector<int> batched, single;
    for (int i = 0; i < n; ++i) {
        const blfls_job& j = jobs[i];
        if (j.iters == 0) {
            if (j.out != j.img) {
                const cudaError_t e = cudaMemcpyAsync(j.out, j.img, sizeof(float) * j.H * j.W * j.C,
                                                      cudaMemcpyDeviceToDevice, user);
                if (e != cudaSuccess) return cuda_fail(e, "copy for iters = 0");
            }
        } else if (j.radius > blf_batch_max_radius()) {
            single.push_back(i);
        } else {
            batched.push_back(i);
        }
    }

    if (!batched.empty()) {
        // --- plans, constants and the scratch arena layout --------------------------------------
        struct Info {
            const FftPlanDev* rp;
            const FftPlanDev* cp;
            float kappa, inv_kappa, cs;
            int lgc, rec, tiles_x, tiles_y, tile_h;
            size_t o_ex, o_ey, o_spec;
        };
        std::vector<Info> info(batched.size());
        size_t arena = 0;
        int max_iters = 0;
        for (size_t k = 0; k < batched.size(); ++k) {
            const blfls_job& j = jobs[batched[k]];
            Info& I = info[k];
            if ((rc = get_plan(h, j.W, &I.rp)) != BLFLS_OK) return rc;
            if ((rc = get_plan(h, j.H, &I.cp)) != BLFLS_OK) return rc;
            blf_constants(j.sigma_s, j.sigma_r, &I.kappa, &I.inv_kappa, &I.cs);
            const int tuned = tuned_col_block(h, I.cp->L);
            I.lgc = solve_fit_lgc(I.cp->L, tuned > 0 ? tuned : h->col_block);
            // The batched column kernel takes the largest block of the batch as its shared
            // memory, so cap every job's block at kBatchColBytes: one long (e.g. Bluestein)
            // column set must not cut the occupancy of every other job's items.
            while (I.lgc > 0 && (sizeof(float2) * (size_t)I.cp->L << I.lgc) > kBatchColBytes) --I.lgc;
            // a column length that needs Bluestein is solved by the recursion, 32 columns a block
            I.rec = I.cp->bluestein && j.lambda <= kRecLamMax ? 1 : 0;
            if (I.rec) I.lgc = 5;
            I.tile_h = blf_tile_height(tuned_tile_h(h, j.radius, j.prec));
            blf_tiles(j.H, j.W, I.tile_h, &I.tiles_x, &I.tiles_y);
            const size_t planes = (size_t)j.C * j.H * j.W;
            I.o_ex = arena;
            arena = align256(arena + sizeof(float) * planes);
            I.o_ey = arena;
            arena = align256(arena + sizeof(float) * planes);
            I.o_spec = arena;
            arena = align256(arena + sizeof(float2) * (size_t)j.C * j.H * (j.W / 2 + 1));
            max_iters = std::max(max_iters, j.iters);
        }
        if ((rc = ensure_state(h, 1)) != BLFLS_OK) return rc;
        BatchState* b = h->batch;
        if ((rc = grow_bytes(h, &b->arena, &b->arena_cap, arena, "batch scratch")) != BLFLS_OK) return rc;
        unsigned char* ar = static_cast<unsigned char*>(b->arena);

        // --- per-pass tables and item lists -------------------------------------------------------
        std::vector<Pass> passes(max_iters);
        size_t blob = 0;
        int max_groups = 1;
        for (int pass = 0; pass < max_iters; ++pass) {
            Pass& P = passes[pass];
            std::map<std::tuple<int, int, int, int>, int> gidx;
            for (size_t k = 0; k < batched.size(); ++k) {
                const blfls_job& j = jobs[batched[k]];
                if (j.iters <= pass) continue;
                const Info& I = info[k];
                BatchJob J{};
                J.src = pass == 0 ? j.img : j.out;
                J.dst = j.out;
                J.ex = reinterpret_cast<float*>(ar + I.o_ex);
                J.ey = reinterpret_cast<float*>(ar + I.o_ey);
                J.spec = reinterpret_cast<float2*>(ar + I.o_spec);
                J.H = j.H;
                J.W = j.W;
                J.C = j.C;
                J.radius = j.radius;
                J.kappa = I.kappa;
                J.inv_kappa = I.inv_kappa;
                J.cs = I.cs;
                J.lam = j.lambda;
                J.scale = 1.0f / ((float)j.H * (float)j.W);
                J.lgc = I.lgc;
                J.rec = I.rec;
                J.tiles_x = I.tiles_x;
                J.tiles_y = I.tiles_y;
                J.tile_h = I.tile_h;
                J.rp = *I.rp;
                J.cp = *I.cp;
                const int entry = (int)P.table.size();
                P.table.push_back(J);
                const int range = std::isfinite(j.sigma_r) ? 1 : 0;
                const auto key = std::make_tuple(j.radius, range, j.prec, I.tile_h);
                auto it = gidx.find(key);
                if (it == gidx.end()) {
                    it = gidx.emplace(key, (int)P.groups.size()).first;
                    P.groups.push_back(Group{j.radius, range, j.prec, I.tile_h, {}, 0});
                }
                Group& G = P.groups[it->second];
                G.items.push_back(make_int2(entry, G.total));
                G.total += j.C * I.tiles_x * I.tiles_y;
                P.rows.push_back(make_int2(entry, P.total_rows));
                P.total_rows += j.C * ((j.H + 1) / 2);
                P.cols.push_back(make_int2(entry, P.total_cols));
                P.total_cols += j.C * ((j.W / 2 + 1 + (1 << I.lgc) - 1) >> I.lgc);
                P.smem_rows = std::max(P.smem_rows, sizeof(float2) * (size_t)row_buf_elems(*I.rp));
                P.max_w = std::max(P.max_w, j.W);
                P.smem_cols = std::max(P.smem_cols, I.rec ? solve_rec_smem(j.H)
                                                           : (sizeof(float2) * (size_t)I.cp->L) << I.lgc);
            }
            max_groups = std::max(max_groups, (int)P.groups.size());
            P.o_table = blob;
            blob = align256(blob + sizeof(BatchJob) * P.table.size());
            P.o_rows = blob;
            blob = align256(blob + sizeof(int2) * P.rows.size());
            P.o_cols = blob;
            blob = align256(blob + sizeof(int2) * P.cols.size());
            for (const Group& G : P.groups) {
                P.o_groups.push_back(blob);
                blob = align256(blob + sizeof(int2) * G.items.size());
            }
        }
        if ((rc = ensure_state(h, max_groups)) != BLFLS_OK) return rc;
        if ((rc = grow_bytes(h, &b->table, &b->table_cap, blob, "batch tables")) != BLFLS_OK) return rc;
        cudaError_t e = cudaEventSynchronize(b->host_free);   // last upload finished reading `host`
        if (e != cudaSuccess) return cuda_fail(e, "batch staging");
        if (blob > b->host_cap) {
            if (b->host) cudaFreeHost(b->host);
            b->host = nullptr;
            b->host_cap = 0;
            if ((e = cudaMallocHost(&b->host, blob)) != cudaSuccess) {
                cudaGetLastError();
                return fail(BLFLS_ENOMEM, std::string("pinned staging: ") + cudaGetErrorString(e));
            }
            b->host_cap = blob;
        }
        unsigned char* hb = static_cast<unsigned char*>(b->host);
        for (const Pass& P : passes) {
            std::memcpy(hb + P.o_table, P.table.data(), sizeof(BatchJob) * P.table.size());
            std::memcpy(hb + P.o_rows, P.rows.data(), sizeof(int2) * P.rows.size());
            std::memcpy(hb + P.o_cols, P.cols.data(), sizeof(int2) * P.cols.size());
            for (size_t g = 0; g < P.groups.size(); ++g)
                std::memcpy(hb + P.o_groups[g], P.groups[g].items.data(),
                            sizeof(int2) * P.groups[g].items.size());
        }

        // --- order after the caller's stream, upload, launch (graph on a repeated shape) ----------
        cudaEventRecord(b->ev_in, user);
        cudaStreamWaitEvent(b->main, b->ev_in, 0);
        if ((e = cudaMemcpyAsync(b->table, b->host, blob, cudaMemcpyHostToDevice, b->main)) != cudaSuccess)
            return cuda_fail(e, "batch table upload");
        cudaEventRecord(b->host_free, b->main);

        std::vector<long long> sig;
        sig.push_back((long long)(size_t)b->table);
        sig.push_back((long long)h->generation);
        for (const Pass& P : passes) {
            sig.push_back((long long)P.table.size());
            sig.push_back(P.total_rows);
            sig.push_back(P.total_cols);
            sig.push_back((long long)P.smem_rows);
            sig.push_back((long long)P.max_w);
            sig.push_back((long long)P.smem_cols);
            sig.push_back((long long)P.o_table);
            sig.push_back((long long)P.o_rows);
            sig.push_back((long long)P.o_cols);
            for (size_t g = 0; g < P.groups.size(); ++g) {
                const Group& G = P.groups[g];
                sig.push_back(((G.radius * 8 + G.range * 4 + G.prec) << 8) + G.tile_h);
                sig.push_back((long long)G.items.size());
                sig.push_back(G.total);
                sig.push_back((long long)P.o_groups[g]);
            }
            sig.push_back(-1);
        }
        auto git = b->graphs.find(sig);
        if (git != b->graphs.end()) {
            if ((e = cudaGraphLaunch(git->second, b->main)) != cudaSuccess) return cuda_fail(e, "graph launch");
        } else if (sig == b->last_sig) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            if ((e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
                return cuda_fail(e, "begin capture");
            const cudaError_t e1 = enqueue(h, passes);
            e = cudaStreamEndCapture(b->main, &graph);
            if (e1 != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                return cuda_fail(e1, "batched launch (capture)");
            }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
            if (b->graphs.size() >= 16) {
                cudaGraphExecDestroy(b->graphs.begin()->second);
                b->graphs.erase(b->graphs.begin());
            }
            b->graphs.emplace(sig, exec);
            if ((e = cudaGraphLaunch(exec, b->main)) != cudaSuccess) return cuda_fail(e, "graph launch");
        } else {
            if ((e = enqueue(h, passes)) != cudaSuccess) return cuda_fail(e, "batched launch");
            b->last_sig = sig;
        }
        cudaEventRecord(b->ev_out, b->main);
        if ((e = cudaStreamWaitEvent(user, b->ev_out, 0)) != cudaSuccess) return cuda_fail(e, "batch join");
    }

    for (int i : single) {
        const blfls_job& j = jobs[i];
        if ((rc = run_smooth(h, j.img, j.out, j.H, j.W, j.C, j.lambda, j.sigma_s, j.sigma_r,
                             j.radius, j.iters, j.prec, user)) != BLFLS_OK)
            return rc;
    }
    return BLFLS_OK;
}

}  // namespace blfls
