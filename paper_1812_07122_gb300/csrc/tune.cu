// Autotuner for the launch shapes of the smoother (no counterpart in the paper).
//
// Two shapes are tuned, each by timing every candidate with CUDA events on a synthetic image
// generated on the device and keeping the fastest:
//   * K1 tile height (8, 16, 32 or 64 rows of the 32-wide bilateral tile), per (radius,
//     precision): taller tiles amortise the halo, shorter ones use less shared memory and raise
//     occupancy;
//   * K3 column block (1..16 columns per CTA), per column-transform length class
//     (ceil(log2 L)): wider blocks make longer contiguous reads, narrower ones fit more CTAs.
// The table is a small JSON file (written by blfls_autotune, read by blfls_create); shapes change
// speed only, never results (the arithmetic per pixel is the same for every shape).
#include "handle.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

namespace blfls {

namespace {

// Smooth periodic pattern plus hashed noise in [0, 1]: gives the range kernel realistic work.
__global__ void synth_field(float* out, int H, int W, int C, unsigned seed)
{
    const size_t n = (size_t)C * H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int x = int(i % W), y = int((i / W) % H), c = int(i / ((size_t)W * H));
        unsigned hsh = (unsigned)i * 2654435761u ^ (seed + 97u * c);
        hsh ^= hsh >> 15;
        hsh *= 2246822519u;
        hsh ^= hsh >> 13;
        const float noise = (hsh & 0xffff) * (1.0f / 65535.0f) - 0.5f;
        const float s = 0.5f + 0.3f * __sinf(6.2831853f * (3.0f * x / W + 2.0f * y / H + 0.1f * c));
        const float step = ((x / 37 + y / 53) & 1) ? 0.2f : 0.f;
        out[i] = fminf(1.f, fmaxf(0.f, s + step + 0.03f * noise));
    }
}

int find_int(const std::string& obj, const char* key, int* out)
{
    const std::string k = std::string("\"") + key + "\"";
    const size_t p = obj.find(k);
    if (p == std::string::npos) return 0;
    const size_t c = obj.find(':', p + k.size());
    if (c == std::string::npos) return 0;
    return std::sscanf(obj.c_str() + c + 1, " %d", out) == 1;
}

int log2_class(int L)
{
    int c = 0;
    while ((1 << c) < L) ++c;
    return c;
}

}  // namespace

int tuned_tile_h(const blfls_handle* h, int radius, int prec)
{
    auto it = h->tune_tile_h.find(std::make_pair(radius, prec));
    return it == h->tune_tile_h.end() ? 32 : it->second;
}

int tuned_col_block(const blfls_handle* h, int L)
{
    auto it = h->tune_col_block.find(log2_class(L));
    return it == h->tune_col_block.end() ? 0 : it->second;
}

int load_tune_table(blfls_handle* h, const char* path)
{
    if (!path) return BLFLS_OK;
    std::ifstream in(path);
    if (!in) return BLFLS_OK;   // a missing table selects the defaults
    std::stringstream ss;
    ss << in.rdbuf();
    const std::string text = ss.str();
    size_t pos = 0;
    while ((pos = text.find('{', pos + 1)) != std::string::npos) {
        const size_t end = text.find('}', pos);
        if (end == std::string::npos) break;
        const std::string obj = text.substr(pos, end - pos + 1);
        int r, p, t, l, cb;
        if (find_int(obj, "radius", &r) && find_int(obj, "prec", &p) && find_int(obj, "tile_h", &t))
            h->tune_tile_h[std::make_pair(r, p)] = blf_tile_height(t);
        else if (find_int(obj, "log2_len", &l) && find_int(obj, "col_block", &cb) && cb >= 1 && cb <= 16)
            h->tune_col_block[l] = cb;
    }
    return BLFLS_OK;
}

int save_tune_table(const blfls_handle* h, const char* path)
{
    std::ofstream out(path);
    if (!out) return fail(BLFLS_EINVAL, std::string("cannot write tune table ") + path);
    out << "{\"blfls_tune_table\": 1,\n \"k1_tile_h\": [";
    bool first = true;
    for (const auto& kv : h->tune_tile_h) {
        out << (first ? "\n  " : ",\n  ") << "{\"radius\": " << kv.first.first << ", \"prec\": "
            << kv.first.second << ", \"tile_h\": " << kv.second << "}";
        first = false;
    }
    out << "],\n \"k3_col_block\": [";
    first = true;
    for (const auto& kv : h->tune_col_block) {
        out << (first ? "\n  " : ",\n  ") << "{\"log2_len\": " << kv.first
            << ", \"col_block\": " << kv.second << "}";
        first = false;
    }
    out << "]}\n";
    return out ? BLFLS_OK : fail(BLFLS_EINVAL, "writing the tune table failed");
}

}  // namespace blfls

using namespace blfls;

extern "C" int blfls_autotune(blfls_handle* h, int H, int W, int C, int radius, int prec,
                              const char* table_path)
{
    if (!h) return fail(BLFLS_EINVAL, "handle is NULL");
    int rc;
    if (H < 1 || W < 1 || H > BLFLS_MAX_DIM || W > BLFLS_MAX_DIM || C < 1 || C > BLFLS_MAX_CHANNELS)
        return fail(BLFLS_EINVAL, "bad autotune image size");
    if ((rc = check_blf_args(H, W, 2.0f, 0.1f, radius, prec)) != BLFLS_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return fail(BLFLS_ECUDA, "cudaSetDevice failed");
    const size_t n = (size_t)C * H * W;
    float* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 3 * n * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BLFLS_ENOMEM, std::string("autotune buffers: ") + cudaGetErrorString(e));
    }
    float* img = buf;
    float* ex = buf + n;
    float* ey = buf + 2 * n;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    synth_field<<<256, 256, 0, s>>>(img, H, W, C, 12345u);

    auto time_it = [&](auto&& launch) -> float {
        launch();   // warm-up
        float best = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a, s);
            launch();
            cudaEventRecord(b, s);
            cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            best = std::min(best, ms);
        }
        return best;
    };

    // K1 tile height (radii handled by the unrolled kernels only)
    if (radius <= blf_batch_max_radius()) {
        const int cands[4] = {8, 16, 32, 64};
        int best_t = 32;
        float best_ms = 1e30f;
        for (int t : cands) {
            if (2 * radius + 1 > H && t > 8) continue;
            const BlfParams bp{H, W, radius, 2.0f + radius / 2.0f, 0.1f, prec, t};
            const float ms = time_it([&] { launch_blf_residual(img, ex, ey, C, bp, nullptr, s); });
            if (ms < best_ms) {
                best_ms = ms;
                best_t = t;
            }
        }
        h->tune_tile_h[std::make_pair(radius, prec)] = best_t;
    }

    // K3 column block for the column-transform length H
    const FftPlanDev *rp = nullptr, *cp = nullptr;
    if ((rc = get_plan(h, W, &rp)) == BLFLS_OK && (rc = get_plan(h, H, &cp)) == BLFLS_OK) {
        float2* spec = nullptr;
        e = cudaMalloc(&spec, sizeof(float2) * (size_t)H * (W / 2 + 1));
        if (e == cudaSuccess) {
            int best_cb = 0;
            float best_ms = 1e30f;
            std::vector<int> timed;
            for (int cb : {1, 2, 4, 7, 8, 13, 16}) {
                // each block size a column driver really takes, once
                const int eff = solve_effective_col_block(*cp, W, cb, h->num_sms);
                if (eff != cb || std::find(timed.begin(), timed.end(), eff) != timed.end()) continue;
                timed.push_back(eff);
                const SolveParams sp{H, W, 30.0f, cb};
                const float ms = time_it([&] {
                    launch_solve_residual(img, ex, ey, img + 0 * n, spec, *rp, *cp, rp->lap,
                                          cp->lap, sp, s, h->num_sms);
                });
                if (ms < best_ms) {
                    best_ms = ms;
                    best_cb = cb;
                }
            }
            if (best_cb > 0) h->tune_col_block[log2_class(cp->L)] = best_cb;
            cudaFree(spec);
        } else {
            cudaGetLastError();
        }
    }
    e = cudaStreamSynchronize(s);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamDestroy(s);
    cudaFree(buf);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (rc != BLFLS_OK) return rc;
    if (table_path) return save_tune_table(h, table_path);
    return BLFLS_OK;
}
