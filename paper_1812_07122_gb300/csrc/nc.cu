// NC-LS (Section III-D): BLF-LS with the bilateral filter replaced by the normalised convolution
// of the domain transform.  Per channel and gradient field g (the periodic forward difference of
// the image along x or y), with a = sigma_s / sigma_r:
//   k8_grad      g for both fields;
//   k8_dt_rows   ct_h[y][x] = sum_{x' = 1..x} (1 + a |g[y][x'] - g[y][x'-1]|), and the row period
//                T_h[y] = ct_h[y][W-1] + 1 + a |g[y][0] - g[y][W-1]|, summed sequentially in FP32
//                by one thread per row (rows staged 32 x 32 through shared memory so the loads are
//                coalesced);
//   k8_dt_cols   the same down every column (one thread per column, coalesced);
//   k8_nc_rows / k8_nc_cols  one box pass of radius r: the mean of the samples j of the periodic
//                line with |(ct[j] + k T) - ct[i]| <= r (k = the period of j; a contiguous run
//                scanned outward from i), N iterations with
//                r_k = sigma_s sqrt(3) 2^(N-k) / sqrt(4^N - 1) sqrt(3), rows then columns; the last
//                column pass writes the residual e = v - g for the Fourier solve.
// Inclusion is a floating-point decision: increments are one FP32 multiply then one add (no fused
// multiply-add), the running sum is sequential, the test is FP32 -- the operations the FP64
// oracle takes in FP32.  All passes are HBM/L1-bound streams.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace blfls {

namespace {

constexpr int kNcThreads = 256;

__global__ void __launch_bounds__(kNcThreads) k8_grad(const float* __restrict__ f,
                                                     float* __restrict__ gx,
                                                     float* __restrict__ gy, int H, int W)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const float c = f[i];
        gx[i] = f[(size_t)y * W + (x + 1 == W ? 0 : x + 1)] - c;
        gy[i] = f[(size_t)(y + 1 == H ? 0 : y + 1) * W + x] - c;
    }
}

__device__ __forceinline__ float dt_step(float a, float cur, float prev)
{
    return __fadd_rn(1.0f, __fmul_rn(a, fabsf(cur - prev)));
}

// One warp per 32 rows.
__global__ void __launch_bounds__(32) k8_dt_rows(const float* __restrict__ g,
                                                 float* __restrict__ ct, float* __restrict__ T,
                                                 int H, int W, float a)
{
    __shared__ float tile[32][33];
    const int lane = threadIdx.x;
    const int y0 = blockIdx.x * 32;
    const int my = y0 + lane;
    float acc = 0.f, prev = 0.f, first = 0.f;
    for (int x0 = 0; x0 < W; x0 += 32) {
        for (int r = 0; r < 32; ++r) {
            const int y = y0 + r, x = x0 + lane;
            tile[r][lane] = (y < H && x < W) ? g[(size_t)y * W + x] : 0.f;
        }
        __syncwarp();
        const int n = min(32, W - x0);
        for (int c = 0; c < n; ++c) {
            const float v = tile[lane][c];
            if (x0 + c == 0) {
                first = v;
            } else {
                acc = __fadd_rn(acc, dt_step(a, v, prev));
            }
            prev = v;
            tile[lane][c] = acc;
        }
        __syncwarp();
        for (int r = 0; r < 32; ++r) {
            const int y = y0 + r, x = x0 + lane;
            if (y < H && x < W) ct[(size_t)y * W + x] = tile[r][lane];
        }
        __syncwarp();
    }
    if (my < H) T[my] = __fadd_rn(acc, dt_step(a, first, prev));
}

__global__ void __launch_bounds__(kNcThreads) k8_dt_cols(const float* __restrict__ g,
                                                        float* __restrict__ ct,
                                                        float* __restrict__ T, int H, int W,
                                                        float a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    float acc = 0.f;
    const float first = g[x];
    float prev = first;
    ct[x] = 0.f;
    for (int y = 1; y < H; ++y) {
        const float v = g[(size_t)y * W + x];
        acc = __fadd_rn(acc, dt_step(a, v, prev));
        ct[(size_t)y * W + x] = acc;
        prev = v;
    }
    T[x] = __fadd_rn(acc, dt_step(a, first, prev));
}

// The transform grows by at least 1 per sample (strictly increasing, also in FP32 below 2^24), so
// the samples inside a box form one run around i: each side is scanned outward until the first
// sample outside, with the period index k tracked by counting wraps.  The included set is the
// one the per-sample test gives.
__device__ __forceinline__ void box_side(const float* c, const float* v, size_t stride, int n,
                                         int i, int step, float ci, float Tp, float r, int R,
                                         float& acc, float& cnt)
{
    int j = i, k = 0;
    for (int d = 1; d <= R; ++d) {
        j += step;
        if (j == n) { j = 0; ++k; }
        if (j < 0) { j = n - 1; --k; }
        const float cj = __fadd_rn(c[(size_t)j * stride], __fmul_rn((float)k, Tp));
        if (fabsf(cj - ci) > r) break;
        acc += v[(size_t)j * stride];
        cnt += 1.f;
    }
}

// Box pass along x of radius r (R = floor(r)).
__global__ void __launch_bounds__(kNcThreads) k8_nc_rows(const float* __restrict__ v,
                                                        const float* __restrict__ ct,
                                                        const float* __restrict__ T,
                                                        float* __restrict__ out, int H, int W,
                                                        float r, int R)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const float* crow = ct + (size_t)y * W;
        const float* vrow = v + (size_t)y * W;
        const float ci = crow[x], Ty = T[y];
        float acc = vrow[x], cnt = 1.f;
        box_side(crow, vrow, 1, W, x, 1, ci, Ty, r, R, acc, cnt);
        box_side(crow, vrow, 1, W, x, -1, ci, Ty, r, R, acc, cnt);
        out[i] = acc / cnt;
    }
}

// Box pass along y; when g is not null the output is the residual (mean - g).
__global__ void __launch_bounds__(kNcThreads) k8_nc_cols(const float* __restrict__ v,
                                                        const float* __restrict__ ct,
                                                        const float* __restrict__ T,
                                                        float* __restrict__ out,
                                                        const float* __restrict__ g, int H,
                                                        int W, float r, int R)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const float ci = ct[i], Tx = T[x];
        float acc = v[i], cnt = 1.f;
        box_side(ct + x, v + x, (size_t)W, H, y, 1, ci, Tx, r, R, acc, cnt);
        box_side(ct + x, v + x, (size_t)W, H, y, -1, ci, Tx, r, R, acc, cnt);
        const float m = acc / cnt;
        out[i] = g ? m - g[i] : m;
    }
}

int nc_blocks(size_t n, int num_sms)
{
    const size_t want = (n + kNcThreads - 1) / kNcThreads;
    return (int)std::max<size_t>(1, std::min(want, (size_t)num_sms * 8));
}

}  // namespace

cudaError_t launch_nc_residuals(const float* f, float* ex, float* ey, int H, int W,
                                float sigma_s, float sigma_r, int n_iter, float* scratch,
                                cudaStream_t s, int num_sms)
{
    const size_t plane = (size_t)H * W;
    float* gx = scratch;
    float* gy = gx + plane;
    float* ct_h = gy + plane;
    float* ct_v = ct_h + plane;
    float* va = ct_v + plane;
    float* vb = va + plane;
    float* T_h = vb + plane;
    float* T_v = T_h + H;
    const float a = std::isfinite(sigma_r) ? sigma_s / sigma_r : 0.0f;   // FP32 division
    const int nb = nc_blocks(plane, num_sms);
    k8_grad<<<nb, kNcThreads, 0, s>>>(f, gx, gy, H, W);
    for (int field = 0; field < 2; ++field) {
        const float* g = field == 0 ? gx : gy;
        float* e = field == 0 ? ex : ey;
        k8_dt_rows<<<(H + 31) / 32, 32, 0, s>>>(g, ct_h, T_h, H, W, a);
        k8_dt_cols<<<(W + kNcThreads - 1) / kNcThreads, kNcThreads, 0, s>>>(g, ct_v, T_v, H, W, a);
        const float* cur = g;
        for (int k = 1; k <= n_iter; ++k) {
            const double rk = (double)sigma_s * std::sqrt(3.0) * std::pow(2.0, n_iter - k) /
                              std::sqrt(std::pow(4.0, n_iter) - 1.0) * std::sqrt(3.0);
            const float r = (float)rk;
            const int R = (int)std::floor(r);
            k8_nc_rows<<<nb, kNcThreads, 0, s>>>(cur, ct_h, T_h, va, H, W, r, R);
            const bool last = k == n_iter;
            k8_nc_cols<<<nb, kNcThreads, 0, s>>>(va, ct_v, T_v, last ? e : vb, last ? g : nullptr,
                                                 H, W, r, R);
            cur = vb;
        }
    }
    return cudaGetLastError();
}

size_t nc_scratch_floats(int H, int W) { return 6 * (size_t)H * W + (size_t)H + (size_t)W; }

}  // namespace blfls
