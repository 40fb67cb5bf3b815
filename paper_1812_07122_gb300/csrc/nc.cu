// NC-LS (Section III-D): BLF-LS with the bilateral filter replaced by the normalised convolution
// of the domain transform.  Per channel and gradient field g (the periodic forward difference of
// the image along x or y), with a = sigma_s / sigma_r:
//   k8_grad      g for both fields;
//   k8_dt_rows   ct_h[y][x] = sum_{x' = 1..x} (1 + a |g[y][x'] - g[y][x'-1]|) and the row period
//                T_h[y] = ct_h[y][W-1] + 1 + a |g[y][0] - g[y][W-1]|: one CTA per row, a block scan
//                over 2048-sample chunks staged in shared memory;
//   k8_dt_cols   the same down every column: a CTA per 32 columns, each warp one segment of rows
//                (segment totals first, then the segments re-scanned from their offsets);
//   k8_nc_rows / k8_nc_cols  one box pass of radius r: the mean of the samples j of the periodic
//                line with |(ct[j] + k T) - ct[i]| <= r (k = the period of j; a contiguous run
//                around i), tiles staged in shared memory and one thread per strip of 8 samples
//                holding the strip and its neighbourhood in registers, N iterations with
//                r_k = sigma_s sqrt(3) 2^(N-k) / sqrt(4^N - 1) sqrt(3), rows then columns; the last
//                column pass writes the residual e = v - g for the Fourier solve.
// The transform is exact, so which samples enter a box does not depend on the summation order:
// an increment is one FP32 multiply then one add (no fused multiply-add), capped at 2^20 (beyond
// every box radius, so no decision changes); being an FP32 value >= 1 it is a multiple of 2^-23,
// and ct and T are held as 64-bit integers in units of 2^-23 (at most 2^43 per step, 2^56 per
// line); the box test is an integer comparison against floor(r 2^23).
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace blfls {

namespace {

constexpr int kNcThreads = 256;
constexpr float kIncCap = 1048576.0f;      // 2^20
constexpr float kUnit = 8388608.0f;        // 2^23
constexpr int kDtPer = 8;                  // row scan: samples per thread
constexpr int kDtChunk = kNcThreads * kDtPer;
constexpr int kColSegs = 32;               // column scan: row segments (warps) per CTA

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

// One step of the transform in units of 2^-23 (exact: v 2^23 is an integer below 2^44).
__device__ __forceinline__ long long dt_inc(float a, float cur, float prev)
{
    const float v = fminf(__fadd_rn(1.0f, __fmul_rn(a, fabsf(cur - prev))), kIncCap);
    return __float2ll_rz(v * kUnit);
}

// Exclusive block scan of one value per thread (kNcThreads threads); *total receives the sum.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* warp_sums,
                                                     long long* total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_sums[w] = inc;
    __syncthreads();
    long long before = 0, all = 0;
#pragma unroll
    for (int k = 0; k < kNcThreads / 32; ++k) {
        const long long s = warp_sums[k];
        before += k < w ? s : 0;
        all += s;
    }
    __syncthreads();   // warp_sums may be rewritten by the next call
    *total = all;
    return before + inc - v;
}

// padded shared-memory slots: conflict-free reads of 8 consecutive samples per thread
__device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// One CTA per row.
__global__ void __launch_bounds__(kNcThreads) k8_dt_rows(const float* __restrict__ g,
                                                        long long* __restrict__ ct,
                                                        long long* __restrict__ T, int H, int W,
                                                        float a)
{
    __shared__ float sg[kDtChunk + kDtChunk / 32 + 1];
    __shared__ long long sc[kDtChunk + kDtChunk / 16];
    __shared__ long long warp_sums[kNcThreads / 32];
    const int y = blockIdx.x;
    const float* row = g + (size_t)y * W;
    long long* crow = ct + (size_t)y * W;
    long long carry = 0;
    for (int x0 = 0; x0 < W; x0 += kDtChunk) {
        const int n = min(kDtChunk, W - x0);
        for (int i = threadIdx.x; i < n; i += kNcThreads) sg[pad32(i)] = row[x0 + i];
        __syncthreads();
        const int b = threadIdx.x * kDtPer;
        long long loc[kDtPer];
        long long sum = 0;
        float prev = b == 0 ? (x0 > 0 ? row[x0 - 1] : 0.f) : sg[pad32(b - 1)];
#pragma unroll
        for (int k = 0; k < kDtPer; ++k) {
            const int i = b + k;
            const float cur = i < n ? sg[pad32(i)] : prev;
            if (i < n && x0 + i > 0) sum += dt_inc(a, cur, prev);
            loc[k] = sum;
            prev = cur;
        }
        long long chunk_total;
        const long long before = carry + block_excl_scan(sum, warp_sums, &chunk_total);
#pragma unroll
        for (int k = 0; k < kDtPer; ++k)
            if (b + k < n) sc[pad16(b + k)] = before + loc[k];
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += kNcThreads) crow[x0 + i] = sc[pad16(i)];
        carry += chunk_total;
        __syncthreads();   // sg and sc are refilled by the next chunk
    }
    if (threadIdx.x == 0) T[y] = carry + dt_inc(a, row[0], row[W - 1]);
}

// A CTA per 32 columns; warp w takes rows [w S, (w + 1) S) of them, S = ceil(H / kColSegs).
__global__ void __launch_bounds__(32 * kColSegs) k8_dt_cols(const float* __restrict__ g,
                                                           long long* __restrict__ ct,
                                                           long long* __restrict__ T, int H,
                                                           int W, float a)
{
    __shared__ long long seg[kColSegs][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int S = (H + kColSegs - 1) / kColSegs;
    const int y0 = w * S, y1 = min(H, y0 + S);
    const bool live = x < W && y0 < y1;
    const float* col = g + x;
    long long sum = 0;
    if (live) {
        float prev = y0 > 0 ? col[(size_t)(y0 - 1) * W] : 0.f;
#pragma unroll 16
        for (int y = y0; y < y1; ++y) {
            const float cur = col[(size_t)y * W];
            if (y > 0) sum += dt_inc(a, cur, prev);
            prev = cur;
        }
    }
    seg[w][lane] = sum;
    __syncthreads();
    long long off = 0, total = 0;
#pragma unroll
    for (int k = 0; k < kColSegs; ++k) {
        off += k < w ? seg[k][lane] : 0;
        total += seg[k][lane];
    }
    if (live) {
        float prev = y0 > 0 ? col[(size_t)(y0 - 1) * W] : 0.f;
        long long acc = off;
#pragma unroll 16
        for (int y = y0; y < y1; ++y) {
            const float cur = col[(size_t)y * W];
            if (y > 0) acc += dt_inc(a, cur, prev);
            ct[(size_t)y * W + x] = acc;
            prev = cur;
        }
    }
    if (w == 0 && x < W) T[x] = total + dt_inc(a, col[0], col[(size_t)(H - 1) * W]);
}

// Box means by a sliding window.  The transform grows by at least 1 per sample (strictly
// increasing, copies of the line one period over shifted by T), so the samples j inside the box
// of sample i, |ct(j) - ct(i)| <= r, form one run [lo(i), hi(i)] of the unwrapped line, and both
// ends only move forward as i does.  A thread takes kNcRun consecutive samples of one line: it
// finds the first sample's run by scanning outward, then for every next sample advances hi over
// the samples that have come inside and lo past those that have left, keeping the run's sum
// (Neumaier-compensated FP32) and count.  The set is exactly the per-sample test's; only the
// order of the additions differs from summing the run afresh.
constexpr int kNcRun = 32;

struct LinePos {   // position p of the unwrapped line: index p mod n and the shift k T
    int m;
    long long shift;
};

__device__ __forceinline__ void step_fwd(LinePos& q, int n, long long Tp)
{
    if (++q.m == n) { q.m = 0; q.shift += Tp; }
}
__device__ __forceinline__ void step_back(LinePos& q, int n, long long Tp)
{
    if (--q.m < 0) { q.m = n - 1; q.shift -= Tp; }
}

__device__ __forceinline__ void nsum_add(float& s, float& comp, float x)
{
    const float t = __fadd_rn(s, x);
    comp += fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
    s = t;
}

// Samples [i0, i1) of one line (length n, element stride st): out = box mean, minus g when given.
__device__ __forceinline__ void box_run(const long long* __restrict__ c,
                                        const float* __restrict__ v, size_t st, int n,
                                        long long Tp, long long rq, int i0, int i1,
                                        float* __restrict__ out, const float* __restrict__ g)
{
    auto C = [&](const LinePos& q) { return c[(size_t)q.m * st] + q.shift; };
    LinePos lo{i0, 0}, hi{i0, 0};
    long long ci = c[(size_t)i0 * st];
    float sum = v[(size_t)i0 * st], comp = 0.f;
    int cnt = 1;
    for (;;) {   // the first sample's run, upwards
        LinePos nx = hi;
        step_fwd(nx, n, Tp);
        if (C(nx) - ci > rq) break;
        hi = nx;
        nsum_add(sum, comp, v[(size_t)hi.m * st]);
        ++cnt;
    }
    for (;;) {   // and downwards
        LinePos pv = lo;
        step_back(pv, n, Tp);
        if (ci - C(pv) > rq) break;
        lo = pv;
        nsum_add(sum, comp, v[(size_t)lo.m * st]);
        ++cnt;
    }
    for (int i = i0;;) {
        const float m = (sum + comp) / (float)cnt;
        out[(size_t)i * st] = g ? m - g[(size_t)i * st] : m;
        if (++i >= i1) break;
        ci = c[(size_t)i * st];
        for (;;) {   // samples that have come inside at the top
            LinePos nx = hi;
            step_fwd(nx, n, Tp);
            if (C(nx) - ci > rq) break;
            hi = nx;
            nsum_add(sum, comp, v[(size_t)hi.m * st]);
            ++cnt;
        }
        while (ci - C(lo) > rq) {   // and those that have left at the bottom (lo <= i stays)
            nsum_add(sum, comp, -v[(size_t)lo.m * st]);
            --cnt;
            step_fwd(lo, n, Tp);
        }
    }
}

// Box means for radii up to RM samples (R = floor(r) <= RM): a thread takes a strip of kNcStrip
// consecutive samples of one line and holds the strip plus RM samples on either side in
// registers (one load per sample instead of one per sample and neighbour); each sample's run is
// then scanned outward over the registers, every comparison taken (predicated, no early exit).
constexpr int kNcStrip = 8;

template <int RM>
__device__ __forceinline__ void strip_means(const long long (&cw)[kNcStrip + 2 * RM],
                                            const float (&vw)[kNcStrip + 2 * RM], long long rq,
                                            float (&mean)[kNcStrip])
{
#pragma unroll
    for (int j = 0; j < kNcStrip; ++j) {
        const long long top = cw[RM + j] + rq, bottom = cw[RM + j] - rq;
        float acc = vw[RM + j], cnt = 1.f;
        bool up = true, dn = true;
#pragma unroll
        for (int d = 1; d <= RM; ++d) {
            up = up && cw[RM + j + d] <= top;
            dn = dn && cw[RM + j - d] >= bottom;
            if (up) { acc += vw[RM + j + d]; cnt += 1.f; }
            if (dn) { acc += vw[RM + j - d]; cnt += 1.f; }
        }
        mean[j] = acc / cnt;
    }
}

// Along x: a CTA stages a tile of 32 rows x 64 columns of the transform and the values, with RM
// samples of periodic neighbourhood on either side, in shared memory with coalesced loads;
// thread (lane, warp) takes row `lane` of the tile and a strip of kNcStrip columns (warp) and
// reads the strip's window from shared memory (odd pitches put the lanes' rows in distinct
// banks); the means go back through shared memory for coalesced stores.
constexpr int kTileLong = kNcStrip * (kNcThreads / 32);   // 64 samples along the row
constexpr int kTileWide = 32;                             // 32 rows
template <int RM>
__global__ void __launch_bounds__(kNcThreads) k8_nc_rows_strip(const float* __restrict__ v,
                                                              const long long* __restrict__ ct,
                                                              const long long* __restrict__ T,
                                                              float* __restrict__ out, int H,
                                                              int W, long long rq)
{
    constexpr int NW = kNcStrip + 2 * RM;
    constexpr int SPAN = kTileLong + 2 * RM;
    constexpr int PC = SPAN | 1, PO = kTileLong + 1;
    __shared__ long long sc[kTileWide * PC];
    __shared__ float sv[kTileWide * PC];
    __shared__ float so[kTileWide * PO];
    const int tiles_x = (W + kTileLong - 1) / kTileLong;
    const int y0 = (blockIdx.x / tiles_x) * kTileWide, x0 = (blockIdx.x % tiles_x) * kTileLong;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = w; r < kTileWide; r += kNcThreads / 32) {
        const int y = y0 + r;
        if (y >= H) break;
        const long long Ty = T[y];
        for (int q = lane; q < SPAN; q += 32) {
            int p = x0 - RM + q;                   // unwrapped column
            long long sh = 0;
            while (p < 0) { p += W; sh -= Ty; }
            while (p >= W) { p -= W; sh += Ty; }
            sc[r * PC + q] = ct[(size_t)y * W + p] + sh;
            sv[r * PC + q] = v[(size_t)y * W + p];
        }
    }
    __syncthreads();
    if (y0 + lane < H) {
        long long cw[NW];
        float vw[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            cw[q] = sc[lane * PC + w * kNcStrip + q];
            vw[q] = sv[lane * PC + w * kNcStrip + q];
        }
        float mean[kNcStrip];
        strip_means<RM>(cw, vw, rq, mean);
#pragma unroll
        for (int j = 0; j < kNcStrip; ++j) so[lane * PO + w * kNcStrip + j] = mean[j];
    }
    __syncthreads();
    for (int r = w; r < kTileWide; r += kNcThreads / 32) {
        const int y = y0 + r;
        if (y >= H) break;
        for (int q = lane; q < kTileLong; q += 32)
            if (x0 + q < W) out[(size_t)y * W + x0 + q] = so[r * PO + q];
    }
}

// Along y: one thread per strip of kNcStrip rows of one column, adjacent threads on adjacent
// columns, the window loaded straight from global memory (coalesced across the warp; the
// neighbouring strips' overlap comes from L1/L2); when g is not null the output is the
// residual (mean - g).
template <int RM>
__global__ void __launch_bounds__(kNcThreads) k8_nc_cols_strip(const float* __restrict__ v,
                                                              const long long* __restrict__ ct,
                                                              const long long* __restrict__ T,
                                                              float* __restrict__ out,
                                                              const float* __restrict__ g,
                                                              int H, int W, long long rq)
{
    constexpr int NW = kNcStrip + 2 * RM;
    const int strips = (H + kNcStrip - 1) / kNcStrip;
    const size_t total = (size_t)W * strips;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / W), x = (int)(t - (size_t)k * W);
        const long long Tx = T[x];
        int m = k * kNcStrip - RM;
        long long sh = 0;
        while (m < 0) { m += H; sh -= Tx; }
        long long cw[NW];
        float vw[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            cw[q] = ct[(size_t)m * W + x] + sh;
            vw[q] = v[(size_t)m * W + x];
            if (++m == H) { m = 0; sh += Tx; }
        }
        float mean[kNcStrip];
        strip_means<RM>(cw, vw, rq, mean);
#pragma unroll
        for (int j = 0; j < kNcStrip; ++j) {
            const int y = k * kNcStrip + j;
            if (y < H) {
                const size_t i = (size_t)y * W + x;
                out[i] = g ? mean[j] - g[i] : mean[j];
            }
        }
    }
}

// Radii above the strip kernels: one thread per run of kNcRun samples with a sliding window.
__global__ void __launch_bounds__(kNcThreads) k8_nc_rows(const float* __restrict__ v,
                                                        const long long* __restrict__ ct,
                                                        const long long* __restrict__ T,
                                                        float* __restrict__ out, int H, int W,
                                                        long long rq)
{
    const int runs = (W + kNcRun - 1) / kNcRun;
    const size_t total = (size_t)H * runs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(t / runs), k = (int)(t - (size_t)y * runs);
        const size_t row = (size_t)y * W;
        box_run(ct + row, v + row, 1, W, T[y], rq, k * kNcRun, min(W, (k + 1) * kNcRun),
                out + row, nullptr);
    }
}

__global__ void __launch_bounds__(kNcThreads) k8_nc_cols(const float* __restrict__ v,
                                                        const long long* __restrict__ ct,
                                                        const long long* __restrict__ T,
                                                        float* __restrict__ out,
                                                        const float* __restrict__ g, int H,
                                                        int W, long long rq)
{
    const int runs = (H + kNcRun - 1) / kNcRun;
    const size_t total = (size_t)W * runs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / W), x = (int)(t - (size_t)k * W);
        box_run(ct + x, v + x, (size_t)W, H, T[x], rq, k * kNcRun, min(H, (k + 1) * kNcRun),
                out + x, g ? g + x : nullptr);
    }
}

int nc_blocks(size_t n, int num_sms)
{
    const size_t want = (n + kNcThreads - 1) / kNcThreads;
    return (int)std::max<size_t>(1, std::min(want, (size_t)num_sms * 8));
}

template <int RM>
void box_pass_strips(const float* v, const long long* ct_h, const long long* T_h, float* mid,
                     const long long* ct_v, const long long* T_v, float* out, const float* g,
                     int H, int W, long long rq, int num_sms, cudaStream_t s)
{
    const int row_tiles = ((H + kTileWide - 1) / kTileWide) * ((W + kTileLong - 1) / kTileLong);
    k8_nc_rows_strip<RM><<<row_tiles, kNcThreads, 0, s>>>(v, ct_h, T_h, mid, H, W, rq);
    const size_t strips = (size_t)W * ((H + kNcStrip - 1) / kNcStrip);
    k8_nc_cols_strip<RM><<<nc_blocks(strips, num_sms), kNcThreads, 0, s>>>(mid, ct_v, T_v, out, g,
                                                                          H, W, rq);
}

// One iteration: box means along the rows of v into mid, then along the columns of mid into out
// (minus g when given).  Strip kernels for R <= 16, sliding windows above.
void nc_box_pass(const float* v, const long long* ct_h, const long long* T_h, float* mid,
                 const long long* ct_v, const long long* T_v, float* out, const float* g, int H,
                 int W, long long rq, int R, int num_sms, cudaStream_t s)
{
    if (R <= 1) return box_pass_strips<1>(v, ct_h, T_h, mid, ct_v, T_v, out, g, H, W, rq, num_sms, s);
    if (R <= 2) return box_pass_strips<2>(v, ct_h, T_h, mid, ct_v, T_v, out, g, H, W, rq, num_sms, s);
    if (R <= 4) return box_pass_strips<4>(v, ct_h, T_h, mid, ct_v, T_v, out, g, H, W, rq, num_sms, s);
    if (R <= 8) return box_pass_strips<8>(v, ct_h, T_h, mid, ct_v, T_v, out, g, H, W, rq, num_sms, s);
    if (R <= 16) return box_pass_strips<16>(v, ct_h, T_h, mid, ct_v, T_v, out, g, H, W, rq, num_sms, s);
    k8_nc_rows<<<nc_blocks((size_t)H * ((W + kNcRun - 1) / kNcRun), num_sms), kNcThreads, 0, s>>>(
        v, ct_h, T_h, mid, H, W, rq);
    k8_nc_cols<<<nc_blocks((size_t)W * ((H + kNcRun - 1) / kNcRun), num_sms), kNcThreads, 0, s>>>(
        mid, ct_v, T_v, out, g, H, W, rq);
}

}  // namespace

cudaError_t launch_nc_residuals(const float* f, float* ex, float* ey, int H, int W,
                                float sigma_s, float sigma_r, int n_iter, float* scratch,
                                cudaStream_t s, int num_sms)
{
    const size_t plane = (size_t)H * W;
    long long* ct_h = reinterpret_cast<long long*>(scratch);   // 8-byte aligned (device allocation)
    long long* ct_v = ct_h + plane;
    long long* T_h = ct_v + plane;
    long long* T_v = T_h + H;
    float* gx = reinterpret_cast<float*>(T_v + W);
    float* gy = gx + plane;
    float* va = gy + plane;
    float* vb = va + plane;
    const float a = std::isfinite(sigma_r) ? sigma_s / sigma_r : 0.0f;   // FP32 division
    const int nb = nc_blocks(plane, num_sms);
    k8_grad<<<nb, kNcThreads, 0, s>>>(f, gx, gy, H, W);
    for (int field = 0; field < 2; ++field) {
        const float* g = field == 0 ? gx : gy;
        float* e = field == 0 ? ex : ey;
        k8_dt_rows<<<H, kNcThreads, 0, s>>>(g, ct_h, T_h, H, W, a);
        k8_dt_cols<<<(W + 31) / 32, 32 * kColSegs, 0, s>>>(g, ct_v, T_v, H, W, a);
        const float* cur = g;
        for (int k = 1; k <= n_iter; ++k) {
            const double rk = (double)sigma_s * std::sqrt(3.0) * std::pow(2.0, n_iter - k) /
                              std::sqrt(std::pow(4.0, n_iter) - 1.0) * std::sqrt(3.0);
            const float r = (float)rk;
            const long long rq = (long long)std::floor((double)r * 8388608.0);
            const int R = (int)std::floor(r);
            const bool last = k == n_iter;
            nc_box_pass(cur, ct_h, T_h, va, ct_v, T_v, last ? e : vb, last ? g : nullptr, H, W,
                        rq, R, num_sms, s);
            cur = vb;
        }
    }
    return cudaGetLastError();
}

// two int64 transform planes and periods, four float planes
size_t nc_scratch_floats(int H, int W) { return 8 * (size_t)H * W + 2 * ((size_t)H + (size_t)W); }

}  // namespace blfls
