// NC-LS (Section III-D): BLF-LS with the bilateral filter replaced by the normalised convolution
// of the domain transform.  Per channel and gradient field g (the periodic forward difference of
// the image along x or y), with a = sigma_s / sigma_r, the transform of a periodic line is the
// running sum ct[i] = sum_{j=1..i} (1 + a |g[j] - g[j-1]|), and one box pass of radius r averages,
// for every sample i, the samples j with |ct(j) - ct(i)| <= r (the line's copies one period over
// shifted by the period T).  Since the transform grows by at least 1 per sample, those samples
// form one run around i, and ct(j) - ct(i) is the sum of the steps between i and j: the box
// passes need only the steps, never ct itself.
//
//   k8_grad_steps  the two fields and, for each field, its steps along x and along y;
//   k8_nc_rows_tile  one box pass of radius r along rows for R = floor(r) <= 64: tiles of values
//                and steps (with R samples of neighbourhood) staged in shared memory, each
//                pixel's run scanned outward there;
//   k8_nc_cols_strip  the pass along columns for R <= 16: a thread holds a strip of 8 samples and
//                its neighbourhood in registers (coalesced loads straight from global memory);
//   k8_nc_rows / k8_nc_cols  larger radii: a sliding window per run of 32 samples;
// N iterations with r_k = sigma_s sqrt(3) 2^(N-k) / sqrt(4^N - 1) sqrt(3), rows then columns; the
// last column pass writes the residual e = v - g for the Fourier solve.
//
// Box decisions follow the real-valued transform: a step 1 + a |dg| is formed from the exact
// second difference of the FP32 image (error-free sums, so dg is exact) and a = sigma_s / sigma_r
// (FP64, split into two FP32 words) as a double-float, and stored as a 32-bit integer number of
// units of 2^-q rounded down, q the largest integer <= 30 with rq_1 + 1 < 2^32 (rq_k =
// floor(r_k 2^q), r_k in FP64; rq_1 of the first, widest iteration).  Steps are clamped to
// rq_1 + 1: a run containing such a step exceeds every radius either way.  Sums of steps are
// exact in 64-bit integers in any order, and the box test "sum <= rq_k" differs from the exact
// test "transform distance <= r_k" only when that distance lies within (number of steps) x 2^-q
// of r_k.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dcheck.cuh"
#include "internal.h"

namespace blfls {

namespace {

constexpr int kNcThreads = 256;
// Error-free transformation: hi + lo == a + b exactly (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& hi, float& lo)
{
    hi = __fadd_rn(a, b);
    const float bb = __fsub_rn(hi, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(b, bb));
}

// One step 1 + a |(p1 - p0) - (q1 - q0)| (the difference of two consecutive gradient samples,
// each the difference of two image values), a = ah + al, in units of 2^-q (`scale` = 2^q) rounded
// down and clamped to `clamp`.  The difference is exact as a double-float; the product and the
// sum carry about 2^-46 relative error, the conversion less than one unit.
__device__ __forceinline__ unsigned step_units(float p1, float p0, float q1, float q0, float ah,
                                               float al, float scale, unsigned long long clamp)
{
    float d1h, d1l, d0h, d0l, dh, dl;
    two_sum(p1, -p0, d1h, d1l);
    two_sum(q1, -q0, d0h, d0l);
    two_sum(d1h, -d0h, dh, dl);
    dl = __fadd_rn(dl, __fsub_rn(d1l, d0l));
    float nh, nl;
    two_sum(dh, dl, nh, nl);                         // normalise
    float ph = nh;
    if (ph < 0.0f) { ph = -ph; nl = -nl; }
    // m = a |d| as a double-float
    const float mh = __fmul_rn(ah, ph);
    const float ml = __fadd_rn(__fmaf_rn(ah, ph, -mh), __fmaf_rn(ah, nl, __fmul_rn(al, ph)));
    // step = 1 + m
    float sh, se;
    two_sum(1.0f, mh, sh, se);
    const float sl = __fadd_rn(se, ml);
    const float xh = __fmul_rn(sh, scale), xl = __fmul_rn(sl, scale);   // exact scalings
    if (xh >= (float)clamp) return (unsigned)clamp;
    const float n = floorf(xh);
    const long long u = (long long)n + (long long)floorf(__fadd_rn(__fsub_rn(xh, n), xl));
    return (unsigned)(u < 0 ? 0 : ((unsigned long long)u < clamp ? u : (long long)clamp));
}

// g for both fields, and the steps of each field: sh_* between (y, x-1) and (y, x), sv_*
// between (y-1, x) and (y, x), periodic.
__global__ void __launch_bounds__(kNcThreads) k8_grad_steps(const float* __restrict__ f,
                                                           float* __restrict__ gx,
                                                           float* __restrict__ gy,
                                                           unsigned* __restrict__ shx,
                                                           unsigned* __restrict__ svx,
                                                           unsigned* __restrict__ shy,
                                                           unsigned* __restrict__ svy, int H,
                                                           int W, float ah, float al, float scale,
                                                           unsigned long long clamp)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const int xl = x == 0 ? W - 1 : x - 1, xr = x + 1 == W ? 0 : x + 1;
        const int yu = y == 0 ? H - 1 : y - 1, yd = y + 1 == H ? 0 : y + 1;
        const float* r0 = f + (size_t)y * W;
        const float* ru = f + (size_t)yu * W;
        const float* rd = f + (size_t)yd * W;
        const float c = r0[x], cr = r0[xr], cl = r0[xl], cd = rd[x], cu = ru[x];
        const float dl = rd[xl], ur = ru[xr];
        gx[i] = cr - c;    // the fields at (y, x)
        gy[i] = cd - c;
        // steps between (y, x-1) and (y, x), and between (y-1, x) and (y, x), of each field
        shx[i] = step_units(cr, c, c, cl, ah, al, scale, clamp);     // g_x(y,x) - g_x(y,x-1)
        svx[i] = step_units(cr, c, ur, cu, ah, al, scale, clamp);    // g_x(y,x) - g_x(y-1,x)
        shy[i] = step_units(cd, c, dl, cl, ah, al, scale, clamp);    // g_y(y,x) - g_y(y,x-1)
        svy[i] = step_units(cd, c, c, cu, ah, al, scale, clamp);     // g_y(y,x) - g_y(y-1,x)
    }
}

// ---------------------------------------------------------------------------------------------
// Box means for R = floor(r) <= kNcTileMaxR from shared-memory tiles.  A CTA stages a tile of the
// values and the steps, with R samples of periodic neighbourhood on either side along the pass,
// with coalesced loads; each thread then takes pixels whose lanes are adjacent along the tile's
// fast axis (conflict-free reads) and scans each pixel's run outward in shared memory, adding
// the steps until the distance exceeds the radius (at most R steps a side).
// ---------------------------------------------------------------------------------------------
constexpr int kNcTileMaxR = 64;
constexpr int kTileLong = 64;   // samples along the pass per tile
constexpr int kTileWide = 32;   // lines per tile
constexpr int kLoadBatch = 4;   // tile rows each warp loads with all their loads in flight

// One pixel's box mean: sample i of a staged line (s[p]: the step into p; v[p]: the value);
// `st` is the distance between consecutive samples in shared memory.
__device__ __forceinline__ float tile_mean(const unsigned* __restrict__ s,
                                           const float* __restrict__ v, int st, int i, int R,
                                           unsigned long long rq)
{
    float acc = v[i * st], cnt = 1.f;
    unsigned long long d = 0;
    for (int k = 1; k <= R; ++k) {   // upwards
        d += s[(i + k) * st];
        if (d > rq) break;
        acc += v[(i + k) * st];
        cnt += 1.f;
    }
    d = 0;
    for (int k = 1; k <= R; ++k) {   // downwards: the step into i - k + 1
        d += s[(i - k + 1) * st];
        if (d > rq) break;
        acc += v[(i - k) * st];
        cnt += 1.f;
    }
    return acc / cnt;
}

// Along x: tiles of 32 rows x 64 columns; thread (lane, warp) takes columns lane and lane + 32
// of rows warp, warp + 8, ... (coalesced stores).
__global__ void __launch_bounds__(kNcThreads) k8_nc_rows_tile(const float* __restrict__ v,
                                                             const unsigned* __restrict__ sh,
                                                             float* __restrict__ out, int H,
                                                             int W, int R, long long rq)
{
    extern __shared__ __align__(16) unsigned char nc_smem[];
    const int span = kTileLong + 2 * R;
    unsigned* ss = reinterpret_cast<unsigned*>(nc_smem);
    float* sv = reinterpret_cast<float*>(ss + kTileWide * span);
    const int tiles_x = (W + kTileLong - 1) / kTileLong;
    const int y0 = (blockIdx.x / tiles_x) * kTileWide, x0 = (blockIdx.x % tiles_x) * kTileLong;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // the tile's rows in groups of kLoadBatch per warp, all loads of a group in flight together
    for (int r0 = w; r0 < kTileWide; r0 += kLoadBatch * (kNcThreads / 32)) {
        for (int q = lane; q < span; q += 32) {
            int p = x0 - R + q;                    // unwrapped column
            while (p < 0) p += W;
            while (p >= W) p -= W;
            unsigned a[kLoadBatch];
            float b[kLoadBatch];
#pragma unroll
            for (int u = 0; u < kLoadBatch; ++u) {
                const int y = y0 + r0 + u * (kNcThreads / 32);
                if (r0 + u * (kNcThreads / 32) < kTileWide && y < H) {
                    a[u] = sh[(size_t)y * W + p];
                    b[u] = v[(size_t)y * W + p];
                }
            }
#pragma unroll
            for (int u = 0; u < kLoadBatch; ++u) {
                const int r = r0 + u * (kNcThreads / 32);
                if (r < kTileWide && y0 + r < H) {
                    ss[r * span + q] = a[u];
                    sv[r * span + q] = b[u];
                }
            }
        }
    }
    __syncthreads();
    for (int r = w; r < kTileWide; r += kNcThreads / 32) {
        const int y = y0 + r;
        if (y >= H) break;
        for (int q = lane; q < kTileLong; q += 32) {
            const int x = x0 + q;
            if (x < W && BLFLS_DCHECK(q + 2 * R < span, kDcNcTile))
                out[(size_t)y * W + x] = tile_mean(ss + r * span, sv + r * span, 1, R + q, R,
                                                   (unsigned long long)rq);
        }
    }
}

// Along y the columns are loaded straight from global memory instead (adjacent threads on
// adjacent columns, so every load is coalesced): a thread takes a strip of kNcStrip samples of
// one column and holds the strip and RM neighbours on either side (values and steps) in
// registers, with one load per sample; the running sum of the steps over that window gives the
// window-relative transform, and each sample's run is scanned outward over the registers with
// every comparison predicated (R = floor(r) <= RM).
constexpr int kNcStrip = 8;

template <int RM>
__device__ __forceinline__ void strip_means(const unsigned (&sw)[kNcStrip + 2 * RM],
                                            const float (&vw)[kNcStrip + 2 * RM], long long rq,
                                            float (&mean)[kNcStrip])
{
    constexpr int NW = kNcStrip + 2 * RM;
    long long cw[NW];   // running sum of the steps over the window (window-relative transform)
    cw[0] = 0;
#pragma unroll
    for (int q = 1; q < NW; ++q) cw[q] = cw[q - 1] + (long long)sw[q];
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

// Along y: one thread per strip of kNcStrip rows of one column, adjacent threads on adjacent
// columns, the window loaded straight from global memory (coalesced across the warp; the
// neighbouring strips' overlap comes from L1/L2); when g is not null the output is the
// residual (mean - g).
template <int RM>
__global__ void __launch_bounds__(kNcThreads) k8_nc_cols_strip(const float* __restrict__ v,
                                                              const unsigned* __restrict__ svs,
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
        int m = k * kNcStrip - RM;
        while (m < 0) m += H;
        unsigned sw[NW];
        float vw[NW];
#pragma unroll
        for (int q = 0; q < NW; ++q) {
            sw[q] = svs[(size_t)m * W + x];
            vw[q] = v[(size_t)m * W + x];
            if (++m == H) m = 0;
        }
        float mean[kNcStrip];
        strip_means<RM>(sw, vw, rq, mean);
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

// ---------------------------------------------------------------------------------------------
// Larger radii: a sliding window.  Both ends of a sample's run only move forward as the sample
// does, so a thread takes kNcRun consecutive samples of one line, finds the first sample's run by
// scanning outward, then for every next sample drops the samples that have left at the bottom and
// adds those that have come inside at the top, keeping the run's sum (Neumaier-compensated FP32),
// its count, and the transform distances from the current sample to both ends.
// ---------------------------------------------------------------------------------------------
constexpr int kNcRun = 32;

__device__ __forceinline__ void nsum_add(float& s, float& comp, float x)
{
    const float t = __fadd_rn(s, x);
    comp += fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s);
    s = t;
}

// Samples [i0, i1) of one line (length n, element stride st); stp[p] is the step into sample p.
__device__ __forceinline__ void box_run(const unsigned* __restrict__ stp,
                                        const float* __restrict__ v, size_t st, int n,
                                        long long rq, int i0, int i1, float* __restrict__ out,
                                        const float* __restrict__ g)
{
    auto wrap = [n](int p) { return p >= n ? p - n : (p < 0 ? p + n : p); };
    int lo = i0, hi = i0;                 // line indices of the run's ends (periodic)
    long long dlo = 0, dhi = 0;           // transform distances from the sample to lo and to hi
    float sum = v[(size_t)i0 * st], comp = 0.f;
    int cnt = 1;
    for (;;) {   // the first sample's run, upwards
        const int nx = wrap(hi + 1);
        const long long d = dhi + (long long)stp[(size_t)nx * st];
        if (d > rq) break;
        hi = nx;
        dhi = d;
        nsum_add(sum, comp, v[(size_t)hi * st]);
        ++cnt;
    }
    for (;;) {   // and downwards
        const long long d = dlo + (long long)stp[(size_t)lo * st];
        if (d > rq) break;
        lo = wrap(lo - 1);
        dlo = d;
        nsum_add(sum, comp, v[(size_t)lo * st]);
        ++cnt;
    }
    for (int i = i0;;) {
        const float m = (sum + comp) / (float)cnt;
        out[(size_t)i * st] = g ? m - g[(size_t)i * st] : m;
        if (++i >= i1) break;
        if (dhi == 0) {   // the previous run ended at the previous sample: i starts a new run
            lo = hi = i;
            dlo = 0;
            sum = v[(size_t)i * st];
            comp = 0.f;
            cnt = 1;
        } else {          // i is inside the previous run
            const long long step = stp[(size_t)i * st];
            dhi -= step;
            dlo += step;
            while (dlo > rq) {   // samples that have left at the bottom
                const int nl = wrap(lo + 1);
                dlo -= (long long)stp[(size_t)nl * st];
                nsum_add(sum, comp, -v[(size_t)lo * st]);
                --cnt;
                lo = nl;
            }
        }
        for (;;) {   // samples that have come inside at the top
            const int nx = wrap(hi + 1);
            const long long d = dhi + (long long)stp[(size_t)nx * st];
            if (d > rq) break;
            hi = nx;
            dhi = d;
            nsum_add(sum, comp, v[(size_t)hi * st]);
            ++cnt;
        }
    }
}

// Box pass along x: one thread per run of kNcRun samples of a row.
__global__ void __launch_bounds__(kNcThreads) k8_nc_rows(const float* __restrict__ v,
                                                        const unsigned* __restrict__ sh,
                                                        float* __restrict__ out, int H, int W,
                                                        long long rq)
{
    const int runs = (W + kNcRun - 1) / kNcRun;
    const size_t total = (size_t)H * runs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(t / runs), k = (int)(t - (size_t)y * runs);
        const size_t row = (size_t)y * W;
        box_run(sh + row, v + row, 1, W, rq, k * kNcRun, min(W, (k + 1) * kNcRun), out + row,
                nullptr);
    }
}

// Box pass along y: one thread per run of kNcRun samples of a column.
__global__ void __launch_bounds__(kNcThreads) k8_nc_cols(const float* __restrict__ v,
                                                        const unsigned* __restrict__ svs,
                                                        float* __restrict__ out,
                                                        const float* __restrict__ g, int H,
                                                        int W, long long rq)
{
    const int runs = (H + kNcRun - 1) / kNcRun;
    const size_t total = (size_t)W * runs;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
         t += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / W), x = (int)(t - (size_t)k * W);
        box_run(svs + x, v + x, (size_t)W, H, rq, k * kNcRun, min(H, (k + 1) * kNcRun), out + x,
                g ? g + x : nullptr);
    }
}

int nc_blocks(size_t n, int num_sms)
{
    const size_t want = (n + kNcThreads - 1) / kNcThreads;
    return (int)std::max<size_t>(1, std::min(want, (size_t)num_sms * 8));
}

size_t nc_tile_smem(int R) { return (size_t)(kTileLong + 2 * R) * kTileWide * 8; }

template <int RM>
void cols_strips(const float* mid, const unsigned* sv, float* out, const float* g, int H, int W,
                 long long rq, int num_sms, cudaStream_t s)
{
    const size_t strips = (size_t)W * ((H + kNcStrip - 1) / kNcStrip);
    k8_nc_cols_strip<RM><<<nc_blocks(strips, num_sms), kNcThreads, 0, s>>>(mid, sv, out, g, H, W,
                                                                          rq);
}

// One iteration: box means along the rows of v into mid, then along the columns of mid into out
// (minus g when given).  Rows: shared-memory tiles for R <= kNcTileMaxR; columns: register strips
// for R <= 16; sliding windows above.
void nc_box_pass(const float* v, const unsigned* sh, float* mid, const unsigned* sv, float* out,
                 const float* g, int H, int W, long long rq, int R, int num_sms, cudaStream_t s)
{
    if (R <= kNcTileMaxR) {
        const int row_tiles = ((H + kTileWide - 1) / kTileWide) * ((W + kTileLong - 1) / kTileLong);
        k8_nc_rows_tile<<<row_tiles, kNcThreads, nc_tile_smem(R), s>>>(v, sh, mid, H, W, R, rq);
    } else {
        k8_nc_rows<<<nc_blocks((size_t)H * ((W + kNcRun - 1) / kNcRun), num_sms), kNcThreads, 0,
                     s>>>(v, sh, mid, H, W, rq);
    }
    if (R <= 1) return cols_strips<1>(mid, sv, out, g, H, W, rq, num_sms, s);
    if (R <= 2) return cols_strips<2>(mid, sv, out, g, H, W, rq, num_sms, s);
    if (R <= 4) return cols_strips<4>(mid, sv, out, g, H, W, rq, num_sms, s);
    if (R <= 8) return cols_strips<8>(mid, sv, out, g, H, W, rq, num_sms, s);
    if (R <= 16) return cols_strips<16>(mid, sv, out, g, H, W, rq, num_sms, s);
    k8_nc_cols<<<nc_blocks((size_t)W * ((H + kNcRun - 1) / kNcRun), num_sms), kNcThreads, 0, s>>>(
        mid, sv, out, g, H, W, rq);
}

}  // namespace

BLFLS_DCHECK_TU(nc)

cudaError_t launch_nc_residuals(const float* f, float* ex, float* ey, int H, int W,
                                float sigma_s, float sigma_r, int n_iter, float* scratch,
                                cudaStream_t s, int num_sms)
{
    const size_t plane = (size_t)H * W;
    float* gx = scratch;
    float* gy = gx + plane;
    float* va = gy + plane;
    float* vb = va + plane;
    unsigned* shx = reinterpret_cast<unsigned*>(vb + plane);
    unsigned* svx = shx + plane;
    unsigned* shy = svx + plane;
    unsigned* svy = shy + plane;
    const double a = std::isfinite(sigma_r) ? (double)sigma_s / (double)sigma_r : 0.0;
    const float ah = (float)a, al = (float)(a - (double)ah);
    std::vector<double> r(n_iter);
    for (int k = 1; k <= n_iter; ++k)
        r[k - 1] = (double)sigma_s * std::sqrt(3.0) * std::pow(2.0, n_iter - k) /
                   std::sqrt(std::pow(4.0, n_iter) - 1.0) * std::sqrt(3.0);
    // units of 2^-q: the largest q <= 30 with rq_1 + 1 < 2^32 (r_1 is the widest radius)
    int q = 30;
    while (q > 0 && std::floor(std::ldexp(r[0], q)) + 1.0 >= 4294967296.0) --q;
    const auto units = [q](double rk) { return (long long)std::floor(std::ldexp(rk, q)); };
    const unsigned long long clamp = (unsigned long long)units(r[0]) + 1;
    if (clamp > 0xffffffffull) return cudaErrorInvalidValue;
    k8_grad_steps<<<nc_blocks(plane, num_sms), kNcThreads, 0, s>>>(f, gx, gy, shx, svx, shy, svy,
                                                                  H, W, ah, al, (float)std::ldexp(1.0, q),
                                                                  clamp);
    for (int field = 0; field < 2; ++field) {
        const float* g = field == 0 ? gx : gy;
        const unsigned* sh = field == 0 ? shx : shy;
        const unsigned* sv = field == 0 ? svx : svy;
        float* e = field == 0 ? ex : ey;
        const float* cur = g;
        for (int k = 1; k <= n_iter; ++k) {
            const bool last = k == n_iter;
            nc_box_pass(cur, sh, va, sv, last ? e : vb, last ? g : nullptr, H, W, units(r[k - 1]),
                        (int)std::floor(r[k - 1]), num_sms, s);
            cur = vb;
        }
    }
    return cudaGetLastError();
}

// four float planes (the two fields, two pass buffers) and four planes of steps
size_t nc_scratch_floats(int H, int W) { return 8 * (size_t)H * W; }

}  // namespace blfls
