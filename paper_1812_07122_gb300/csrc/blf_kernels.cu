// Step 1 of BLF-LS (Section III-A): the bilateral filter of Eq. 1 on the periodic forward-
// difference gradients (Section II-B), emitted as residuals e_* = f_BLF(g_*) - g_*.
//
// K1 (tiled): one CTA per 32x32 output tile of one channel.  It loads the image tile with an
// (r+1)-pixel periodic halo into shared memory, forms both gradient fields on the tile + r halo
// (pre-scaled by kappa = sqrt(log2(e) / (2 sigma_r^2)) so that a range weight is a single
// exp2(a - d^2)), and then each thread filters a vertical strip of 8 pixels of both fields.
// For every window column dx the thread streams the 8 + 2r field values of that column once
// from shared memory and reuses each against every strip pixel it reaches, so the inner loop
// is register-resident: per tap one subtract, one FMA for the exponent (the spatial log-weight
// of (dx, dy) folded in), one MUFU ex2 and two accumulations.
// Radii up to kMaxTemplR are compiled with the window fully unrolled per column; larger radii up
// to kMaxTiledR use the same tiling with a runtime window loop; above that a plain per-pixel
// kernel reads precomputed gradients from global memory.
#include "internal.h"

#include <cmath>

namespace blfls {

namespace {

constexpr int kTW = 32;          // tile width  (one warp across)
constexpr int kTH = 32;          // tile height
constexpr int kStrip = 8;        // pixels per thread (vertical strip)
constexpr int kThreads = kTW * kTH / kStrip;  // 128
constexpr int kMaxTemplR = 16;
constexpr int kMaxTiledR = 48;
constexpr float kLog2e = 1.4426950408889634f;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ int wrap_idx(int i, int n)
{
    int m = i % n;
    return m < 0 ? m + n : m;
}

// Shared-memory layout of a tile for radius R: f on (TH+2R+1) x (TW+2R+1), then g_x, g_y on
// (TH+2R) x (TW+2R).
__host__ __device__ __forceinline__ int f_pitch(int R) { return kTW + 2 * R + 1; }
__host__ __device__ __forceinline__ int g_pitch(int R) { return kTW + 2 * R; }
__host__ __device__ __forceinline__ size_t tile_smem_bytes(int R)
{
    return sizeof(float) * ((size_t)(kTH + 2 * R + 1) * f_pitch(R) +
                            2 * (size_t)(kTH + 2 * R) * g_pitch(R));
}

// Load the periodic tile and form kappa * gradients.  Returns pointers into shared memory.
__device__ __forceinline__ void load_tile_gradients(const float* __restrict__ f, int H, int W,
                                                    int x0, int y0, int R, float kappa,
                                                    float* sm, float*& gx, float*& gy)
{
    const int fp = f_pitch(R), fr = kTH + 2 * R + 1;
    const int gp = g_pitch(R), gr = kTH + 2 * R;
    float* sf = sm;
    gx = sm + fr * fp;
    gy = gx + gr * gp;
    for (int i = threadIdx.x; i < fr * fp; i += blockDim.x) {
        const int r = i / fp, c = i - r * fp;
        const int yy = wrap_idx(y0 - R + r, H), xx = wrap_idx(x0 - R + c, W);
        sf[i] = __ldg(f + (size_t)yy * W + xx);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < gr * gp; i += blockDim.x) {
        const int r = i / gp, c = i - r * gp;
        const float v = sf[r * fp + c];
        gx[i] = kappa * (sf[r * fp + c + 1] - v);
        gy[i] = kappa * (sf[(r + 1) * fp + c] - v);
    }
    __syncthreads();
}

__device__ __forceinline__ void store_residuals(float* __restrict__ ex, float* __restrict__ ey,
                                                int H, int W, int x, int ybase,
                                                const float (&ax)[kStrip], const float (&zx)[kStrip],
                                                const float (&sx)[kStrip], const float (&ay)[kStrip],
                                                const float (&zy)[kStrip], const float (&sy)[kStrip],
                                                float inv_kappa)
{
    if (x >= W) return;
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        const int y = ybase + j;
        if (y < H) {
            ex[(size_t)y * W + x] = (__fdiv_rn(ax[j], zx[j]) - sx[j]) * inv_kappa;
            ey[(size_t)y * W + x] = (__fdiv_rn(ay[j], zy[j]) - sy[j]) * inv_kappa;
        }
    }
}

// Tiled kernel, window fully unrolled per column for a compile-time radius R.
template <int R, bool RANGE>
__global__ void __launch_bounds__(kThreads) k1_blf_tiled(const float* __restrict__ img,
                                                         float* __restrict__ ex,
                                                         float* __restrict__ ey, int H, int W,
                                                         float kappa, float inv_kappa, float cs)
{
    extern __shared__ float sm[];
    const size_t plane = (size_t)H * W;
    const float* f = img + blockIdx.z * plane;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    float *gx, *gy;
    load_tile_gradients(f, H, W, x0, y0, R, kappa, sm, gx, gy);

    constexpr int gp = kTW + 2 * R;
    const int cx = threadIdx.x & (kTW - 1);
    const int r0 = (threadIdx.x / kTW) * kStrip;
    float sx[kStrip], sy[kStrip], ax[kStrip], ay[kStrip], zx[kStrip], zy[kStrip];
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        sx[j] = gx[(R + r0 + j) * gp + R + cx];
        sy[j] = gy[(R + r0 + j) * gp + R + cx];
        ax[j] = ay[j] = zx[j] = zy[j] = 0.f;
    }
    // spatial log2-weights: a(dx, dy) = -(dx^2 + dy^2) * cs
    float sa[2 * R + 1];
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) sa[d] = -float((d - R) * (d - R)) * cs;

#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
        const float adx = -float(dx * dx) * cs;
        float ra[2 * R + 1];
#pragma unroll
        for (int d = 0; d <= 2 * R; ++d) ra[d] = adx + sa[d];
        const float* colx = gx + r0 * gp + R + cx + dx;
        const float* coly = gy + r0 * gp + R + cx + dx;
#pragma unroll
        for (int i = 0; i < kStrip + 2 * R; ++i) {
            const float tx = colx[i * gp];
            const float ty = coly[i * gp];
#pragma unroll
            for (int j = 0; j < kStrip; ++j) {
                const int d = i - j;  // dy + R
                if (d < 0 || d > 2 * R) continue;
                float wx, wy;
                if (RANGE) {
                    const float qx = tx - sx[j];
                    const float qy = ty - sy[j];
                    wx = ex2_approx(fmaf(-qx, qx, ra[d]));
                    wy = ex2_approx(fmaf(-qy, qy, ra[d]));
                } else {
                    wx = wy = ex2_approx(ra[d]);
                }
                ax[j] = fmaf(wx, tx, ax[j]);
                zx[j] += wx;
                ay[j] = fmaf(wy, ty, ay[j]);
                zy[j] += wy;
            }
        }
    }
    store_residuals(ex + blockIdx.z * plane, ey + blockIdx.z * plane, H, W, x0 + cx, y0 + r0,
                    ax, zx, sx, ay, zy, sy, inv_kappa);
}

// Tiled kernel with a runtime radius (kMaxTemplR < R <= kMaxTiledR): one shared-memory read per
// tap instead of register reuse across the strip.
template <bool RANGE>
__global__ void __launch_bounds__(kThreads) k1_blf_tiled_rt(const float* __restrict__ img,
                                                            float* __restrict__ ex,
                                                            float* __restrict__ ey, int H, int W,
                                                            int R, float kappa, float inv_kappa,
                                                            float cs)
{
    extern __shared__ float sm[];
    const size_t plane = (size_t)H * W;
    const float* f = img + blockIdx.z * plane;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
    float *gx, *gy;
    load_tile_gradients(f, H, W, x0, y0, R, kappa, sm, gx, gy);
    const int gp = g_pitch(R);
    const int cx = threadIdx.x & (kTW - 1);
    const int r0 = (threadIdx.x / kTW) * kStrip;
    float sx[kStrip], sy[kStrip], ax[kStrip], ay[kStrip], zx[kStrip], zy[kStrip];
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        sx[j] = gx[(R + r0 + j) * gp + R + cx];
        sy[j] = gy[(R + r0 + j) * gp + R + cx];
        ax[j] = ay[j] = zx[j] = zy[j] = 0.f;
    }
    for (int dy = -R; dy <= R; ++dy) {
        for (int dx = -R; dx <= R; ++dx) {
            const float a = -float(dx * dx + dy * dy) * cs;
            const float* px = gx + (R + r0 + dy) * gp + R + cx + dx;
            const float* py = gy + (R + r0 + dy) * gp + R + cx + dx;
#pragma unroll
            for (int j = 0; j < kStrip; ++j) {
                const float tx = px[j * gp], ty = py[j * gp];
                float wx, wy;
                if (RANGE) {
                    const float qx = tx - sx[j], qy = ty - sy[j];
                    wx = ex2_approx(fmaf(-qx, qx, a));
                    wy = ex2_approx(fmaf(-qy, qy, a));
                } else {
                    wx = wy = ex2_approx(a);
                }
                ax[j] = fmaf(wx, tx, ax[j]);
                zx[j] += wx;
                ay[j] = fmaf(wy, ty, ay[j]);
                zy[j] += wy;
            }
        }
    }
    store_residuals(ex + blockIdx.z * plane, ey + blockIdx.z * plane, H, W, x0 + cx, y0 + r0,
                    ax, zx, sx, ay, zy, sy, inv_kappa);
}

// Radii above the tiled limit: gradients precomputed to global memory, one pixel per thread.
__global__ void k1_gradients(const float* __restrict__ img, float* __restrict__ g, int H, int W,
                             float kappa)
{
    const size_t plane = (size_t)H * W;
    const float* f = img + blockIdx.y * plane;
    float* gx = g + blockIdx.y * 2 * plane;
    float* gy = gx + plane;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = int(i / W), x = int(i - (size_t)y * W);
        const float v = f[i];
        gx[i] = kappa * (f[(size_t)y * W + (x + 1 == W ? 0 : x + 1)] - v);
        gy[i] = kappa * (f[(size_t)(y + 1 == H ? 0 : y + 1) * W + x] - v);
    }
}

template <bool RANGE>
__global__ void k1_blf_global(const float* __restrict__ g, float* __restrict__ ex,
                              float* __restrict__ ey, int H, int W, int R, float inv_kappa,
                              float cs)
{
    const size_t plane = (size_t)H * W;
    const float* gx = g + blockIdx.y * 2 * plane;
    const float* gy = gx + plane;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = int(i / W), x = int(i - (size_t)y * W);
        const float sx = gx[i], sy = gy[i];
        float ax = 0.f, ay = 0.f, zx = 0.f, zy = 0.f;
        for (int dy = -R; dy <= R; ++dy) {
            const size_t row = (size_t)wrap_idx(y + dy, H) * W;
            for (int dx = -R; dx <= R; ++dx) {
                const size_t t = row + wrap_idx(x + dx, W);
                const float a = -float(dx * dx + dy * dy) * cs;
                const float tx = __ldg(gx + t), ty = __ldg(gy + t);
                float wx, wy;
                if (RANGE) {
                    const float qx = tx - sx, qy = ty - sy;
                    wx = ex2_approx(fmaf(-qx, qx, a));
                    wy = ex2_approx(fmaf(-qy, qy, a));
                } else {
                    wx = wy = ex2_approx(a);
                }
                ax = fmaf(wx, tx, ax);
                zx += wx;
                ay = fmaf(wy, ty, ay);
                zy += wy;
            }
        }
        ex[blockIdx.y * plane + i] = (__fdiv_rn(ax, zx) - sx) * inv_kappa;
        ey[blockIdx.y * plane + i] = (__fdiv_rn(ay, zy) - sy) * inv_kappa;
    }
}

using TiledFn = void (*)(const float*, float*, float*, int, int, float, float, float);

template <int R>
TiledFn pick_tiled(int r, bool range)
{
    if constexpr (R > kMaxTemplR) {
        return nullptr;
    } else {
        if (r == R) return range ? k1_blf_tiled<R, true> : k1_blf_tiled<R, false>;
        return pick_tiled<R + 1>(r, range);
    }
}

}  // namespace

int blf_tiled_max_radius() { return kMaxTiledR; }

void init_blf_kernel_attributes()
{
    for (int r = 0; r <= kMaxTemplR; ++r)
        for (int range = 0; range < 2; ++range)
            cudaFuncSetAttribute(pick_tiled<0>(r, range), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes(r));
    cudaFuncSetAttribute(k1_blf_tiled_rt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_smem_bytes(kMaxTiledR));
    cudaFuncSetAttribute(k1_blf_tiled_rt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tile_smem_bytes(kMaxTiledR));
}

cudaError_t launch_blf_residual(const float* img, float* ex, float* ey, int C, const BlfParams& p,
                                float* gscratch, cudaStream_t s)
{
    const bool range = std::isfinite(p.sigma_r);
    const double kappa_d = range ? std::sqrt(1.4426950408889634 / (2.0 * (double)p.sigma_r * p.sigma_r)) : 1.0;
    const float kappa = (float)kappa_d;
    const float inv_kappa = (float)(1.0 / kappa_d);
    const float cs = std::isfinite(p.sigma_s)
                         ? (float)(1.4426950408889634 / (2.0 * (double)p.sigma_s * p.sigma_s))
                         : 0.0f;
    const int R = p.radius;
    if (R <= kMaxTiledR) {
        dim3 grid((p.W + kTW - 1) / kTW, (p.H + kTH - 1) / kTH, C);
        const size_t smem = tile_smem_bytes(R);
        if (R <= kMaxTemplR) {
            TiledFn fn = pick_tiled<0>(R, range);
            fn<<<grid, kThreads, smem, s>>>(img, ex, ey, p.H, p.W, kappa, inv_kappa, cs);
        } else if (range) {
            k1_blf_tiled_rt<true><<<grid, kThreads, smem, s>>>(img, ex, ey, p.H, p.W, R, kappa, inv_kappa, cs);
        } else {
            k1_blf_tiled_rt<false><<<grid, kThreads, smem, s>>>(img, ex, ey, p.H, p.W, R, kappa, inv_kappa, cs);
        }
        return cudaGetLastError();
    }
    if (!gscratch) return cudaErrorInvalidValue;
    const size_t plane = (size_t)p.H * p.W;
    const int blocks = (int)std::min<size_t>((plane + 255) / 256, 4096);
    for (int c = 0; c < C; ++c) {
        k1_gradients<<<dim3(blocks, 1), 256, 0, s>>>(img + c * plane, gscratch, p.H, p.W, kappa);
        if (range)
            k1_blf_global<true><<<dim3(blocks, 1), 256, 0, s>>>(gscratch, ex + c * plane, ey + c * plane, p.H, p.W, R, inv_kappa, cs);
        else
            k1_blf_global<false><<<dim3(blocks, 1), 256, 0, s>>>(gscratch, ex + c * plane, ey + c * plane, p.H, p.W, R, inv_kappa, cs);
    }
    return cudaGetLastError();
}

}  // namespace blfls
