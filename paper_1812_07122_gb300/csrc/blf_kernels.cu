// Step 1 of BLF-LS (Section III-A): dispatch of the bilateral kernels, plus the kernels for radii
// above the unrolled range (a scalar tiled kernel with a runtime window, and a per-pixel kernel
// over precomputed gradients).  The unrolled kernels live in blf_tile.cuh and are instantiated
// per precision in blf_f32.cu, blf_f16.cu and blf_bf16.cu.
#include "blf_tile.cuh"

namespace blfls {

TiledFn pick_tiled_f32_entry(int r, bool range);
TiledFn pick_tiled_f16_entry(int r, bool range);
TiledFn pick_tiled_bf16_entry(int r, bool range);
BatchFn pick_batch_f32_entry(int r, bool range);
BatchFn pick_batch_f16_entry(int r, bool range);
BatchFn pick_batch_bf16_entry(int r, bool range);
JointFn pick_joint_f32_entry(int r);
JointFn pick_joint_f16_entry(int r);
JointFn pick_joint_bf16_entry(int r);

BLFLS_DCHECK_TU(blf_kernels)

JointFn pick_joint_prec(int prec, int r)
{
    if (prec == 1) return pick_joint_f16_entry(r);
    if (prec == 2) return pick_joint_bf16_entry(r);
    return pick_joint_f32_entry(r);
}

TiledFn pick_tiled_prec(int prec, int r, bool range)
{
    if (prec == 1) return pick_tiled_f16_entry(r, range);
    if (prec == 2) return pick_tiled_bf16_entry(r, range);
    return pick_tiled_f32_entry(r, range);
}

BatchFn pick_batch_prec(int prec, int r, bool range)
{
    if (prec == 1) return pick_batch_f16_entry(r, range);
    if (prec == 2) return pick_batch_bf16_entry(r, range);
    return pick_batch_f32_entry(r, range);
}

namespace {

// ---------------------------------------------------------------------------------------------
// Radii above kMaxTemplR: scalar FP32 tiles with a runtime window (one shared load per tap).
// ---------------------------------------------------------------------------------------------
template <bool RANGE>
__global__ void __launch_bounds__(kMaxThreads) k1_blf_tiled_rt(const float* __restrict__ img,
                                                               float* __restrict__ ex,
                                                               float* __restrict__ ey, int H,
                                                               int W, int R, int th, const Kap k0,
                                                               float cs,
                                                               const float4* __restrict__ kdev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const Kap k = kap_of(k0, kdev, blockIdx.z);
    const int fp = f_pitch(R), gp = g_pitch(R), gr = g_rows(R, th);
    float* sf = reinterpret_cast<float*>(smem);
    float* gx = reinterpret_cast<float*>(smem + f_bytes(R, th));
    float* gy = gx + gr * gp;
    const size_t plane = (size_t)H * W;
    const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * th;
    load_f_tile(img + blockIdx.z * plane, H, W, x0, y0, R, th, sf);
    __syncthreads();
    for (int i = threadIdx.x; i < gr * gp; i += blockDim.x) {
        const int r = i / gp, c = i - r * gp;
        gx[i] = grad_x(sf, fp, r, c, k.x);
        gy[i] = grad_y(sf, fp, r, c, k.y);
    }
    __syncthreads();
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
            if (!BLFLS_DCHECK(R + cx + dx >= 0 && R + cx + dx < gp && r0 + dy + R >= 0 &&
                              (R + r0 + dy + kStrip - 1) * gp + R + cx + dx < gr * gp,
                              kDcTileWindow))
                continue;
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
    store_strip(ex + blockIdx.z * plane, ey + blockIdx.z * plane, H, W, x0 + cx, y0 + r0, ax, zx,
                sx, ay, zy, sy, k);
}

// Radii above the tiled limit: gradients precomputed to global memory, one pixel per thread.
// kdev (when set) holds this channel's range constants (kx, ky, 1/kx, 1/ky).
__global__ void k1_gradients(const float* __restrict__ img, float* __restrict__ g, int H, int W,
                             float kx, float ky, const float4* __restrict__ kdev)
{
    if (kdev) {
        kx = kdev->x;
        ky = kdev->y;
    }
    const size_t plane = (size_t)H * W;
    float* gx = g;
    float* gy = g + plane;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = int(i / W), x = int(i - (size_t)y * W);
        const float v = img[i];
        gx[i] = kx * (img[(size_t)y * W + (x + 1 == W ? 0 : x + 1)] - v);
        gy[i] = ky * (img[(size_t)(y + 1 == H ? 0 : y + 1) * W + x] - v);
    }
}

// `hg`, when not null, holds the guidance image's gradients (same layout): the range weights
// compare them instead of the input's (joint filter).
template <bool RANGE>
__global__ void k1_blf_global(const float* __restrict__ g, const float* __restrict__ hg,
                              float* __restrict__ ex, float* __restrict__ ey, int H, int W, int R,
                              float inv_kx, float inv_ky, float cs, const float4* __restrict__ kdev)
{
    if (kdev) {
        inv_kx = kdev->z;
        inv_ky = kdev->w;
    }
    const size_t plane = (size_t)H * W;
    const float* gx = g;
    const float* gy = g + plane;
    const float* hx = hg ? hg : gx;
    const float* hy = hg ? hg + plane : gy;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = int(i / W), x = int(i - (size_t)y * W);
        const float sx = gx[i], sy = gy[i];
        const float hsx = hx[i], hsy = hy[i];
        float ax = 0.f, ay = 0.f, zx = 0.f, zy = 0.f;
        for (int dy = -R; dy <= R; ++dy) {
            const size_t row = (size_t)wrap_idx(y + dy, H) * W;
            for (int dx = -R; dx <= R; ++dx) {
                const size_t t = row + wrap_idx(x + dx, W);
                const float a = -float(dx * dx + dy * dy) * cs;
                const float tx = __ldg(gx + t), ty = __ldg(gy + t);
                float wx, wy;
                if (RANGE) {
                    const float qx = __ldg(hx + t) - hsx, qy = __ldg(hy + t) - hsy;
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
        ex[i] = (__fdiv_rn(ax, zx) - sx) * inv_kx;
        ey[i] = (__fdiv_rn(ay, zy) - sy) * inv_ky;
    }
}


}  // namespace

size_t blf_templ_smem_bytes(int R, int prec, int th, bool joint)
{
    // one tile of (g_x, g_y) pairs (two for the joint filter: input and guidance): half2 for
    // FP16W, float2 for FP32 and BF16W
    const size_t pair = (prec == 1) ? sizeof(__half2) : sizeof(float2);
    return f_bytes(R, th) + (joint ? 2 : 1) * pair * (size_t)g_rows(R, th) * g_pitch(R);
}

int blf_tile_height(int th)
{
    return (th == 8 || th == 16 || th == 32 || th == 64) ? th : 32;
}

int blf_tiled_max_radius() { return kMaxTiledR; }
int blf_joint_tiled_max_radius() { return kMaxTemplR; }

void init_blf_kernel_attributes()
{
    for (int r = 0; r <= kMaxTemplR; ++r)
        for (int range = 0; range < 2; ++range)
            for (int prec = 0; prec < 3; ++prec) {
                cudaFuncSetAttribute(pick_tiled_prec(prec, r, range),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)blf_templ_smem_bytes(r, prec, kMaxTH));
                cudaFuncSetAttribute(pick_batch_prec(prec, r, range),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)blf_templ_smem_bytes(r, prec, kMaxTH));
                if (range)
                    cudaFuncSetAttribute(pick_joint_prec(prec, r),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)blf_templ_smem_bytes(r, prec, kMaxTH, true));
            }
    const int rt = (int)tile_smem_bytes(kMaxTiledR, sizeof(float), 32);
    cudaFuncSetAttribute(k1_blf_tiled_rt<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rt);
    cudaFuncSetAttribute(k1_blf_tiled_rt<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rt);
}

void blf_constants(float sigma_s, float sigma_r, float* kappa, float* inv_kappa, float* cs)
{
    const bool range = std::isfinite(sigma_r);
    const double kappa_d = range ? std::sqrt(1.4426950408889634 / (2.0 * (double)sigma_r * sigma_r)) : 1.0;
    *kappa = (float)kappa_d;
    *inv_kappa = (float)(1.0 / kappa_d);
    *cs = std::isfinite(sigma_s) ? (float)(1.4426950408889634 / (2.0 * (double)sigma_s * sigma_s))
                                 : 0.0f;
}

cudaError_t launch_blf_residual(const float* img, float* ex, float* ey, int C, const BlfParams& p,
                                float* gscratch, cudaStream_t s)
{
    const bool range = std::isfinite(p.sigma_r);
    const bool joint = p.guide != nullptr && range;   // without a range kernel the guide is moot
    float kx, ikx, ky, iky, cs;
    blf_constants(p.sigma_s, p.sigma_r * p.range_scale_x, &kx, &ikx, &cs);
    blf_constants(p.sigma_s, p.sigma_r * p.range_scale_y, &ky, &iky, &cs);
    const Kap k{kx, ky, ikx, iky};
    const int R = p.radius;
    const size_t plane = (size_t)p.H * p.W;
    if (joint ? R <= kMaxTemplR : R <= kMaxTiledR) {
        const int th = (R <= kMaxTemplR) ? blf_tile_height(p.tile_h) : 32;
        const int threads = kTW * th / kStrip;
        dim3 grid((p.W + kTW - 1) / kTW, (p.H + th - 1) / th, C);
        if (joint) {
            JointFn fn = pick_joint_prec(p.prec, R);
            fn<<<grid, threads, blf_templ_smem_bytes(R, p.prec, th, true), s>>>(
                img, p.guide, p.guide_stride, ex, ey, p.H, p.W, th, k, cs);
        } else if (R <= kMaxTemplR) {
            TiledFn fn = pick_tiled_prec(p.prec, R, range);
            fn<<<grid, threads, blf_templ_smem_bytes(R, p.prec, th), s>>>(img, ex, ey, p.H, p.W, th,
                                                                         k, cs, p.kap_dev);
        } else {
            if (p.prec != 0) return cudaErrorNotSupported;
            const size_t smem = tile_smem_bytes(R, sizeof(float), th);
            if (range)
                k1_blf_tiled_rt<true><<<grid, threads, smem, s>>>(img, ex, ey, p.H, p.W, R, th, k, cs, p.kap_dev);
            else
                k1_blf_tiled_rt<false><<<grid, threads, smem, s>>>(img, ex, ey, p.H, p.W, R, th, k, cs, p.kap_dev);
        }
        return cudaGetLastError();
    }
    // per-pixel kernel over gradients in global memory (the guidance's after the input's)
    if (p.prec != 0) return cudaErrorNotSupported;
    if (!gscratch) return cudaErrorInvalidValue;
    const int blocks = (int)std::min<size_t>((plane + 255) / 256, 4096);
    float* hg = joint ? gscratch + 2 * plane : nullptr;
    for (int c = 0; c < C; ++c) {
        const float4* kd = p.kap_dev ? p.kap_dev + c : nullptr;
        k1_gradients<<<blocks, 256, 0, s>>>(img + c * plane, gscratch, p.H, p.W, kx, ky, kd);
        if (joint) k1_gradients<<<blocks, 256, 0, s>>>(p.guide + c * p.guide_stride, hg, p.H, p.W, kx, ky, kd);
        if (range)
            k1_blf_global<true><<<blocks, 256, 0, s>>>(gscratch, hg, ex + c * plane, ey + c * plane, p.H, p.W, R, ikx, iky, cs, kd);
        else
            k1_blf_global<false><<<blocks, 256, 0, s>>>(gscratch, nullptr, ex + c * plane, ey + c * plane, p.H, p.W, R, ikx, iky, cs, kd);
    }
    return cudaGetLastError();
}

int blf_batch_max_radius() { return kMaxTemplR; }

void blf_tiles(int H, int W, int th, int* tiles_x, int* tiles_y)
{
    th = blf_tile_height(th);
    *tiles_x = (W + kTW - 1) / kTW;
    *tiles_y = (H + th - 1) / th;
}

cudaError_t launch_blf_batch(const BatchJob* jobs, const int2* grp, int ngrp, int total, int radius,
                             bool range, int prec, int th, int num_sms, cudaStream_t s)
{
    if (total <= 0) return cudaSuccess;
    BatchFn fn = pick_batch_prec(prec, radius, range);
    if (!fn) return cudaErrorNotSupported;
    th = blf_tile_height(th);
    const int threads = kTW * th / kStrip;
    const size_t smem = blf_templ_smem_bytes(radius, prec, th);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    const int grid = std::max(1, std::min(total, num_sms * std::max(occ, 1)));
    fn<<<grid, threads, smem, s>>>(jobs, grp, ngrp, total);
    return cudaGetLastError();
}

}  // namespace blfls
