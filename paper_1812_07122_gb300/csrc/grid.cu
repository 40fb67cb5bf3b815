// Bilateral-grid approximation of the BLF of Eq. 1 (the fast filter the paper uses in its
// experiments, Section III-A / IV), on the two periodic forward-difference gradient fields of a
// channel; the output is the residual e = BLF_grid(g) - g consumed by the Fourier solve.
//
// For one field g (H x W), with spatial and range sampling steps s_s = sigma_s, s_r = sigma_r and
// a padding of P = 2 cells, the grid holds (sum of g, count) pairs over
// Gz x Gy x Gx = (floor((max g - min g) / s_r) + 1 + 2P) x (floor((H-1)/s_s) + 1 + 2P) x
// (floor((W-1)/s_s) + 1 + 2P) cells, z-major:
//   k6_minmax   min and max of both fields of every channel (order-preserving integer keys, so the
//               atomics are exact and the result does not depend on their order);
//   k6_splat    one thread per spatial cell walks the pixels whose nearest cell it is and adds
//               (g, 1) to the range bin of each, in a fixed order (deterministic, no atomics);
//   k6_blur     the 3-tap kernel (e^-1/2, 1, e^-1/2) along x, y, then z (zero outside);
//   k6_slice    trilinear interpolation at (z, y / s_s + P, x / s_s + P): e = sum / count - g.
// Cell indices are floor(t + 1/2) of the real t: FP32 decides away from rounding boundaries, FP64
// near them (see cell_of), so the cells are those of the FP64 definition on the FP32 gradients.
// Grid passes are HBM/L2-bound streams.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "dcheck.cuh"
#include "internal.h"

namespace blfls {

namespace {

constexpr int kGridThreads = 256;
constexpr int kPad = 2;

__device__ __forceinline__ int f2key(float v)
{
    const int i = __float_as_int(v);
    return i ^ ((i >> 31) & 0x7fffffff);
}

__device__ __forceinline__ float grad_at(const float* f, int H, int W, int y, int x, int field)
{
    const float c = f[(size_t)y * W + x];
    return field == 0 ? f[(size_t)y * W + (x + 1 == W ? 0 : x + 1)] - c
                      : f[(size_t)(y + 1 == H ? 0 : y + 1) * W + x] - c;
}

__global__ void k6_init_keys(int* keys, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = (i & 1) ? INT_MIN : INT_MAX;
}

// keys[4c + 2 field + 0] = min key, keys[4c + 2 field + 1] = max key; blockIdx.y = channel
__global__ void __launch_bounds__(kGridThreads) k6_minmax(const float* __restrict__ img, int H,
                                                         int W, int* keys)
{
    const size_t plane = (size_t)H * W;
    const float* f = img + blockIdx.y * plane;
    int mn[2] = {INT_MAX, INT_MAX}, mx[2] = {INT_MIN, INT_MIN};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
#pragma unroll
        for (int fl = 0; fl < 2; ++fl) {
            const int k = f2key(grad_at(f, H, W, y, x, fl));
            mn[fl] = min(mn[fl], k);
            mx[fl] = max(mx[fl], k);
        }
    }
#pragma unroll
    for (int fl = 0; fl < 2; ++fl) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[fl] = min(mn[fl], __shfl_xor_sync(0xffffffffu, mn[fl], o));
            mx[fl] = max(mx[fl], __shfl_xor_sync(0xffffffffu, mx[fl], o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(keys + 4 * blockIdx.y + 2 * fl, mn[fl]);
            atomicMax(keys + 4 * blockIdx.y + 2 * fl + 1, mx[fl]);
        }
    }
}

struct GridGeom {
    int H, W, gx, gy, gz;
    float ss, sr, lo;
    int field;
};

// floor((a - b) / den + 1/2) of the exact real value for FP32 operands: the FP32 evaluation
// (relative error below 2.5e-7) decides when it lies more than 1e-6 (relative) away from both
// neighbouring integers; otherwise FP64 decides (a - b exact, one correctly rounded division), so
// a pixel near a rounding boundary goes where the FP64 definition puts it.
__device__ __forceinline__ int cell_of(float a, float b, float den)
{
    const float q = __fadd_rn(__fdiv_rn(__fsub_rn(a, b), den), 0.5f);
    const float n = floorf(q);
    const float margin = fmaxf(fabsf(q), 1.0f) * 1.0e-6f;
    if (q - n > margin && (n + 1.0f) - q > margin) return (int)n;
    return (int)floor(__dadd_rn(__ddiv_rn(__dsub_rn((double)a, (double)b), (double)den), 0.5));
}

// One thread per spatial cell (cy, cx) that a pixel can round to: floor((W-1)/s_s) + 2 cells per
// axis (the last pixel can round up into the first padding cell).
__global__ void __launch_bounds__(kGridThreads) k6_splat(const float* __restrict__ f,
                                                        float2* __restrict__ grid, GridGeom G)
{
    const int nx = G.gx - 2 * kPad + 1, ny = G.gy - 2 * kPad + 1;
    const size_t slab = (size_t)G.gy * G.gx;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nx * ny; t += gridDim.x * blockDim.x) {
        const int ky = t / nx, kx = t - ky * nx;
        // candidates around (k - 1/2) s .. (k + 1/2) s; each checked with the cell decision itself
        const int y0 = max(0, (int)floorf((ky - 0.5f) * G.ss) - 1);
        const int y1 = min(G.H - 1, (int)ceilf((ky + 0.5f) * G.ss) + 1);
        const int x0 = max(0, (int)floorf((kx - 0.5f) * G.ss) - 1);
        const int x1 = min(G.W - 1, (int)ceilf((kx + 0.5f) * G.ss) + 1);
        float2* col = grid + (size_t)(ky + kPad) * G.gx + (kx + kPad);
        for (int y = y0; y <= y1; ++y) {
            if (cell_of((float)y, 0.0f, G.ss) != ky) continue;
            for (int x = x0; x <= x1; ++x) {
                if (cell_of((float)x, 0.0f, G.ss) != kx) continue;
                const float g = grad_at(f, G.H, G.W, y, x, G.field);
                const int z = cell_of(g, G.lo, G.sr) + kPad;
                if (!BLFLS_DCHECK(z >= 0 && z < G.gz && ky + kPad < G.gy && kx + kPad < G.gx,
                                  kDcGridCell))
                    continue;
                float2* c = col + (size_t)z * slab;
                c->x += g;
                c->y += 1.f;
            }
        }
    }
}

// out[i] = in[i] + e (in[i - stride] + in[i + stride]) along one axis (zero outside).
__global__ void __launch_bounds__(kGridThreads) k6_blur(const float2* __restrict__ in,
                                                       float2* __restrict__ out, int gx, int gy,
                                                       int gz, int axis)
{
    const float e = 0.60653065971263342f;   // exp(-1/2)
    const size_t n = (size_t)gx * gy * gz;
    const size_t stride = axis == 0 ? 1 : axis == 1 ? (size_t)gx : (size_t)gx * gy;
    const int len = axis == 0 ? gx : axis == 1 ? gy : gz;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int pos = (int)((i / stride) % (size_t)len);
        float2 a = in[i];
        float2 s = make_float2(0.f, 0.f);
        if (pos > 0) { const float2 b = in[i - stride]; s.x += b.x; s.y += b.y; }
        if (pos + 1 < len) { const float2 b = in[i + stride]; s.x += b.x; s.y += b.y; }
        out[i] = make_float2(fmaf(e, s.x, a.x), fmaf(e, s.y, a.y));
    }
}

__global__ void __launch_bounds__(kGridThreads) k6_slice(const float* __restrict__ f,
                                                        const float2* __restrict__ grid,
                                                        float* __restrict__ e, GridGeom G)
{
    const size_t plane = (size_t)G.H * G.W;
    const size_t slab = (size_t)G.gy * G.gx;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / G.W), x = (int)(i - (size_t)y * G.W);
        const float g = grad_at(f, G.H, G.W, y, x, G.field);
        const float zf = __fdiv_rn(g - G.lo, G.sr) + kPad;
        const float yf = __fdiv_rn((float)y, G.ss) + kPad;
        const float xf = __fdiv_rn((float)x, G.ss) + kPad;
        const int z0 = min((int)zf, G.gz - 2), y0 = min((int)yf, G.gy - 2), x0 = min((int)xf, G.gx - 2);
        const float fz = zf - z0, fy = yf - y0, fx = xf - x0;
        float sw = 0.f, sc = 0.f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const float w = (dz ? fz : 1.f - fz) * (dy ? fy : 1.f - fy) * (dx ? fx : 1.f - fx);
                    const float2 c = grid[(size_t)(z0 + dz) * slab + (size_t)(y0 + dy) * G.gx + (x0 + dx)];
                    sw = fmaf(w, c.x, sw);
                    sc = fmaf(w, c.y, sc);
                }
        e[i] = __fdiv_rn(sw, sc) - g;
    }
}

__device__ __forceinline__ float key_to_float(int key)
{
    return __int_as_float(key ^ ((key >> 31) & 0x7fffffff));
}

// Range constants of every channel for normalised gradients: each field's range R = max - min
// (1 for a constant field), sigma_r R in FP32, then kappa = sqrt(log2(e) / (2 (sigma_r R)^2)) and
// 1 / kappa in FP64 rounded to FP32 -- the host's blf_constants, operation for operation.
__global__ void k6_range_kappa(const int* __restrict__ keys, int C, float sigma_r,
                               float4* __restrict__ kap)
{
    const int c = threadIdx.x;
    if (c >= C) return;
    float k[2], ik[2];
#pragma unroll
    for (int fl = 0; fl < 2; ++fl) {
        const float lo = key_to_float(keys[4 * c + 2 * fl]);
        const float hi = key_to_float(keys[4 * c + 2 * fl + 1]);
        const float range = hi - lo;
        const float sr = sigma_r * (range > 0.f ? range : 1.0f);
        double kd = 1.0;
        if (isfinite(sr)) kd = sqrt(1.4426950408889634 / (2.0 * (double)sr * sr));
        k[fl] = (float)kd;
        ik[fl] = (float)(1.0 / kd);
    }
    kap[c] = make_float4(k[0], k[1], ik[0], ik[1]);
}

int stream_blocks(size_t n, int num_sms)
{
    const size_t want = (n + kGridThreads - 1) / kGridThreads;
    return (int)std::max<size_t>(1, std::min(want, (size_t)num_sms * 8));
}

}  // namespace

BLFLS_DCHECK_TU(grid)

cudaError_t launch_grid_minmax(const float* img, int H, int W, int C, int* keys, cudaStream_t s,
                               int num_sms)
{
    k6_init_keys<<<1, 32, 0, s>>>(keys, 4 * C);
    dim3 grid(stream_blocks((size_t)H * W, num_sms) / std::max(1, C) + 1, C);
    k6_minmax<<<grid, kGridThreads, 0, s>>>(img, H, W, keys);
    return cudaGetLastError();
}

cudaError_t launch_range_kappa(const int* keys, int C, float sigma_r, float4* kap, cudaStream_t s)
{
    k6_range_kappa<<<1, 32, 0, s>>>(keys, C, sigma_r, kap);
    return cudaGetLastError();
}

float grid_key_to_float(int key)
{
    const int i = key ^ ((key >> 31) & 0x7fffffff);
    float v;
    std::memcpy(&v, &i, sizeof v);
    return v;
}

void grid_dims(int H, int W, float lo, float hi, float sigma_s, float sigma_r, int* gx, int* gy,
               int* gz)
{
    const double ss = sigma_s, sr = sigma_r;
    *gx = (int)std::floor((W - 1) / ss) + 1 + 2 * kPad;
    *gy = (int)std::floor((H - 1) / ss) + 1 + 2 * kPad;
    *gz = (int)std::floor(((double)hi - (double)lo) / sr) + 1 + 2 * kPad;
}

cudaError_t launch_grid_residual(const float* f, float* e, int field, int H, int W, float sigma_s,
                                 float sigma_r, float lo, int gx, int gy, int gz, float2* ga,
                                 float2* gb, cudaStream_t s, int num_sms)
{
    const size_t cells = (size_t)gx * gy * gz;
    cudaError_t err = cudaMemsetAsync(ga, 0, cells * sizeof(float2), s);
    if (err != cudaSuccess) return err;
    const GridGeom G{H, W, gx, gy, gz, sigma_s, sigma_r, lo, field};
    const int nsp = (gx - 2 * kPad + 1) * (gy - 2 * kPad + 1);
    k6_splat<<<stream_blocks((size_t)nsp, num_sms), kGridThreads, 0, s>>>(f, ga, G);
    const int nb = stream_blocks(cells, num_sms);
    k6_blur<<<nb, kGridThreads, 0, s>>>(ga, gb, gx, gy, gz, 0);
    k6_blur<<<nb, kGridThreads, 0, s>>>(gb, ga, gx, gy, gz, 1);
    k6_blur<<<nb, kGridThreads, 0, s>>>(ga, gb, gx, gy, gz, 2);
    k6_slice<<<stream_blocks((size_t)H * W, num_sms), kGridThreads, 0, s>>>(f, gb, e, G);
    return cudaGetLastError();
}

}  // namespace blfls
