// Bilateral-grid approximation of the BLF of Eq. 1 (the fast filter the paper uses in its
// experiments, Section III-A / IV), on the two periodic forward-difference gradient fields of a
// channel; the output is the residual e = BLF_grid(g) - g consumed by the Fourier solve.
//
// For one field g (H x W), with spatial and range sampling steps s_s = sigma_s, s_r = sigma_r and
// a padding of P = 2 cells, the grid holds (sum of g, count) pairs over
// Gz x Gy x Gx = (floor((max g - min g) / s_r) + 1 + 2P) x (floor((H-1)/s_s) + 1 + 2P) x
// (floor((W-1)/s_s) + 1 + 2P) cells, z-major:
//   k6_minmax      min and max of both fields of every channel (order-preserving integer keys, so
//                  the atomics are exact and the result does not depend on their order);
//   k6_*0         the first chunk of range levels of one field, one launch per phase, the levels
//                 from the range keys on the device: clear; splat (one thread per spatial cell
//                 walks the pixels whose nearest cell it is and adds (g, 1) to the range level of
//                 each, in a fixed order: deterministic, no atomics); the 3-tap blur (e^-1/2, 1,
//                 e^-1/2) along x, y, then z (zero outside); the trilinear slice at
//                 (z, y / s_s + P, x / s_s + P): e = sum / count - g;
//   k6_chunks     the further chunks of a wider field (one cooperative launch, grid-wide
//                 barriers between the phases; it returns at once for one chunk).
// The range is never read back to the host: the buffers hold a chunk of levels whose size the
// host fixes, and a wider range takes more chunks.
// Cell indices are floor(t + 1/2) of the real t: FP32 decides away from rounding boundaries, FP64
// near them (see cell_of), so the cells are those of the FP64 definition on the FP32 gradients.
// Grid passes are HBM/L2-bound streams.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "blfls.h"
#include "dcheck.cuh"
#include "internal.h"

namespace blfls {

namespace cg = cooperative_groups;

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

__device__ __forceinline__ float key_to_float(int key)
{
    return __int_as_float(key ^ ((key >> 31) & 0x7fffffff));
}

// One field's grid, computed in chunks of range levels so that the buffers have a size the host
// knows before the range is known: chunk k holds the levels z in [zb - 1, zb + zc] of the grid
// (zb = k (zc - 1); buffer level l = z - zb + 1), and slices the pixels whose lower trilinear
// level z0 lies in [zb, zb + zc - 1), so the chunks partition the pixels.  Every cell of a chunk
// is the same sum, blurred in the same order, as in the whole grid (the levels just outside a
// chunk are splatted too), so the result does not depend on zc.
struct GridChunk {
    const float* f;
    float* e;
    const int4* lev;    // this field's levels (k6_levels): lo (bits), gz, chunks, ok
    float2* ga;
    float2* gb;         // (zc + 2) x gy x gx cells each
    int H, W, gx, gy, zc, field;
    float ss, sr;
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

// Splat: one thread per spatial cell (cy, cx) that a pixel can round to (floor((W-1)/s_s) + 2
// cells per axis: the last pixel can round up into the first padding cell) walks its pixels in
// order and adds (g, 1) to the range level of each that falls in the chunk.
__device__ __forceinline__ void grid_splat(const GridChunk& P, float lo, int gz, int zb,
                                           size_t tid, size_t nthreads)
{
    const int nx = P.gx - 2 * kPad + 1, ny = P.gy - 2 * kPad + 1;
    const size_t slab = (size_t)P.gy * P.gx;
    for (size_t t = tid; t < (size_t)nx * ny; t += nthreads) {
        const int ky = (int)(t / nx), kx = (int)(t - (size_t)ky * nx);
        // candidates around (k - 1/2) s .. (k + 1/2) s; each checked with the cell decision itself
        const int y0 = max(0, (int)floorf((ky - 0.5f) * P.ss) - 1);
        const int y1 = min(P.H - 1, (int)ceilf((ky + 0.5f) * P.ss) + 1);
        const int x0 = max(0, (int)floorf((kx - 0.5f) * P.ss) - 1);
        const int x1 = min(P.W - 1, (int)ceilf((kx + 0.5f) * P.ss) + 1);
        float2* col = P.ga + (size_t)(ky + kPad) * P.gx + (kx + kPad);
        for (int y = y0; y <= y1; ++y) {
            if (cell_of((float)y, 0.0f, P.ss) != ky) continue;
            for (int x = x0; x <= x1; ++x) {
                if (cell_of((float)x, 0.0f, P.ss) != kx) continue;
                const float g = grad_at(P.f, P.H, P.W, y, x, P.field);
                const int l = cell_of(g, lo, P.sr) + kPad - zb + 1;
                if (l < 0 || l > P.zc + 1) continue;   // another chunk's level
                if (!BLFLS_DCHECK(l - 1 + zb < gz && ky + kPad < P.gy && kx + kPad < P.gx,
                                  kDcGridCell))
                    continue;
                float2* c = col + (size_t)l * slab;
                c->x += g;
                c->y += 1.f;
            }
        }
    }
}

// The range levels of a field's grid from its range keys, as the FP64 definition
// floor((max - min) / s_r) + 1 + 2P, and the chunks that cover them (chunk k: zb = k (zc - 1)).
// A range of more than max_cells cells of s_r, or a NaN range, cannot be gridded (ok = 0).
// One thread per field (k6_levels); the phase kernels read the result.
struct GridLevels {
    float lo;
    int gz, nchunks;
    bool ok;
};
__global__ void k6_levels(const int* __restrict__ keys, int nfields, float sigma_r, int zc,
                          int max_cells, int4* __restrict__ lev)
{
    const int q = threadIdx.x;
    if (q >= nfields) return;
    const float lo = key_to_float(keys[2 * q]);
    const float hi = key_to_float(keys[2 * q + 1]);
    const double span = floor(((double)hi - (double)lo) / (double)sigma_r);
    const bool ok = span >= 0.0 && span <= (double)max_cells;
    const int gz = ok ? (int)span + 1 + 2 * kPad : 0;
    const int nchunks = ok ? (gz - 1 + zc - 2) / (zc - 1) : 0;   // chunks of z0 in [0, gz - 2]
    lev[q] = make_int4(__float_as_int(lo), gz, nchunks, ok ? 1 : 0);
}
__device__ __forceinline__ GridLevels grid_levels(const GridChunk& P)
{
    const int4 v = __ldg(P.lev);
    return GridLevels{__int_as_float(v.x), v.y, v.z, v.w != 0};
}

// Buffer levels chunk zb fills: l in [l0, l1), global z = zb + l - 1 inside the grid's [0, gz)
// (l0 = 0 below the first chunk's bottom level, l1 up to zc + 2 over its top one: the levels just
// outside a chunk are its z blur's neighbours; levels outside the grid are never read).
struct ChunkLevels {
    int l0, l1;
};
__device__ __forceinline__ ChunkLevels chunk_levels(const GridChunk& P, int gz, int zb)
{
    return ChunkLevels{zb == 0 ? 1 : 0, min(P.zc + 2, gz - zb + 1)};
}

// A chunk holds fewer than 2^32 cells (its buffers are bounded by BLFLS_GRID_MAX_BYTES), so the
// cell loops use 32-bit indices.
__device__ __forceinline__ void grid_clear(const GridChunk& P, ChunkLevels cl, unsigned tid,
                                           unsigned nthreads)
{
    const unsigned slab = (unsigned)P.gx * P.gy;
    const unsigned first = slab * (unsigned)cl.l0, n = slab * (unsigned)(cl.l1 - cl.l0);
    for (unsigned k = tid; k < n; k += nthreads) P.ga[first + k] = make_float2(0.f, 0.f);
}

// out = in + e (in[-stride] + in[+stride]) along x (axis 0) or y (axis 1) of the chunk's levels,
// or along z (axis 2) for its interior levels inside the grid; zero outside the whole grid.
__device__ __forceinline__ void grid_blur(const float2* __restrict__ in, float2* __restrict__ out,
                                          const GridChunk& P, int gz, int zb, ChunkLevels cl,
                                          int axis, unsigned tid, unsigned nthreads)
{
    const float e = 0.60653065971263342f;   // exp(-1/2)
    const unsigned gx = (unsigned)P.gx, gy = (unsigned)P.gy;
    const unsigned slab = gx * gy;
    const int la = axis == 2 ? 1 : cl.l0;
    const int lb = axis == 2 ? min(P.zc + 1, gz - zb + 1) : cl.l1;
    const unsigned first = slab * (unsigned)la;
    const unsigned n = lb > la ? slab * (unsigned)(lb - la) : 0u;
    const unsigned stride = axis == 0 ? 1u : axis == 1 ? gx : slab;
    for (unsigned k = tid; k < n; k += nthreads) {
        const unsigned i = first + k;
        int pos, len;
        if (axis == 0) {
            pos = (int)(i % gx);
            len = P.gx;
        } else if (axis == 1) {
            pos = (int)((i / gx) % gy);
            len = P.gy;
        } else {
            pos = (int)(i / slab) - 1 + zb;   // global level
            len = gz;
        }
        const float2 a = in[i];
        float2 s = make_float2(0.f, 0.f);
        if (pos > 0) { const float2 b = in[i - stride]; s.x += b.x; s.y += b.y; }
        if (pos + 1 < len) { const float2 b = in[i + stride]; s.x += b.x; s.y += b.y; }
        out[i] = make_float2(fmaf(e, s.x, a.x), fmaf(e, s.y, a.y));
    }
}

// Slice: trilinear interpolation at (z, y / s_s + P, x / s_s + P) for the pixels whose lower
// level z0 lies in [zb, zb + zc - 1): e = sum / count - g.
__device__ __forceinline__ void grid_slice(const GridChunk& P, float lo, int gz, int zb,
                                           size_t tid, size_t nthreads)
{
    const size_t plane = (size_t)P.H * P.W;
    const size_t slab = (size_t)P.gy * P.gx;
    for (size_t i = tid; i < plane; i += nthreads) {
        const int y = (int)(i / P.W), x = (int)(i - (size_t)y * P.W);
        const float g = grad_at(P.f, P.H, P.W, y, x, P.field);
        const float zf = __fdiv_rn(g - lo, P.sr) + kPad;
        const int z0 = min((int)zf, gz - 2);
        if (z0 < zb || z0 >= zb + P.zc - 1) continue;   // another chunk's pixel
        const float yf = __fdiv_rn((float)y, P.ss) + kPad;
        const float xf = __fdiv_rn((float)x, P.ss) + kPad;
        const int y0 = min((int)yf, P.gy - 2), x0 = min((int)xf, P.gx - 2);
        const float fz = zf - z0, fy = yf - y0, fx = xf - x0;
        const float2* base = P.gb + (size_t)(z0 - zb + 1) * slab;
        float sw = 0.f, sc = 0.f;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const float w = (dz ? fz : 1.f - fz) * (dy ? fy : 1.f - fy) * (dx ? fx : 1.f - fx);
                    const float2 c = base[(size_t)dz * slab + (size_t)(y0 + dy) * P.gx + (x0 + dx)];
                    sw = fmaf(w, c.x, sw);
                    sc = fmaf(w, c.y, sc);
                }
        P.e[i] = __fdiv_rn(sw, sc) - g;
    }
}

__device__ __forceinline__ unsigned gtid() { return blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ unsigned gthreads() { return gridDim.x * blockDim.x; }

// The first chunk (the only one for a field of range up to 2 and the chunk size the host picks)
// in one launch per phase: each kernel reads the levels from the range keys.
__global__ void __launch_bounds__(kGridThreads) k6_clear0(GridChunk P)
{
    const GridLevels G = grid_levels(P);
    if (G.ok) grid_clear(P, chunk_levels(P, G.gz, 0), gtid(), gthreads());
}
__global__ void __launch_bounds__(kGridThreads) k6_splat0(GridChunk P)
{
    const GridLevels G = grid_levels(P);
    if (G.ok) grid_splat(P, G.lo, G.gz, 0, gtid(), gthreads());
}
__global__ void __launch_bounds__(kGridThreads) k6_blur0(GridChunk P, int axis)
{
    const GridLevels G = grid_levels(P);
    if (!G.ok) return;
    const float2* in = axis == 1 ? P.gb : P.ga;
    float2* out = axis == 1 ? P.ga : P.gb;
    grid_blur(in, out, P, G.gz, 0, chunk_levels(P, G.gz, 0), axis, gtid(), gthreads());
}
__global__ void __launch_bounds__(kGridThreads) k6_slice0(GridChunk P)
{
    const GridLevels G = grid_levels(P);
    if (!G.ok) {
        const size_t plane = (size_t)P.H * P.W;
        for (size_t i = gtid(); i < plane; i += gthreads()) P.e[i] = __int_as_float(0x7fc00000);
        return;
    }
    grid_slice(P, G.lo, G.gz, 0, gtid(), gthreads());
}

// The remaining chunks of a wider field, in one cooperative launch with a grid-wide barrier
// between the phases (returns at once when the first chunk covered the field).  Every block
// takes the same branches, so every block reaches every barrier.
__global__ void __launch_bounds__(kGridThreads) k6_chunks(GridChunk P)
{
    const GridLevels G = grid_levels(P);
    if (G.nchunks <= 1) return;
    cg::grid_group grid = cg::this_grid();
    const unsigned tid = gtid(), nthreads = gthreads();
    for (int k = 1; k < G.nchunks; ++k) {
        const int zb = k * (P.zc - 1);
        const ChunkLevels cl = chunk_levels(P, G.gz, zb);
        grid.sync();   // the previous chunk's slice has read the buffers
        grid_clear(P, cl, tid, nthreads);
        grid.sync();
        grid_splat(P, G.lo, G.gz, zb, tid, nthreads);
        grid.sync();
        grid_blur(P.ga, P.gb, P, G.gz, zb, cl, 0, tid, nthreads);
        grid.sync();
        grid_blur(P.gb, P.ga, P, G.gz, zb, cl, 1, tid, nthreads);
        grid.sync();
        grid_blur(P.ga, P.gb, P, G.gz, zb, cl, 2, tid, nthreads);
        grid.sync();
        grid_slice(P, G.lo, G.gz, zb, tid, nthreads);
    }
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

void grid_spatial_dims(int H, int W, float sigma_s, int* gx, int* gy)
{
    const double ss = sigma_s;
    *gx = (int)std::floor((W - 1) / ss) + 1 + 2 * kPad;
    *gy = (int)std::floor((H - 1) / ss) + 1 + 2 * kPad;
}

int grid_chunk_levels(float sigma_r, int gx, int gy)
{
    // the levels a field of range 2 needs (gradients of an image in [0, 1]), at most 256 MiB of
    // cells per buffer, at least 8
    const double want = std::floor(2.0 / (double)sigma_r) + 1 + 2 * kPad;
    const double budget = std::floor((256.0 * 1024 * 1024) / (sizeof(float2) * (double)gx * gy)) - 2;
    return (int)std::max(8.0, std::min(want, budget));
}

cudaError_t launch_grid_levels(const int* keys, int C, float sigma_r, int zc, int4* lev,
                               cudaStream_t s)
{
    k6_levels<<<1, 2 * BLFLS_MAX_CHANNELS, 0, s>>>(keys, 2 * C, sigma_r, zc,
                                                    BLFLS_GRID_MAX_RANGE_CELLS, lev);
    return cudaGetLastError();
}

cudaError_t launch_grid_field(const float* f, float* e, int field, int H, int W, float sigma_s,
                              float sigma_r, const int4* lev, int gx, int gy, int zc, float2* ga,
                              float2* gb, cudaStream_t s, int num_sms)
{
    const GridChunk P{f, e, lev, ga, gb, H, W, gx, gy, zc, field, sigma_s, sigma_r};
    const size_t cells = (size_t)gx * gy * (size_t)(zc + 2);
    const int nsp = (gx - 2 * kPad + 1) * (gy - 2 * kPad + 1);
    const int nb = stream_blocks(cells, num_sms);
    k6_clear0<<<nb, kGridThreads, 0, s>>>(P);
    k6_splat0<<<stream_blocks((size_t)nsp, num_sms), kGridThreads, 0, s>>>(P);
    for (int axis = 0; axis < 3; ++axis) k6_blur0<<<nb, kGridThreads, 0, s>>>(P, axis);
    k6_slice0<<<stream_blocks((size_t)H * W, num_sms), kGridThreads, 0, s>>>(P);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    // one block per SM: the launch returns at once in the usual case of a single chunk
    void* args[] = {(void*)&P};
    return cudaLaunchCooperativeKernel((const void*)k6_chunks, dim3((unsigned)num_sms),
                                       dim3(kGridThreads), args, 0, s);
}

}  // namespace blfls
