// Shared device code of step 1 of BLF-LS (Section III-A): the bilateral filter of Eq. 1 on the periodic forward-
// difference gradients (Section II-B), emitted as residuals e_* = f_BLF(g_*) - g_*.
//
// K1 (tiled): one CTA per 32 x th output tile of one channel (4 th threads).  The CTA loads the
// image tile with an (r+1)-pixel periodic halo into shared memory and forms both gradient fields
// on the tile + r halo, pre-scaled by kappa = sqrt(log2(e) / (2 sigma_r^2)) so that a range
// weight is a single exp2(-(t' - s')^2).  Each thread filters a vertical strip of 8 pixels of
// both fields: for every window column dx it streams the 8 + 2r values of that column once and
// applies each to every strip pixel in reach.  The spatial weight is split as
// exp2(a_dx) * exp2(a_dy): the dy part sits in the exponent (a per-kernel register table), the
// dx part multiplies the tap value once per row.  The FP32 form packs the two gradient fields
// into the two lanes of sm_100 f32x2 arithmetic (the tile stores (g_x', g_y') pairs): per tap pair
// one packed subtract, one packed FMA (the exponent), two MUFU ex2 and two packed FMAs (sum of
// weighted values and sum of weights) -- three instructions per tap.
//
// Precision forms (same tiling):
//   FP16W: the same field packing in half2 lanes: tile, exponent, weights and products in half2
//          (ex2.approx.f16x2 gives both fields' weights per MUFU operation); the products and
//          weights of one window column are summed in half2 and flushed into FP32 accumulators
//          (scaled by exp2(a_dx)) after every column.
//   BF16W: as FP32 but the weights are rounded to BF16 by ex2.approx.ftz.bf16x2, then widened
//          (exactly) to FP32 for the products and sums.
// Radii up to kMaxTemplR are compiled with the window unrolled per column; larger radii up to
// kMaxTiledR use a scalar FP32 kernel with a runtime window; above that a per-pixel kernel reads
// precomputed gradients from global memory.
#pragma once
#include "dcheck.cuh"
#include "internal.h"

#include <cmath>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace blfls {
namespace {

constexpr int kTW = 32;          // tile width  (one warp across)
constexpr int kMaxTH = 64;       // tallest tile (rows); the height is a launch parameter
constexpr int kStrip = 8;        // pixels per thread (vertical strip)
constexpr int kPairs = kStrip / 2;
constexpr int kMaxThreads = kTW * kMaxTH / kStrip;  // 256: 32 threads per 8 rows
constexpr int kMaxTemplR = 16;
constexpr int kMaxTiledR = 48;
constexpr float kBig = 1e30f;    // exponent offset that turns a weight into exactly 0

using u64 = unsigned long long;

// Range scaling of the two gradient fields: x' = kx g_x, y' = ky g_y (kappa of Eq. 1's range
// kernel, see blf_constants; the fields differ only when each is normalised to its own range),
// and the inverses that map residuals back.
struct Kap {
    float x, y, ix, iy;
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ __half2 ex2_h2(__half2 x)
{
    unsigned xi = *reinterpret_cast<unsigned*>(&x), yi;
    asm("ex2.approx.f16x2 %0, %1;" : "=r"(yi) : "r"(xi));
    return *reinterpret_cast<__half2*>(&yi);
}
__device__ __forceinline__ __nv_bfloat162 ex2_bf2(__nv_bfloat162 x)
{
    unsigned xi = *reinterpret_cast<unsigned*>(&x), yi;
    asm("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(yi) : "r"(xi));
    return *reinterpret_cast<__nv_bfloat162*>(&yi);
}
// packed FP32 pairs (sm_100+ f32x2 arithmetic)
__device__ __forceinline__ u64 pk(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(u64 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ int wrap_idx(int i, int n)
{
    int m = i % n;
    return m < 0 ? m + n : m;
}

// Shared-memory layout of a tile for radius R: f on (TH+2R+1) x (TW+2R+1) floats, then the two
// gradient tiles of (TH+2R) x (TW+2R) elements of `elem` bytes each.
__host__ __device__ __forceinline__ int f_pitch(int R) { return kTW + 2 * R + 1; }
__host__ __device__ __forceinline__ int f_rows(int R, int th) { return th + 2 * R + 1; }
__host__ __device__ __forceinline__ int g_pitch(int R) { return kTW + 2 * R; }
__host__ __device__ __forceinline__ int g_rows(int R, int th) { return th + 2 * R; }
__host__ __device__ __forceinline__ size_t f_bytes(int R, int th)
{
    return ((sizeof(float) * (size_t)f_rows(R, th) * f_pitch(R)) + 15) & ~size_t(15);
}
__host__ __device__ __forceinline__ size_t tile_smem_bytes(int R, size_t elem, int th)
{
    return f_bytes(R, th) + 2 * elem * (size_t)g_rows(R, th) * g_pitch(R);
}

// The image tile with its periodic halo: rows y0 - R .., columns x0 - R .. (fr x fp values).
// Each warp takes whole tile rows with its lanes along the row (coalesced loads); a lane wraps
// its columns once and a warp each of its rows once, instead of wrapping every element.
constexpr int kTileColsPerLane = (kTW + 2 * kMaxTiledR + 1 + 31) / 32;

__device__ __forceinline__ void load_f_tile(const float* __restrict__ f, int H, int W, int x0,
                                            int y0, int R, int th, float* sf)
{
    const int fp = f_pitch(R), fr = f_rows(R, th);
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    int xs[kTileColsPerLane];
#pragma unroll
    for (int k = 0; k < kTileColsPerLane; ++k) xs[k] = wrap_idx(x0 - R + lane + 32 * k, W);
    for (int r = threadIdx.x >> 5; r < fr; r += nw) {
        const int yy = wrap_idx(y0 - R + r, H);
        if (!BLFLS_DCHECK(yy >= 0 && yy < H, kDcTileLoad)) continue;
        const float* row = f + (size_t)yy * W;
        float* srow = sf + r * fp;
#pragma unroll
        for (int k = 0; k < kTileColsPerLane; ++k) {
            const int c = lane + 32 * k;
            if (c < fp && BLFLS_DCHECK(xs[k] >= 0 && xs[k] < W, kDcTileLoad))
                srow[c] = __ldg(row + xs[k]);
        }
    }
}

// kappa-scaled gradient at tile position (r, c) of the g tiles (FP32, from the f tile)
__device__ __forceinline__ float grad_x(const float* sf, int fp, int r, int c, float kappa)
{
    return kappa * (sf[r * fp + c + 1] - sf[r * fp + c]);
}
__device__ __forceinline__ float grad_y(const float* sf, int fp, int r, int c, float kappa)
{
    return kappa * (sf[(r + 1) * fp + c] - sf[r * fp + c]);
}

// e = (acc / Z - s') / kappa (per field) for the strip (FP32 accumulators), guarded against the image edge.
__device__ __forceinline__ void store_strip(float* __restrict__ ex, float* __restrict__ ey, int H,
                                            int W, int x, int ybase, const float* ax,
                                            const float* zx, const float* sx, const float* ay,
                                            const float* zy, const float* sy, const Kap k)
{
    if (x >= W || !BLFLS_DCHECK(x >= 0 && ybase >= 0, kDcTileStore)) return;
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        const int y = ybase + j;
        if (y < H) {
            ex[(size_t)y * W + x] = (__fdiv_rn(ax[j], zx[j]) - sx[j]) * k.ix;
            ey[(size_t)y * W + x] = (__fdiv_rn(ay[j], zy[j]) - sy[j]) * k.iy;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// FP32 and BF16-weight forms, packed f32x2 with the two gradient fields in the two lanes: the
// tile holds interleaved (g_x', g_y') pairs, so one 64-bit shared load gives both fields' value
// of a tap, both lanes share the tap's spatial weight, and per tap pair the work is one packed
// subtract, one packed FMA (exponent), two ex2, and two packed FMAs (weighted sum, weight sum).
// BF16W rounds the weights to BF16 (ex2.approx.ftz.bf16x2) and widens them back exactly.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ u64 bf2_to_f2(__nv_bfloat162 w)
{
    const unsigned b = *reinterpret_cast<unsigned*>(&w);
    return pk(__uint_as_float(b << 16), __uint_as_float(b & 0xffff0000u));
}

template <int R, bool RANGE, bool BF16W, bool JOINT>
__device__ __forceinline__ void tile_pair_fields(const float* __restrict__ f,
                                                 const float* __restrict__ guide,
                                                 float* __restrict__ ex, float* __restrict__ ey,
                                                 int H, int W, int x0, int y0, int th,
                                                 const Kap k, float cs,
                                                 unsigned char* smem)
{
    constexpr int fp = kTW + 2 * R + 1, gp = kTW + 2 * R;
    const int gr = th + 2 * R;
    float* sf = reinterpret_cast<float*>(smem);
    float2* g = reinterpret_cast<float2*>(smem + f_bytes(R, th));   // (g_x', g_y') per position
    float2* hg = JOINT ? g + gr * gp : g;                            // range-term values
    load_f_tile(f, H, W, x0, y0, R, th, sf);
    __syncthreads();
    for (int i = threadIdx.x; i < gr * gp; i += blockDim.x) {
        const int r = i / gp, c = i - r * gp;
        g[i] = make_float2(grad_x(sf, fp, r, c, k.x), grad_y(sf, fp, r, c, k.y));
    }
    if constexpr (JOINT) {   // the guidance image's gradients, through the same f buffer
        __syncthreads();
        load_f_tile(guide, H, W, x0, y0, R, th, sf);
        __syncthreads();
        for (int i = threadIdx.x; i < gr * gp; i += blockDim.x) {
            const int r = i / gp, c = i - r * gp;
            hg[i] = make_float2(grad_x(sf, fp, r, c, k.x), grad_y(sf, fp, r, c, k.y));
        }
    }
    __syncthreads();

    const int cx = threadIdx.x & (kTW - 1);
    const int r0 = (threadIdx.x / kTW) * kStrip;
    u64 S[kStrip], A[kStrip], Z[kStrip];
    const u64* own = reinterpret_cast<const u64*>(hg + (R + r0) * gp + R + cx);
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        S[j] = own[j * gp];
        A[j] = Z[j] = 0ull;
    }
    // NA[d] = (n, n), n = (d - R)^2 cs: the dy part of the spatial log2-weight of both lanes
    u64 NA[2 * R + 1];
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) {
        const float n = float((d - R) * (d - R)) * cs;
        NA[d] = pk(n, n);
        asm volatile("" : "+l"(NA[d]));   // keep the table in registers (no per-use recompute)
    }

#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
        // this column's reads: rows r0 .. r0 + kStrip + 2R - 1 of tile column R + cx + dx
        if (!BLFLS_DCHECK(R + cx + dx >= 0 && R + cx + dx < gp &&
                          (r0 + kStrip + 2 * R - 1) * gp + R + cx + dx < gr * gp, kDcTileWindow))
            continue;
        const float gdx = ex2_approx(-float(dx * dx) * cs);     // the dx part of the weight
        const u64 GD = pk(gdx, gdx);
        const u64* col = reinterpret_cast<const u64*>(g + r0 * gp + R + cx + dx);
        const u64* rcol = reinterpret_cast<const u64*>(hg + r0 * gp + R + cx + dx);
#pragma unroll
        for (int i = 0; i < kStrip + 2 * R; ++i) {
            const u64 T = col[i * gp];
            const u64 TR = JOINT ? rcol[i * gp] : T;   // the value the range weight compares
            const u64 TG = mul2(T, GD);
#pragma unroll
            for (int j = 0; j < kStrip; ++j) {
                const int d = i - j;  // dy + R
                if (d < 0 || d > 2 * R) continue;
                float e0, e1;
                if (RANGE) {
                    const u64 Q = sub2(TR, S[j]);
                    upk(fma2(Q, Q, NA[d]), e0, e1);
                } else {
                    upk(NA[d], e0, e1);
                }
                u64 Wt;
                if (BF16W) Wt = bf2_to_f2(ex2_bf2(__floats2bfloat162_rn(-e0, -e1)));
                else Wt = pk(ex2_approx(-e0), ex2_approx(-e1));
                A[j] = fma2(Wt, TG, A[j]);
                Z[j] = fma2(Wt, GD, Z[j]);
            }
        }
    }
    float ax[kStrip], zx[kStrip], sx[kStrip], ay[kStrip], zy[kStrip], sy[kStrip];
    const u64* own_g = reinterpret_cast<const u64*>(g + (R + r0) * gp + R + cx);
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        upk(A[j], ax[j], ay[j]);
        upk(Z[j], zx[j], zy[j]);
        upk(JOINT ? own_g[j * gp] : S[j], sx[j], sy[j]);   // the input's own gradient
    }
    store_strip(ex, ey, H, W, x0 + cx, y0 + r0, ax, zx, sx, ay, zy, sy, k);
}

template <int R, bool RANGE, bool JOINT>
__device__ __forceinline__ void tile_f32(const float* __restrict__ f, const float* __restrict__ guide,
                                         float* __restrict__ ex,
                                         float* __restrict__ ey, int H, int W, int x0, int y0,
                                         int th, const Kap k, float cs,
                                         unsigned char* smem)
{
    tile_pair_fields<R, RANGE, false, JOINT>(f, guide, ex, ey, H, W, x0, y0, th, k, cs, smem);
}

template <int R, bool RANGE, bool JOINT>
__device__ __forceinline__ void tile_bf16(const float* __restrict__ f, const float* __restrict__ guide,
                                          float* __restrict__ ex,
                                          float* __restrict__ ey, int H, int W, int x0, int y0,
                                          int th, const Kap k, float cs,
                                          unsigned char* smem)
{
    tile_pair_fields<R, RANGE, true, JOINT>(f, guide, ex, ey, H, W, x0, y0, th, k, cs, smem);
}

// ---------------------------------------------------------------------------------------------
// FP16 weights: the two gradient fields in the two half2 lanes; exponent, weights and products
// in half2 (ex2.approx.f16x2 gives both fields' weights in one MUFU operation); each window
// column's sums of w t and w are kept in half2 and flushed into FP32 accumulators (scaled by
// the column's spatial factor exp2(a_dx)) after every column.
// ---------------------------------------------------------------------------------------------
template <int R, bool RANGE, bool JOINT>
__device__ __forceinline__ void tile_f16(const float* __restrict__ f, const float* __restrict__ guide,
                                         float* __restrict__ ex,
                                         float* __restrict__ ey, int H, int W, int x0,
                                         int y0, int th, const Kap k,
                                         float cs, unsigned char* smem)
{
    constexpr int fp = kTW + 2 * R + 1, gp = kTW + 2 * R;
    const int gr = th + 2 * R;
    float* sf = reinterpret_cast<float*>(smem);
    __half2* g = reinterpret_cast<__half2*>(smem + f_bytes(R, th));   // (g_x', g_y') per position
    __half2* hg = JOINT ? g + gr * gp : g;                            // range-term values
    load_f_tile(f, H, W, x0, y0, R, th, sf);
    __syncthreads();
    for (int i = threadIdx.x; i < gr * gp; i += blockDim.x) {
        const int r = i / gp, c = i - r * gp;
        g[i] = __floats2half2_rn(grad_x(sf, fp, r, c, k.x), grad_y(sf, fp, r, c, k.y));
    }

    const int cx = threadIdx.x & (kTW - 1);
    const int r0 = (threadIdx.x / kTW) * kStrip;
    __half2 S[kStrip];
    u64 A[kStrip], Z[kStrip];
    float sxs[kStrip], sys[kStrip];
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        sxs[j] = grad_x(sf, fp, R + r0 + j, R + cx, k.x);   // FP32 centre values of the input
        sys[j] = grad_y(sf, fp, R + r0 + j, R + cx, k.y);
        A[j] = Z[j] = 0ull;
    }
    if constexpr (JOINT) {   // the guidance image's gradients, through the same f buffer
        __syncthreads();
        load_f_tile(guide, H, W, x0, y0, R, th, sf);
        __syncthreads();
        for (int i = threadIdx.x; i < gr * gp; i += blockDim.x) {
            const int r = i / gp, c = i - r * gp;
            hg[i] = __floats2half2_rn(grad_x(sf, fp, r, c, k.x), grad_y(sf, fp, r, c, k.y));
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kStrip; ++j) S[j] = hg[(R + r0 + j) * gp + R + cx];
    // AD[d] = (a, a), a = -(d - R)^2 cs: the dy part of the spatial log2-weight of both lanes
    __half2 AD[2 * R + 1];
#pragma unroll
    for (int d = 0; d <= 2 * R; ++d) {
        AD[d] = __float2half2_rn(-float((d - R) * (d - R)) * cs);
        asm volatile("" : "+r"(*reinterpret_cast<unsigned*>(&AD[d])));
    }
    const __half2 hz = __float2half2_rn(0.f);

#pragma unroll 1
    for (int dx = -R; dx <= R; ++dx) {
        if (!BLFLS_DCHECK(R + cx + dx >= 0 && R + cx + dx < gp &&
                          (r0 + kStrip + 2 * R - 1) * gp + R + cx + dx < gr * gp, kDcTileWindow))
            continue;
        const float gdx = ex2_approx(-float(dx * dx) * cs);
        const u64 GD = pk(gdx, gdx);
        __half2 P[kStrip], Q[kStrip];    // this column's sums of w t and w
#pragma unroll
        for (int j = 0; j < kStrip; ++j) P[j] = Q[j] = hz;
        const __half2* col = g + r0 * gp + R + cx + dx;
        const __half2* rcol = hg + r0 * gp + R + cx + dx;
#pragma unroll
        for (int i = 0; i < kStrip + 2 * R; ++i) {
            const __half2 T = col[i * gp];
            const __half2 TR = JOINT ? rcol[i * gp] : T;   // the value the range weight compares
#pragma unroll
            for (int j = 0; j < kStrip; ++j) {
                const int d = i - j;  // dy + R
                if (d < 0 || d > 2 * R) continue;
                __half2 Wt;
                if (RANGE) {
                    const __half2 D = __hsub2(TR, S[j]);
                    Wt = ex2_h2(__hfma2(__hneg2(D), D, AD[d]));
                } else {
                    Wt = ex2_h2(AD[d]);
                }
                P[j] = __hfma2(Wt, T, P[j]);
                Q[j] = __hadd2(Q[j], Wt);
            }
        }
#pragma unroll
        for (int j = 0; j < kStrip; ++j) {
            const float2 pf = __half22float2(P[j]), qf = __half22float2(Q[j]);
            A[j] = fma2(GD, pk(pf.x, pf.y), A[j]);
            Z[j] = fma2(GD, pk(qf.x, qf.y), Z[j]);
        }
    }
    float ax[kStrip], zx[kStrip], ay[kStrip], zy[kStrip];
#pragma unroll
    for (int j = 0; j < kStrip; ++j) {
        upk(A[j], ax[j], ay[j]);
        upk(Z[j], zx[j], zy[j]);
    }
    store_strip(ex, ey, H, W, x0 + cx, y0 + r0, ax, zx, sxs, ay, zy, sys, k);
}

// JOINT: the range weights compare the gradients of `guide` (the joint filter of Section III-D);
// the values averaged are still the gradients of f.
template <int R, bool RANGE, int PREC, bool JOINT = false>
__device__ __forceinline__ void blf_tile(const float* f, const float* guide, float* ex, float* ey,
                                         int H, int W, int x0, int y0, int th, const Kap k,
                                         float cs, unsigned char* smem)
{
    if constexpr (PREC == 1) tile_f16<R, RANGE, JOINT>(f, guide, ex, ey, H, W, x0, y0, th, k, cs, smem);
    else if constexpr (PREC == 2) tile_bf16<R, RANGE, JOINT>(f, guide, ex, ey, H, W, x0, y0, th, k, cs, smem);
    else tile_f32<R, RANGE, JOINT>(f, guide, ex, ey, H, W, x0, y0, th, k, cs, smem);
}

// The range constants of channel z: from the device when kdev is set, else the launch's.
__device__ __forceinline__ Kap kap_of(const Kap k, const float4* __restrict__ kdev, int z)
{
    if (!kdev) return k;
    const float4 v = kdev[z];
    return Kap{v.x, v.y, v.z, v.w};
}

// One CTA per 32 x th tile (4 th threads); blockIdx.z selects the channel.  The FP32 and BF16W
// forms are held to 64 registers so that four 256-thread CTAs fit on an SM; FP16W to 128 (two).
template <int R, bool RANGE, int PREC>
__global__ void __launch_bounds__(kMaxThreads, PREC == 1 ? 2 : 4) k1_blf(const float* __restrict__ img,
                                                      float* __restrict__ ex,
                                                      float* __restrict__ ey, int H, int W,
                                                      int th, const Kap k, float cs,
                                                      const float4* __restrict__ kdev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t plane = (size_t)H * W;
    blf_tile<R, RANGE, PREC>(img + blockIdx.z * plane, nullptr, ex + blockIdx.z * plane,
                             ey + blockIdx.z * plane, H, W, blockIdx.x * kTW, blockIdx.y * th,
                             th, kap_of(k, kdev, blockIdx.z), cs, smem);
}

// Joint form: as k1_blf with the range kernel on, guided by channel z of `guide` (channel
// stride gstride floats; 0 shares one guidance channel among all channels).
template <int R, int PREC>
__global__ void __launch_bounds__(kMaxThreads) k1_blf_joint(const float* __restrict__ img,
                                                            const float* __restrict__ guide,
                                                            size_t gstride,
                                                            float* __restrict__ ex,
                                                            float* __restrict__ ey, int H, int W,
                                                            int th, const Kap k, float cs)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t plane = (size_t)H * W;
    blf_tile<R, true, PREC, true>(img + blockIdx.z * plane, guide + blockIdx.z * gstride,
                                  ex + blockIdx.z * plane, ey + blockIdx.z * plane, H, W,
                                  blockIdx.x * kTW, blockIdx.y * th, th, k, cs, smem);
}

// Batched form: a persistent grid walks every tile of every channel of the jobs of one
// (radius, range kernel, precision) group.  grp[g] = (job index, first item of that job).
template <int R, bool RANGE, int PREC>
__global__ void __launch_bounds__(kMaxThreads) k1_blf_batch(const BatchJob* __restrict__ jobs,
                                                         const int2* __restrict__ grp, int ngrp,
                                                         int total)
{
    extern __shared__ __align__(16) unsigned char smem[];
    int g = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        while (g + 1 < ngrp && __ldg(&grp[g + 1].y) <= item) ++g;
        const BatchJob& J = jobs[__ldg(&grp[g].x)];
        const int local = item - __ldg(&grp[g].y);
        const int per_plane = J.tiles_x * J.tiles_y;
        const int c = local / per_plane, rem = local - c * per_plane;
        const int ty = rem / J.tiles_x, tx = rem - ty * J.tiles_x;
        const size_t plane = (size_t)J.H * J.W;
        __syncthreads();   // the previous tile's readers are done with shared memory
        blf_tile<R, RANGE, PREC>(J.src + c * plane, nullptr, J.ex + c * plane, J.ey + c * plane,
                                 J.H, J.W, tx * kTW, ty * J.tile_h, J.tile_h,
                                 Kap{J.kappa, J.kappa, J.inv_kappa, J.inv_kappa}, J.cs, smem);
    }
}

}  // namespace

using TiledFn = void (*)(const float*, float*, float*, int, int, int, const Kap, float,
                         const float4*);
using BatchFn = void (*)(const BatchJob*, const int2*, int, int);
using JointFn = void (*)(const float*, const float*, size_t, float*, float*, int, int, int,
                         const Kap, float);

// Kernel pointers of one precision (defined in blf_f32.cu, blf_f16.cu, blf_bf16.cu).
TiledFn pick_tiled_prec(int prec, int r, bool range);
BatchFn pick_batch_prec(int prec, int r, bool range);
JointFn pick_joint_prec(int prec, int r);
size_t blf_templ_smem_bytes(int R, int prec, int th, bool joint = false);

}  // namespace blfls
