// Fourier solve of Eq. 8 in residual form (the step after the bilateral filter):
//
//   u = f + F^-1[ lam * F(r) / (1 + lam (|F d_x|^2 + |F d_y|^2)) ],
//   r = D_x^T e_x + D_y^T e_y,   e_* = f_BLF(g_*) - g_*,
//
// which is Eq. 8 rewritten by linearity (D_* f = g_*): subtracting (1 + lam L) F(f) from the
// numerator of Eq. 8 leaves lam * sum conj(F d_*) F(e_*), i.e. lam F(D^T e).  |F d_x|^2 =
// 4 sin^2(pi k_x / W) and |F d_y|^2 = 4 sin^2(pi k_y / H) are the eigenvalues of the periodic
// Laplacian (tables computed in FP64 on the host, stored FP32, in each plan's `lap`).
//
// K2 (rows, forward): builds r for two rows at once from e_x, e_y (backward differences with
//    wrap), packs them as one complex row z = r_a + i r_b, FFTs it and splits the result into the
//    two half spectra (W/2+1 bins each).
// K3 (columns): FFT down each column of the half spectrum, multiply by
//    lam / (H W (1 + lam (sx + sy))), inverse FFT down the column.
// K4 (rows, inverse): rebuilds the full row spectrum of two rows from their halves (Hermitian
//    symmetry), inverse FFT, and writes u = f + result (real part row a, imaginary part row b).
//
// Each phase is written once as a per-item compute function (a row pair, or a block of columns)
// and driven by one of three persistent grids: the staged single-image drivers (each CTA walks a
// contiguous band of items and copies the next item into shared memory with cp.async while it
// transforms the current one, double-buffered); the plain single-image drivers (loads then
// transform, twiddles staged in shared memory once per CTA), used when the staged buffers do not
// fit; and the batched drivers over the items of many jobs.  All run the same arithmetic, so a
// job's result does not depend on the driver or the batch it ran in.
#include "fft_device.cuh"

namespace blfls {

namespace {

// Shared-memory budget of one solve CTA; twiddles share it with the data when they fit.
constexpr size_t kSmemCap = 220 * 1024;
// Column block of the staged column drivers when no tuned value is given.
constexpr int kDefaultColBlock = 4;

__device__ __forceinline__ const float2* stage_twiddles(float2* tw_smem, const FftPlanDev& p,
                                                        bool in_smem)
{
    if (!in_smem) return p.tw;
    for (int i = threadIdx.x; i < p.L; i += blockDim.x) tw_smem[i] = __ldg(p.tw + i);
    __syncthreads();
    return tw_smem;
}

// K2, first half: r = D_x^T e_x + D_y^T e_y for rows y0 and y1 (given in global or shared memory)
// packed as z = r0 + i r1 into `data`.  Ends synchronised, so the rows may be overwritten after.
__device__ __forceinline__ void k2_build(const float* ex0, const float* ex1, const float* eym,
                                         const float* ey0, const float* ey1, bool has1, int W,
                                         const FftPlanDev& rp, float2* data)
{
    if ((W & 3) == 0 && ((reinterpret_cast<uintptr_t>(ex0) | reinterpret_cast<uintptr_t>(ex1) |
                          reinterpret_cast<uintptr_t>(eym) | reinterpret_cast<uintptr_t>(ey0) |
                          reinterpret_cast<uintptr_t>(ey1)) & 15) == 0) {
        // four pixels per thread from 16-byte loads; the padded positions of x..x+3 are
        // contiguous when the padding block S is a multiple of 4 (or there is no padding)
        const bool contig = (rp.pad_span & 3) == 0;
        for (int q = threadIdx.x; q < (W >> 2); q += blockDim.x) {
            const int x = q << 2;
            const float4 a = *reinterpret_cast<const float4*>(ex0 + x);
            const float4 m = *reinterpret_cast<const float4*>(eym + x);
            const float4 e0 = *reinterpret_cast<const float4*>(ey0 + x);
            const float l0 = ex0[x == 0 ? W - 1 : x - 1];
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f), e1 = b;
            float l1 = 0.f;
            if (has1) {
                b = *reinterpret_cast<const float4*>(ex1 + x);
                e1 = *reinterpret_cast<const float4*>(ey1 + x);
                l1 = ex1[x == 0 ? W - 1 : x - 1];
            }
            // (D_x^T e_x)[x] = e_x[x-1] - e_x[x];  (D_y^T e_y)[y] = e_y[y-1] - e_y[y]
            const float2 z0 = make_float2((l0 - a.x) + (m.x - e0.x), has1 ? (l1 - b.x) + (e0.x - e1.x) : 0.f);
            const float2 z1 = make_float2((a.x - a.y) + (m.y - e0.y), has1 ? (b.x - b.y) + (e0.y - e1.y) : 0.f);
            const float2 z2 = make_float2((a.y - a.z) + (m.z - e0.z), has1 ? (b.y - b.z) + (e0.z - e1.z) : 0.f);
            const float2 z3 = make_float2((a.z - a.w) + (m.w - e0.w), has1 ? (b.z - b.w) + (e0.w - e1.w) : 0.f);
            if (contig) {
                float2* d = data + row_pos(rp, x);
                d[0] = z0;
                d[1] = z1;
                d[2] = z2;
                d[3] = z3;
            } else {
                data[row_pos(rp, x)] = z0;
                data[row_pos(rp, x + 1)] = z1;
                data[row_pos(rp, x + 2)] = z2;
                data[row_pos(rp, x + 3)] = z3;
            }
        }
        __syncthreads();
        return;
    }
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int xm = (x == 0) ? W - 1 : x - 1;
        // (D_x^T e_x)[y][x] = e_x[y][x-1] - e_x[y][x];  (D_y^T e_y)[y][x] = e_y[y-1][x] - e_y[y][x]
        const float r0 = (ex0[xm] - ex0[x]) + (eym[x] - ey0[x]);
        float r1 = 0.f;
        if (has1) r1 = (ex1[xm] - ex1[x]) + (ey0[x] - ey1[x]);
        data[row_pos(rp, x)] = make_float2(r0, r1);
    }
    __syncthreads();
}

// K2, second half: forward FFT of z, split into the two half spectra s0, s1 (W/2+1 bins each).
// P: a compile-time plan matching rp, or void.
template <class P = void>
__device__ __forceinline__ void k2_transform(bool has1, int W, float2* s0, float2* s1,
                                             const FftPlanDev& rp, const float2* tw, float2* data)
{
    const int Wh = W / 2 + 1;
    fft_forward_p<P, 0, true>(data, 0, rp, tw);
#pragma unroll 4
    for (int k = threadIdx.x; k < Wh; k += blockDim.x) {
        const int kn = (k == 0) ? 0 : W - k;
        const float2 zk = data[row_pos(rp, __ldg(rp.perm + k))];
        const float2 zn = data[row_pos(rp, __ldg(rp.perm + kn))];
        // A = (Z_k + conj Z_{W-k}) / 2,  B = (Z_k - conj Z_{W-k}) / (2i)
        s0[k] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        if (has1) s1[k] = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    }
    __syncthreads();
}

// K2 on one row pair: rows y0 and y1 packed as z = r0 + i r1, forward FFT, half spectra.
__device__ __forceinline__ void k2_rows(const float* ex0, const float* ex1, const float* eym,
                                        const float* ey0, const float* ey1, bool has1, int W,
                                        float2* s0, float2* s1, const FftPlanDev& rp,
                                        const float2* tw, float2* data)
{
    k2_build(ex0, ex1, eym, ey0, ey1, has1, W, rp, data);
    k2_transform(has1, W, s0, s1, rp, tw, data);
}

// K2: row pair `pair` (rows 2 pair, 2 pair + 1) of one channel, read from global memory.
__device__ __forceinline__ void k2_item(const float* __restrict__ ex, const float* __restrict__ ey,
                                        float2* __restrict__ spec, int H, int W, int pair,
                                        const FftPlanDev& rp, const float2* tw, float2* data)
{
    const int Wh = W / 2 + 1;
    const int y0 = 2 * pair, y1 = y0 + 1;
    const bool has1 = y1 < H;
    const int ym = (y0 == 0) ? H - 1 : y0 - 1;
    const int yb = has1 ? y1 : y0;
    k2_rows(ex + (size_t)y0 * W, ex + (size_t)yb * W, ey + (size_t)ym * W, ey + (size_t)y0 * W,
            ey + (size_t)yb * W, has1, W, spec + (size_t)y0 * Wh, spec + (size_t)yb * Wh, rp, tw,
            data);
}

// ---- column solve by recursion (column lengths without a mixed-radix plan) ----------------------
// Along a column of fixed x frequency kx, Eq. 8's column DFT, divide by 1 + lam (sx + sy) and
// inverse DFT is the solve of the cyclic tridiagonal system
//     (1 + lam sx) Z - lam (Z[n+1] - 2 Z[n] + Z[n-1]) = lam R        (periodic in n),
// because the DFT diagonalises the periodic second difference with eigenvalues sy.  The operator
// factors as (lam / r) (1 - r S)(1 - r S^-1), S the cyclic shift and r in [0, 1) the smaller root
// of lam r^2 - d r + lam = 0, d = 1 + lam sx + 2 lam, so Z = r (1 - r S^-1)^-1 (1 - r S)^-1 R
// (times the H / (HW) the unnormalised transforms would apply): a causal and an anticausal
// first-order recursion, each cyclic.  Every column is split into segments of kRecSeg rows: each
// segment runs its recursion from zero, the segments' carries are chained per column (the cyclic
// start value from the geometric sum over the whole column), and each segment adds its carry's
// decay.  The segments depend only on H, so a column's result does not depend on how columns
// are grouped.  The recursion amplifies rounding by about 1 / (1 - r), largest at kx = 0; it is
// used while lam <= kRecLamMax (1 / (1 - r) below about 100), Bluestein column transforms above.

// r, r^kRecSeg, r^(rows of the last segment) and 1 / (1 - r^H) of a column
struct RecCoef {
    float r, rseg, rlast, icyc;
};
__device__ __forceinline__ RecCoef rec_coef(float lam, float sxv, int H)
{
    static_assert(kRecSeg == 32, "r^kRecSeg by five squarings");
    const float a = fmaf(lam, sxv, 1.0f);                       // 1 + lam sx
    const float d = fmaf(2.0f, lam, a);                         // 1 + lam sx + 2 lam
    // r = (d - sqrt(d^2 - 4 lam^2)) / (2 lam), written without the cancellation
    const float r = __fdiv_rn(2.0f * lam, d + sqrtf(a * fmaf(4.0f, lam, a)));
    float rseg = r;
#pragma unroll
    for (int k = 0; k < 5; ++k) rseg *= rseg;
    const int nseg = (H + kRecSeg - 1) / kRecSeg;
    const int last = H - (nseg - 1) * kRecSeg;
    float rlast = 1.0f;
    for (int k = 0; k < last; ++k) rlast *= r;
    float rh = rlast;
    for (int k = 1; k < nseg; ++k) rh *= rseg;
    return RecCoef{r, rseg, rlast, __fdiv_rn(1.0f, 1.0f - rh)};
}

// Cyclic carries of one column from its segments' values from zero: forward (causal, carry into
// segment s from the left) or backward (anticausal, from the right).
template <bool BACKWARD>
__device__ __forceinline__ void rec_carries(const RecCoef& k, int nseg, const float2* part,
                                            float2* carry, int stride)
{
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < nseg; ++q) {
        const int sg = BACKWARD ? nseg - 1 - q : q;
        const float rl = sg == nseg - 1 ? k.rlast : k.rseg;
        const float2 p = part[sg * stride];
        acc = make_float2(fmaf(rl, acc.x, p.x), fmaf(rl, acc.y, p.y));
    }
    float2 cin = make_float2(acc.x * k.icyc, acc.y * k.icyc);
    for (int q = 0; q < nseg; ++q) {
        const int sg = BACKWARD ? nseg - 1 - q : q;
        carry[sg * stride] = cin;
        const float rl = sg == nseg - 1 ? k.rlast : k.rseg;
        const float2 p = part[sg * stride];
        cin = make_float2(fmaf(rl, cin.x, p.x), fmaf(rl, cin.y, p.y));
    }
}

// Shared memory of the recursion solve of one 32-column block: the segments' values and carries.
__host__ __device__ __forceinline__ size_t rec_smem(int H)
{
    return sizeof(float2) * 2 * 32 * (size_t)((H + kRecSeg - 1) / kRecSeg);
}

// Columns [32 blk, 32 blk + 32) of one channel's half spectrum, solved in place by the recursion:
// lanes on adjacent columns (each row's 32 values are one 256-byte run), warps on segments.  The
// values pass through global memory (L2) between the phases; `sm` holds rec_smem(H) bytes.
__device__ __forceinline__ void k3_rec_item(float2* __restrict__ spec, int H, int W, int blk,
                                            const float* __restrict__ sx, float lam, float scale,
                                            float2* sm)
{
    const int Wh = W / 2 + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int kx = blk * 32 + lane;
    const bool live_col = kx < Wh;
    const int nseg = (H + kRecSeg - 1) / kRecSeg;
    float2* part = sm;                             // [segment][lane]
    float2* carry = sm + (size_t)nseg * 32;        // [segment][lane]
    const RecCoef k = rec_coef(lam, __ldg(sx + min(kx, Wh - 1)), H);
    const float r = k.r;
    float2* col = spec + kx;
    // a live lane's column lies inside the half spectrum (rows n < H of Wh columns)
    const bool live = live_col && BLFLS_DCHECK(kx >= 0 && blk >= 0 && H >= 1, kDcSolveGlobal);
    // causal pass from zero in every segment: w[n] = R[n] + r w[n-1]
    for (int sg = warp; sg < nseg; sg += nw) {
        const int n0 = sg * kRecSeg;
        float2 v[kRecSeg];
#pragma unroll
        for (int t = 0; t < kRecSeg; ++t)
            v[t] = (live && n0 + t < H) ? col[(size_t)(n0 + t) * Wh] : make_float2(0.f, 0.f);
        float2 w = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < kRecSeg; ++t)
            if (n0 + t < H) w = make_float2(fmaf(r, w.x, v[t].x), fmaf(r, w.y, v[t].y));
        part[sg * 32 + lane] = w;
    }
    __syncthreads();
    if (warp == 0) rec_carries<false>(k, nseg, part + lane, carry + lane, 32);
    __syncthreads();
    // complete the causal pass; anticausal pass from zero: z[n] = w[n] + r z[n+1], stored
    for (int sg = warp; sg < nseg; sg += nw) {
        const int n0 = sg * kRecSeg;
        float2 v[kRecSeg];
#pragma unroll
        for (int t = 0; t < kRecSeg; ++t)
            v[t] = (live && n0 + t < H) ? col[(size_t)(n0 + t) * Wh] : make_float2(0.f, 0.f);
        const float2 cin = carry[sg * 32 + lane];
        float2 p = make_float2(r * cin.x, r * cin.y);
        float2 w = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < kRecSeg; ++t)
            if (n0 + t < H) {
                w = make_float2(fmaf(r, w.x, v[t].x), fmaf(r, w.y, v[t].y));
                v[t] = make_float2(w.x + p.x, w.y + p.y);
                p = make_float2(r * p.x, r * p.y);
            }
        float2 z = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = kRecSeg - 1; t >= 0; --t)
            if (n0 + t < H) {
                z = make_float2(fmaf(r, z.x, v[t].x), fmaf(r, z.y, v[t].y));
                if (live) col[(size_t)(n0 + t) * Wh] = z;
            }
        part[sg * 32 + lane] = z;
    }
    __syncthreads();
    if (warp == 0) rec_carries<true>(k, nseg, part + lane, carry + lane, 32);
    __syncthreads();
    // complete the anticausal pass: Z = r z times H / (H W)
    const float m = r * (scale * (float)H);
    for (int sg = warp; sg < nseg; sg += nw) {
        const int n0 = sg * kRecSeg;
        const float2 cin = carry[sg * 32 + lane];
        float2 p = make_float2(r * cin.x, r * cin.y);
#pragma unroll
        for (int t = kRecSeg - 1; t >= 0; --t)
            if (n0 + t < H) {
                if (live) {
                    const float2 z = col[(size_t)(n0 + t) * Wh];
                    col[(size_t)(n0 + t) * Wh] = make_float2((z.x + p.x) * m, (z.y + p.y) * m);
                }
                p = make_float2(r * p.x, r * p.y);
            }
    }
    __syncthreads();
}

// K3 by recursion for one channel: one 32-column block per CTA (grid-stride).
__global__ void __launch_bounds__(512) k3_cols_rec(float2* __restrict__ spec, int H, int W,
                                                   const float* __restrict__ sx, float lam,
                                                   float scale)
{
    extern __shared__ float2 smem[];
    const int nblk = (W / 2 + 1 + 31) / 32;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x)
        k3_rec_item(spec, H, W, blk, sx, lam, scale, smem);
}

// K3 on one column block already in `data` (rows n < H; the caller synchronised): forward FFT
// down the columns, spectral divide (Eq. 8 denominator, F(1) = 1, with lam and the 1/(HW) of the
// inverse), inverse FFT.  Ends synchronised.
// `syp`, when given, holds sy[iperm[p]] for every work position p (staged once per CTA).
// P: a compile-time plan matching cp, or void.
template <int LGC = -1, class P = void>
__device__ __forceinline__ void k3_solve_block(float2* data, int H, int W, int kx0, int lgc,
                                               const FftPlanDev& cp, const float* __restrict__ sx,
                                               const float* __restrict__ sy, float lam,
                                               float scale, const float2* tw,
                                               const float* syp = nullptr)
{
    const int CB = 1 << lgc;
    const int Wh = W / 2 + 1;
    if (LGC >= 0) lgc = LGC;
    fft_forward_p<P, LGC, false>(data, lgc, cp, tw);
    const int nfreq = cp.bluestein ? H : cp.L;
    // every launch uses a multiple of 32 threads, so a thread's column i & (CB - 1) is the same
    // in every iteration and its x eigenvalue is read once
    const float sxv = __ldg(sx + min(kx0 + (int)(threadIdx.x & (CB - 1)), Wh - 1));
    for (int i = threadIdx.x; i < (nfreq << lgc); i += blockDim.x) {
        const int p = i >> lgc;
        const float syv = syp ? syp[p] : __ldg(sy + __ldg(cp.iperm + p));
        const float den = fmaf(lam, sxv + syv, 1.0f);
        const float m = __fdividef(scale, den) * lam;
        const float2 v = data[i];
        data[i] = make_float2(v.x * m, v.y * m);
    }
    __syncthreads();
    fft_inverse_p<P, LGC, false>(data, lgc, cp, tw);
}

// K3: columns [blk * 2^lgc, (blk + 1) * 2^lgc) of the half spectrum of one channel.
__device__ __forceinline__ void k3_item(float2* __restrict__ spec, int H, int W, int blk,
                                        const FftPlanDev& cp, const float* __restrict__ sx,
                                        const float* __restrict__ sy, float lam, float scale,
                                        int lgc, const float2* tw, float2* data)
{
    const int CB = 1 << lgc;
    const int Wh = W / 2 + 1;
    const int kx0 = blk * CB;
    for (int i = threadIdx.x; i < (H << lgc); i += blockDim.x) {
        const int n = i >> lgc, c = i & (CB - 1);
        const int kx = kx0 + c;
        data[i] = (kx < Wh && BLFLS_DCHECK(n < H && kx >= 0, kDcSolveGlobal))
                      ? spec[(size_t)n * Wh + kx] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    k3_solve_block(data, H, W, kx0, lgc, cp, sx, sy, lam, scale, tw);
    for (int i = threadIdx.x; i < (H << lgc); i += blockDim.x) {
        const int n = i >> lgc, c = i & (CB - 1);
        const int kx = kx0 + c;
        if (kx < Wh) spec[(size_t)n * Wh + kx] = data[i];
    }
    __syncthreads();
}

// K4, first half: rebuild Z = A + i B over all W bins of a row pair from its half spectra
// (global or shared memory), in the digit-reversed order the inverse FFT reads.  Ends synchronised.
__device__ __forceinline__ void k4_rebuild(const float2* s0, const float2* s1, bool has1, int W,
                                           const FftPlanDev& rp, float2* data)
{
#pragma unroll 4
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        const bool upper = k > W / 2;
        const int kk = upper ? W - k : k;
        float2 a = s0[kk];
        float2 b = has1 ? s1[kk] : make_float2(0.f, 0.f);
        if (upper) { a.y = -a.y; b.y = -b.y; }
        if (k == 0 || 2 * k == W) { a.y = 0.f; b.y = 0.f; }  // real bins of a real row
        // Z = A + i B
        data[row_pos(rp, __ldg(rp.perm + k))] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
}

// K4, last step (after the inverse FFT): u = f + result, real part row a, imaginary part row b.
__device__ __forceinline__ void k4_output(bool has1, const float* f0, const float* f1, float* o0,
                                          float* o1, int W, const FftPlanDev& rp,
                                          const float2* data)
{
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const float2 z = data[row_pos(rp, x)];
        o0[x] = f0[x] + z.x;
        if (has1) o1[x] = f1[x] + z.y;
    }
    __syncthreads();
}

// K4 on one row pair: rebuild, inverse FFT, u = f + result.
__device__ __forceinline__ void k4_rows(const float2* s0, const float2* s1, bool has1,
                                        const float* f0, const float* f1, float* o0, float* o1,
                                        int W, const FftPlanDev& rp, const float2* tw,
                                        float2* data)
{
    k4_rebuild(s0, s1, has1, W, rp, data);
    fft_inverse<0, true>(data, 0, rp, tw);
    k4_output(has1, f0, f1, o0, o1, W, rp, data);
}

// K4: row pair `pair` of one channel, read from global memory.
__device__ __forceinline__ void k4_item(const float2* __restrict__ spec, const float* f, float* out,
                                        int H, int W, int pair, const FftPlanDev& rp,
                                        const float2* tw, float2* data)
{
    const int Wh = W / 2 + 1;
    const int y0 = 2 * pair, y1 = y0 + 1;
    const bool has1 = y1 < H;
    const int yb = has1 ? y1 : y0;
    k4_rows(spec + (size_t)y0 * Wh, spec + (size_t)yb * Wh, has1, f + (size_t)y0 * W,
            f + (size_t)yb * W, out + (size_t)y0 * W, out + (size_t)yb * W, W, rp, tw, data);
}

// ---- asynchronous staging (cp.async) --------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async4(void* s, const void* g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async16(void* s, const void* g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage n floats (a row) into shared memory: 16-byte copies when src and dst are 16-byte aligned
// and n % 4 == 0 (`vec`), else 4-byte copies.
__device__ __forceinline__ void stage_floats(float* dst, const float* src, int n, bool vec)
{
    if (vec) {
        for (int i = threadIdx.x; i < (n >> 2); i += blockDim.x) cp_async16(dst + 4 * i, src + 4 * i);
    } else {
        for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async4(dst + i, src + i);
    }
}
// Stage n complex values: 16-byte copies (which bypass L1) when src and dst share their
// alignment modulo 16 bytes, with at most one 8-byte copy at either end; else 8-byte copies.
__device__ __forceinline__ void stage_complex(float2* dst, const float2* src, int n)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(src), d = reinterpret_cast<uintptr_t>(dst);
    if (((a ^ d) & 15) != 0) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) cp_async8(dst + i, src + i);
        return;
    }
    const int lead = (a & 15) ? 1 : 0;
    const int npairs = (n - lead) >> 1;
    if (threadIdx.x == 0) {
        if (lead && n > 0) cp_async8(dst, src);
        if (((n - lead) & 1) && n > lead) cp_async8(dst + n - 1, src + n - 1);
    }
    for (int i = threadIdx.x; i < npairs; i += blockDim.x)
        cp_async16(dst + lead + 2 * i, src + lead + 2 * i);
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Contiguous band of items [b0, b1) of a CTA when n items are split over gridDim.x CTAs.
__device__ __forceinline__ void band(int n, int& b0, int& b1)
{
    const int per = (n + gridDim.x - 1) / gridDim.x;
    b0 = min(n, blockIdx.x * per);
    b1 = min(n, b0 + per);
}

// ---- single image --------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k2_rows_forward(
    const float* __restrict__ ex, const float* __restrict__ ey, float2* __restrict__ spec,
    int H, int W, FftPlanDev rp, int tw_in_smem)
{
    extern __shared__ float2 smem[];
    const float2* tw = stage_twiddles(smem + row_buf_elems(rp), rp, tw_in_smem);
    const int npairs = (H + 1) / 2;
    for (int pair = blockIdx.x; pair < npairs; pair += gridDim.x)
        k2_item(ex, ey, spec, H, W, pair, rp, tw, smem);
}

__global__ void __launch_bounds__(512) k3_cols_solve(
    float2* __restrict__ spec, int H, int W, FftPlanDev cp, const float* __restrict__ sx,
    const float* __restrict__ sy, float lam, float scale, int lgc, int tw_in_smem)
{
    extern __shared__ float2 smem[];
    const float2* tw = stage_twiddles(smem + ((size_t)cp.L << lgc), cp, tw_in_smem);
    const int nblk = (W / 2 + 1 + (1 << lgc) - 1) >> lgc;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x)
        k3_item(spec, H, W, blk, cp, sx, sy, lam, scale, lgc, tw, smem);
}

__global__ void __launch_bounds__(512) k4_rows_inverse(
    const float2* __restrict__ spec, const float* f, float* out, int H, int W, FftPlanDev rp,
    int tw_in_smem)
{
    extern __shared__ float2 smem[];
    const float2* tw = stage_twiddles(smem + row_buf_elems(rp), rp, tw_in_smem);
    const int npairs = (H + 1) / 2;
    for (int pair = blockIdx.x; pair < npairs; pair += gridDim.x)
        k4_item(spec, f, out, H, W, pair, rp, tw, smem);
}

// ---- single image, staged: each CTA walks a contiguous band of items.  Its input rows sit in
// one staging buffer, which is refilled with cp.async for the next item as soon as the current
// one has been read out of it, so the copy runs under the FFT.  256 threads (a 3840-point row
// has 240 radix-16 or 256 radix-15 butterflies per stage) and two CTAs per SM. ------------------

constexpr int kStagedThreads = 256;

__host__ __device__ __forceinline__ size_t row_floats(int W) { return (size_t)((W + 3) & ~3); }
// K2: [5][Wp] floats (e_x rows y0, y1 and e_y rows y0-1, y0, y1), then the FFT buffer.
__host__ __device__ __forceinline__ size_t k2s_stage_bytes(int W) { return sizeof(float) * 5 * row_floats(W); }
__host__ __device__ __forceinline__ size_t k2s_smem(int W, const FftPlanDev& rp)
{
    return k2s_stage_bytes(W) + sizeof(float2) * (size_t)row_buf_elems(rp);
}
// K4: [2][Wh] half spectra, [2][Wp] floats of f, then the FFT buffer.
__host__ __device__ __forceinline__ size_t k4s_spec_bytes(int W) { return align16(sizeof(float2) * 2 * (size_t)(W / 2 + 1)); }
__host__ __device__ __forceinline__ size_t k4s_smem(int W, const FftPlanDev& rp)
{
    return k4s_spec_bytes(W) + sizeof(float) * 2 * row_floats(W) + sizeof(float2) * (size_t)row_buf_elems(rp);
}
// K3: two column blocks (double-buffered; the FFT runs in place in one of them), the plan's
// twiddle table, and the column eigenvalues in work-position order (sy[iperm[p]]).
__host__ __device__ __forceinline__ size_t k3s_smem(int L, int lgc)
{
    return 2 * (sizeof(float2) * (size_t)L << lgc) + sizeof(float2) * (size_t)L +
           sizeof(float) * (size_t)L;
}

template <class P>
__global__ void __launch_bounds__(kStagedThreads, 2) k2_rows_staged(const float* __restrict__ ex,
                                                                    const float* __restrict__ ey,
                                                                    float2* __restrict__ spec,
                                                                    int H, int W, FftPlanDev rp,
                                                                    int vec)
{
    extern __shared__ __align__(16) unsigned char staged_smem[];
    float* st = reinterpret_cast<float*>(staged_smem);
    const size_t Wp = row_floats(W);
    float2* data = reinterpret_cast<float2*>(staged_smem + k2s_stage_bytes(W));
    const int Wh = W / 2 + 1;
    const int npairs = (H + 1) / 2;
    int p0, p1;
    band(npairs, p0, p1);
    if (p0 >= p1) return;
    auto issue = [&](int p) {
        const int y0 = 2 * p, y1 = y0 + 1;
        const int ym = (y0 == 0) ? H - 1 : y0 - 1;
        stage_floats(st, ex + (size_t)y0 * W, W, vec);
        stage_floats(st + 2 * Wp, ey + (size_t)ym * W, W, vec);
        stage_floats(st + 3 * Wp, ey + (size_t)y0 * W, W, vec);
        if (y1 < H) {
            stage_floats(st + Wp, ex + (size_t)y1 * W, W, vec);
            stage_floats(st + 4 * Wp, ey + (size_t)y1 * W, W, vec);
        }
        cp_commit();
    };
    issue(p0);
    for (int p = p0; p < p1; ++p) {
        cp_wait<0>();
        __syncthreads();
        const int y0 = 2 * p, y1 = y0 + 1;
        const bool has1 = y1 < H;
        k2_build(st, st + Wp, st + 2 * Wp, st + 3 * Wp, st + 4 * Wp, has1, W, rp, data);
        if (p + 1 < p1) issue(p + 1);   // the rows of pair p have been read out
        k2_transform<P>(has1, W, spec + (size_t)y0 * Wh, spec + (size_t)(has1 ? y1 : y0) * Wh,
                        rp, rp.tw, data);
    }
}

template <class P>
__global__ void __launch_bounds__(kStagedThreads, 2) k4_rows_staged(const float2* __restrict__ spec,
                                                                    const float* f, float* out,
                                                                    int H, int W, FftPlanDev rp,
                                                                    int vec)
{
    extern __shared__ __align__(16) unsigned char staged_smem[];
    const int Wh = W / 2 + 1;
    const size_t Wp = row_floats(W);
    float2* ss = reinterpret_cast<float2*>(staged_smem);
    float* sf = reinterpret_cast<float*>(staged_smem + k4s_spec_bytes(W));
    float2* data = reinterpret_cast<float2*>(staged_smem + k4s_spec_bytes(W) + sizeof(float) * 2 * Wp);
    const int npairs = (H + 1) / 2;
    int p0, p1;
    band(npairs, p0, p1);
    if (p0 >= p1) return;
    auto issue_spec = [&](int p) {
        const int y0 = 2 * p, y1 = y0 + 1;
        stage_complex(ss, spec + (size_t)y0 * Wh, Wh);
        if (y1 < H) stage_complex(ss + Wh, spec + (size_t)y1 * Wh, Wh);
        cp_commit();
    };
    auto issue_f = [&](int p) {
        const int y0 = 2 * p, y1 = y0 + 1;
        stage_floats(sf, f + (size_t)y0 * W, W, vec);
        if (y1 < H) stage_floats(sf + Wp, f + (size_t)y1 * W, W, vec);
        cp_commit();
    };
    // Copy groups complete in issue order: spectra(p), f(p), spectra(p+1), f(p+1), ...
    issue_spec(p0);
    issue_f(p0);
    for (int p = p0; p < p1; ++p) {
        cp_wait<1>();                 // spectra(p) landed; f(p) may still be in flight
        __syncthreads();
        const int y0 = 2 * p, y1 = y0 + 1;
        const bool has1 = y1 < H;
        k4_rebuild(ss, ss + Wh, has1, W, rp, data);
        const bool more = p + 1 < p1;
        if (more) issue_spec(p + 1);  // the spectra of pair p have been read out
        fft_inverse_p<P, 0, true>(data, 0, rp, rp.tw);
        if (more) cp_wait<1>(); else cp_wait<0>();   // f(p) landed
        __syncthreads();
        k4_output(has1, sf, sf + Wp, out + (size_t)y0 * W, out + (size_t)(has1 ? y1 : y0) * W, W,
                  rp, data);
        if (more) issue_f(p + 1);
    }
}

// Launched with any block size up to kColThreadsMax (chosen per plan, see col_threads).
constexpr int kColThreadsMax = 768;   // keeps 85 registers per thread available

template <int LGC, class P>
__global__ void __launch_bounds__(kColThreadsMax) k3_cols_staged(float2* __restrict__ spec, int H,
                                                                 int W, FftPlanDev cp,
                                                                 const float* __restrict__ sx,
                                                                 const float* __restrict__ sy,
                                                                 float lam, float scale)
{
    constexpr int lgc = LGC;
    extern __shared__ __align__(16) unsigned char staged_smem[];
    const int CB = 1 << lgc;
    const int Wh = W / 2 + 1;
    const size_t blk_elems = (size_t)cp.L << lgc;
    float2* bufs = reinterpret_cast<float2*>(staged_smem);
    float2* tws = bufs + 2 * blk_elems;
    float* syp = reinterpret_cast<float*>(tws + cp.L);
    const int nblk = (Wh + CB - 1) >> lgc;
    int b0, b1;
    band(nblk, b0, b1);
    if (b0 >= b1) return;
    auto issue = [&](int b, float2* buf) {
        const int kx0 = b * CB;
        for (int i = threadIdx.x; i < (H << lgc); i += blockDim.x) {
            const int n = i >> lgc, c = i & (CB - 1);
            const int kx = kx0 + c;
            if (kx < Wh) cp_async8(buf + i, spec + (size_t)n * Wh + kx);
            else buf[i] = make_float2(0.f, 0.f);
        }
    };
    issue(b0, bufs);
    cp_commit();
    for (int i = threadIdx.x; i < cp.L; i += blockDim.x) {
        tws[i] = __ldg(cp.tw + i);
        syp[i] = __ldg(sy + __ldg(cp.iperm + i) % H);   // positions >= H (Bluestein scratch) unused
    }
    for (int b = b0; b < b1; ++b) {
        float2* data = bufs + ((b - b0) & 1) * blk_elems;
        if (b + 1 < b1) {
            issue(b + 1, bufs + (((b - b0) & 1) ^ 1) * blk_elems);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const int kx0 = b * CB;
        k3_solve_block<LGC, P>(data, H, W, kx0, lgc, cp, sx, sy, lam, scale, tws, syp);
        for (int i = threadIdx.x; i < (H << lgc); i += blockDim.x) {
            const int n = i >> lgc, c = i & (CB - 1);
            const int kx = kx0 + c;
            if (kx < Wh) spec[(size_t)n * Wh + kx] = data[i];
        }
        __syncthreads();
    }
}

// ---- single image, compile-time plans, fused stage endpoints --------------------------------
// The same transforms as the staged drivers, operation for operation (bit-identical results),
// with the first and last stages moving their data between registers and global memory or the
// staging buffers directly, so shared memory sees only the exchanges between stages:
//   K2: each first-stage butterfly forms its inputs r = D_x^T e_x + D_y^T e_y from the staged rows
//       in registers (no build pass);
//   K3: the first stage reads the spectrum from global memory, the last forward stage, the
//       spectral divide and the first inverse stage run in registers (one butterfly, no exchange
//       between them), and the last inverse stage writes the spectrum back (no staging buffer,
//       so more CTAs fit on an SM);
//   K4: the first inverse stage gathers its inputs straight from the staged half spectra
//       (Hermitian rebuild in registers) and the last one writes u = f + result.

template <class P>
__global__ void __launch_bounds__(kStagedThreads, 2) k2_rows_fused(const float* __restrict__ ex,
                                                                   const float* __restrict__ ey,
                                                                   float2* __restrict__ spec,
                                                                   int H, int W, FftPlanDev rp,
                                                                   int vec)
{
    static_assert(P::nst >= 2, "fused drivers need two or more stages");
    constexpr int PADS = P::L / P::radix[0];
    constexpr int R0 = P::radix[0];
    constexpr unsigned M0 = P::span(0);
    using S0 = CtStageOf<P, 0, 1, PADS>;
    extern __shared__ __align__(16) unsigned char staged_smem[];
    float* st = reinterpret_cast<float*>(staged_smem);
    const size_t Wp = row_floats(W);
    float2* data = reinterpret_cast<float2*>(staged_smem + k2s_stage_bytes(W));
    const int Wh = W / 2 + 1;
    const int npairs = (H + 1) / 2;
    int p0, p1;
    band(npairs, p0, p1);
    if (p0 >= p1) return;
    // Staging slots: e_x rows y0, y1, e_y row y0, and two e_y slots that alternate: pair i of the
    // band (i = p - p0) stages its e_y row y1 in slot i mod 2, which is the row y0 - 1 the next
    // pair needs, so each e_y row is copied once (the band's first pair also copies its y0 - 1).
    auto eyslot = [&](int k) { return st + (3 + (k & 1)) * Wp; };
    auto issue = [&](int p) {
        const int i = p - p0;
        const int y0 = 2 * p, y1 = y0 + 1;
        stage_floats(st, ex + (size_t)y0 * W, W, vec);
        stage_floats(st + 2 * Wp, ey + (size_t)y0 * W, W, vec);
        if (i == 0) {
            const int ym = (y0 == 0) ? H - 1 : y0 - 1;
            stage_floats(eyslot(1), ey + (size_t)ym * W, W, vec);
        }
        if (y1 < H) {
            stage_floats(st + Wp, ex + (size_t)y1 * W, W, vec);
            stage_floats(eyslot(i), ey + (size_t)y1 * W, W, vec);
        }
        cp_commit();
    };
    const float* ex0 = st;
    const float* ex1 = st + Wp;
    const float* ey0 = st + 2 * Wp;
    issue(p0);
    for (int p = p0; p < p1; ++p) {
        cp_wait<0>();
        __syncthreads();
        const int y0 = 2 * p, y1 = y0 + 1;
        const bool has1 = y1 < H;
        const float* eym = eyslot(p - p0 + 1);
        const float* ey1 = eyslot(p - p0);
        for (unsigned b = threadIdx.x; b < S0::total; b += blockDim.x) {
            unsigned nat, j, col;
            S0::locate(b, nat, j, col);
            if (!S0::in_buffer(S0::offset(nat, col)) ||
                !BLFLS_DCHECK(nat + (R0 - 1) * M0 < (unsigned)W, kDcSolveGlobal))
                continue;
            float2 v[R0];
#pragma unroll
            for (int t = 0; t < R0; ++t) {
                const int x = (int)(nat + t * M0);
                const int xm = (x == 0) ? W - 1 : x - 1;
                // (D_x^T e_x)[x] = e_x[x-1] - e_x[x];  (D_y^T e_y)[y] = e_y[y-1] - e_y[y]
                const float r0 = (ex0[xm] - ex0[x]) + (eym[x] - ey0[x]);
                const float r1 = has1 ? (ex1[xm] - ex1[x]) + (ey0[x] - ey1[x]) : 0.f;
                v[t] = make_float2(r0, r1);
            }
            float2 o[R0];
            S0::fwd(v, o, rp.tw, j);
            float2* xb = data + S0::offset(nat, col);
#pragma unroll
            for (int q = 0; q < R0; ++q) xb[q * S0::st] = o[q];
        }
        __syncthreads();
        if (p + 1 < p1) issue(p + 1);   // the rows of pair p have been read out
        ct_forward_range<P, 1, PADS, 1>(data, rp.tw, std::make_integer_sequence<int, P::nst - 1>{});
        float2* s0 = spec + (size_t)y0 * Wh;
        float2* s1 = spec + (size_t)(has1 ? y1 : y0) * Wh;
#pragma unroll 4
        for (int k = threadIdx.x; k < Wh; k += blockDim.x) {
            const int kn = (k == 0) ? 0 : W - k;
            const float2 zk = data[S0::offset(ct_position<P>((unsigned)k), 0)];
            const float2 zn = data[S0::offset(ct_position<P>((unsigned)kn), 0)];
            // A = (Z_k + conj Z_{W-k}) / 2,  B = (Z_k - conj Z_{W-k}) / (2i)
            s0[k] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
            if (has1) s1[k] = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
        }
        __syncthreads();
    }
}

// NC columns per block: any count, so that the column blocks can be balanced over the SMs (see
// fused_col_block).
template <int NC, class P>
__global__ void __launch_bounds__(kColThreadsMax) k3_cols_fused(float2* __restrict__ spec, int H,
                                                                int W, FftPlanDev cp,
                                                                const float* __restrict__ sx,
                                                                float lam, float scale)
{
    static_assert(P::nst >= 2, "fused drivers need two or more stages");
    constexpr int R0 = P::radix[0];
    constexpr unsigned M0 = P::span(0);
    constexpr int NL = P::nst - 1;
    constexpr int RL = P::radix[NL];
    using S0 = CtStageOf<P, 0, NC, 0>;
    using SL = CtStageOf<P, NL, NC, 0>;
    extern __shared__ __align__(16) unsigned char staged_smem[];
    float2* data = reinterpret_cast<float2*>(staged_smem);
    constexpr int CB = NC;
    const int Wh = W / 2 + 1;
    const int nblk = (Wh + CB - 1) / CB;
    const float2* tw = cp.tw;
    int b0, b1;
    band(nblk, b0, b1);
    for (int blk = b0; blk < b1; ++blk) {
        const int kx0 = blk * CB;
        // first forward stage, inputs from the spectrum in global memory
        for (unsigned b = threadIdx.x; b < S0::total; b += blockDim.x) {
            unsigned nat, j, col;
            S0::locate(b, nat, j, col);
            const int kx = kx0 + (int)col;
            if (!S0::in_buffer(S0::offset(nat, col)) ||
                !BLFLS_DCHECK(nat + (R0 - 1) * M0 < (unsigned)H, kDcSolveGlobal))
                continue;
            float2 v[R0];
#pragma unroll
            for (int t = 0; t < R0; ++t)
                v[t] = kx < Wh ? spec[(size_t)(nat + t * M0) * Wh + kx] : make_float2(0.f, 0.f);
            float2 o[R0];
            S0::fwd(v, o, tw, j);
            float2* xb = data + S0::offset(nat, col);
#pragma unroll
            for (int q = 0; q < R0; ++q) xb[q * S0::st] = o[q];
        }
        __syncthreads();
        ct_forward_range<P, NC, 0, 1>(data, tw, std::make_integer_sequence<int, NL - 1>{});
        // last forward stage, spectral divide (Eq. 8 denominator, F(1) = 1, with lam and the
        // 1/(HW) of the inverse), first inverse stage -- all in registers
        for (unsigned b = threadIdx.x; b < SL::total; b += blockDim.x) {
            unsigned nat, j, col;
            SL::locate(b, nat, j, col);
            if (!SL::in_buffer(SL::offset(nat, col))) continue;
            float2* xb = data + SL::offset(nat, col);
            float2 v[RL], y[RL], o[RL];
#pragma unroll
            for (int t = 0; t < RL; ++t) v[t] = xb[t * SL::st];
            SL::fwd(v, y, tw, j);
            const float sxv = __ldg(sx + min(kx0 + (int)col, Wh - 1));
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                const float syv = __ldg(cp.lapp + nat + q);
                const float den = fmaf(lam, sxv + syv, 1.0f);
                const float m = __fdividef(scale, den) * lam;
                y[q] = make_float2(y[q].x * m, y[q].y * m);
            }
            SL::inv(y, o, tw, j);
#pragma unroll
            for (int t = 0; t < RL; ++t) xb[t * SL::st] = o[t];
        }
        __syncthreads();
        ct_inverse_range<P, NC, 0, NL>(data, tw, std::make_integer_sequence<int, NL - 1>{});
        // last inverse stage, outputs to the spectrum in global memory
        for (unsigned b = threadIdx.x; b < S0::total; b += blockDim.x) {
            unsigned nat, j, col;
            S0::locate(b, nat, j, col);
            const int kx = kx0 + (int)col;
            if (!S0::in_buffer(S0::offset(nat, col)) ||
                !BLFLS_DCHECK(nat + (R0 - 1) * M0 < (unsigned)H, kDcSolveGlobal))
                continue;
            const float2* xb = data + S0::offset(nat, col);
            float2 a[R0], o[R0];
#pragma unroll
            for (int q = 0; q < R0; ++q) a[q] = xb[q * S0::st];
            S0::inv(a, o, tw, j);
            if (kx < Wh) {
#pragma unroll
                for (int t = 0; t < R0; ++t) spec[(size_t)(nat + t * M0) * Wh + kx] = o[t];
            }
        }
        __syncthreads();
    }
}

template <class P>
__global__ void __launch_bounds__(kStagedThreads, 2) k4_rows_fused(const float2* __restrict__ spec,
                                                                   const float* f, float* out,
                                                                   int H, int W, FftPlanDev rp,
                                                                   int vec)
{
    static_assert(P::nst >= 2, "fused drivers need two or more stages");
    constexpr int PADS = P::L / P::radix[0];
    constexpr int R0 = P::radix[0];
    constexpr unsigned M0 = P::span(0);
    constexpr int NL = P::nst - 1;
    constexpr int RL = P::radix[NL];
    using S0 = CtStageOf<P, 0, 1, PADS>;
    using SL = CtStageOf<P, NL, 1, PADS>;
    extern __shared__ __align__(16) unsigned char staged_smem[];
    const int Wh = W / 2 + 1;
    const size_t Wp = row_floats(W);
    float2* ss = reinterpret_cast<float2*>(staged_smem);
    float* sf = reinterpret_cast<float*>(staged_smem + k4s_spec_bytes(W));
    float2* data = reinterpret_cast<float2*>(staged_smem + k4s_spec_bytes(W) + sizeof(float) * 2 * Wp);
    const int npairs = (H + 1) / 2;
    int p0, p1;
    band(npairs, p0, p1);
    if (p0 >= p1) return;
    auto issue_spec = [&](int p) {
        const int y0 = 2 * p, y1 = y0 + 1;
        stage_complex(ss, spec + (size_t)y0 * Wh, Wh);
        if (y1 < H) stage_complex(ss + Wh, spec + (size_t)y1 * Wh, Wh);
        cp_commit();
    };
    auto issue_f = [&](int p) {
        const int y0 = 2 * p, y1 = y0 + 1;
        stage_floats(sf, f + (size_t)y0 * W, W, vec);
        if (y1 < H) stage_floats(sf + Wp, f + (size_t)y1 * W, W, vec);
        cp_commit();
    };
    // Copy groups complete in issue order: spectra(p), f(p), spectra(p+1), f(p+1), ...
    issue_spec(p0);
    issue_f(p0);
    for (int p = p0; p < p1; ++p) {
        cp_wait<1>();                 // spectra(p) landed; f(p) may still be in flight
        __syncthreads();
        const int y0 = 2 * p, y1 = y0 + 1;
        const bool has1 = y1 < H;
        // first inverse stage (the last stage's inverse, span 1), its inputs Z = A + i B rebuilt
        // from the two half spectra by Hermitian symmetry at the frequencies of its positions.
        // Butterfly b = q0 (L / (R0 R_last)) + rest holds frequencies whose lowest digit is q0, so
        // thread i takes q0 = i mod R0: adjacent lanes read adjacent frequencies of the staged
        // spectra (no bank conflicts), and write positions L / R0 apart (padded: no conflicts).
        for (unsigned i = threadIdx.x; i < SL::total; i += blockDim.x) {
            const unsigned b = (i % (unsigned)R0) * (SL::total / (unsigned)R0) + i / (unsigned)R0;
            unsigned nat, j, col;
            SL::locate(b, nat, j, col);
            if (!SL::in_buffer(SL::offset(nat, col))) continue;
            float2 v[RL], o[RL];
            // the last stage has span 1: position nat + q holds frequency k(nat) + q R_0..R_{NL-1}
            const int k0 = ct_frequency<P>(nat);
            static_assert(P::span(NL) == 1, "the last stage has span 1");
            constexpr int wl = P::L / RL;
#pragma unroll
            for (int q = 0; q < RL; ++q) {
                const int k = k0 + q * wl;
                const bool upper = k > W / 2;
                const int kk = upper ? W - k : k;
                float2 a = ss[kk];
                float2 bb = has1 ? ss[Wh + kk] : make_float2(0.f, 0.f);
                if (upper) { a.y = -a.y; bb.y = -bb.y; }
                if (k == 0 || 2 * k == W) { a.y = 0.f; bb.y = 0.f; }  // real bins of a real row
                v[q] = make_float2(a.x - bb.y, a.y + bb.x);            // Z = A + i B
            }
            SL::inv(v, o, rp.tw, j);
            float2* xb = data + SL::offset(nat, col);
#pragma unroll
            for (int t = 0; t < RL; ++t) xb[t * SL::st] = o[t];
        }
        __syncthreads();
        const bool more = p + 1 < p1;
        if (more) issue_spec(p + 1);  // the spectra of pair p have been read out
        ct_inverse_range<P, 1, PADS, NL>(data, rp.tw, std::make_integer_sequence<int, NL - 1>{});
        if (more) cp_wait<1>(); else cp_wait<0>();   // f(p) landed
        __syncthreads();
        // last inverse stage (stage 0): u = f + result, real part row a, imaginary part row b
        float* o0 = out + (size_t)y0 * W;
        float* o1 = out + (size_t)(has1 ? y1 : y0) * W;
        for (unsigned b = threadIdx.x; b < S0::total; b += blockDim.x) {
            unsigned nat, j, col;
            S0::locate(b, nat, j, col);
            if (!S0::in_buffer(S0::offset(nat, col)) ||
                !BLFLS_DCHECK(nat + (R0 - 1) * M0 < (unsigned)W, kDcSolveGlobal))
                continue;
            const float2* xb = data + S0::offset(nat, col);
            float2 a[R0], z[R0];
#pragma unroll
            for (int q = 0; q < R0; ++q) a[q] = xb[q * S0::st];
            S0::inv(a, z, rp.tw, j);
#pragma unroll
            for (int t = 0; t < R0; ++t) {
                const int x = (int)(nat + t * M0);
                o0[x] = sf[x] + z[t].x;
                if (has1) o1[x] = sf[Wp + x] + z[t].y;
            }
        }
        __syncthreads();
        if (more) issue_f(p + 1);
    }
}

// ---- batched: items of many jobs ------------------------------------------------------------
__device__ __forceinline__ int find_group(const int2* grp, int ngrp, int item, int g)
{
    while (g + 1 < ngrp && __ldg(&grp[g + 1].y) <= item) ++g;
    return g;
}

__global__ void __launch_bounds__(512) k2_batch(const BatchJob* __restrict__ jobs,
                                                const int2* __restrict__ grp, int ngrp, int total)
{
    extern __shared__ float2 smem[];
    int g = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        g = find_group(grp, ngrp, item, g);
        const BatchJob& J = jobs[__ldg(&grp[g].x)];
        const int npairs = (J.H + 1) / 2;
        const int local = item - __ldg(&grp[g].y);
        const int c = local / npairs, pair = local - c * npairs;
        const size_t plane = (size_t)J.H * J.W;
        k2_item(J.ex + c * plane, J.ey + c * plane, J.spec + c * (size_t)J.H * (J.W / 2 + 1), J.H,
                J.W, pair, J.rp, J.rp.tw, smem);
    }
}

__global__ void __launch_bounds__(512) k3_batch(const BatchJob* __restrict__ jobs,
                                                const int2* __restrict__ grp, int ngrp, int total)
{
    extern __shared__ float2 smem[];
    int g = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        g = find_group(grp, ngrp, item, g);
        const BatchJob& J = jobs[__ldg(&grp[g].x)];
        const int Wh = J.W / 2 + 1;
        const int nblk = (Wh + (1 << J.lgc) - 1) >> J.lgc;
        const int local = item - __ldg(&grp[g].y);
        const int c = local / nblk, blk = local - c * nblk;
        if (J.rec)   // 32-column blocks (lgc = 5) solved by the recursion
            k3_rec_item(J.spec + c * (size_t)J.H * Wh, J.H, J.W, blk, J.rp.lap, J.lam, J.scale,
                        smem);
        else
            k3_item(J.spec + c * (size_t)J.H * Wh, J.H, J.W, blk, J.cp, J.rp.lap, J.cp.lap, J.lam,
                    J.scale, J.lgc, J.cp.tw, smem);
    }
}

__global__ void __launch_bounds__(512) k4_batch(const BatchJob* __restrict__ jobs,
                                                const int2* __restrict__ grp, int ngrp, int total)
{
    extern __shared__ float2 smem[];
    int g = 0;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        g = find_group(grp, ngrp, item, g);
        const BatchJob& J = jobs[__ldg(&grp[g].x)];
        const int npairs = (J.H + 1) / 2;
        const int local = item - __ldg(&grp[g].y);
        const int c = local / npairs, pair = local - c * npairs;
        const size_t plane = (size_t)J.H * J.W;
        k4_item(J.spec + c * (size_t)J.H * (J.W / 2 + 1), J.src + c * plane, J.dst + c * plane,
                J.H, J.W, pair, J.rp, J.rp.tw, smem);
    }
}

// ---- batched, staged: the row drivers of the single image over the row pairs of many jobs,
// taken with a grid stride; the staging buffer and the FFT buffer are sized for the widest row
// of the batch. ---------------------------------------------------------------------------------

// Row pair `item` of the jobs: job entry, channel plane offset and pair index.
struct RowItem {
    const BatchJob* J;
    int c, pair;
};

__device__ __forceinline__ RowItem row_item(const BatchJob* __restrict__ jobs,
                                            const int2* __restrict__ grp, int ngrp, int item,
                                            int& g)
{
    while (g + 1 < ngrp && __ldg(&grp[g + 1].y) <= item) ++g;
    const BatchJob* J = jobs + __ldg(&grp[g].x);
    const int npairs = (J->H + 1) / 2;
    const int local = item - __ldg(&grp[g].y);
    const int c = local / npairs;
    return RowItem{J, c, local - c * npairs};
}

__device__ __forceinline__ bool aligned16(const void* p)
{
    return (reinterpret_cast<uintptr_t>(p) & 15) == 0;
}

__global__ void __launch_bounds__(kStagedThreads, 2) k2_batch_staged(const BatchJob* __restrict__ jobs,
                                                                     const int2* __restrict__ grp,
                                                                     int ngrp, int total, int Wp)
{
    extern __shared__ __align__(16) unsigned char staged_smem[];
    float* st = reinterpret_cast<float*>(staged_smem);
    float2* data = reinterpret_cast<float2*>(staged_smem + sizeof(float) * 5 * (size_t)Wp);
    // items blockIdx.x, blockIdx.x + gridDim.x, ...: the costs of the jobs' row pairs differ
    // widely (widths, Bluestein rows), and a stride spreads them evenly over the CTAs
    const int i0 = blockIdx.x, step = gridDim.x;
    if (i0 >= total) return;
    int gc = 0, gn = 0;   // group cursors of the current and the next item
    auto issue = [&](const RowItem& it) {
        const BatchJob& J = *it.J;
        const int H = J.H, W = J.W;
        const size_t plane = (size_t)H * W;
        const float* ex = J.ex + it.c * plane;
        const float* ey = J.ey + it.c * plane;
        const int y0 = 2 * it.pair, y1 = y0 + 1;
        const int ym = (y0 == 0) ? H - 1 : y0 - 1;
        const bool vec = (W & 3) == 0 && aligned16(ex) && aligned16(ey);
        stage_floats(st, ex + (size_t)y0 * W, W, vec);
        stage_floats(st + 2 * Wp, ey + (size_t)ym * W, W, vec);
        stage_floats(st + 3 * Wp, ey + (size_t)y0 * W, W, vec);
        if (y1 < H) {
            stage_floats(st + Wp, ex + (size_t)y1 * W, W, vec);
            stage_floats(st + 4 * Wp, ey + (size_t)y1 * W, W, vec);
        }
        cp_commit();
    };
    RowItem cur = row_item(jobs, grp, ngrp, i0, gc);
    gn = gc;
    issue(cur);
    for (int item = i0; item < total; item += step) {
        cp_wait<0>();
        __syncthreads();
        const BatchJob& J = *cur.J;
        const int W = J.W, Wh = W / 2 + 1;
        const int y0 = 2 * cur.pair, y1 = y0 + 1;
        const bool has1 = y1 < J.H;
        k2_build(st, st + Wp, st + 2 * Wp, st + 3 * Wp, st + 4 * Wp, has1, W, J.rp, data);
        RowItem next{};
        if (item + step < total) {
            next = row_item(jobs, grp, ngrp, item + step, gn);
            issue(next);   // the rows of this pair have been read out
        }
        float2* spec = J.spec + cur.c * (size_t)J.H * Wh;
        k2_transform(has1, W, spec + (size_t)y0 * Wh, spec + (size_t)(has1 ? y1 : y0) * Wh, J.rp,
                     J.rp.tw, data);
        cur = next;
    }
}

__global__ void __launch_bounds__(kStagedThreads, 2) k4_batch_staged(const BatchJob* __restrict__ jobs,
                                                                     const int2* __restrict__ grp,
                                                                     int ngrp, int total, int Wp)
{
    extern __shared__ __align__(16) unsigned char staged_smem[];
    const size_t spec_bytes = align16(sizeof(float2) * 2 * (size_t)(Wp / 2 + 1));
    float2* ss = reinterpret_cast<float2*>(staged_smem);
    float* sf = reinterpret_cast<float*>(staged_smem + spec_bytes);
    float2* data = reinterpret_cast<float2*>(staged_smem + spec_bytes + sizeof(float) * 2 * (size_t)Wp);
    const int i0 = blockIdx.x, step = gridDim.x;   // strided items, as in k2_batch_staged
    if (i0 >= total) return;
    int gc = 0, gn = 0;
    auto issue_spec = [&](const RowItem& it) {
        const BatchJob& J = *it.J;
        const int Wh = J.W / 2 + 1;
        const float2* spec = J.spec + it.c * (size_t)J.H * Wh;
        const int y0 = 2 * it.pair, y1 = y0 + 1;
        stage_complex(ss, spec + (size_t)y0 * Wh, Wh);
        if (y1 < J.H) stage_complex(ss + Wh, spec + (size_t)y1 * Wh, Wh);
        cp_commit();
    };
    auto issue_f = [&](const RowItem& it) {
        const BatchJob& J = *it.J;
        const int W = J.W;
        const float* f = J.src + it.c * (size_t)J.H * W;
        const int y0 = 2 * it.pair, y1 = y0 + 1;
        const bool vec = (W & 3) == 0 && aligned16(f);
        stage_floats(sf, f + (size_t)y0 * W, W, vec);
        if (y1 < J.H) stage_floats(sf + Wp, f + (size_t)y1 * W, W, vec);
        cp_commit();
    };
    // copy groups complete in issue order: spectra(p), f(p), spectra(p+1), f(p+1), ...
    RowItem cur = row_item(jobs, grp, ngrp, i0, gc);
    gn = gc;
    issue_spec(cur);
    issue_f(cur);
    for (int item = i0; item < total; item += step) {
        cp_wait<1>();   // spectra of this pair landed; its f may still be in flight
        __syncthreads();
        const BatchJob& J = *cur.J;
        const int W = J.W, Wh = W / 2 + 1;
        const int y0 = 2 * cur.pair, y1 = y0 + 1;
        const bool has1 = y1 < J.H;
        k4_rebuild(ss, ss + Wh, has1, W, J.rp, data);
        const bool more = item + step < total;
        RowItem next{};
        if (more) {
            next = row_item(jobs, grp, ngrp, item + step, gn);
            issue_spec(next);   // the spectra of this pair have been read out
        }
        fft_inverse<0, true>(data, 0, J.rp, J.rp.tw);
        if (more) cp_wait<1>(); else cp_wait<0>();   // f of this pair landed
        __syncthreads();
        float* out = J.dst + cur.c * (size_t)J.H * W;
        k4_output(has1, sf, sf + Wp, out + (size_t)y0 * W, out + (size_t)(has1 ? y1 : y0) * W, W,
                  J.rp, data);
        if (more) issue_f(next);
        cur = next;
    }
}

int threads_for(int work)
{
    int t = 128;
    while (t < 512 && t * 4 < work) t *= 2;
    return t;
}

}  // namespace

BLFLS_DCHECK_TU(solve_kernels)

static void set_staged_attributes();   // below, with the plan pickers

void init_solve_kernel_attributes()
{
    cudaFuncSetAttribute(k2_rows_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k3_cols_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k4_rows_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k2_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k3_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k4_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    set_staged_attributes();
    cudaFuncSetAttribute(k2_batch_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k4_batch_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

size_t solve_smem_rows(const FftPlanDev& rp)
{
    const size_t data = sizeof(float2) * row_buf_elems(rp);
    const size_t tw = sizeof(float2) * rp.L;
    return data + tw <= kSmemCap ? data + tw : data;
}

size_t solve_smem_cols(const FftPlanDev& cp, int col_block)
{
    const size_t data = sizeof(float2) * (size_t)cp.L * col_block;
    const size_t tw = sizeof(float2) * cp.L;
    return data + tw <= kSmemCap ? data + tw : data;
}

int solve_fit_lgc(int L, int col_block)
{
    int lgc = 0;
    while ((1 << lgc) < col_block) ++lgc;
    while (lgc > 0 && sizeof(float2) * (size_t)L * (1u << lgc) > kSmemCap) --lgc;
    return lgc;
}

// Block size of the staged column driver.  Stage s of the plan has (L / radix_s) << lgc
// butterflies and every thread takes ceil(butterflies / threads) of them, so a block size that
// leaves a few butterflies over doubles that stage.  Pick the size (a multiple of 32 up to
// kColThreadsMax) with the least sum over stages of ceil(butterflies / threads) divided by the
// number of CTAs that fit on an SM.
typedef void (*ColsStagedFn)(float2*, int, int, FftPlanDev, const float*, const float*, float, float);
typedef void (*RowsK2Fn)(const float*, const float*, float2*, int, int, FftPlanDev, int);
typedef void (*RowsK4Fn)(const float2*, const float*, float*, int, int, FftPlanDev, int);

// Compile-time plans of the staged drivers: row lengths 3840 and 1920, column lengths 2160 and
// 1080 (the radix sequences factor_direct gives them); other lengths use the runtime plan.
using RowPlanA = CtPlan<16, 16, 15>;   // 3840
using RowPlanB = CtPlan<16, 8, 15>;    // 1920
using ColPlanA = CtPlan<16, 15, 9>;    // 2160
using ColPlanB = CtPlan<8, 15, 9>;     // 1080

template <class P>
static bool plan_is(const FftPlanDev& p)
{
    if (p.bluestein || p.nst != P::nst || p.L != P::L) return false;
    for (int s = 0; s < P::nst; ++s)
        if (p.radix[s] != P::radix[s]) return false;
    return true;
}

static RowsK2Fn rows_k2_kernel(const FftPlanDev& rp)
{
    if (plan_is<RowPlanA>(rp)) return k2_rows_fused<RowPlanA>;
    if (plan_is<RowPlanB>(rp)) return k2_rows_fused<RowPlanB>;
    return k2_rows_staged<void>;
}
static RowsK4Fn rows_k4_kernel(const FftPlanDev& rp)
{
    if (plan_is<RowPlanA>(rp)) return k4_rows_fused<RowPlanA>;
    if (plan_is<RowPlanB>(rp)) return k4_rows_fused<RowPlanB>;
    return k4_rows_staged<void>;
}

template <class P>
static ColsStagedFn cols_staged_kernel_p(int lgc)
{
    switch (lgc) {
        case 0: return k3_cols_staged<0, P>;
        case 1: return k3_cols_staged<1, P>;
        case 2: return k3_cols_staged<2, P>;
        case 3: return k3_cols_staged<3, P>;
        default: return k3_cols_staged<4, P>;   // col_block is at most 16
    }
}
typedef void (*ColsFusedFn)(float2*, int, int, FftPlanDev, const float*, float, float);
// Column counts the fused column driver is compiled for.  13 columns of 2160 points fill one
// CTA's shared memory, and the 1921 columns of a 3840-wide spectrum then make 148 blocks: one
// round over the 152 SMs.
constexpr int kFusedBlocks[] = {1, 2, 4, 7, 8, 13, 16};
template <class P>
static ColsFusedFn cols_fused_kernel_p(int nc)
{
    switch (nc) {
        case 1: return k3_cols_fused<1, P>;
        case 2: return k3_cols_fused<2, P>;
        case 4: return k3_cols_fused<4, P>;
        case 7: return k3_cols_fused<7, P>;
        case 8: return k3_cols_fused<8, P>;
        case 13: return k3_cols_fused<13, P>;
        case 16: return k3_cols_fused<16, P>;
        default: return nullptr;
    }
}
static bool fused_plan(const FftPlanDev& cp) { return plan_is<ColPlanA>(cp) || plan_is<ColPlanB>(cp); }
// The fused column driver of a compile-time plan for nc columns per block, or nullptr (runtime
// plans: staged driver).
static ColsFusedFn cols_fused_kernel(int nc, const FftPlanDev& cp)
{
    if (plan_is<ColPlanA>(cp)) return cols_fused_kernel_p<ColPlanA>(nc);
    if (plan_is<ColPlanB>(cp)) return cols_fused_kernel_p<ColPlanB>(nc);
    return nullptr;
}
static ColsStagedFn cols_staged_kernel(int lgc, const FftPlanDev& cp)
{
    (void)cp;
    return cols_staged_kernel_p<void>(lgc);
}
// Shared memory of the fused column driver: one block of nc columns.
static size_t k3f_smem(int L, int nc) { return sizeof(float2) * (size_t)L * nc; }

// Columns per block of the fused column driver.  A block size from a tune table (col_block > 0)
// is taken as the largest compiled count not above it that fits; otherwise the count that
// minimises ceil(blocks / SMs) x columns per block (the columns the busiest SM transforms), the
// larger count winning ties.
static int fused_col_block(const FftPlanDev& cp, int W, int col_block, int num_sms)
{
    const int ncols = W / 2 + 1;
    int best = 1;
    long best_cost = -1;
    for (int nc : kFusedBlocks) {
        if (k3f_smem(cp.L, nc) > kSmemCap) continue;
        if (col_block > 0) {
            if (nc <= col_block) best = nc;
            continue;
        }
        const long blocks = (ncols + nc - 1) / nc;
        const long cost = (blocks + num_sms - 1) / num_sms * nc;
        if (best_cost < 0 || cost <= best_cost) {
            best_cost = cost;
            best = nc;
        }
    }
    return best;
}

static void set_staged_attributes()
{
    const int big = 227 * 1024;
    for (RowsK2Fn f : {k2_rows_staged<void>, k2_rows_fused<RowPlanA>, k2_rows_fused<RowPlanB>})
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    for (RowsK4Fn f : {k4_rows_staged<void>, k4_rows_fused<RowPlanA>, k4_rows_fused<RowPlanB>})
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    for (int lgc = 0; lgc <= 4; ++lgc)
        cudaFuncSetAttribute(cols_staged_kernel_p<void>(lgc),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    for (int nc : kFusedBlocks)
        for (ColsFusedFn f : {cols_fused_kernel_p<ColPlanA>(nc), cols_fused_kernel_p<ColPlanB>(nc)})
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k3_cols_rec, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// Block size of a column driver (fn: its kernel); see the comment above.
static int col_threads(const void* fn, const FftPlanDev& cp, int ncol, size_t smem, int* occ_out)
{
    int best_t = 128, best_occ = 1;
    double best = 1e30;
    for (int t = 128; t <= kColThreadsMax; t += 32) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, t, smem);
        if (occ < 1) continue;
        long rounds = 0;
        for (int st = 0; st < cp.nst; ++st) {
            const long nb = (long)(cp.L / cp.radix[st]) * ncol;
            rounds += (nb + t - 1) / t;
        }
        const double cost = (double)rounds / occ;
        if (cost < best - 1e-9) { best = cost; best_t = t; best_occ = occ; }
    }
    *occ_out = best_occ;
    return best_t;
}

size_t solve_rec_smem(int H) { return rec_smem(H); }

int solve_effective_col_block(const FftPlanDev& cp, int W, int col_block, int num_sms)
{
    if (fused_plan(cp)) return fused_col_block(cp, W, col_block, num_sms);
    int lgc = solve_fit_lgc(cp.L, col_block > 0 ? col_block : kDefaultColBlock);
    while (lgc > 0 && k3s_smem(cp.L, lgc) > kSmemCap) --lgc;
    return 1 << lgc;
}

cudaError_t launch_solve_residual(const float* f, const float* ex, const float* ey, float* out,
                                  float2* spec, const FftPlanDev& rp, const FftPlanDev& cp,
                                  const float* sx, const float* sy, const SolveParams& p,
                                  cudaStream_t s, int num_sms, const cudaEvent_t* marks)
{
    const int H = p.H, W = p.W;
    const float scale = 1.0f / ((float)H * (float)W);
    // Staged drivers when their shared memory fits; rows of floats are copied 16 bytes at a time
    // when every row start is 16-byte aligned.
    const size_t cap = kSmemCap;
    const bool al16 = (W % 4 == 0) && ((reinterpret_cast<uintptr_t>(ex) | reinterpret_cast<uintptr_t>(ey) |
                                        reinterpret_cast<uintptr_t>(f)) % 16 == 0);
    const bool rows_staged = k2s_smem(W, rp) <= cap && k4s_smem(W, rp) <= cap;
    // the fused column driver on compile-time plans (any column count, see fused_col_block),
    // else the staged driver on a power-of-two block (col_block 0: no tuned value, the default)
    const int nc = fused_plan(cp) ? fused_col_block(cp, W, p.col_block, num_sms) : 0;
    const ColsFusedFn k3f = nc > 0 ? cols_fused_kernel(nc, cp) : nullptr;
    const bool cols_fused = k3f != nullptr && k3f_smem(cp.L, nc) <= cap;
    int lgc = solve_fit_lgc(cp.L, p.col_block > 0 ? p.col_block : kDefaultColBlock);
    while (lgc > 0 && k3s_smem(cp.L, lgc) > cap) --lgc;
    const bool cols_staged = !cols_fused && k3s_smem(cp.L, lgc) <= cap;
    const int CB = 1 << lgc;
    const int npairs = (H + 1) / 2;
    const int nblk = (W / 2 + 1 + CB - 1) / CB;

    if (rows_staged) {
        const size_t sm2 = k2s_smem(W, rp);
        int occ = 0;
        const RowsK2Fn k2 = rows_k2_kernel(rp);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2, kStagedThreads, sm2);
        const int grid = std::max(1, std::min(npairs, num_sms * std::max(occ, 1)));
        k2<<<grid, kStagedThreads, sm2, s>>>(ex, ey, spec, H, W, rp, al16 ? 1 : 0);
    } else {
        const size_t smem_r = solve_smem_rows(rp);
        const int tw_r = smem_r > sizeof(float2) * row_buf_elems(rp);
        const int thr_r = threads_for(rp.L / 4);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2_rows_forward, thr_r, smem_r);
        const int grid_r = std::max(1, std::min(npairs, num_sms * std::max(occ, 1)));
        k2_rows_forward<<<grid_r, thr_r, smem_r, s>>>(ex, ey, spec, H, W, rp, tw_r);
    }
    if (marks) cudaEventRecord(marks[0], s);
    if (cp.bluestein && p.lambda <= kRecLamMax) {
        const int nb = (W / 2 + 1 + 31) / 32;
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k3_cols_rec, 512, rec_smem(H));
        const int grid = std::max(1, std::min(nb, num_sms * std::max(occ, 1)));
        k3_cols_rec<<<grid, 512, rec_smem(H), s>>>(spec, H, W, sx, p.lambda, scale);
    } else if (cols_fused) {
        const size_t sm3 = k3f_smem(cp.L, nc);
        int occ = 0;
        const int thr = col_threads((const void*)k3f, cp, nc, sm3, &occ);
        const int nblk_f = (W / 2 + 1 + nc - 1) / nc;
        const int grid = std::max(1, std::min(nblk_f, num_sms * std::max(occ, 1)));
        k3f<<<grid, thr, sm3, s>>>(spec, H, W, cp, sx, p.lambda, scale);
    } else if (cols_staged) {
        const size_t sm3 = k3s_smem(cp.L, lgc);
        int occ = 0;
        const ColsStagedFn k3 = cols_staged_kernel(lgc, cp);
        const int thr = col_threads((const void*)k3, cp, 1 << lgc, sm3, &occ);
        const int grid = std::max(1, std::min(nblk, num_sms * std::max(occ, 1)));
        k3<<<grid, thr, sm3, s>>>(spec, H, W, cp, sx, sy, p.lambda, scale);
    } else {
        const int lgc1 = solve_fit_lgc(cp.L, p.col_block > 0 ? p.col_block : kDefaultColBlock);
        const int CB1 = 1 << lgc1;
        const size_t smem_c = solve_smem_cols(cp, CB1);
        const int tw_c = smem_c > sizeof(float2) * (size_t)cp.L * CB1;
        const int thr_c = threads_for((cp.L * CB1) / 4);
        int occ_c = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k3_cols_solve, thr_c, smem_c);
        const int nblk1 = (W / 2 + 1 + CB1 - 1) / CB1;
        const int grid_c = std::max(1, std::min(nblk1, num_sms * std::max(occ_c, 1)));
        k3_cols_solve<<<grid_c, thr_c, smem_c, s>>>(spec, H, W, cp, sx, sy, p.lambda, scale, lgc1, tw_c);
    }
    if (marks) cudaEventRecord(marks[1], s);
    if (rows_staged) {
        const size_t sm4 = k4s_smem(W, rp);
        int occ = 0;
        const RowsK4Fn k4 = rows_k4_kernel(rp);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k4, kStagedThreads, sm4);
        const int grid = std::max(1, std::min(npairs, num_sms * std::max(occ, 1)));
        k4<<<grid, kStagedThreads, sm4, s>>>(spec, f, out, H, W, rp, al16 ? 1 : 0);
    } else {
        const size_t smem_r = solve_smem_rows(rp);
        const int tw_r = smem_r > sizeof(float2) * row_buf_elems(rp);
        const int thr_r = threads_for(rp.L / 4);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k4_rows_inverse, thr_r, smem_r);
        const int grid_r = std::max(1, std::min(npairs, num_sms * std::max(occ, 1)));
        k4_rows_inverse<<<grid_r, thr_r, smem_r, s>>>(spec, f, out, H, W, rp, tw_r);
    }
    return cudaGetLastError();
}

cudaError_t launch_solve_batch(const BatchJob* jobs, int njobs, const int2* grp_rows,
                               int total_rows, const int2* grp_cols, int total_cols,
                               size_t smem_rows, size_t smem_cols, int max_w, int num_sms,
                               cudaStream_t s, const cudaEvent_t* marks)
{
    if (total_rows <= 0) return cudaSuccess;
    const int thr = 256;
    // staged row drivers when their buffers (sized for the widest row) fit
    const int Wp = (int)row_floats(max_w);
    const size_t sm2 = sizeof(float) * 5 * (size_t)Wp + smem_rows;
    const size_t sm4 = align16(sizeof(float2) * 2 * (size_t)(Wp / 2 + 1)) + sizeof(float) * 2 * (size_t)Wp + smem_rows;
    const bool staged = sm2 <= kSmemCap && sm4 <= kSmemCap;
    int occ_r = 0, occ_c = 0, occ_2 = 0, occ_4 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k3_batch, thr, smem_cols);
    const int grid_c = std::max(1, std::min(total_cols, num_sms * std::max(occ_c, 1)));
    if (staged) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_2, k2_batch_staged, kStagedThreads, sm2);
        const int grid_2 = std::max(1, std::min(total_rows, num_sms * std::max(occ_2, 1)));
        k2_batch_staged<<<grid_2, kStagedThreads, sm2, s>>>(jobs, grp_rows, njobs, total_rows, Wp);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_r, k2_batch, thr, smem_rows);
        const int grid_r = std::max(1, std::min(total_rows, num_sms * std::max(occ_r, 1)));
        k2_batch<<<grid_r, thr, smem_rows, s>>>(jobs, grp_rows, njobs, total_rows);
    }
    if (marks) cudaEventRecord(marks[0], s);
    k3_batch<<<grid_c, thr, smem_cols, s>>>(jobs, grp_cols, njobs, total_cols);
    if (marks) cudaEventRecord(marks[1], s);
    if (staged) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_4, k4_batch_staged, kStagedThreads, sm4);
        const int grid_4 = std::max(1, std::min(total_rows, num_sms * std::max(occ_4, 1)));
        k4_batch_staged<<<grid_4, kStagedThreads, sm4, s>>>(jobs, grp_rows, njobs, total_rows, Wp);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_r, k4_batch, thr, smem_rows);
        const int grid_r = std::max(1, std::min(total_rows, num_sms * std::max(occ_r, 1)));
        k4_batch<<<grid_r, thr, smem_rows, s>>>(jobs, grp_rows, njobs, total_rows);
    }
    return cudaGetLastError();
}

}  // namespace blfls
