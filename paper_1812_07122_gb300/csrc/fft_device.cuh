// CTA-wide in-place FFTs on shared memory, used by the Fourier solve of Eq. 8.
//
// A "column set" is `ncols` interleaved transforms: element n of column c sits at
// x[n * ncols + c] (ncols a power of two; 1 for a single row).  All threads of the CTA take part;
// every routine starts by assuming its input is visible to all threads (the caller synchronised)
// and ends with a __syncthreads().
//
// Direct transforms (length L = product of the plan's radices 16, 15, 9, 8, 4, 2, 3, 5, 7;
// 15 and 9 are two-level butterflies 3x5 and 3x3):
//   forward: decimation in frequency, natural input -> output in digit-reversed order
//            (frequency k at position perm[k]);
//   inverse: the conjugate stages in reverse order, digit-reversed input -> natural output,
//            unnormalised (a forward-then-inverse pair multiplies by L).
// Bluestein transforms (length N not 7-smooth) convert the length-N DFT into a cyclic
// convolution of length L = 2^k >= 2N-1 carried out by the direct transforms; input and output
// are in natural order, positions [N, L) are scratch.
#pragma once

#include "internal.h"

namespace blfls {

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// -i * a (forward rotation) or +i * a (inverse rotation)
template <bool INV>
__device__ __forceinline__ float2 rot_i(float2 a)
{
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi k / R) and sin(2 pi k / R) for the odd radices (mathematical constants).
__device__ __forceinline__ constexpr float root_cos(int R, int k)
{
    return R == 3 ? -0.5f
         : R == 5 ? (k == 1 ? 0.309016994374947424f : -0.809016994374947424f)
         : /* 7 */  (k == 1 ? 0.623489801858733531f
                   : k == 2 ? -0.222520933956314404f : -0.900968867902419126f);
}
__device__ __forceinline__ constexpr float root_sin(int R, int k)
{
    return R == 3 ? 0.866025403784438647f
         : R == 5 ? (k == 1 ? 0.951056516295153572f : 0.587785252292473129f)
         : /* 7 */  (k == 1 ? 0.781831482468029809f
                   : k == 2 ? 0.974927912181823607f : 0.433883739117558120f);
}

// cos(2 pi k / 16), k = 0..4 (mathematical constants)
__device__ __forceinline__ constexpr float c16(int k)
{
    return k == 0 ? 1.0f : k == 1 ? 0.923879532511286756f : k == 2 ? 0.707106781186547524f
         : k == 3 ? 0.382683432365089772f : 0.0f;
}
// w16^e = exp(-+2 pi i e / 16) for e = 0..15 as (cos, sin) with the sign of the transform
template <bool INV>
__device__ __forceinline__ float2 w16(int e)
{
    e &= 15;
    const int q = e & 3, quad = e >> 2;      // e = 4 quad + q
    // exp(-2 pi i e/16) = (-i)^quad * (cos(2 pi q/16) - i sin(2 pi q/16))
    float cr = c16(q), ci = -c16(4 - q);
    for (int t = 0; t < quad; ++t) {          // multiply by -i: (a, b) -> (b, -a)
        const float a = cr;
        cr = ci;
        ci = -a;
    }
    return INV ? make_float2(cr, -ci) : make_float2(cr, ci);
}

// In-register 4-point DFT on v[o], v[o+st], v[o+2st], v[o+3st].
template <bool INV, int N>
__device__ __forceinline__ void dft4_at(float2 (&v)[N], int o, int st)
{
    const float2 a = cadd(v[o], v[o + 2 * st]), b = csub(v[o], v[o + 2 * st]);
    const float2 c = cadd(v[o + st], v[o + 3 * st]), d = rot_i<INV>(csub(v[o + st], v[o + 3 * st]));
    v[o] = cadd(a, c);
    v[o + 2 * st] = csub(a, c);
    v[o + st] = cadd(b, d);
    v[o + 3 * st] = csub(b, d);
}

// In-register R-point DFT, y_q = sum_t x_t w^(t q), w = exp(-+2 pi i / R).
template <int R, bool INV>
__device__ __forceinline__ void small_dft(float2 (&v)[R])
{
    if constexpr (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        dft4_at<INV>(v, 0, 1);
    } else if constexpr (R == 8) {
        // 8 = 4 x 2: t = 2 t1 + t2; DFT4 over t1 (stride 2) for each t2, twiddle w8^(t2 k1),
        // DFT2 over t2; y[k1 + 4 k2] lands at v[2 k1 + k2] before the final reorder.
        dft4_at<INV>(v, 0, 2);
        dft4_at<INV>(v, 1, 2);
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1) v[2 * k1 + 1] = cmul(v[2 * k1 + 1], w16<INV>(2 * k1));
        float2 y[8];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            y[k1] = cadd(v[2 * k1], v[2 * k1 + 1]);
            y[k1 + 4] = csub(v[2 * k1], v[2 * k1 + 1]);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = y[k];
    } else if constexpr (R == 16) {
        // 16 = 4 x 4: t = 4 t1 + t2; DFT4 over t1 (stride 4) for each t2, twiddle
        // w16^(t2 k1), DFT4 over t2; y[k1 + 4 k2] lands at v[4 k1 + k2] before the reorder.
#pragma unroll
        for (int t2 = 0; t2 < 4; ++t2) dft4_at<INV>(v, t2, 4);
        // after the first pass v[4 k1 + t2] holds sub-DFT output k1 of column t2
#pragma unroll
        for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
            for (int t2 = 1; t2 < 4; ++t2) v[4 * k1 + t2] = cmul(v[4 * k1 + t2], w16<INV>(k1 * t2));
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4_at<INV>(v, 4 * k1, 1);
        float2 y[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = y[k];
    } else {
        // odd R: pair t with R-t; y_q = x0 + sum_t [(x_t + x_{R-t}) cos -/+ i (x_t - x_{R-t}) sin]
        constexpr int h = (R - 1) / 2;
        float2 s[h + 1], d[h + 1];
#pragma unroll
        for (int t = 1; t <= h; ++t) {
            s[t] = cadd(v[t], v[R - t]);
            d[t] = csub(v[t], v[R - t]);
        }
        const float2 x0 = v[0];
        float2 y0 = x0;
#pragma unroll
        for (int t = 1; t <= h; ++t) y0 = cadd(y0, s[t]);
#pragma unroll
        for (int q = 1; q <= h; ++q) {
            float2 re = x0, im = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 1; t <= h; ++t) {
                const int k = (t * q) % R;
                const float c = root_cos(R, k <= h ? k : R - k);
                const float sn = (k <= h ? 1.f : -1.f) * root_sin(R, k <= h ? k : R - k);
                re.x = fmaf(s[t].x, c, re.x);
                re.y = fmaf(s[t].y, c, re.y);
                im.x = fmaf(d[t].x, sn, im.x);
                im.y = fmaf(d[t].y, sn, im.y);
            }
            const float2 r = rot_i<INV>(im);  // -i*im forward, +i*im inverse
            v[q] = cadd(re, r);
            v[R - q] = csub(re, r);
        }
        v[0] = y0;
    }
}

// One decimation-in-frequency stage over blocks of length R*m:
//   inputs x[base + t m], base = blk*(R m) + j;  R-point DFT;  output q times w_(R m)^(j q).
// blk = b / m comes from a multiply-high by the plan's magic number (no integer division).
template <int R>
__device__ __forceinline__ void dif_stage(float2* __restrict__ x, int lgc, int Lw, int m,
                                          unsigned magic, int tw_step,
                                          const float2* __restrict__ tw)
{
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(Lw / R) << lgc;
    const unsigned um = (unsigned)m, lblk = um * R;
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned bi = b >> lgc;
        const unsigned blk = magic ? __umulhi(bi, magic) : bi;
        const unsigned j = bi - blk * um;
        const unsigned base = blk * lblk + j;
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = x[((base + t * um) << lgc) + col];
        small_dft<R, false>(v);
        const unsigned jt = j * (unsigned)tw_step;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 w = q ? tw[q * jt] : make_float2(1.f, 0.f);
            x[((base + q * um) << lgc) + col] = q ? cmul(v[q], w) : v[q];
        }
    }
}

// The inverse of dif_stage (up to the factor R): inputs times conj(w_(R m)^(j q)), inverse DFT.
template <int R>
__device__ __forceinline__ void dit_inv_stage(float2* __restrict__ x, int lgc, int Lw, int m,
                                              unsigned magic, int tw_step,
                                              const float2* __restrict__ tw)
{
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(Lw / R) << lgc;
    const unsigned um = (unsigned)m, lblk = um * R;
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned bi = b >> lgc;
        const unsigned blk = magic ? __umulhi(bi, magic) : bi;
        const unsigned j = bi - blk * um;
        const unsigned base = blk * lblk + j;
        const unsigned jt = j * (unsigned)tw_step;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 a = x[((base + q * um) << lgc) + col];
            v[q] = q ? cmulc(a, tw[q * jt]) : a;
        }
        small_dft<R, true>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) x[((base + t * um) << lgc) + col] = v[t];
    }
}

// Two-level radix R = R1 x R2 (R1, R2 in {3, 5}): t = R2 t1 + t2, k = k1 + R1 k2.
//   Y[t2][k1] = DFT_R1 over t1 of x[R2 t1 + t2];  Y[t2][k1] *= w_R^(t2 k1);
//   y[k1 + R1 k2] = DFT_R2 over t2 of Y[t2][k1].
// w_R^e = tw[e L / R] from the plan's twiddle table (L is a multiple of R). The result stays in
// v with y[k] at v[two_level_slot<R1, R2>(k)], so no second register array is needed.
template <int R1, int R2>
__device__ __forceinline__ constexpr int two_level_slot(int k)
{
    return R2 * (k % R1) + k / R1;
}

template <int R1, int R2, bool INV>
__device__ __forceinline__ void dft_two_level(float2 (&v)[R1 * R2], const float2* __restrict__ tw,
                                              unsigned lr)
{
#pragma unroll
    for (int t2 = 0; t2 < R2; ++t2) {
        float2 a[R1];
#pragma unroll
        for (int t1 = 0; t1 < R1; ++t1) a[t1] = v[R2 * t1 + t2];
        small_dft<R1, INV>(a);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            float2 y = a[k1];
            if (t2 != 0 && k1 != 0) {
                const float2 w = tw[(unsigned)(t2 * k1) * lr];
                y = INV ? cmulc(y, w) : cmul(y, w);
            }
            v[R2 * k1 + t2] = y;
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 b[R2];
#pragma unroll
        for (int t2 = 0; t2 < R2; ++t2) b[t2] = v[R2 * k1 + t2];
        small_dft<R2, INV>(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[R2 * k1 + k2] = b[k2];
    }
}

template <int R1, int R2>
__device__ __forceinline__ void dif_stage2(float2* __restrict__ x, int lgc, int Lw, int m,
                                           unsigned magic, int tw_step,
                                           const float2* __restrict__ tw)
{
    constexpr int R = R1 * R2;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(Lw / R) << lgc;
    const unsigned um = (unsigned)m, lblk = um * R, lr = (unsigned)(Lw / R);
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned bi = b >> lgc;
        const unsigned blk = magic ? __umulhi(bi, magic) : bi;
        const unsigned j = bi - blk * um;
        const unsigned base = blk * lblk + j;
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = x[((base + t * um) << lgc) + col];
        dft_two_level<R1, R2, false>(v, tw, lr);
        const unsigned jt = j * (unsigned)tw_step;
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 y = v[two_level_slot<R1, R2>(q)];
            x[((base + q * um) << lgc) + col] = q ? cmul(y, tw[q * jt]) : y;
        }
    }
}

template <int R1, int R2>
__device__ __forceinline__ void dit_inv_stage2(float2* __restrict__ x, int lgc, int Lw, int m,
                                               unsigned magic, int tw_step,
                                               const float2* __restrict__ tw)
{
    constexpr int R = R1 * R2;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(Lw / R) << lgc;
    const unsigned um = (unsigned)m, lblk = um * R, lr = (unsigned)(Lw / R);
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned bi = b >> lgc;
        const unsigned blk = magic ? __umulhi(bi, magic) : bi;
        const unsigned j = bi - blk * um;
        const unsigned base = blk * lblk + j;
        const unsigned jt = j * (unsigned)tw_step;
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 a = x[((base + q * um) << lgc) + col];
            v[q] = q ? cmulc(a, tw[q * jt]) : a;
        }
        dft_two_level<R1, R2, true>(v, tw, lr);
#pragma unroll
        for (int t = 0; t < R; ++t) x[((base + t * um) << lgc) + col] = v[two_level_slot<R1, R2>(t)];
    }
}

__device__ __forceinline__ void direct_forward(float2* x, int lgc, const FftPlanDev& p,
                                               const float2* tw)
{
    const int Lw = p.L;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s], m = p.span[s];
        const unsigned mg = p.magic[s];
        const int tw_step = Lw / (m * R);
        switch (R) {
            case 16: dif_stage<16>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 15: dif_stage2<3, 5>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 9: dif_stage2<3, 3>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 8: dif_stage<8>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 4: dif_stage<4>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 2: dif_stage<2>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 3: dif_stage<3>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 5: dif_stage<5>(x, lgc, Lw, m, mg, tw_step, tw); break;
            default: dif_stage<7>(x, lgc, Lw, m, mg, tw_step, tw); break;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void direct_inverse(float2* x, int lgc, const FftPlanDev& p,
                                               const float2* tw)
{
    const int Lw = p.L;
    for (int s = p.nst - 1; s >= 0; --s) {
        const int R = p.radix[s], m = p.span[s];
        const unsigned mg = p.magic[s];
        const int tw_step = Lw / (m * R);
        switch (R) {
            case 16: dit_inv_stage<16>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 15: dit_inv_stage2<3, 5>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 9: dit_inv_stage2<3, 3>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 8: dit_inv_stage<8>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 4: dit_inv_stage<4>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 2: dit_inv_stage<2>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 3: dit_inv_stage<3>(x, lgc, Lw, m, mg, tw_step, tw); break;
            case 5: dit_inv_stage<5>(x, lgc, Lw, m, mg, tw_step, tw); break;
            default: dit_inv_stage<7>(x, lgc, Lw, m, mg, tw_step, tw); break;
        }
        __syncthreads();
    }
}

// Bluestein: X_k = c_k sum_n (x_n c_n) conj(c_{k-n}),  c_n = exp(-i pi n^2 / N).
// The inverse transform conjugates input and output.
template <bool INV>
__device__ __forceinline__ void bluestein(float2* x, int lgc, const FftPlanDev& p,
                                          const float2* tw)
{
    const int ncols = 1 << lgc;
    const int N = p.N, Lw = p.L;
    for (int i = threadIdx.x; i < (Lw << lgc); i += blockDim.x) {
        const int n = i >> lgc;
        float2 v = make_float2(0.f, 0.f);
        if (n < N) {
            float2 a = x[i];
            if (INV) a = cconj(a);
            v = cmul(a, __ldg(p.chirp + n));
        }
        x[i] = v;
    }
    __syncthreads();
    direct_forward(x, lgc, p, tw);
    for (int i = threadIdx.x; i < (Lw << lgc); i += blockDim.x)
        x[i] = cmul(x[i], __ldg(p.bhat + (i >> lgc)));
    __syncthreads();
    direct_inverse(x, lgc, p, tw);
    for (int i = threadIdx.x; i < (N << lgc); i += blockDim.x) {
        const float2 v = cmul(x[i], __ldg(p.chirp + (i >> lgc)));
        x[i] = INV ? cconj(v) : v;
    }
    __syncthreads();
    (void)ncols;
}

// Forward DFT of every column: natural input; frequency k ends at position perm[k].
__device__ __forceinline__ void fft_forward(float2* x, int lgc, const FftPlanDev& p,
                                            const float2* tw)
{
    if (p.bluestein) bluestein<false>(x, lgc, p, tw);
    else direct_forward(x, lgc, p, tw);
}

// Unnormalised inverse DFT: frequency k read from position perm[k]; natural output.
__device__ __forceinline__ void fft_inverse(float2* x, int lgc, const FftPlanDev& p,
                                            const float2* tw)
{
    if (p.bluestein) bluestein<true>(x, lgc, p, tw);
    else direct_inverse(x, lgc, p, tw);
}

}  // namespace blfls
