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
// convolution of length L >= 2N-1 (the smallest 7-smooth such L) carried out by the direct
// transforms; input and output are in natural order, positions [N, L) are scratch.
#pragma once

#include "dcheck.cuh"
#include "internal.h"

#include <type_traits>
#include <utility>

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
// Complex add / subtract as one packed f32x2 operation (two IEEE round-to-nearest FP32 results,
// the same values as two scalar operations in half the issue slots).
__device__ __forceinline__ float2 cadd(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\tmov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
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

// a * w16^e (e = 0..15, sign of the transform); the roots +-1 and +-i as a swap and signs.
template <bool INV>
__device__ __forceinline__ float2 mul_w16(float2 a, int e)
{
    e &= 15;
    if (e == 0) return a;
    if ((e & 3) == 0) {
        // exp(-+i pi e / 8) = (-+i)^(e / 4)
        const int quad = e >> 2;
        if (quad == 2) return make_float2(-a.x, -a.y);
        return (quad == 1) != INV ? rot_i<false>(a) : rot_i<true>(a);
    }
    return cmul(a, w16<INV>(e));
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
        for (int k1 = 1; k1 < 4; ++k1) v[2 * k1 + 1] = mul_w16<INV>(v[2 * k1 + 1], 2 * k1);
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
            for (int t2 = 1; t2 < 4; ++t2) v[4 * k1 + t2] = mul_w16<INV>(v[4 * k1 + t2], k1 * t2);
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

// cos and sin of 2 pi e / R for the internal twiddles of the two-level butterflies
// (R = 15: e = 1, 2, 3, 4, 6, 8; R = 9: e = 1, 2, 4; mathematical constants).
__device__ __forceinline__ constexpr float root2_cos(int R, int e)
{
    return R == 15 ? (e == 1 ? 0.913545457642600895502f : e == 2 ? 0.669130606358858213826f
                    : e == 3 ? 0.309016994374947424102f : e == 4 ? -0.104528463267653471400f
                    : e == 6 ? -0.809016994374947424102f : -0.978147600733805637929f)
                   : (e == 1 ? 0.766044443118978035202f : e == 2 ? 0.173648177666930348852f
                    : -0.939692620785908384054f);
}
__device__ __forceinline__ constexpr float root2_sin(int R, int e)
{
    return R == 15 ? (e == 1 ? 0.406736643075800207754f : e == 2 ? 0.743144825477394235015f
                    : e == 3 ? 0.951056516295153572116f : e == 4 ? 0.994521895368273336923f
                    : e == 6 ? 0.587785252292473129169f : -0.207911690817759337102f)
                   : (e == 1 ? 0.642787609686539326323f : e == 2 ? 0.984807753012208059367f
                    : 0.342020143325668733044f);
}

// Two-level radix R = R1 x R2 (R1, R2 in {3, 5}): t = R2 t1 + t2, k = k1 + R1 k2.
//   Y[t2][k1] = DFT_R1 over t1 of x[R2 t1 + t2];  Y[t2][k1] *= w_R^(t2 k1);
//   y[k1 + R1 k2] = DFT_R2 over t2 of Y[t2][k1].
// The result stays in v with y[k] at v[slot(k)], so no second register array is needed.
template <int R1, int R2>
struct TwoLevel {
    static constexpr int R = R1 * R2;
    static constexpr int F = R1;   // outer twiddles from w^e and w^(R1 e), see twiddle_powers
    static __device__ __forceinline__ constexpr int slot(int k) { return R2 * (k % R1) + k / R1; }
    template <bool INV>
    static __device__ __forceinline__ void dft(float2 (&v)[R])
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
                    const int e = t2 * k1;   // w_R^e = (cos, -sin) forward, (cos, sin) inverse
                    const float2 w = make_float2(root2_cos(R, e), root2_sin(R, e));
                    y = INV ? cmul(y, w) : cmulc(y, w);
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
};

// A plain R-point butterfly in the same interface (output k at v[k]).
template <int R_>
struct OneLevel {
    static constexpr int R = R_;
    // outer twiddles from w^e and w^(4 e) for R = 4, 8, 16; table loads for the small odd radices
    static constexpr int F = (R_ == 4 || R_ == 8 || R_ == 16) ? 4 : 0;
    static __device__ __forceinline__ constexpr int slot(int k) { return k; }
    template <bool INV>
    static __device__ __forceinline__ void dft(float2 (&v)[R]) { small_dft<R, INV>(v); }
};

// Outer twiddles w^(e q), q = 0..R-1, of one butterfly.  With F > 0 only two table entries are
// read, a = w^e and b = w^(F e), and w^(e q) = a^(q mod F) * b^(q div F): each is a product of
// at most four rounded factors (a few ulps), and the table reads drop from R-1 to 2.  With F = 0
// every w^(e q) is read from the table.  e < L / R, so F e < L stays inside the table.
template <int R, int F>
__device__ __forceinline__ void twiddle_powers(float2 (&w)[R], const float2* __restrict__ tw,
                                               unsigned e)
{
    if constexpr (F == 0) {
        w[0] = make_float2(1.f, 0.f);
#pragma unroll
        for (int q = 1; q < R; ++q) w[q] = tw[q * e];
    } else {
        constexpr int G = (R + F - 1) / F;
        float2 ap[F], bp[G];
        ap[0] = make_float2(1.f, 0.f);
        ap[1] = tw[e];
#pragma unroll
        for (int k = 2; k < F; ++k) ap[k] = (k % 2 == 0) ? cmul(ap[k / 2], ap[k / 2]) : cmul(ap[k - 1], ap[1]);
        bp[0] = make_float2(1.f, 0.f);
        if constexpr (G > 1) {
            bp[1] = tw[F * e];
#pragma unroll
            for (int k = 2; k < G; ++k) bp[k] = (k % 2 == 0) ? cmul(bp[k / 2], bp[k / 2]) : cmul(bp[k - 1], bp[1]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int k1 = q % F, k2 = q / F;
            w[q] = k2 == 0 ? ap[k1] : k1 == 0 ? bp[k2] : cmul(ap[k1], bp[k2]);
        }
    }
}

// One decimation-in-frequency stage over blocks of length R*m:
//   inputs x[base + t m], base = blk*(R m) + j;  R-point DFT;  output q times w_(R m)^(j q).
// blk = b / m comes from a multiply-high by the plan's magic number (no integer division).
// The last stage (m = 1) has j = 0, so its twiddles are all 1 and are skipped.
// LGC >= 0 fixes the column-set shift at compile time; LGC = -1 takes it from `lgc_rt`.
// PAD (rows, lgc = 0) addresses a row buffer padded as described at FftPlanDev::pad_span.
template <class B, int LGC, bool PAD>
__device__ __forceinline__ void dif_stage(float2* __restrict__ x, int lgc_rt, int Lw, int m,
                                          unsigned magic, int tw_step,
                                          const float2* __restrict__ tw, int pad_span,
                                          unsigned pad_magic)
{
    constexpr int R = B::R;
    const int lgc = LGC >= 0 ? LGC : lgc_rt;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(Lw / R) << lgc;
    const unsigned um = (unsigned)m, lblk = um * R;
    const bool twiddled = m > 1;
    const bool pad = PAD && pad_span > 0;
    const unsigned limit = ((unsigned)Lw << lgc) + (pad ? (unsigned)(Lw / pad_span) : 0u);
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned bi = b >> lgc;
        const unsigned blk = magic ? __umulhi(bi, magic) : bi;
        const unsigned j = bi - blk * um;
        unsigned base = blk * lblk + j;
        unsigned st = um << lgc;
        if (pad) {   // the butterfly lies inside one span-S block (stage 0: one element per block)
            base += __umulhi(base, pad_magic);
            if (um == (unsigned)pad_span) st = um + 1;
        }
        if (!BLFLS_DCHECK((base << lgc) + col + (R - 1) * st < limit, kDcFftStage)) continue;
        float2* xb = x + ((base << lgc) + col);
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = xb[t * st];
        B::template dft<false>(v);
        if (twiddled) {
            float2 w[R];
            twiddle_powers<R, B::F>(w, tw, j * (unsigned)tw_step);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float2 y = v[B::slot(q)];
                xb[q * st] = q ? cmul(y, w[q]) : y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) xb[q * st] = v[B::slot(q)];
        }
    }
}

// The inverse of dif_stage (up to the factor R): inputs times conj(w_(R m)^(j q)), inverse DFT.
template <class B, int LGC, bool PAD>
__device__ __forceinline__ void dit_inv_stage(float2* __restrict__ x, int lgc_rt, int Lw, int m,
                                              unsigned magic, int tw_step,
                                              const float2* __restrict__ tw, int pad_span,
                                              unsigned pad_magic)
{
    constexpr int R = B::R;
    const int lgc = LGC >= 0 ? LGC : lgc_rt;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(Lw / R) << lgc;
    const unsigned um = (unsigned)m, lblk = um * R;
    const bool twiddled = m > 1;
    const bool pad = PAD && pad_span > 0;
    const unsigned limit = ((unsigned)Lw << lgc) + (pad ? (unsigned)(Lw / pad_span) : 0u);
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned bi = b >> lgc;
        const unsigned blk = magic ? __umulhi(bi, magic) : bi;
        const unsigned j = bi - blk * um;
        unsigned base = blk * lblk + j;
        unsigned st = um << lgc;
        if (pad) {   // the butterfly lies inside one span-S block (stage 0: one element per block)
            base += __umulhi(base, pad_magic);
            if (um == (unsigned)pad_span) st = um + 1;
        }
        if (!BLFLS_DCHECK((base << lgc) + col + (R - 1) * st < limit, kDcFftStage)) continue;
        float2* xb = x + ((base << lgc) + col);
        float2 v[R];
        if (twiddled) {
            float2 w[R];
            twiddle_powers<R, B::F>(w, tw, j * (unsigned)tw_step);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float2 a = xb[q * st];
                v[q] = q ? cmulc(a, w[q]) : a;
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = xb[q * st];
        }
        B::template dft<true>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) xb[t * st] = v[B::slot(t)];
    }
}

template <int LGC, bool PAD>
__device__ __forceinline__ void direct_forward(float2* x, int lgc, const FftPlanDev& p,
                                               const float2* tw)
{
    const int Lw = p.L;
    for (int s = 0; s < p.nst; ++s) {
        const int R = p.radix[s], m = p.span[s];
        const unsigned mg = p.magic[s];
        const int tw_step = Lw / (m * R);
        switch (R) {
            case 16: dif_stage<OneLevel<16>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 15: dif_stage<TwoLevel<3, 5>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 9: dif_stage<TwoLevel<3, 3>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 8: dif_stage<OneLevel<8>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 4: dif_stage<OneLevel<4>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 2: dif_stage<OneLevel<2>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 3: dif_stage<OneLevel<3>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 5: dif_stage<OneLevel<5>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            default: dif_stage<OneLevel<7>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
        }
        __syncthreads();
    }
}

template <int LGC, bool PAD>
__device__ __forceinline__ void direct_inverse(float2* x, int lgc, const FftPlanDev& p,
                                               const float2* tw)
{
    const int Lw = p.L;
    for (int s = p.nst - 1; s >= 0; --s) {
        const int R = p.radix[s], m = p.span[s];
        const unsigned mg = p.magic[s];
        const int tw_step = Lw / (m * R);
        switch (R) {
            case 16: dit_inv_stage<OneLevel<16>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 15: dit_inv_stage<TwoLevel<3, 5>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 9: dit_inv_stage<TwoLevel<3, 3>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 8: dit_inv_stage<OneLevel<8>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 4: dit_inv_stage<OneLevel<4>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 2: dit_inv_stage<OneLevel<2>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 3: dit_inv_stage<OneLevel<3>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            case 5: dit_inv_stage<OneLevel<5>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
            default: dit_inv_stage<OneLevel<7>, LGC, PAD>(x, lgc, Lw, m, mg, tw_step, tw, p.pad_span, p.pad_magic); break;
        }
        __syncthreads();
    }
}

// Bluestein: X_k = c_k sum_n (x_n c_n) conj(c_{k-n}),  c_n = exp(-i pi n^2 / N).
// The inverse transform conjugates input and output.
template <bool INV, int LGC>
__device__ __forceinline__ void bluestein(float2* x, int lgc, const FftPlanDev& p,
                                          const float2* tw)
{
    if (LGC >= 0) lgc = LGC;
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
    direct_forward<LGC, false>(x, lgc, p, tw);
    for (int i = threadIdx.x; i < (Lw << lgc); i += blockDim.x)
        x[i] = cmul(x[i], __ldg(p.bhat + (i >> lgc)));
    __syncthreads();
    direct_inverse<LGC, false>(x, lgc, p, tw);
    for (int i = threadIdx.x; i < (N << lgc); i += blockDim.x) {
        const float2 v = cmul(x[i], __ldg(p.chirp + (i >> lgc)));
        x[i] = INV ? cconj(v) : v;
    }
    __syncthreads();
}

// ---- Bluestein with its pointwise passes folded into the stages ---------------------------
// The same values as `bluestein` (operation for operation), in 2 nst - 1 passes over shared
// memory instead of 2 nst + 3: the chirp pre-multiply (and the zero padding beyond N) is taken in
// the loads of the first forward stage, the multiply by the kernel spectrum between the last
// forward stage and the first inverse stage (one butterfly, in registers: that stage has span 1),
// and the chirp post-multiply in the stores of the last inverse stage.  Plans of two or more
// stages (a one-stage plan takes `bluestein`).

template <class F>
__device__ __forceinline__ void with_radix(int R, F&& f)
{
    switch (R) {
        case 16: f(OneLevel<16>{}); break;
        case 15: f(TwoLevel<3, 5>{}); break;
        case 9: f(TwoLevel<3, 3>{}); break;
        case 8: f(OneLevel<8>{}); break;
        case 4: f(OneLevel<4>{}); break;
        case 2: f(OneLevel<2>{}); break;
        case 3: f(OneLevel<3>{}); break;
        case 5: f(OneLevel<5>{}); break;
        default: f(OneLevel<7>{}); break;
    }
}

// Forward stage 0 with the chirp in its loads: input n is conj^INV(x_n) c_n for n < N, 0 beyond.
template <class B, bool INV>
__device__ __forceinline__ void blue_first_stage(float2* __restrict__ x, int lgc,
                                                 const FftPlanDev& p, const float2* __restrict__ tw)
{
    constexpr int R = B::R;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned m = (unsigned)p.span[0];
    const unsigned total = (unsigned)(p.L / R) << lgc;
    const unsigned st = m << lgc;
    const unsigned N = (unsigned)p.N;
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned j = b >> lgc;                       // stage 0: one block, base = j
        if (!BLFLS_DCHECK(((j + (R - 1) * m) << lgc) + col < ((unsigned)p.L << lgc), kDcFftStage))
            continue;
        float2* xb = x + ((j << lgc) + col);
        float2 v[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const unsigned n = j + t * m;
            float2 a = make_float2(0.f, 0.f);
            if (n < N) {
                a = xb[t * st];
                if (INV) a = cconj(a);
                a = cmul(a, __ldg(p.chirp + n));
            }
            v[t] = a;
        }
        B::template dft<false>(v);
        float2 w[R];
        twiddle_powers<R, B::F>(w, tw, j);                 // tw_step of stage 0 is 1
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 y = v[B::slot(q)];
            xb[q * st] = q ? cmul(y, w[q]) : y;
        }
    }
    __syncthreads();
}

// Last forward stage (span 1), times the kernel spectrum, then its inverse.
template <class B>
__device__ __forceinline__ void blue_middle_stage(float2* __restrict__ x, int lgc,
                                                  const FftPlanDev& p)
{
    constexpr int R = B::R;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned total = (unsigned)(p.L / R) << lgc;
    const unsigned st = 1u << lgc;
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned base = (b >> lgc) * R;
        if (!BLFLS_DCHECK(((base + R - 1) << lgc) + col < ((unsigned)p.L << lgc), kDcFftStage))
            continue;
        float2* xb = x + ((base << lgc) + col);
        float2 v[R], a[R];
#pragma unroll
        for (int t = 0; t < R; ++t) v[t] = xb[t * st];
        B::template dft<false>(v);
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = cmul(v[B::slot(q)], __ldg(p.bhat + base + q));
        B::template dft<true>(a);
#pragma unroll
        for (int t = 0; t < R; ++t) xb[t * st] = a[B::slot(t)];
    }
    __syncthreads();
}

// Inverse stage 0 with the chirp in its stores: output n < N becomes conj^INV(y_n c_n).
template <class B, bool INV>
__device__ __forceinline__ void blue_last_stage(float2* __restrict__ x, int lgc,
                                                const FftPlanDev& p, const float2* __restrict__ tw)
{
    constexpr int R = B::R;
    const unsigned mask = (1u << lgc) - 1u;
    const unsigned m = (unsigned)p.span[0];
    const unsigned total = (unsigned)(p.L / R) << lgc;
    const unsigned st = m << lgc;
    const unsigned N = (unsigned)p.N;
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b & mask;
        const unsigned j = b >> lgc;
        if (!BLFLS_DCHECK(((j + (R - 1) * m) << lgc) + col < ((unsigned)p.L << lgc), kDcFftStage))
            continue;
        float2* xb = x + ((j << lgc) + col);
        float2 w[R], v[R];
        twiddle_powers<R, B::F>(w, tw, j);
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const float2 a = xb[q * st];
            v[q] = q ? cmulc(a, w[q]) : a;
        }
        B::template dft<true>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const unsigned n = j + t * m;
            if (n < N) {
                const float2 o = cmul(v[B::slot(t)], __ldg(p.chirp + n));
                xb[t * st] = INV ? cconj(o) : o;
            }
        }
    }
    __syncthreads();
}

// Not inlined: one copy serves every driver (the runtime column shift), which keeps the nine
// radices of its five stage kinds out of each kernel's compilation.
template <bool INV>
__device__ __noinline__ void bluestein_fused(float2* x, int lgc, const FftPlanDev& p,
                                             const float2* tw)
{
    const int Lw = p.L, nl = p.nst - 1;
    with_radix(p.radix[0], [&](auto bf) { blue_first_stage<decltype(bf), INV>(x, lgc, p, tw); });
    for (int s = 1; s < nl; ++s) {
        const int R = p.radix[s], m = p.span[s];
        const unsigned mg = p.magic[s];
        with_radix(R, [&](auto bf) {
            dif_stage<decltype(bf), -1, false>(x, lgc, Lw, m, mg, Lw / (m * R), tw, 0, 0u);
        });
        __syncthreads();
    }
    with_radix(p.radix[nl], [&](auto bf) { blue_middle_stage<decltype(bf)>(x, lgc, p); });
    for (int s = nl - 1; s >= 1; --s) {
        const int R = p.radix[s], m = p.span[s];
        const unsigned mg = p.magic[s];
        with_radix(R, [&](auto bf) {
            dit_inv_stage<decltype(bf), -1, false>(x, lgc, Lw, m, mg, Lw / (m * R), tw, 0, 0u);
        });
        __syncthreads();
    }
    with_radix(p.radix[0], [&](auto bf) { blue_last_stage<decltype(bf), INV>(x, lgc, p, tw); });
}

// Forward DFT of every column: natural input; frequency k ends at position perm[k].
// LGC >= 0 fixes lgc at compile time (rows: 0); LGC = -1 reads it at run time.  PAD: x is a
// padded row buffer (Bluestein plans have no padding).
template <int LGC = -1, bool PAD = false>
__device__ __forceinline__ void fft_forward(float2* x, int lgc, const FftPlanDev& p,
                                            const float2* tw)
{
    if (p.bluestein) {
        if (p.nst >= 2) bluestein_fused<false>(x, LGC >= 0 ? LGC : lgc, p, tw);
        else bluestein<false, LGC>(x, lgc, p, tw);
    } else {
        direct_forward<LGC, PAD>(x, lgc, p, tw);
    }
}

// Unnormalised inverse DFT: frequency k read from position perm[k]; natural output.
template <int LGC = -1, bool PAD = false>
__device__ __forceinline__ void fft_inverse(float2* x, int lgc, const FftPlanDev& p,
                                            const float2* tw)
{
    if (p.bluestein) {
        if (p.nst >= 2) bluestein_fused<true>(x, LGC >= 0 ? LGC : lgc, p, tw);
        else bluestein<true, LGC>(x, lgc, p, tw);
    } else {
        direct_inverse<LGC, PAD>(x, lgc, p, tw);
    }
}

// Buffer index of work position q in a padded row buffer.
__device__ __forceinline__ unsigned row_pos(const FftPlanDev& p, unsigned q)
{
    return p.pad_span ? q + __umulhi(q, p.pad_magic) : q;
}

// ---------------------------------------------------------------------------------------------
// Compile-time plans.  For the common lengths the radix sequence is a template argument, so the
// butterfly spans, strides, twiddle steps, the divisions that locate a butterfly and the row
// padding are all constants (shared-memory offsets become immediates, divisions become
// multiply-shifts).  The arithmetic is the runtime plan's, operation for operation: the same
// butterflies, twiddle-table entries and memory layout, so the results are bit-identical.
// ---------------------------------------------------------------------------------------------
template <int... Rs>
struct CtPlan {
    static constexpr int nst = sizeof...(Rs);
    static constexpr int radix[nst] = {Rs...};
    static constexpr int L = (Rs * ...);
    static constexpr int span(int s)
    {
        int m = L;
        for (int k = 0; k <= s; ++k) m /= radix[k];
        return m;
    }
};

template <int R> struct Bfly { using type = OneLevel<R>; };
template <> struct Bfly<15> { using type = TwoLevel<3, 5>; };
template <> struct Bfly<9> { using type = TwoLevel<3, 3>; };

// One stage of a compile-time plan of length L: radix R, span M, NC interleaved columns
// (element n of column c at n NC + c; NC = 1 for a row), row padding span PADS (0: none); INV
// selects the inverse (dit_inv_stage) form.
template <int R, int M, int L, int NC, int PADS, bool INV>
__device__ __forceinline__ void ct_stage(float2* __restrict__ x, const float2* __restrict__ tw)
{
    using B = typename Bfly<R>::type;
    constexpr unsigned total = (unsigned)(L / R) * NC;
    constexpr unsigned lblk = (unsigned)M * R;
    constexpr unsigned st = (PADS > 0 && M == PADS) ? (unsigned)M + 1 : (unsigned)M * NC;
    constexpr unsigned tw_step = (unsigned)(L / (M * R));
    constexpr unsigned limit = (unsigned)L * NC + (PADS > 0 ? (unsigned)(L / PADS) : 0u);
    for (unsigned b = threadIdx.x; b < total; b += blockDim.x) {
        const unsigned col = b % (unsigned)NC;
        const unsigned bi = b / (unsigned)NC;
        const unsigned blk = bi / (unsigned)M;
        const unsigned j = bi - blk * (unsigned)M;
        unsigned base = blk * lblk + j;
        if constexpr (PADS > 0) base += base / (unsigned)PADS;
        if (!BLFLS_DCHECK(base * NC + col + (R - 1) * st < limit, kDcFftStage)) continue;
        float2* xb = x + (base * NC + col);
        float2 v[R];
        if constexpr (!INV) {
#pragma unroll
            for (int t = 0; t < R; ++t) v[t] = xb[t * st];
            B::template dft<false>(v);
            if constexpr (M > 1) {
                float2 w[R];
                twiddle_powers<R, B::F>(w, tw, j * tw_step);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float2 y = v[B::slot(q)];
                    xb[q * st] = q ? cmul(y, w[q]) : y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < R; ++q) xb[q * st] = v[B::slot(q)];
            }
        } else {
            if constexpr (M > 1) {
                float2 w[R];
                twiddle_powers<R, B::F>(w, tw, j * tw_step);
#pragma unroll
                for (int q = 0; q < R; ++q) {
                    const float2 a = xb[q * st];
                    v[q] = q ? cmulc(a, w[q]) : a;
                }
            } else {
#pragma unroll
                for (int q = 0; q < R; ++q) v[q] = xb[q * st];
            }
            B::template dft<true>(v);
#pragma unroll
            for (int t = 0; t < R; ++t) xb[t * st] = v[B::slot(t)];
        }
    }
    __syncthreads();
}

// Butterfly geometry of stage (R, M) of a compile-time plan, for drivers that move a
// butterfly's data between global memory, staging buffers and registers themselves (the first
// and last stages of a transform) instead of through ct_stage.  Butterfly b covers column
// `col` (b mod NC) and the natural positions nat + t M, t = 0..R-1; its elements sit at buffer
// offsets off + t st.  fwd / inv apply the butterfly and its twiddles in registers exactly as
// ct_stage does (same operations, same results).
template <int R, int M, int L, int NC, int PADS>
struct CtStage {
    using B = typename Bfly<R>::type;
    static constexpr unsigned total = (unsigned)(L / R) * NC;   // butterflies of all columns
    static constexpr unsigned st = (PADS > 0 && M == PADS) ? (unsigned)M + 1 : (unsigned)M * NC;
    static constexpr unsigned tw_step = (unsigned)(L / (M * R));
    static __device__ __forceinline__ void locate(unsigned b, unsigned& nat, unsigned& j,
                                                  unsigned& col)
    {
        col = b % (unsigned)NC;
        const unsigned bi = b / (unsigned)NC;
        const unsigned blk = bi / (unsigned)M;
        j = bi - blk * (unsigned)M;
        nat = blk * (unsigned)M * R + j;
    }
    static __device__ __forceinline__ unsigned offset(unsigned nat, unsigned col)
    {
        unsigned base = nat;
        if constexpr (PADS > 0) base += base / (unsigned)PADS;
        return base * NC + col;
    }
    // the butterfly at buffer offset off stays inside the transform buffer
    static __device__ __forceinline__ bool in_buffer(unsigned off)
    {
        constexpr unsigned limit = (unsigned)L * NC + (PADS > 0 ? (unsigned)(L / PADS) : 0u);
        return BLFLS_DCHECK(off + (R - 1) * st < limit, kDcFftStage);
    }
    // forward (decimation in frequency): v in input order t -> out[q] = DFT(v)_q w^(j q)
    static __device__ __forceinline__ void fwd(float2 (&v)[R], float2 (&out)[R],
                                               const float2* __restrict__ tw, unsigned j)
    {
        B::template dft<false>(v);
        if constexpr (M > 1) {
            float2 w[R];
            twiddle_powers<R, B::F>(w, tw, j * tw_step);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const float2 y = v[B::slot(q)];
                out[q] = q ? cmul(y, w[q]) : y;
            }
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) out[q] = v[B::slot(q)];
        }
    }
    // inverse: a in output order q -> out[t] = IDFT(a conj(w^(j q)))_t
    static __device__ __forceinline__ void inv(float2 (&a)[R], float2 (&out)[R],
                                               const float2* __restrict__ tw, unsigned j)
    {
        float2 v[R];
        if constexpr (M > 1) {
            float2 w[R];
            twiddle_powers<R, B::F>(w, tw, j * tw_step);
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = q ? cmulc(a[q], w[q]) : a[q];
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) v[q] = a[q];
        }
        B::template dft<true>(v);
#pragma unroll
        for (int t = 0; t < R; ++t) out[t] = v[B::slot(t)];
    }
};

// Frequency held at work position p after the forward transform of plan P (the digit reversal:
// p = sum_s q_s span(s)  <->  k = sum_s q_s R_0 ... R_{s-1}); the same as the plan's iperm table.
template <class P, int... S>
__device__ __forceinline__ int ct_frequency_digits(unsigned p, std::integer_sequence<int, S...>)
{
    int k = 0, w = 1;
    ((k += (int)(p / (unsigned)P::span(S)) * w, p %= (unsigned)P::span(S), w *= P::radix[S]), ...);
    return k;
}
template <class P>
__device__ __forceinline__ int ct_frequency(unsigned p)
{
    return ct_frequency_digits<P>(p, std::make_integer_sequence<int, P::nst>{});
}

// Work position of frequency k after the forward transform of plan P (the inverse of
// ct_frequency; the same as the plan's perm table).
template <class P, int... S>
__device__ __forceinline__ unsigned ct_position_digits(unsigned k, std::integer_sequence<int, S...>)
{
    unsigned p = 0;
    ((p += (k % (unsigned)P::radix[S]) * (unsigned)P::span(S), k /= (unsigned)P::radix[S]), ...);
    return p;
}
template <class P>
__device__ __forceinline__ unsigned ct_position(unsigned k)
{
    return ct_position_digits<P>(k, std::make_integer_sequence<int, P::nst>{});
}

// Stage s of plan P as a CtStage (NC interleaved columns).
template <class P, int S, int NC, int PADS>
using CtStageOf = CtStage<P::radix[S], P::span(S), P::L, NC, PADS>;

// Middle stages [S0, S1) of plan P through shared memory (forward, in order).
template <class P, int NC, int PADS, int S0, int... S>
__device__ __forceinline__ void ct_forward_range(float2* x, const float2* tw,
                                                 std::integer_sequence<int, S...>)
{
    (ct_stage<P::radix[S0 + S], P::span(S0 + S), P::L, NC, PADS, false>(x, tw), ...);
}
// Inverse stages S1-1 .. S0 of plan P through shared memory (in the inverse order).
template <class P, int NC, int PADS, int S1, int... S>
__device__ __forceinline__ void ct_inverse_range(float2* x, const float2* tw,
                                                 std::integer_sequence<int, S...>)
{
    (ct_stage<P::radix[S1 - 1 - S], P::span(S1 - 1 - S), P::L, NC, PADS, true>(x, tw), ...);
}

template <class P, int LGC, int PADS, int... S>
__device__ __forceinline__ void ct_forward_stages(float2* x, const float2* tw,
                                                  std::integer_sequence<int, S...>)
{
    (ct_stage<P::radix[S], P::span(S), P::L, (1 << LGC), PADS, false>(x, tw), ...);
}
template <class P, int LGC, int PADS, int... S>
__device__ __forceinline__ void ct_inverse_stages(float2* x, const float2* tw,
                                                  std::integer_sequence<int, S...>)
{
    (ct_stage<P::radix[P::nst - 1 - S], P::span(P::nst - 1 - S), P::L, (1 << LGC), PADS, true>(x, tw), ...);
}

// Forward / unnormalised inverse DFT of every column with plan P (PAD: a padded row buffer,
// lgc = 0; the padding span is L / radix[0] for plans of two or more stages).
template <class P, int LGC, bool PAD>
__device__ __forceinline__ void ct_forward(float2* x, const float2* tw)
{
    constexpr int PADS = (PAD && P::nst >= 2) ? P::L / P::radix[0] : 0;
    ct_forward_stages<P, LGC, PADS>(x, tw, std::make_integer_sequence<int, P::nst>{});
}
template <class P, int LGC, bool PAD>
__device__ __forceinline__ void ct_inverse(float2* x, const float2* tw)
{
    constexpr int PADS = (PAD && P::nst >= 2) ? P::L / P::radix[0] : 0;
    ct_inverse_stages<P, LGC, PADS>(x, tw, std::make_integer_sequence<int, P::nst>{});
}

// Forward / inverse through plan P when it is a CtPlan, else through the runtime plan `p`.
template <class P, int LGC, bool PAD>
__device__ __forceinline__ void fft_forward_p(float2* x, int lgc, const FftPlanDev& p,
                                              const float2* tw)
{
    if constexpr (std::is_void_v<P>) fft_forward<LGC, PAD>(x, lgc, p, tw);
    else ct_forward<P, LGC, PAD>(x, tw);
}
template <class P, int LGC, bool PAD>
__device__ __forceinline__ void fft_inverse_p(float2* x, int lgc, const FftPlanDev& p,
                                              const float2* tw)
{
    if constexpr (std::is_void_v<P>) fft_inverse<LGC, PAD>(x, lgc, p, tw);
    else ct_inverse<P, LGC, PAD>(x, tw);
}

}  // namespace blfls
