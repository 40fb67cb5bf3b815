// FFT plans for the Fourier solve of Eq. 8: factorisation, twiddles, digit-reversal tables and
// Bluestein chirps.  Every table is computed in FP64 on the host and stored as FP32.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

namespace blfls {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Digit-reversed position of every frequency for an in-place decimation-in-frequency FFT with
// stages radices[0..m-1]: k = q0 + R0 q1 + R0 R1 q2 + ...  sits at  sum_s q_s * (N / (R0..Rs)).
std::vector<int> dif_positions(int N, const std::vector<int>& radices)
{
    std::vector<int> pos(N);
    for (int k = 0; k < N; ++k) {
        int rem = k, span = N, p = 0;
        for (int R : radices) {
            const int q = rem % R;
            rem /= R;
            span /= R;
            p += q * span;
        }
        pos[k] = p;
    }
    return pos;
}

// Plain FP64 mixed-radix FFT for lengths whose prime factors are 2, 3, 5 and 7 (recursive
// decimation in time: n = p m with p the smallest prime factor), forward sign exp(-2 pi i nk/N).
// Roots come from one table of the L-th roots of unity (w_n^e = root[e L / n]), so a plan costs
// L cosines and sines.  `tmp` is scratch of n elements.
void fft_smooth_rec(std::complex<double>* a, size_t n, const std::vector<std::complex<double>>& root,
                    size_t rstep, std::complex<double>* tmp)
{
    if (n <= 1) return;
    size_t p = n;
    for (size_t q : {2, 3, 5, 7})
        if (n % q == 0) { p = q; break; }
    const size_t m = n / p;
    for (size_t r = 0; r < p; ++r)
        for (size_t t = 0; t < m; ++t) tmp[r * m + t] = a[t * p + r];
    for (size_t r = 0; r < p; ++r) fft_smooth_rec(tmp + r * m, m, root, rstep * p, a);
    // X[k + m q] = sum_r w_n^(r (k + m q)) S_r[k]
    for (size_t k = 0; k < m; ++k)
        for (size_t q = 0; q < p; ++q) {
            const size_t kk = k + m * q;
            std::complex<double> acc = tmp[k];
            for (size_t r = 1; r < p; ++r) acc += root[((r * kk) % n) * rstep] * tmp[r * m + k];
            a[kk] = acc;
        }
}

void host_fft_smooth(std::vector<std::complex<double>>& a)
{
    const size_t n = a.size();
    if (n <= 1) return;
    std::vector<std::complex<double>> root(n), tmp(n);
    for (size_t j = 0; j < n; ++j) {
        const double ang = -2.0 * kPi * double(j) / double(n);
        root[j] = std::complex<double>(std::cos(ang), std::sin(ang));
    }
    fft_smooth_rec(a.data(), n, root, 1, tmp.data());
}

// Work length of a Bluestein transform of length N: the smallest 7-smooth L >= 2N - 1 (the
// cyclic convolution needs L >= 2N - 1; the direct FFT handles every 7-smooth length).
int bluestein_length(int N)
{
    for (int L = std::max(1, 2 * N - 1);; ++L) {
        int r = L;
        for (int q : {2, 3, 5, 7})
            while (r % q == 0) r /= q;
        if (r == 1) return L;
    }
}

}  // namespace

bool factor_direct(int N, std::vector<int>& radices)
{
    radices.clear();
    if (N < 1) return false;
    int n = N;
    while (n % 16 == 0) { radices.push_back(16); n /= 16; }
    if (n % 8 == 0) { radices.push_back(8); n /= 8; }
    if (n % 4 == 0) { radices.push_back(4); n /= 4; }
    if (n % 2 == 0) { radices.push_back(2); n /= 2; }
    while (n % 15 == 0) { radices.push_back(15); n /= 15; }
    while (n % 9 == 0) { radices.push_back(9); n /= 9; }
    while (n % 3 == 0) { radices.push_back(3); n /= 3; }
    while (n % 5 == 0) { radices.push_back(5); n /= 5; }
    while (n % 7 == 0) { radices.push_back(7); n /= 7; }
    return n == 1 && int(radices.size()) <= kMaxStages;
}

// Row-buffer padding (see FftPlanDev::pad_span), with its multiply-high checked for every p < L.
static bool fill_padding(FftPlanDev& d)
{
    d.pad_span = 0;
    d.pad_magic = 0;
    if (d.bluestein || d.nst < 2) return true;
    const unsigned S = (unsigned)(d.L / d.radix[0]);
    const unsigned magic = (unsigned)((((unsigned long long)1 << 32) + S - 1) / S);
    for (unsigned q = 0; q < (unsigned)d.L; ++q)
        if ((unsigned)(((unsigned long long)q * magic) >> 32) != q / S) return false;
    d.pad_span = (int)S;
    d.pad_magic = magic;
    return true;
}

bool fill_stage_division(FftPlanDev& d)
{
    int span = d.L;
    for (int s = 0; s < d.nst; ++s) {
        span /= d.radix[s];
        d.span[s] = span;
        d.magic[s] = span == 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + span - 1) / span);
        if (span > 1) {
            // butterfly indices of one column reach L / radix[s]: check every quotient
            const unsigned nb = (unsigned)(d.L / d.radix[s]);
            for (unsigned b = 0; b < nb; ++b)
                if ((unsigned)(((unsigned long long)b * d.magic[s]) >> 32) != b / (unsigned)span)
                    return false;
        }
    }
    return true;
}

cudaError_t build_fft_plan(int N, FftPlanHost& out)
{
    out = FftPlanHost{};
    std::vector<unsigned char> blob;
    FftPlanDev rel;
    if (!build_fft_tables_host(N, blob, rel)) return cudaErrorInvalidValue;
    void* dmem = nullptr;
    cudaError_t e = cudaMalloc(&dmem, blob.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(dmem, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dmem);
        return e;
    }
    out.dev = bind_fft_tables(rel, dmem);
    out.dmem = dmem;
    out.bytes = blob.size();
    return cudaSuccess;
}

void free_fft_plan(FftPlanHost& p)
{
    if (p.dmem) cudaFree(p.dmem);
    p = FftPlanHost{};
}

// Every table of the plan of length N (twiddles, digit-reversal positions, Bluestein chirp and
// kernel spectrum, Laplacian eigenvalues), computed in FP64 and stored FP32, laid out in one host
// blob: tw | chirp | bhat | perm | iperm | lap | lapp, each 256-byte aligned.  `rel` receives the plan
// with every table pointer holding its byte offset inside the blob; bind_fft_tables turns those
// offsets into addresses once the blob sits at `base` (build_fft_plan uploads it to its own
// allocation, the allocation-free solve into its static array).
bool build_fft_tables_host(int N, std::vector<unsigned char>& blob, FftPlanDev& rel)
{
    rel = FftPlanDev{};
    rel.N = N;
    std::vector<int> radices;
    const bool direct = factor_direct(N, radices);
    int L = N;
    if (!direct) {
        L = bluestein_length(N);
        if (!factor_direct(L, radices)) return false;
    }
    if (L > kMaxFftLen) return false;
    rel.L = L;
    rel.bluestein = direct ? 0 : 1;
    rel.nst = int(radices.size());
    for (int s = 0; s < rel.nst; ++s) rel.radix[s] = radices[s];
    if (!fill_stage_division(rel) || !fill_padding(rel)) return false;

    std::vector<float2> tw(L);
    for (int m = 0; m < L; ++m) {
        const double ang = -2.0 * kPi * double(m) / double(L);
        tw[m] = make_float2(float(std::cos(ang)), float(std::sin(ang)));
    }
    const std::vector<int> posL = dif_positions(L, radices);
    std::vector<int> iperm(L);
    for (int k = 0; k < L; ++k) iperm[posL[k]] = k;
    std::vector<int> perm(N);
    std::vector<float2> chirp, bhat;
    if (direct) {
        perm = posL;
    } else {
        for (int k = 0; k < N; ++k) perm[k] = k;
        for (int p = 0; p < L; ++p) iperm[p] = p;
        // c_n = exp(-i pi n^2 / N), with n^2 reduced mod 2N in integers to keep the angle exact.
        std::vector<std::complex<double>> c(N);
        chirp.resize(N);
        for (int n = 0; n < N; ++n) {
            const long long q = (long long)n * n % (2LL * N);
            const double ang = -kPi * double(q) / double(N);
            c[n] = std::complex<double>(std::cos(ang), std::sin(ang));
            chirp[n] = make_float2(float(c[n].real()), float(c[n].imag()));
        }
        std::vector<std::complex<double>> b(L, 0.0);
        for (int n = 0; n < N; ++n) {
            b[n] = std::conj(c[n]);
            if (n > 0) b[L - n] = std::conj(c[n]);
        }
        host_fft_smooth(b);
        bhat.resize(L);
        for (int k = 0; k < L; ++k) {
            const std::complex<double> v = b[k] / double(L);
            bhat[posL[k]] = make_float2(float(v.real()), float(v.imag()));
        }
    }
    std::vector<float> lap(N);
    for (int k = 0; k < N; ++k) {
        const double sn = std::sin(kPi * double(k) / double(N));
        lap[k] = float(4.0 * sn * sn);
    }
    const size_t o_tw = 0;
    const size_t o_chirp = align256(o_tw + sizeof(float2) * L);
    const size_t o_bhat = align256(o_chirp + sizeof(float2) * chirp.size());
    const size_t o_perm = align256(o_bhat + sizeof(float2) * bhat.size());
    const size_t o_iperm = align256(o_perm + sizeof(int) * N);
    std::vector<float> lapp(L);
    for (int p = 0; p < L; ++p) lapp[p] = lap[iperm[p] % N];
    const size_t o_lap = align256(o_iperm + sizeof(int) * L);
    const size_t o_lapp = align256(o_lap + sizeof(float) * N);
    const size_t bytes = align256(o_lapp + sizeof(float) * L);
    blob.assign(bytes, 0);
    std::memcpy(blob.data() + o_tw, tw.data(), sizeof(float2) * L);
    if (!chirp.empty()) std::memcpy(blob.data() + o_chirp, chirp.data(), sizeof(float2) * N);
    if (!bhat.empty()) std::memcpy(blob.data() + o_bhat, bhat.data(), sizeof(float2) * L);
    std::memcpy(blob.data() + o_perm, perm.data(), sizeof(int) * N);
    std::memcpy(blob.data() + o_iperm, iperm.data(), sizeof(int) * L);
    std::memcpy(blob.data() + o_lap, lap.data(), sizeof(float) * N);
    std::memcpy(blob.data() + o_lapp, lapp.data(), sizeof(float) * L);
    rel.tw = reinterpret_cast<const float2*>(o_tw);
    rel.chirp = chirp.empty() ? nullptr : reinterpret_cast<const float2*>(o_chirp);
    rel.bhat = bhat.empty() ? nullptr : reinterpret_cast<const float2*>(o_bhat);
    rel.perm = reinterpret_cast<const int*>(o_perm);
    rel.iperm = reinterpret_cast<const int*>(o_iperm);
    rel.lap = reinterpret_cast<const float*>(o_lap);
    rel.lapp = reinterpret_cast<const float*>(o_lapp);
    return true;
}

FftPlanDev bind_fft_tables(const FftPlanDev& rel, const void* base)
{
    const unsigned char* b = static_cast<const unsigned char*>(base);
    FftPlanDev d = rel;
    d.tw = reinterpret_cast<const float2*>(b + reinterpret_cast<size_t>(rel.tw));
    d.chirp = rel.chirp ? reinterpret_cast<const float2*>(b + reinterpret_cast<size_t>(rel.chirp)) : nullptr;
    d.bhat = rel.bhat ? reinterpret_cast<const float2*>(b + reinterpret_cast<size_t>(rel.bhat)) : nullptr;
    d.perm = reinterpret_cast<const int*>(b + reinterpret_cast<size_t>(rel.perm));
    d.iperm = reinterpret_cast<const int*>(b + reinterpret_cast<size_t>(rel.iperm));
    d.lap = reinterpret_cast<const float*>(b + reinterpret_cast<size_t>(rel.lap));
    d.lapp = reinterpret_cast<const float*>(b + reinterpret_cast<size_t>(rel.lapp));
    return d;
}

}  // namespace blfls
