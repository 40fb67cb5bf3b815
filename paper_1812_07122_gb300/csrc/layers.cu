// Elementwise kernels of the LS model and of the base/detail applications.
//
// * k0_ls_residuals: the LS model of Section II-B (Eqs. 5-6) is BLF-LS with the guidance
//   gradients set to zero, so its residuals are e_x = 0 - D_x f and e_y = 0 - D_y f, and the
//   Fourier solve (K2-K4) then returns u = f + F^-1[lam F(D^T e) / (1 + lam L)]
//   = F^-1[F(f) / (1 + lam L)], which is Eq. 6.
// * k5_log: l = ln(max(f, floor)), the logarithmic image of the tone-mapping framework
//   (Section IV).
// * k5_layers: the epilogues of Section IV, detail enhancement out = f + m (f - u) and
//   log-domain tone mapping out = exp(c b + (l - b)).
// * k5_gauss_rows / k5_gauss_cols: the periodic separable Gaussian that gives rolling guidance
//   its first guidance image (Section III-D), rows then columns.
// All are HBM-bound streams (12 bytes per pixel for the first three); grid-stride loops over a
// persistent grid of a few CTAs per SM.
#include <algorithm>

#include "internal.h"

namespace blfls {

namespace {

constexpr int kStreamThreads = 256;

__global__ void __launch_bounds__(kStreamThreads) k0_ls_residuals(const float* __restrict__ f,
                                                                 float* __restrict__ ex,
                                                                 float* __restrict__ ey, int H,
                                                                 int W)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const float c = f[i];
        const float right = f[(size_t)y * W + (x + 1 == W ? 0 : x + 1)];
        const float down = f[(size_t)(y + 1 == H ? 0 : y + 1) * W + x];
        ex[i] = c - right;   // -(D_x f)
        ey[i] = c - down;    // -(D_y f)
    }
}

__global__ void __launch_bounds__(kStreamThreads) k5_log(const float* __restrict__ f,
                                                        float* __restrict__ l, size_t n,
                                                        float floor_v)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        l[i] = logf(fmaxf(f[i], floor_v));
}

// mode 0: out = f + s (f - u);  mode 1: out = exp(s u + (f - u)) with f the log image, u its base.
__global__ void __launch_bounds__(kStreamThreads) k5_layers(const float* f, const float* u,
                                                           float* out, size_t n, int mode, float s)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const float a = f[i], b = u[i];
        out[i] = mode == 0 ? fmaf(s, a - b, a) : expf(fmaf(s, b, a - b));
    }
}

struct GaussTaps {
    int R;
    float w[2 * kMaxGaussR + 1];
};

__device__ __forceinline__ int wrap_mod(int i, int n)
{
    const int m = i % n;
    return m < 0 ? m + n : m;
}

__global__ void __launch_bounds__(kStreamThreads) k5_gauss_rows(const float* __restrict__ in,
                                                               float* __restrict__ out, int H,
                                                               int W, GaussTaps t)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        const float* row = in + (size_t)y * W;
        float acc = 0.f;
        for (int k = -t.R; k <= t.R; ++k) acc = fmaf(t.w[k + t.R], __ldg(row + wrap_mod(x + k, W)), acc);
        out[i] = acc;
    }
}

__global__ void __launch_bounds__(kStreamThreads) k5_gauss_cols(const float* __restrict__ in,
                                                               float* __restrict__ out, int H,
                                                               int W, GaussTaps t)
{
    const size_t n = (size_t)H * W;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / W), x = (int)(i - (size_t)y * W);
        float acc = 0.f;
        for (int k = -t.R; k <= t.R; ++k)
            acc = fmaf(t.w[k + t.R], __ldg(in + (size_t)wrap_mod(y + k, H) * W + x), acc);
        out[i] = acc;
    }
}

int stream_grid(size_t n, int num_sms)
{
    const size_t want = (n + kStreamThreads - 1) / kStreamThreads;
    const size_t cap = (size_t)num_sms * 8;
    return (int)std::max<size_t>(1, std::min(want, cap));
}

}  // namespace

cudaError_t launch_ls_residuals(const float* f, float* ex, float* ey, int H, int W,
                                cudaStream_t s, int num_sms)
{
    k0_ls_residuals<<<stream_grid((size_t)H * W, num_sms), kStreamThreads, 0, s>>>(f, ex, ey, H, W);
    return cudaGetLastError();
}

cudaError_t launch_log_image(const float* f, float* l, size_t n, float floor_v, cudaStream_t s,
                             int num_sms)
{
    k5_log<<<stream_grid(n, num_sms), kStreamThreads, 0, s>>>(f, l, n, floor_v);
    return cudaGetLastError();
}

cudaError_t launch_layer_epilogue(int mode, const float* f, const float* u, float* out, size_t n,
                                  float strength, cudaStream_t s, int num_sms)
{
    k5_layers<<<stream_grid(n, num_sms), kStreamThreads, 0, s>>>(f, u, out, n, mode, strength);
    return cudaGetLastError();
}

cudaError_t launch_gaussian(const float* in, float* tmp, float* out, int H, int W, const float* w,
                            int R, cudaStream_t s, int num_sms)
{
    if (R < 0 || R > kMaxGaussR) return cudaErrorInvalidValue;
    GaussTaps t;
    t.R = R;
    for (int k = 0; k <= 2 * R; ++k) t.w[k] = w[k];
    const int grid = stream_grid((size_t)H * W, num_sms);
    k5_gauss_rows<<<grid, kStreamThreads, 0, s>>>(in, tmp, H, W, t);
    k5_gauss_cols<<<grid, kStreamThreads, 0, s>>>(tmp, out, H, W, t);
    return cudaGetLastError();
}

}  // namespace blfls
