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
// Each phase is written once as a per-item device function (a row pair, or a block of columns)
// and driven either by a single-image persistent grid (twiddles staged in shared memory once per
// CTA) or by a batched persistent grid over the items of many jobs (twiddles read through L1,
// since consecutive items may belong to different transform lengths).  Both drivers run the
// same arithmetic, so a job's result does not depend on the batch it ran in.
#include "fft_device.cuh"

namespace blfls {

namespace {

// Shared-memory budget of one solve CTA; twiddles share it with the data when they fit.
constexpr size_t kSmemCap = 220 * 1024;

__device__ __forceinline__ const float2* stage_twiddles(float2* tw_smem, const FftPlanDev& p,
                                                        bool in_smem)
{
    if (!in_smem) return p.tw;
    for (int i = threadIdx.x; i < p.L; i += blockDim.x) tw_smem[i] = __ldg(p.tw + i);
    __syncthreads();
    return tw_smem;
}

// K2: row pair `pair` (rows 2 pair, 2 pair + 1) of one channel.
__device__ __forceinline__ void k2_item(const float* __restrict__ ex, const float* __restrict__ ey,
                                        float2* __restrict__ spec, int H, int W, int pair,
                                        const FftPlanDev& rp, const float2* tw, float2* data)
{
    const int Wh = W / 2 + 1;
    const int y0 = 2 * pair, y1 = y0 + 1;
    const bool has1 = y1 < H;
    const int ym = (y0 == 0) ? H - 1 : y0 - 1;
    const float* ex0 = ex + (size_t)y0 * W;
    const float* ey0 = ey + (size_t)y0 * W;
    const float* eym = ey + (size_t)ym * W;
    const float* ex1 = ex + (size_t)(has1 ? y1 : y0) * W;
    const float* ey1 = ey + (size_t)(has1 ? y1 : y0) * W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const int xm = (x == 0) ? W - 1 : x - 1;
        // (D_x^T e_x)[y][x] = e_x[y][x-1] - e_x[y][x];  (D_y^T e_y)[y][x] = e_y[y-1][x] - e_y[y][x]
        const float r0 = (__ldg(ex0 + xm) - __ldg(ex0 + x)) + (__ldg(eym + x) - __ldg(ey0 + x));
        float r1 = 0.f;
        if (has1) r1 = (__ldg(ex1 + xm) - __ldg(ex1 + x)) + (__ldg(ey0 + x) - __ldg(ey1 + x));
        data[x] = make_float2(r0, r1);
    }
    __syncthreads();
    fft_forward(data, 0, rp, tw);
    float2* s0 = spec + (size_t)y0 * Wh;
    float2* s1 = spec + (size_t)(has1 ? y1 : y0) * Wh;
    for (int k = threadIdx.x; k < Wh; k += blockDim.x) {
        const int kn = (k == 0) ? 0 : W - k;
        const float2 zk = data[__ldg(rp.perm + k)];
        const float2 zn = data[__ldg(rp.perm + kn)];
        // A = (Z_k + conj Z_{W-k}) / 2,  B = (Z_k - conj Z_{W-k}) / (2i)
        s0[k] = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
        if (has1) s1[k] = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    }
    __syncthreads();
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
        data[i] = (kx < Wh) ? spec[(size_t)n * Wh + kx] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_forward(data, lgc, cp, tw);
    // spectral divide (Eq. 8 denominator, F(1) = 1), with lam and the 1/(HW) of the inverse
    const int nfreq = cp.bluestein ? H : cp.L;
    for (int i = threadIdx.x; i < (nfreq << lgc); i += blockDim.x) {
        const int p = i >> lgc, c = i & (CB - 1);
        const int kx = min(kx0 + c, Wh - 1);
        const int ky = __ldg(cp.iperm + p);
        const float den = fmaf(lam, __ldg(sx + kx) + __ldg(sy + ky), 1.0f);
        const float m = __fdividef(scale, den) * lam;
        const float2 v = data[i];
        data[i] = make_float2(v.x * m, v.y * m);
    }
    __syncthreads();
    fft_inverse(data, lgc, cp, tw);
    for (int i = threadIdx.x; i < (H << lgc); i += blockDim.x) {
        const int n = i >> lgc, c = i & (CB - 1);
        const int kx = kx0 + c;
        if (kx < Wh) spec[(size_t)n * Wh + kx] = data[i];
    }
    __syncthreads();
}

// K4: row pair `pair` of one channel: u = f + inverse row FFT of the corrected spectrum.
__device__ __forceinline__ void k4_item(const float2* __restrict__ spec, const float* f, float* out,
                                        int H, int W, int pair, const FftPlanDev& rp,
                                        const float2* tw, float2* data)
{
    const int Wh = W / 2 + 1;
    const int y0 = 2 * pair, y1 = y0 + 1;
    const bool has1 = y1 < H;
    const float2* s0 = spec + (size_t)y0 * Wh;
    const float2* s1 = spec + (size_t)(has1 ? y1 : y0) * Wh;
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
        const bool upper = k > W / 2;
        const int kk = upper ? W - k : k;
        float2 a = s0[kk];
        float2 b = has1 ? s1[kk] : make_float2(0.f, 0.f);
        if (upper) { a.y = -a.y; b.y = -b.y; }
        if (k == 0 || 2 * k == W) { a.y = 0.f; b.y = 0.f; }  // real bins of a real row
        // Z = A + i B
        data[__ldg(rp.perm + k)] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    fft_inverse(data, 0, rp, tw);
    const float* f0 = f + (size_t)y0 * W;
    float* o0 = out + (size_t)y0 * W;
    for (int x = threadIdx.x; x < W; x += blockDim.x) {
        const float2 z = data[x];
        o0[x] = f0[x] + z.x;
        if (has1) out[(size_t)y1 * W + x] = f[(size_t)y1 * W + x] + z.y;
    }
    __syncthreads();
}

// ---- single image --------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k2_rows_forward(
    const float* __restrict__ ex, const float* __restrict__ ey, float2* __restrict__ spec,
    int H, int W, FftPlanDev rp, int tw_in_smem)
{
    extern __shared__ float2 smem[];
    const float2* tw = stage_twiddles(smem + rp.L, rp, tw_in_smem);
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
    const float2* tw = stage_twiddles(smem + rp.L, rp, tw_in_smem);
    const int npairs = (H + 1) / 2;
    for (int pair = blockIdx.x; pair < npairs; pair += gridDim.x)
        k4_item(spec, f, out, H, W, pair, rp, tw, smem);
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

int threads_for(int work)
{
    int t = 128;
    while (t < 512 && t * 4 < work) t *= 2;
    return t;
}

}  // namespace

void init_solve_kernel_attributes()
{
    cudaFuncSetAttribute(k2_rows_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k3_cols_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k4_rows_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k2_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k3_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(k4_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

size_t solve_smem_rows(const FftPlanDev& rp)
{
    const size_t data = sizeof(float2) * rp.L;
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

cudaError_t launch_solve_residual(const float* f, const float* ex, const float* ey, float* out,
                                  float2* spec, const FftPlanDev& rp, const FftPlanDev& cp,
                                  const float* sx, const float* sy, const SolveParams& p,
                                  cudaStream_t s, int num_sms, const cudaEvent_t* marks)
{
    const int H = p.H, W = p.W;
    const int lgc = solve_fit_lgc(cp.L, p.col_block);
    const int CB = 1 << lgc;

    const size_t smem_r = solve_smem_rows(rp);
    const int tw_r = smem_r > sizeof(float2) * rp.L;
    const int thr_r = threads_for(rp.L / 4);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2_rows_forward, thr_r, smem_r);
    const int npairs = (H + 1) / 2;
    const int grid_r = std::max(1, std::min(npairs, num_sms * std::max(occ, 1)));

    const size_t smem_c = solve_smem_cols(cp, CB);
    const int tw_c = smem_c > sizeof(float2) * (size_t)cp.L * CB;
    const int thr_c = threads_for((cp.L * CB) / 4);
    int occ_c = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k3_cols_solve, thr_c, smem_c);
    const int nblk = (W / 2 + 1 + CB - 1) / CB;
    const int grid_c = std::max(1, std::min(nblk, num_sms * std::max(occ_c, 1)));

    k2_rows_forward<<<grid_r, thr_r, smem_r, s>>>(ex, ey, spec, H, W, rp, tw_r);
    if (marks) cudaEventRecord(marks[0], s);
    const float scale = 1.0f / ((float)H * (float)W);
    k3_cols_solve<<<grid_c, thr_c, smem_c, s>>>(spec, H, W, cp, sx, sy, p.lambda, scale, lgc, tw_c);
    if (marks) cudaEventRecord(marks[1], s);
    k4_rows_inverse<<<grid_r, thr_r, smem_r, s>>>(spec, f, out, H, W, rp, tw_r);
    return cudaGetLastError();
}

cudaError_t launch_solve_batch(const BatchJob* jobs, int njobs, const int2* grp_rows,
                               int total_rows, const int2* grp_cols, int total_cols,
                               size_t smem_rows, size_t smem_cols, int num_sms, cudaStream_t s,
                               const cudaEvent_t* marks)
{
    if (total_rows <= 0) return cudaSuccess;
    const int thr = 256;
    int occ_r = 0, occ_c = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_r, k2_batch, thr, smem_rows);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, k3_batch, thr, smem_cols);
    const int grid_r = std::max(1, std::min(total_rows, num_sms * std::max(occ_r, 1)));
    const int grid_c = std::max(1, std::min(total_cols, num_sms * std::max(occ_c, 1)));
    k2_batch<<<grid_r, thr, smem_rows, s>>>(jobs, grp_rows, njobs, total_rows);
    if (marks) cudaEventRecord(marks[0], s);
    k3_batch<<<grid_c, thr, smem_cols, s>>>(jobs, grp_cols, njobs, total_cols);
    if (marks) cudaEventRecord(marks[1], s);
    k4_batch<<<grid_r, thr, smem_rows, s>>>(jobs, grp_rows, njobs, total_rows);
    return cudaGetLastError();
}

}  // namespace blfls
