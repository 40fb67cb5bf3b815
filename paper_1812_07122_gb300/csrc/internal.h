// Internal declarations shared by the BLF-LS CUDA sources (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace blfls {

// ---------------------------------------------------------------------------------------------
// FFT plans.  A transform of length N is either a direct in-place mixed-radix FFT (N factors
// into 16, 15, 9, 8, 4, 2, 3, 5, 7) or Bluestein's chirp-z algorithm over a direct FFT of the
// smallest 7-smooth length L >= 2N - 1.  The direct forward transform is decimation in
// frequency: natural-order input, output in mixed-radix digit-reversed order, so frequency k
// sits at position perm[k].  The inverse runs the conjugate stages in reverse order and takes
// that order back to natural.  Bluestein transforms use natural order on both sides (perm is
// the identity for its users).  All tables are computed in FP64 on the host and stored as FP32
// (complex as float2).
// ---------------------------------------------------------------------------------------------
constexpr int kMaxStages = 16;
constexpr int kMaxFftLen = 16384;  // longest direct transform (Bluestein work length)

struct FftPlanDev {
    int N;          // transform length
    int L;          // work length in shared memory (N, or the Bluestein length)
    int nst;        // number of direct stages
    int bluestein;  // 0 / 1
    int radix[kMaxStages];
    int span[kMaxStages];            // m_s = L / (radix[0] ... radix[s]): butterfly span of stage s
    unsigned magic[kMaxStages];      // ceil(2^32 / m_s): b / m_s = umulhi(b, magic) (0 when m_s = 1)
    const float2* tw;      // L entries: exp(-2 pi i m / L)
    const int* perm;       // N entries: work position of frequency k (identity for Bluestein)
    const int* iperm;      // L entries: frequency held at work position p (direct only)
    const float2* chirp;   // N entries (Bluestein): exp(-i pi n^2 / N)
    const float2* bhat;    // L entries (Bluestein): DFT_L of the conjugate chirp / L, in the
                           // direct transform's position order
    const float* lap;      // N entries: 4 sin^2(pi k / N), the periodic Laplacian's eigenvalues
    const float* lapp;     // L entries: lap[iperm[p] mod N], the eigenvalue at work position p
    // Row buffers place work position p at p + p / S, S = pad_span = L / radix[0] (direct plans
    // of two or more stages; 0 = no padding), so that positions S apart (the digit-reversed
    // neighbours k, k+1) fall in different shared-memory banks.
    int pad_span;
    unsigned pad_magic;    // ceil(2^32 / S): p / S = umulhi(p, pad_magic) for every p < L
};

// Elements of a padded row buffer for plan p.
__host__ __device__ inline int row_buf_elems(const FftPlanDev& p)
{
    return p.L + (p.pad_span ? p.L / p.pad_span : 0);
}

struct FftPlanHost {
    FftPlanDev dev{};
    void* dmem = nullptr;  // one device allocation holding every table
    size_t bytes = 0;
};

// Factor N for the direct path; returns false when N has a prime factor above 7.
bool factor_direct(int N, std::vector<int>& radices);
// Fill span[] and magic[] from radix[] (and check the magic divisions exhaustively).
bool fill_stage_division(FftPlanDev& d);
// Build the host tables of a plan and upload them (cudaMalloc'd, owned by the caller).
cudaError_t build_fft_plan(int N, FftPlanHost& out);
void free_fft_plan(FftPlanHost& p);
// Host-only variant for callers that place the tables themselves: fills `blob` and returns the
// plan with table offsets in place of pointers; bind_fft_tables rebases them onto `base`.
bool build_fft_tables_host(int N, std::vector<unsigned char>& blob, FftPlanDev& rel);
FftPlanDev bind_fft_tables(const FftPlanDev& rel, const void* base);
// Record the message returned by blfls_last_error() on this thread.
void set_last_error(const std::string& msg);

// ---------------------------------------------------------------------------------------------
// Batched form: one entry per job of the device job table of one pass.
// ---------------------------------------------------------------------------------------------
// K3 solves a column length without a mixed-radix plan (one that needs Bluestein) by the cyclic
// recursion its divide amounts to, in segments of kRecSeg rows, while lambda <= kRecLamMax.
constexpr int kRecSeg = 32;
constexpr float kRecLamMax = 1.0e4f;

struct BatchJob {
    const float* src;   // this pass's input  [C][H][W]
    float* dst;         // this pass's output [C][H][W]
    float* ex;          // residual planes [C][H][W] (scratch)
    float* ey;
    float2* spec;       // half spectra [C][H][W/2+1] (scratch)
    int H, W, C, radius;
    float kappa, inv_kappa, cs;   // bilateral constants (see launch_blf_residual)
    float lam, scale;             // solve: lambda and 1/(H W)
    int lgc;                      // log2 of the column block of K3
    int rec;                      // K3 by recursion (lgc = 5), see kRecLamMax
    int tiles_x, tiles_y;         // K1 tiling
    int tile_h;                   // K1 tile height (rows)
    FftPlanDev rp, cp;            // row (length W) and column (length H) plans
};

// ---------------------------------------------------------------------------------------------
// Bilateral step (K1): for each channel, ex = BLF(D_x f) - D_x f and ey likewise.
// ---------------------------------------------------------------------------------------------
struct BlfParams {
    int H, W;
    int radius;
    float sigma_s, sigma_r;
    int prec;    // blfls_precision
    int tile_h;  // K1 tile height: 8, 16, 32 or 64 rows (others select 32)
    // Joint filter (Section III-D): when set, the range weights compare the gradients of this
    // image instead of the input's; channel c uses guide + c * guide_stride (0 = one shared
    // guidance channel).
    const float* guide = nullptr;
    size_t guide_stride = 0;
    // Range widths per field: field x uses sigma_r * range_scale_x, field y sigma_r *
    // range_scale_y (1 and 1 unless each field is normalised to its own range).
    float range_scale_x = 1.0f, range_scale_y = 1.0f;
    // When set, the range constants (kx, ky, 1/kx, 1/ky) of channel c are read from the device at
    // kap_dev[c] instead (computed there from the fields' ranges, see launch_range_kappa), so the
    // host need not wait for the ranges.
    const float4* kap_dev = nullptr;
};

// Launch K1 over channels [0, C) of img (planes of H*W floats).  `gscratch` must hold
// 2*H*W floats when the radius is above the tiled kernels' limit, 4*H*W for a joint filter of
// radius above blf_joint_tiled_max_radius() (else it may be null).
void init_blf_kernel_attributes();
void init_solve_kernel_attributes();

cudaError_t launch_blf_residual(const float* img, float* ex, float* ey, int C,
                                const BlfParams& p, float* gscratch, cudaStream_t s);
int blf_tiled_max_radius();
int blf_joint_tiled_max_radius();
int blf_batch_max_radius();
void blf_tiles(int H, int W, int tile_h, int* tiles_x, int* tiles_y);
int blf_tile_height(int tile_h);   // the height actually used for a requested one
// Bilateral constants of a job: kappa = sqrt(log2 e / (2 sigma_r^2)) (1 without range kernel),
// cs = log2 e / (2 sigma_s^2) (0 without spatial kernel).
void blf_constants(float sigma_s, float sigma_r, float* kappa, float* inv_kappa, float* cs);
// Persistent K1 over the jobs of one (radius, range, precision) group; grp[g] = (job, first item).
cudaError_t launch_blf_batch(const BatchJob* jobs, const int2* grp, int ngrp, int total, int radius,
                             bool range, int prec, int tile_h, int num_sms, cudaStream_t s);

// ---------------------------------------------------------------------------------------------
// Fourier solve (K2 rows forward, K3 columns forward / divide / inverse, K4 rows inverse).
// spec holds H rows of W/2+1 complex values.
// ---------------------------------------------------------------------------------------------
struct SolveParams {
    int H, W;
    float lambda;
    int col_block;   // columns per CTA in K3 (1..16; 0: the column driver's own choice)
};

// Shared memory of the recursion K3 (kRecSeg) on a 32-column block of columns of length H.
size_t solve_rec_smem(int H);
// The K3 column block a solve launch takes for a requested col_block (0: the column driver's own
// choice) with column plan cp on an image W wide.
int solve_effective_col_block(const FftPlanDev& cp, int W, int col_block, int num_sms);

// `marks` (nullable) receives two events recorded after K2 and after K3.
cudaError_t launch_solve_residual(const float* f, const float* ex, const float* ey, float* out,
                                  float2* spec, const FftPlanDev& rowp, const FftPlanDev& colp,
                                  const float* sx, const float* sy, const SolveParams& p,
                                  cudaStream_t s, int num_sms, const cudaEvent_t* marks = nullptr);

// Smallest/largest shared memory the solve kernels need for these plans (bytes).
size_t solve_smem_rows(const FftPlanDev& rowp);
size_t solve_smem_cols(const FftPlanDev& colp, int col_block);
// Largest column block (log2) whose data fits the K3 shared-memory cap for a plan of length L.
int solve_fit_lgc(int L, int col_block);

// Batched solve phases: persistent grids over the row pairs (K2, K4) or column blocks (K3) of
// every channel of every job; grp arrays as for launch_blf_batch.  smem_* = the largest dynamic
// shared memory any job needs in that phase.
cudaError_t launch_solve_batch(const BatchJob* jobs, int njobs, const int2* grp_rows,
                               int total_rows, const int2* grp_cols, int total_cols,
                               size_t smem_rows, size_t smem_cols, int max_w, int num_sms,
                               cudaStream_t s, const cudaEvent_t* marks = nullptr);

// Elementwise kernels of the LS model and of the base/detail applications (layers.cu).
cudaError_t launch_ls_residuals(const float* f, float* ex, float* ey, int H, int W,
                                cudaStream_t s, int num_sms);
cudaError_t launch_log_image(const float* f, float* l, size_t n, float floor_v, cudaStream_t s,
                             int num_sms);
cudaError_t launch_layer_epilogue(int mode, const float* f, const float* u, float* out, size_t n,
                                  float strength, cudaStream_t s, int num_sms);
// Periodic separable Gaussian of one plane: rows of `in` into `tmp`, then columns into `out`;
// taps w[0..2R] (sum 1), R <= kMaxGaussR.
constexpr int kMaxGaussR = 96;
cudaError_t launch_gaussian(const float* in, float* tmp, float* out, int H, int W, const float* w,
                            int R, cudaStream_t s, int num_sms);

// Bilateral-grid BLF (grid.cu).  launch_grid_minmax: keys[4c + 2 field + {0, 1}] receive the
// order-preserving keys of min / max of field (0: x, 1: y) of channel c.  launch_grid_levels:
// lev[2c + field] = the range levels of that field's grid (zc levels per chunk).
// launch_grid_field: e = BLF_grid(g_field) - g_field for one channel from its levels (lev points
// at this field's entry); ga, gb hold (zc + 2) gx gy float2 each (grid_spatial_dims,
// grid_chunk_levels).
cudaError_t launch_grid_minmax(const float* img, int H, int W, int C, int* keys, cudaStream_t s,
                               int num_sms);
// Normalised gradients: per channel, the range constants (kx, ky, 1/kx, 1/ky) of the two fields
// from their range keys (launch_grid_minmax), sigma_r scaled by each field's range, on the device.
cudaError_t launch_range_kappa(const int* keys, int C, float sigma_r, float4* kap, cudaStream_t s);
void grid_spatial_dims(int H, int W, float sigma_s, int* gx, int* gy);
int grid_chunk_levels(float sigma_r, int gx, int gy);
cudaError_t launch_grid_levels(const int* keys, int C, float sigma_r, int zc, int4* lev,
                               cudaStream_t s);
cudaError_t launch_grid_field(const float* f, float* e, int field, int H, int W, float sigma_s,
                              float sigma_r, const int4* lev, int gx, int gy, int zc, float2* ga,
                              float2* gb, cudaStream_t s, int num_sms);

// NC-LS (nc.cu): ex, ey = NC(g) - g for one channel f, n_iter box iterations; `scratch` holds
// nc_scratch_floats(H, W) floats.
cudaError_t launch_nc_residuals(const float* f, float* ex, float* ey, int H, int W,
                                float sigma_s, float sigma_r, int n_iter, float* scratch,
                                cudaStream_t s, int num_sms);
size_t nc_scratch_floats(int H, int W);

}  // namespace blfls
