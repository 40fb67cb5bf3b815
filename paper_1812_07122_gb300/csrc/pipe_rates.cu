// Per-SM, per-clock throughput of the arithmetic pipes the bilateral kernel leans on, measured
// on the device itself (measurement support for the benchmark's roofline; no counterpart in the
// paper).  Each probe launches one 1024-thread block per SM (a large shared-memory request keeps
// a second block off the SM), runs eight independent dependency chains per thread, and divides
// the operations the block completed by the SM clock cycles (clock64) that the block spent, so
// the result does not depend on the clock frequency.
#include "blfls.h"
#include "internal.h"

#include <algorithm>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <vector>

namespace {

constexpr int kThreads = 1024;
constexpr int kChains = 8;
constexpr int kProbeSmem = 160 * 1024;

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ unsigned ex2h2(unsigned x)
{
    unsigned y;
    asm volatile("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
__device__ __forceinline__ unsigned ex2bf2(unsigned x)
{
    unsigned y;
    asm volatile("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c)
{
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void mma16816(float (&d)[4], unsigned a, unsigned b)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, "
                 "{%4, %4, %4, %4}, {%5, %5}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a), "r"(b));
}

// OP: 0 FFMA, 1 FFMA2 (f32x2), 2 ex2 f32, 3 ex2 f16x2, 4 ex2 bf16x2, 5 HFMA2 (f16x2),
// 6 mma.sync m16n8k16 (f16 inputs, f32 accumulators)
template <int OP>
__global__ void __launch_bounds__(kThreads) pipe_probe(long long* cycles, float* sink, int iters)
{
    extern __shared__ float pad[];
    const float seed = 1e-3f * (threadIdx.x & 31);
    float acc = 0.f;
    __syncthreads();
    long long t0 = clock64();
    if constexpr (OP == 0) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = seed + k;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], 0.999f, 0.001f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += a[k];
    } else if constexpr (OP == 1) {
        unsigned long long a[kChains];
        const unsigned long long m = pack2(0.999f, 0.999f), c = pack2(0.001f, 0.001f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = pack2(seed + k, seed - k);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fma2(a[k], m, c);
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += __uint_as_float((unsigned)a[k]);
    } else if constexpr (OP == 2) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = -seed - 0.01f * k;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = -0.5f * ex2f(a[k]);
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += a[k];
    } else if constexpr (OP == 3) {
        unsigned a[kChains];
        const __half2 mh = __floats2half2_rn(-0.5f, -0.5f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const __half2 v = __floats2half2_rn(-seed, -0.01f * k);
            a[k] = *reinterpret_cast<const unsigned*>(&v);
        }
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                unsigned e = ex2h2(a[k]);
                __half2 v = __hmul2(*reinterpret_cast<__half2*>(&e), mh);
                a[k] = *reinterpret_cast<unsigned*>(&v);
            }
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += __low2float(*reinterpret_cast<__half2*>(&a[k]));
    } else if constexpr (OP == 5) {
        __half2 a[kChains];
        const __half2 m = __floats2half2_rn(0.999f, 0.999f), c = __floats2half2_rn(1e-3f, 1e-3f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = __floats2half2_rn(seed + 0.01f * k, seed);
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = __hfma2(a[k], m, c);
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += __low2float(a[k]);
    } else if constexpr (OP == 6) {
        float d[kChains][4];
        const __half2 ah = __floats2half2_rn(seed, 0.5f), bh = __floats2half2_rn(0.25f, -seed);
        const unsigned a = *reinterpret_cast<const unsigned*>(&ah);
        const unsigned b = *reinterpret_cast<const unsigned*>(&bh);
#pragma unroll
        for (int k = 0; k < kChains; ++k) d[k][0] = d[k][1] = d[k][2] = d[k][3] = 0.f;
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) mma16816(d[k], a, b);
#pragma unroll
        for (int k = 0; k < kChains; ++k) acc += d[k][0] + d[k][3];
    } else {
        unsigned a[kChains];
        const __nv_bfloat162 mb = __floats2bfloat162_rn(-0.5f, -0.5f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const __nv_bfloat162 v = __floats2bfloat162_rn(-seed, -0.01f * k);
            a[k] = *reinterpret_cast<const unsigned*>(&v);
        }
        for (int i = 0; i < iters; ++i)
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                unsigned e = ex2bf2(a[k]);
                __nv_bfloat162 v = __hmul2(*reinterpret_cast<__nv_bfloat162*>(&e), mb);
                a[k] = *reinterpret_cast<unsigned*>(&v);
            }
#pragma unroll
        for (int k = 0; k < kChains; ++k)
            acc += __low2float(*reinterpret_cast<__nv_bfloat162*>(&a[k]));
    }
    __syncthreads();
    const long long t1 = clock64();
    if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
    if (acc == 12345.f) sink[blockIdx.x] = acc + pad[0];  // keeps the chains alive
}

template <int OP>
double run_probe(int num_sms, long long* d_cycles, float* d_sink, int iters)
{
    cudaFuncSetAttribute(pipe_probe<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem);
    pipe_probe<OP><<<num_sms, kThreads, kProbeSmem>>>(d_cycles, d_sink, 16);  // warm-up
    pipe_probe<OP><<<num_sms, kThreads, kProbeSmem>>>(d_cycles, d_sink, iters);
    std::vector<long long> cyc(num_sms);
    if (cudaMemcpy(cyc.data(), d_cycles, sizeof(long long) * num_sms, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return -1.0;
    std::sort(cyc.begin(), cyc.end());
    const double med = (double)cyc[num_sms / 2];
    // results per thread-instruction; an m16n8k16 MMA is 16 * 8 * 16 multiply-adds per warp
    const double per_instr = (OP == 0 || OP == 2) ? 1.0 : OP == 6 ? 2048.0 / 32.0 : 2.0;
    return (double)kThreads * kChains * iters * per_instr / med;
}

}  // namespace

extern "C" int blfls_pipe_rates(int device, double* rates, int n)
{
    if (!rates || n < 1) return BLFLS_EINVAL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return BLFLS_EINVAL;
    int num_sms = 0;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device);
    long long* d_cycles = nullptr;
    float* d_sink = nullptr;
    int rc = BLFLS_OK;
    if (cudaMalloc(&d_cycles, sizeof(long long) * num_sms) != cudaSuccess ||
        cudaMalloc(&d_sink, sizeof(float) * num_sms) != cudaSuccess) {
        rc = BLFLS_ENOMEM;
    } else {
        const int iters = 2048;
        double r[7];
        r[0] = run_probe<0>(num_sms, d_cycles, d_sink, iters);
        r[1] = run_probe<1>(num_sms, d_cycles, d_sink, iters);
        r[2] = run_probe<2>(num_sms, d_cycles, d_sink, iters / 4);
        r[3] = run_probe<3>(num_sms, d_cycles, d_sink, iters / 4);
        r[4] = run_probe<4>(num_sms, d_cycles, d_sink, iters / 4);
        r[5] = run_probe<5>(num_sms, d_cycles, d_sink, iters);
        r[6] = run_probe<6>(num_sms, d_cycles, d_sink, iters / 8);
        for (int i = 0; i < n && i < 7; ++i) rates[i] = r[i];
        if (cudaGetLastError() != cudaSuccess) rc = BLFLS_ECUDA;
    }
    if (d_cycles) cudaFree(d_cycles);
    if (d_sink) cudaFree(d_sink);
    cudaSetDevice(prev);
    return rc;
}
