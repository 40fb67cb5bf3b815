// blfls_solve_residual_noalloc: the Fourier-solve step with no device allocation at all.
//
// Who needs it: callers that must not call cudaMalloc/cudaFree -- a plug-in inside a host
// application that owns every byte of device memory through its own arena, or a real-time video
// path where an allocation (which may synchronise the whole device) would stall the frame.  They
// pass their own inputs and outputs; the scratch this step needs (the half spectrum and the FFT
// tables) lives in one statically sized __device__ array below, which every GPU that loads the
// library keeps until the process exits.
//
// Host code must not hand the array's name to a kernel: on the host that name is only a
// stand-in, not a device address.  The address is fetched once per device with
// cudaGetSymbolAddress (with that device current) and passed to the kernels.
#include "blfls.h"
#include "internal.h"

#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace {

using namespace blfls;

constexpr size_t kSpecBytes = BLFLS_NOALLOC_SPECTRUM_BYTES;
constexpr size_t kTableBytes = BLFLS_NOALLOC_TABLE_BYTES;

// [half spectrum | row-FFT tables | column-FFT tables]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kSpecBytes + kTableBytes];

struct DeviceSlot {
    unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
    int num_sms = 0;
    int rows_n = -1, cols_n = -1;   // transform lengths whose tables are resident
    FftPlanDev rp{}, cp{};
};

struct HostTables {
    std::vector<unsigned char> blob;
    FftPlanDev rel{};
};

std::mutex g_mu;
std::map<int, DeviceSlot> g_slots;       // by device ordinal
std::map<int, HostTables> g_tables;      // by transform length (host memory only)

int fail(int code, const std::string& msg)
{
    set_last_error(msg);
    return code;
}

const HostTables* host_tables(int n)
{
    auto it = g_tables.find(n);
    if (it == g_tables.end()) {
        HostTables t;
        if (!build_fft_tables_host(n, t.blob, t.rel)) return nullptr;
        it = g_tables.emplace(n, std::move(t)).first;
    }
    return &it->second;
}

}  // namespace

extern "C" int blfls_solve_residual_noalloc(const float* img, const float* ex, const float* ey,
                                            float* out, int H, int W, int C, float lambda,
                                            void* stream)
{
    if (!img || !ex || !ey || !out) return fail(BLFLS_EINVAL, "image pointer is NULL");
    if (H < 1 || W < 1 || H > BLFLS_NOALLOC_MAX_DIM || W > BLFLS_NOALLOC_MAX_DIM)
        return fail(BLFLS_EINVAL, "no-allocation solve: H and W must lie in [1, BLFLS_NOALLOC_MAX_DIM]");
    if (C < 1 || C > BLFLS_MAX_CHANNELS) return fail(BLFLS_EINVAL, "C must lie in [1, BLFLS_MAX_CHANNELS]");
    if (!(lambda >= 0.f) || !(lambda <= 3.402823466e38f)) return fail(BLFLS_EINVAL, "lambda must be finite and >= 0");
    const size_t spec_bytes = sizeof(float2) * (size_t)H * (size_t)(W / 2 + 1);
    if (spec_bytes > kSpecBytes)
        return fail(BLFLS_EINVAL, "no-allocation solve: H*(W/2+1) complex values exceed the static "
                                  "scratch (BLFLS_NOALLOC_SPECTRUM_BYTES)");

    std::lock_guard<std::mutex> lock(g_mu);
    const HostTables* rt = host_tables(W);
    const HostTables* ct = host_tables(H);
    if (!rt || !ct) return fail(BLFLS_EINVAL, "no-allocation solve: unsupported transform length");
    if (rt->blob.size() + ct->blob.size() > kTableBytes)
        return fail(BLFLS_EINVAL, "no-allocation solve: FFT tables exceed BLFLS_NOALLOC_TABLE_BYTES");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(BLFLS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    DeviceSlot& slot = g_slots[dev];
    if (!slot.base) {
        // First call on this device: find the array's device address, the SM count and the
        // kernels' shared-memory limits (no allocation involved).
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(BLFLS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        e = cudaDeviceGetAttribute(&slot.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(BLFLS_ECUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
        init_solve_kernel_attributes();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(BLFLS_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
        slot.base = static_cast<unsigned char*>(p);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* spec = slot.base;
    unsigned char* tables = slot.base + kSpecBytes;
    if (slot.rows_n != W || slot.cols_n != H) {
        // Upload the tables of this size pair; stream-ordered after earlier work on `s`.  The
        // copy reads pageable host memory, which a stream capture cannot record: refuse it
        // there rather than break the capture.
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(s, &cap);
        if (e != cudaSuccess) return fail(BLFLS_ECUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
        if (cap != cudaStreamCaptureStatusNone)
            return fail(BLFLS_EINVAL, "no-allocation solve: this size needs new FFT tables, which "
                                      "cannot be uploaded while the stream is capturing");
        e = cudaMemcpyAsync(tables, rt->blob.data(), rt->blob.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tables + rt->blob.size(), ct->blob.data(), ct->blob.size(),
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            slot.rows_n = slot.cols_n = -1;
            return fail(BLFLS_ECUDA, std::string("table upload: ") + cudaGetErrorString(e));
        }
        slot.rp = bind_fft_tables(rt->rel, tables);
        slot.cp = bind_fft_tables(ct->rel, tables + rt->blob.size());
        slot.rows_n = W;
        slot.cols_n = H;
    }
    const size_t plane = (size_t)H * W;
    const SolveParams sp{H, W, lambda, 4};
    for (int c = 0; c < C; ++c) {
        e = launch_solve_residual(img + c * plane, ex + c * plane, ey + c * plane, out + c * plane,
                                  reinterpret_cast<float2*>(spec), slot.rp, slot.cp, slot.rp.lap,
                                  slot.cp.lap, sp, s, slot.num_sms);
        if (e != cudaSuccess) return fail(BLFLS_ECUDA, std::string("solve kernel launch: ") + cudaGetErrorString(e));
    }
    return BLFLS_OK;
}
