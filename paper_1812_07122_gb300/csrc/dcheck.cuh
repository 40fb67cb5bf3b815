// Device-side range checks of the debug build (compiled with -DBLFLS_DEVICE_CHECKS).
//
// BLFLS_DCHECK(cond, site) evaluates to cond.  When a check fails in a debug build it sets bit
// `site` of its translation unit's check word (an atomic OR) and the caller skips the access it
// guards; nothing traps, asserts or waits, so a bad index leaves the context usable and the
// host learns of it through blfls_device_checks.  In a release build the macro is the constant
// true and compiles away.  Each translation unit that uses checks has its own word (a __device__
// variable is per translation unit without relocatable device code) and exports a host function
// that reads and clears it (BLFLS_DCHECK_TU); blfls_device_checks ORs them.
#pragma once

#include <cuda_runtime.h>

namespace blfls {

// Check sites: one bit each.
enum DcheckSite : unsigned {
    kDcTileLoad = 0,      // K1: image tile load (source row / column, shared-memory index)
    kDcTileWindow = 1,    // K1: a window column's reads inside the gradient tile
    kDcTileStore = 2,     // K1: residual store
    kDcFftStage = 3,      // FFT stage: butterfly element offsets inside the transform buffer
    kDcSolveGlobal = 4,   // K2/K3/K4: global spectrum / image indices
    kDcGridCell = 5,      // bilateral grid: splat cell inside the grid
    kDcNcTile = 6,        // NC-LS: tile and strip indices
    kDcStaged = 7,        // staged-copy offsets inside the staging buffers
};

#ifdef BLFLS_DEVICE_CHECKS
static __device__ unsigned int g_blfls_check_word;
__device__ __forceinline__ bool dcheck_fail(unsigned site)
{
    atomicOr(&g_blfls_check_word, 1u << site);
    return false;
}
#define BLFLS_DCHECK(cond, site) ((cond) ? true : ::blfls::dcheck_fail(site))
#define BLFLS_DCHECK_TU(name)                                                                  \
    unsigned int dcheck_fetch_##name()                                                       \
    {                                                                                          \
        unsigned int w = 0, zero = 0;                                                          \
        if (cudaMemcpyFromSymbol(&w, g_blfls_check_word, sizeof w) != cudaSuccess) w = ~0u;   \
        cudaMemcpyToSymbol(g_blfls_check_word, &zero, sizeof zero);                            \
        return w;                                                                              \
    }
#else
#define BLFLS_DCHECK(cond, site) true
#define BLFLS_DCHECK_TU(name)                                                                  \
    unsigned int dcheck_fetch_##name() { return 0u; }
#endif

}  // namespace blfls
