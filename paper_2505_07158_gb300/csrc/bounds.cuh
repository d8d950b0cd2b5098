// Range checks of the checked build.
//
// Compiled with -DFHD_BOUNDS_CHECK, FHD_IN(i, n, site) is true when the index i (taken as an unsigned 64-bit
// value, so that a negative index fails too) is below the extent n.  Otherwise it counts the violation in
// this translation unit's bounds record (the first violation also leaves its site, index and extent there)
// and is false, and the caller skips the access: a skipped load leaves its default value, a skipped store
// writes nothing.  Nothing traps and nothing asserts: the kernel runs to its end and the host reads the
// record afterwards (fhd_bounds_report, cipher_sync_status).
//
// In the default build FHD_IN(i, n, site) is the constant true, so the checks, and the extents computed only
// for them, compile away.
#pragma once
#include "common.cuh"

namespace fhd {
namespace {

#ifdef FHD_BOUNDS_CHECK
__device__ BoundsRecord g_bounds;

__device__ __noinline__ void bounds_fail(unsigned site, unsigned long long i, unsigned long long n) {
    if (atomicAdd(&g_bounds.count, 1u) == 0) {
        g_bounds.site = site;
        g_bounds.index = i;
        g_bounds.limit = n;
    }
}

#define FHD_IN(i, n, site)                                                  \
    ((unsigned long long)(i) < (unsigned long long)(n)                      \
         ? true                                                             \
         : (::fhd::bounds_fail((site), (unsigned long long)(i), (unsigned long long)(n)), false))
#else
#define FHD_IN(i, n, site) true
#endif

}  // namespace
}  // namespace fhd

// Defines cudaError_t fhd::NAME(BoundsRecord *acc): read and clear this translation unit's bounds record
// and add it into *acc (acc's first violation stays if it has one).  One use per translation unit.
#ifdef FHD_BOUNDS_CHECK
#define FHD_BOUNDS_TAKER(NAME)                                                                   \
    namespace fhd {                                                                              \
    cudaError_t NAME(BoundsRecord *acc) {                                                        \
        BoundsRecord r{};                                                                        \
        cudaError_t e = cudaMemcpyFromSymbol(&r, g_bounds, sizeof r);                            \
        if (e != cudaSuccess) return e;                                                          \
        if (r.count) {                                                                           \
            const BoundsRecord z{};                                                              \
            e = cudaMemcpyToSymbol(g_bounds, &z, sizeof z);                                      \
            if (e != cudaSuccess) return e;                                                      \
            if (!acc->count) {                                                                   \
                acc->site = r.site;                                                              \
                acc->index = r.index;                                                            \
                acc->limit = r.limit;                                                            \
            }                                                                                    \
            acc->count += r.count;                                                               \
        }                                                                                        \
        return cudaSuccess;                                                                      \
    }                                                                                            \
    }
#else
#define FHD_BOUNDS_TAKER(NAME)                                  \
    namespace fhd {                                             \
    cudaError_t NAME(BoundsRecord *) { return cudaSuccess; }    \
    }
#endif
