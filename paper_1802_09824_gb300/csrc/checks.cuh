// Debug bounds checks.
//
// Built with -DPHPP_BOUNDS_CHECK (build.py --checked: libphpp_checked.so),
// every index checked with in_bounds() that falls outside its buffer skips
// the access and is recorded -- a count and the site of the first one -- in
// a device word of its translation unit; ph_debug_bounds() sums and clears
// them.  The checks never trap and never wait, so a checked build is safe
// to run on a shared GPU.  In the normal build in_bounds() is `true` and
// compiles away.
#pragma once

#include "phpp_internal.cuh"

namespace phpp {

// Sites (the first one seen is reported).
enum BoundsSite : uint32_t {
    BS_PP_STAGE = 1,      // k_pp / k_pp_walk: staging buffer slot
    BS_PP_ENTRY = 2,      // k_pp: pair-list entry index
    BS_PP_SOURCE = 3,     // k_pp: source particle row
    BS_PP_QUEUE = 4,      // learned k_pp: ring slot
    BS_L1_TABLE = 5,      // learned factor: layer-1 table node
    BS_F_TABLE = 6,       // tabulated factor: node
    BS_PAIR_RUN = 7,      // k_pairs: run of a candidate
    BS_PAIR_LEAF = 8,     // k_pairs: candidate leaf
    BS_SORT_OUT = 9,      // radix scatter: output slot
    BS_BUILD_CELL = 10,   // build: ground cell of a particle
    BS_BUILD_ROW = 11,    // build: leaf / group row
    BS_PM_NODE = 12,      // PM: mesh node
    BS_DOM_ROW = 13,      // device exchange: row of the send or receive buffer
    BS_ORDER = 14,        // group order: output slot
};

#ifdef PHPP_BOUNDS_CHECK
// One pair of words per translation unit: hits, first site.
static __device__ unsigned int g_bounds_words[2];

__device__ __forceinline__ bool in_bounds(long long i, long long n, uint32_t site)
{
    if (i >= 0 && i < n) return true;
    atomicAdd(&g_bounds_words[0], 1u);
    atomicCAS(&g_bounds_words[1], 0u, site);
    return false;
}

// This translation unit's reader of its words, registered with the
// library's registry when the library is loaded (internal linkage: one per
// translation unit).
static int bounds_read_tu(unsigned int *hits, unsigned int *site)
{
    unsigned int w[2] = {0u, 0u};
    cudaError_t e = cudaMemcpyFromSymbol(w, g_bounds_words, sizeof w);
    if (e == cudaSuccess) {
        const unsigned int z[2] = {0u, 0u};
        e = cudaMemcpyToSymbol(g_bounds_words, z, sizeof z);
    }
    *hits = w[0];
    *site = w[1];
    return e == cudaSuccess ? 0 : -1;
}
static const int g_bounds_registered = (register_bounds_reader(&bounds_read_tu), 0);
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long, uint32_t) { return true; }
#endif

}  // namespace phpp
