// Bounds-checked builds.
//
// Compiled with -DQG_BOUNDS_CHECK, the kernels check the indices of their
// shared-memory, global-memory and table accesses against the extents of
// the buffers they address (and the 16-byte rule for TMA box coordinates)
// before each access.  A failed check records its site number in this
// translation unit's error word (the first failure wins) and the access is
// skipped: nothing traps, and the run continues so that the host can read
// the word (qg_bounds_check_result).  In normal builds QG_IN(...) is `true`
// and the checks compile away.
#pragma once

#include <cuda_runtime.h>

#ifdef QG_BOUNDS_CHECK
namespace qg {
namespace {
__device__ int g_bounds_site = 0;
__device__ __forceinline__ bool bounds_ok(long long i, long long n, int site) {
    if (i >= 0 && i < n) return true;
    atomicCAS(&g_bounds_site, 0, site);
    return false;
}
}  // namespace
}  // namespace qg
#define QG_IN(i, n, site) (::qg::bounds_ok((long long)(i), (long long)(n), (site)))
// host side: the site recorded in this translation unit (0: none), cleared
#define QG_BOUNDS_QUERY(fn)                                                       \
    int fn() {                                                                    \
        int v = 0, z = 0;                                                         \
        if (cudaMemcpyFromSymbol(&v, ::qg::g_bounds_site, sizeof(int)) != cudaSuccess) \
            return -1;                                                            \
        cudaMemcpyToSymbol(::qg::g_bounds_site, &z, sizeof(int));                 \
        return v;                                                                 \
    }
#else
#define QG_IN(i, n, site) (true)
#define QG_BOUNDS_QUERY(fn) \
    int fn() { return 0; }
#endif
