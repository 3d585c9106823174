// Index checks of the bounds-check build (nvcc -DGBCG_BOUNDS_CHECK; built as
// libgbcg_check.so beside the normal library).  Every column index a kernel
// gathers through and every staged row range it walks is tested before use;
// a bad one is counted in this translation unit's g_bounds_faults and
// replaced by index 0 (or an empty range), so the access stays in bounds and
// no kernel traps.  cg_bounds_faults() sums the counters.  Normal builds
// compile the checks away (bchk returns its argument).
#pragma once

#include <cuda_runtime.h>

namespace gbcg {

#ifdef GBCG_BOUNDS_CHECK
static __device__ unsigned int g_bounds_faults;

__device__ __forceinline__ int bchk(int i, int lim) {
    if ((unsigned)i >= (unsigned)lim) {
        atomicAdd(&g_bounds_faults, 1u);
        return 0;
    }
    return i;
}
// [k0, k1) must lie in [lo, hi]; otherwise it becomes empty.
__device__ __forceinline__ void bchk_range(int &k0, int &k1, int lo, int hi) {
    if (k0 < lo || k1 > hi || k1 < k0) {
        atomicAdd(&g_bounds_faults, 1u);
        k1 = k0 = lo;
    }
}
// Host: the counter of this translation unit (-1 if it cannot be read).
static inline long long read_bounds_faults() {
    unsigned int v = 0;
    return cudaMemcpyFromSymbol(&v, g_bounds_faults, sizeof v) == cudaSuccess ? (long long)v : -1;
}
#else
__device__ __forceinline__ int bchk(int i, int) { return i; }
__device__ __forceinline__ void bchk_range(int &, int &, int, int) {}
static inline long long read_bounds_faults() { return -1; }
#endif

}  // namespace gbcg
