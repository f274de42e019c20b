// gks_bounds.cuh -- index checks of debug-bounds builds (compiled with
// GKS_DEBUG_BOUNDS). Kernels pass every data-dependent index through
// in_bounds(i, n) before the access; in a debug-bounds build a failed check
// skips the access and sets this translation unit's flag, which the host
// takes after the steps (gks_step, gks_sync and the adjoint calls then return
// GKS_ERR_DEBUG_BOUNDS). In a plain build in_bounds is the constant true and
// costs nothing. Internal header.
#pragma once

#include <cuda_runtime.h>

namespace gks {

#ifdef GKS_DEBUG_BOUNDS
static __device__ int g_bounds_flag;

__device__ __forceinline__ bool in_bounds(long i, long n)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&g_bounds_flag, 1);
    return false;
}

// The flag of this translation unit, cleared (host; synchronises).
static inline int bounds_flag_take()
{
    int v = 0, z = 0;
    cudaMemcpyFromSymbol(&v, g_bounds_flag, sizeof(int));
    cudaMemcpyToSymbol(g_bounds_flag, &z, sizeof(int));
    return v;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(long, long) { return true; }
static inline int bounds_flag_take() { return 0; }
#endif

}  // namespace gks
