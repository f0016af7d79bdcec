// L2 cache hints for loads whose lines are read again soon (kept in L2 with an
// evict-last access policy), used by the complex128 coins that read their
// rows twice.  The streaming counterparts (__ldcs, __stcs) come from CUDA.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

// an L2 access policy that marks the lines a load brings in as evict-last
__device__ __forceinline__ uint64_t l2_evict_last_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// a complex load under an L2 access policy
__device__ __forceinline__ double2 ld_keep(const double2 *p, uint64_t pol)
{
    double2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ float2 ld_keep(const float2 *p, uint64_t pol)
{
    float2 v;
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
