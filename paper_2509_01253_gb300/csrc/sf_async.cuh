// sf_async.cuh -- asynchronous global -> shared copies (cp.async) used to
// double-buffer tiles in the persistent transform kernels.
#pragma once
#include <stdint.h>

__device__ __forceinline__ unsigned sf_smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// 8-byte asynchronous copy (cached in L1 on the way).
__device__ __forceinline__ void sf_cp8(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sf_smem_addr(sdst)), "l"(gsrc) : "memory");
}

// 16-byte asynchronous copy (bypasses L1).
__device__ __forceinline__ void sf_cp16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sf_smem_addr(sdst)), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void sf_cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Wait until at most N of this thread's committed groups are still in flight.
template <int N>
__device__ __forceinline__ void sf_cp_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Hint: bring the 128-byte line holding p into L2 (no data returned).
__device__ __forceinline__ void sf_prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
