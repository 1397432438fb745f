// sf_kernels.cuh -- device helpers shared by the kernel translation units.
#pragma once
#include <algorithm>

#include "sf_internal.h"
#include "sf_tile.cuh"

__device__ __forceinline__ SfGeo ring_geo(const SfRing &R)
{
    SfGeo g;
    g.log_n = R.log_n; g.n = R.n; g.log_r = R.log_r; g.r = R.r; g.log_c = R.log_c; g.c = R.c;
    return g;
}

// NTT slot j holds the evaluation at psi^(2 brev(j) + 1).
__device__ __forceinline__ unsigned slot_exponent(int j, int log_n)
{
    return 2u * (__brev((unsigned)j) >> (32 - log_n)) + 1u;
}

// tau_d in the NTT domain is a permutation: (tau_d a)^[j] = a^[auto_src(j)],
// the slot whose exponent is exponent(j) * d mod 2N.  Unsigned products wrap
// mod 2^32, which preserves the residue mod 2N (a power of two).
__device__ __forceinline__ int auto_src(int j, int d, int log_n)
{
    unsigned e = (slot_exponent(j, log_n) * (unsigned)d) & ((2u << log_n) - 1u);
    return (int)(__brev((e - 1u) >> 1) >> (32 - log_n));
}

// Multiplication by X^s in the NTT domain: slot j is scaled by psi^(s * e_j),
// read from the power table pw[0 .. 2N).
__device__ __forceinline__ unsigned mono_index(int j, unsigned s, int log_n)
{
    return (slot_exponent(j, log_n) * s) & ((2u << log_n) - 1u);
}

#define SF_MAX_JOBS 64
struct SfJobList {
    SfPolyJob j[SF_MAX_JOBS];
};

// floor(x 2^64 / q) for a canonical residue x: 2^64 = one_p q + r_mod, so
// x 2^64 = (x one_p + h) q + (x r_mod - h q) with h = floor(x r_mod / q),
// which Shoup's product by r_mod gives up to one correction.
__device__ __forceinline__ u64 sf_shoup_companion_dev(u64 x, const SfMod &M)
{
    u64 h = sf_mulhi(x, M.r_mod_p);
    const u64 rem = x * M.r_mod - h * M.q;
    if (rem >= M.q) ++h;
    return x * M.one_p + h;
}
