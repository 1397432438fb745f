// sf_arith.cuh -- 64-bit modular arithmetic for moduli q < 2^51.
//
// Residues live in uint64 words.  Three published reductions are used:
//  * Shoup (1996) / Harvey (2014) multiplication by a fixed operand w with the
//    precomputed companion w' = floor(w * 2^64 / q): for any x < 2^64,
//    x*w - floor(x*w'/2^64)*q lies in [0, 2q).
//  * Montgomery (1985) REDC with R = 2^64 for products of two variable
//    residues: for T < q*2^64, (T + m q)/2^64 with m = T * (-q^-1) mod 2^64
//    lies in [0, 2q) and equals T * 2^-64 mod q.
//  * Harvey's lazy butterflies keep inverse-NTT values in [0, 4q); forward
//    values grow by at most 4q per stage (see sf_bfly_ct), far below 2^64.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SF_HD __host__ __device__ __forceinline__
#else
#define SF_HD inline
#endif

typedef uint64_t u64;

SF_HD u64 sf_mulhi(u64 a, u64 b)
{
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (u64)(((unsigned __int128)a * b) >> 64);
#endif
}

// x*w mod q in [0, 2q) for any x < 2^64; w < q, wp = floor(w 2^64 / q).
SF_HD u64 sf_mul_shoup_lazy(u64 x, u64 w, u64 wp, u64 q)
{
    u64 qhat = sf_mulhi(x, wp);
    return x * w - qhat * q;
}

SF_HD u64 sf_mul_shoup(u64 x, u64 w, u64 wp, u64 q)
{
    u64 r = sf_mul_shoup_lazy(x, w, wp, q);
    return r >= q ? r - q : r;
}

SF_HD u64 sf_csub(u64 x, u64 q) { return x >= q ? x - q : x; }

SF_HD u64 sf_add(u64 a, u64 b, u64 q) { return sf_csub(a + b, q); }

SF_HD u64 sf_sub(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator for sums of products (hi, lo).
struct sf_u128 {
    u64 lo, hi;
};

SF_HD void sf_mac128(sf_u128 &acc, u64 a, u64 b)
{
    u64 lo = a * b;
    u64 hi = sf_mulhi(a, b);
    u64 nlo = acc.lo + lo;
    acc.hi += hi + (nlo < lo ? 1 : 0);
    acc.lo = nlo;
}

// Montgomery REDC: returns T * 2^-64 mod q in [0, 2q) for T = hi*2^64 + lo < q*2^64.
// qinv_neg = -q^-1 mod 2^64.
SF_HD u64 sf_redc_lazy(u64 hi, u64 lo, u64 q, u64 qinv_neg)
{
    u64 m = lo * qinv_neg;
    u64 mq_hi = sf_mulhi(m, q);
    // lo + (m*q mod 2^64) == 0 mod 2^64, with a carry out exactly when lo != 0
    return hi + mq_hi + (lo != 0 ? 1 : 0);
}

SF_HD u64 sf_redc(u64 hi, u64 lo, u64 q, u64 qinv_neg)
{
    return sf_csub(sf_redc_lazy(hi, lo, q, qinv_neg), q);
}

// a * b_mont * 2^-64 mod q: with b_mont = b * 2^64 mod q this is a*b mod q.
SF_HD u64 sf_mul_mont(u64 a, u64 b_mont, u64 q, u64 qinv_neg)
{
    return sf_redc(sf_mulhi(a, b_mont), a * b_mont, q, qinv_neg);
}

// High 64 bits of a*b from three of the four 32 x 32-bit partial products:
// the low x low product and the carries out of the two cross products are
// dropped, so the result is the exact high part minus 0, 1 or 2.
SF_HD u64 sf_mulhi_trunc(u64 a, u64 b)
{
#if defined(__CUDA_ARCH__)
    const uint32_t al = (uint32_t)a, ah = (uint32_t)(a >> 32), bl = (uint32_t)b, bh = (uint32_t)(b >> 32);
    return (u64)ah * bh + __umulhi(ah, bl) + __umulhi(al, bh);
#else
    const u64 al = (uint32_t)a, ah = a >> 32, bl = (uint32_t)b, bh = b >> 32;
    return ah * bh + ((ah * bl) >> 32) + ((al * bh) >> 32);
#endif
}

// Shoup's product with the truncated quotient: qhat is the exact
// floor(x w' / 2^64) minus at most 2, so x*w - qhat*q lies in [0, 4q).
SF_HD u64 sf_mul_shoup_lazy4(u64 x, u64 w, u64 wp, u64 q)
{
    return x * w - sf_mulhi_trunc(x, wp) * q;
}

// Forward (Cooley-Tukey) butterfly without reduction: with Y*w mod q taken
// lazily in [0, 4q) (valid for any Y < 2^64), X' = X + T and Y' = X - T + 4q
// grow the bound by at most 4q per stage.  Starting below 4q, a whole
// transform of at most 16 stages stays below 68q < 2^58 for q < 2^51, so no
// conditional subtraction is needed until a consumer wants canonical values
// (every consumer reduces inputs below 2^64, or multiplies them by a residue
// below q with a Montgomery reduction that accepts products below q 2^64).
SF_HD void sf_bfly_ct(u64 &X, u64 &Y, u64 w, u64 wp, u64 q, u64 two_q)
{
    u64 t = sf_mul_shoup_lazy4(Y, w, wp, q);
    u64 x = X;
    X = x + t;
    Y = x - t + 2 * two_q;
}

// Inverse (Gentleman-Sande) lazy butterfly: X, Y in [0, 4q) -> X', Y' in
// [0, 4q).  The sum is brought back below 4q by one conditional subtraction;
// the difference X - Y + 4q (below 8q) is multiplied with the truncated
// quotient, which lands in [0, 4q) for any input.  Every consumer of an
// inverse pass either runs more of these butterflies or finishes with a full
// Shoup product (any input below 2^64, canonical output).
SF_HD void sf_bfly_gs(u64 &X, u64 &Y, u64 w, u64 wp, u64 q, u64 two_q)
{
    const u64 four_q = 2 * two_q;
    u64 x = X + Y;
    u64 t = X - Y + four_q;
    X = x >= four_q ? x - four_q : x;
    Y = sf_mul_shoup_lazy4(t, w, wp, q);
}

// Reduce a lazy value in [0, 4q) to [0, q).
SF_HD u64 sf_reduce4(u64 x, u64 q, u64 two_q)
{
    x = x >= two_q ? x - two_q : x;
    return x >= q ? x - q : x;
}

// Reduce any x < 2^64 to [0, q): Shoup multiplication by 1 (one_p =
// floor(2^64 / q)) lands in [0, 2q), then one conditional subtraction.
SF_HD u64 sf_reduce(u64 x, u64 q, u64 one_p)
{
    return sf_csub(x - sf_mulhi(x, one_p) * q, q);
}
