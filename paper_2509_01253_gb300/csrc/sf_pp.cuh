// sf_pp.cuh -- shared device code of the prime-power rings M = t^alpha
// (Sec. 2.1-2.3, Table 2): the ring and modulus constants, the generic
// and the compile-time length-M radix-t transforms, and the dispatch over
// the compiled rings.  Used by the ring arithmetic and RNS RLWE (sf_pp.cu)
// and by the torus scheme (sf_tq.cu).
#pragma once
#include <utility>
#include <vector>

#include "sf_arith.cuh"
#include "sf_internal.h"

#define SF_PP_THREADS 256
#define SF_PP_MAX_T 7
#define SF_PP_MAX_M 4096

struct SfPpMod {
    u64 q, one_p;            // modulus, floor(2^64 / q)
    u64 qinv_neg, r2;        // -q^-1 mod 2^64, 2^128 mod q (Montgomery products of two residues)
    u64 minv, minv_p;        // M^-1 mod q (Shoup)
    u64 h2, h2_p;            // 2^-1 mod q (Shoup)
    u64 c3, c3_p;            // t = 3: (zeta - zeta^2) / 2, zeta = omega^(M/3) (Shoup)
    u64 qh_inv, qh_inv_p;    // (Q / q_i)^-1 mod q_i (Shoup): the RNS digits of key switching
    u64 rm, rm_p;            // 2^64 mod q (Shoup): companions computed on the device
};

struct SfPpRing {
    int t, alpha, M, N, m, L;
    const u64 *w;            // [L][M] omega_i^e
    const u64 *w_p;          // [L][M] Shoup companions
    const u64 *iw;           // [L][M] omega_i^-e
    const u64 *iw_p;
    const u64 *qhat;         // [L][L][2]: (Q / q_i) mod q_j and its Shoup companion
    const u64 *dftc;         // [L][H][H][4], H = (t-1)/2: C_rk, C_rk', S_rk, S_rk' of the paired t-point DFT
    SfPpMod mod[SF_MAX_MODULI];
};

struct sf_pp_ring {
    int device;
    SfPpRing R;
    std::vector<u64> q;
    u64 *d_tables = nullptr;     // w, w_p, iw, iw_p
    u64 *d_scratch = nullptr;    // trace work buffers
    size_t scratch_words = 0;
    u64 *d_ks = nullptr;         // key-switch and ciphertext work buffers
    size_t ks_words = 0;
};

// a * b mod q for two residues below q (two Montgomery reductions: a b 2^-64,
// then times 2^128 2^-64)
__device__ __forceinline__ u64 pp_mulmod(u64 a, u64 b, const SfPpMod &P)
{
    return sf_mul_mont(sf_mul_mont(a, b, P.q, P.qinv_neg), P.r2, P.q, P.qinv_neg);
}

// one forward (DIF) stage of span len over the block's vector s
__device__ __forceinline__ void pp_stage_fwd(u64 *s, const SfPpRing &R, int i, int len)
{
    const int t = R.t, third = len / t, stride = R.M / len;
    const u64 q = R.mod[i].q, one_p = R.mod[i].one_p;
    const u64 *w = R.w + (size_t)i * R.M, *wp = R.w_p + (size_t)i * R.M;
    const int root_t = R.M / t;   // omega^(M/t): a primitive t-th root
    for (int idx = threadIdx.x; idx < R.M / t; idx += blockDim.x) {
        const int blk = idx / third, j = idx - blk * third;
        const int base = blk * len + j;
        u64 x[SF_PP_MAX_T];
        for (int r = 0; r < t; ++r) x[r] = s[base + r * third];
        for (int k = 0; k < t; ++k) {
            // y_k = sum_r x_r zeta^(r k), zeta = omega^(M/t); lazily below 2 t q
            u64 acc = x[0];
            for (int r = 1; r < t; ++r) {
                const int e = (root_t * ((r * k) % t)) % R.M;
                acc += sf_mul_shoup_lazy(x[r], w[e], wp[e], q);
            }
            u64 y = sf_reduce(acc, q, one_p);
            // twiddle omega_len^(j k) = omega^(stride j k)
            const int e = (int)(((long long)stride * j * k) % R.M);
            if (e) y = sf_mul_shoup(y, w[e], wp[e], q);
            s[base + k * third] = y;
        }
    }
}

// one inverse (DIT) stage of span len: untwiddle, then the inverse t-point DFT
__device__ __forceinline__ void pp_stage_inv(u64 *s, const SfPpRing &R, int i, int len)
{
    const int t = R.t, third = len / t, stride = R.M / len;
    const u64 q = R.mod[i].q, one_p = R.mod[i].one_p;
    const u64 *iw = R.iw + (size_t)i * R.M, *iwp = R.iw_p + (size_t)i * R.M;
    const int root_t = R.M / t;
    for (int idx = threadIdx.x; idx < R.M / t; idx += blockDim.x) {
        const int blk = idx / third, j = idx - blk * third;
        const int base = blk * len + j;
        u64 x[SF_PP_MAX_T];
        for (int k = 0; k < t; ++k) {
            u64 v = s[base + k * third];
            const int e = (int)(((long long)stride * j * k) % R.M);
            x[k] = e ? sf_mul_shoup(v, iw[e], iwp[e], q) : v;
        }
        for (int r = 0; r < t; ++r) {
            u64 acc = x[0];
            for (int k = 1; k < t; ++k) {
                const int e = (root_t * ((r * k) % t)) % R.M;
                acc += sf_mul_shoup_lazy(x[k], iw[e], iwp[e], q);
            }
            s[base + r * third] = sf_reduce(acc, q, one_p);
        }
    }
}

__device__ __forceinline__ void pp_forward(u64 *s, const SfPpRing &R, int i)
{
    for (int len = R.M; len >= R.t; len /= R.t) {
        pp_stage_fwd(s, R, i, len);
        __syncthreads();
    }
}

__device__ __forceinline__ void pp_inverse(u64 *s, const SfPpRing &R, int i)
{
    for (int len = R.t; len <= R.M; len *= R.t) {
        pp_stage_inv(s, R, i, len);
        __syncthreads();
    }
    const SfPpMod &P = R.mod[i];
    for (int e = threadIdx.x; e < R.M; e += blockDim.x) s[e] = sf_mul_shoup(s[e], P.minv, P.minv_p, P.q);
    __syncthreads();
}

// X^(N + e) = -sum_{k < t-1} X^(e + k m): fold positions N .. M-1 into 0 .. N-1
__device__ __forceinline__ void pp_reduce_phi(u64 *s, const SfPpRing &R, int i)
{
    const u64 q = R.mod[i].q;
    for (int e = threadIdx.x; e < R.m; e += blockDim.x) {
        const u64 v = s[R.N + e];
        for (int k = 0; k < R.t - 1; ++k) s[e + k * R.m] = sf_sub(s[e + k * R.m], v, q);
    }
    __syncthreads();
}

// ---- compile-time rings (Table 2: 3^7, 7^4, 5^5, and the smaller test rings)
// The same stages with t and alpha as template parameters: every span, stride
// and root index is a constant, the t values of a butterfly stay in
// registers, and one thread runs one butterfly per stage (M / t threads,
// rounded up to whole warps).  Twiddle exponents need no reduction: for span
// len, j < len / t and k < t give (M / len) j k < M.
template <int T, int ALPHA>
struct SfPpT {
    static constexpr int M = T == 3 ? (ALPHA == 2 ? 9 : ALPHA == 3 ? 27 : ALPHA == 4 ? 81 : ALPHA == 5 ? 243 : ALPHA == 6 ? 729 : 2187)
                           : T == 5 ? (ALPHA == 2 ? 25 : ALPHA == 3 ? 125 : ALPHA == 4 ? 625 : 3125)
                                    : (ALPHA == 2 ? 49 : ALPHA == 3 ? 343 : 2401);
    static constexpr int BFLY = M / T;
    static constexpr int THREADS = (BFLY + 31) / 32 * 32;
};

// the 3-point DFT with two products: with zeta + zeta^2 = -1,
// y1, y2 = x0 - (x1 + x2) / 2 +- c (x1 - x2), c = (zeta - zeta^2) / 2
// (the inverse transform's root zeta^-1 flips the sign of c)
template <bool INV>
__device__ __forceinline__ void ppt_dft3(u64 &x0, u64 &x1, u64 &x2, const SfPpMod &P)
{
    const u64 q = P.q;
    const u64 sm = sf_add(x1, x2, q), df = sf_sub(x1, x2, q);
    const u64 u = sf_sub(x0, sf_mul_shoup(sm, P.h2, P.h2_p, q), q);
    const u64 v = sf_mul_shoup(df, P.c3, P.c3_p, q);
    x0 = sf_add(x0, sm, q);
    x1 = INV ? sf_sub(u, v, q) : sf_add(u, v, q);
    x2 = INV ? sf_add(u, v, q) : sf_sub(u, v, q);
}

// The t-point DFT for odd t >= 5 by conjugate pairs: with A_r = x_r + x_(t-r),
// B_r = x_r - x_(t-r) (r = 1 .. H, H = (t-1)/2),
//   y_k, y_(t-k) = x_0 + sum_r A_r C_rk +- sum_r B_r S_rk,
// C_rk = (zeta^(rk) + zeta^(-rk)) / 2, S_rk = (zeta^(rk) - zeta^(-rk)) / 2, so
// (t-1)^2 / 2 products instead of t (t-1); the inverse (root zeta^-1) flips S.
template <int T, bool INV>
__device__ __forceinline__ void ppt_dft_pairs(u64 *x, const u64 *dc, u64 q, u64 one_p)
{
    constexpr int H = (T - 1) / 2;
    u64 A[H], B[H];
    u64 y0 = x[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
        A[r - 1] = sf_add(x[r], x[T - r], q);
        B[r - 1] = sf_sub(x[r], x[T - r], q);
        y0 = sf_add(y0, A[r - 1], q);
    }
    u64 y[T];
    y[0] = y0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        u64 U = 0, V = 0;   // lazy: H terms below 2q each
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const u64 *c = dc + 4 * ((r - 1) * H + (k - 1));
            U += sf_mul_shoup_lazy(A[r - 1], __ldg(c), __ldg(c + 1), q);
            V += sf_mul_shoup_lazy(B[r - 1], __ldg(c + 2), __ldg(c + 3), q);
        }
        const u64 base = sf_add(x[0], sf_reduce(U, q, one_p), q);
        V = sf_reduce(V, q, one_p);
        y[k] = INV ? sf_sub(base, V, q) : sf_add(base, V, q);
        y[T - k] = INV ? sf_add(base, V, q) : sf_sub(base, V, q);
    }
#pragma unroll
    for (int k = 0; k < T; ++k) x[k] = y[k];
}

// one forward stage reading its inputs through ld(index) (the block's vector
// itself, or a producer for the first stage) and writing them to s
template <int T, int M, int LEN, class LD>
__device__ __forceinline__ void ppt_stage_fwd_ld(u64 *s, LD ld, const u64 *w, const u64 *wp, const u64 *dc, u64 q,
                                                 u64 one_p, const SfPpMod &P)
{
    static_assert(T >= 3 && (T & 1), "compiled rings have an odd prime t");
    constexpr int THIRD = LEN / T, STRIDE = M / LEN;
    const int idx = threadIdx.x;
    if (idx < M / T) {
        const int blk = idx / THIRD, j = idx - blk * THIRD;
        const int base = blk * LEN + j;
        u64 x[T];
#pragma unroll
        for (int r = 0; r < T; ++r) x[r] = ld(base + r * THIRD);
        if constexpr (T == 3) {
            ppt_dft3<false>(x[0], x[1], x[2], P);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int e = STRIDE * j * k;
                s[base + k * THIRD] = e ? sf_mul_shoup(x[k], __ldg(w + e), __ldg(wp + e), q) : x[k];
            }
        } else {
            ppt_dft_pairs<T, false>(x, dc, q, one_p);
#pragma unroll
            for (int k = 0; k < T; ++k) {
                const int e = STRIDE * j * k;
                s[base + k * THIRD] = e ? sf_mul_shoup(x[k], __ldg(w + e), __ldg(wp + e), q) : x[k];
            }
        }
    }
}

template <int T, int M, int LEN>
__device__ __forceinline__ void ppt_stage_fwd(u64 *s, const u64 *w, const u64 *wp, const u64 *dc, u64 q, u64 one_p,
                                              const SfPpMod &P)
{
    ppt_stage_fwd_ld<T, M, LEN>(s, [s](int i) { return s[i]; }, w, wp, dc, q, one_p, P);
}

template <int T, int M, int LEN>
__device__ __forceinline__ void ppt_stage_inv(u64 *s, const u64 *iw, const u64 *iwp, const u64 *dc, u64 q, u64 one_p,
                                              const SfPpMod &P)
{
    static_assert(T >= 3 && (T & 1), "compiled rings have an odd prime t");
    constexpr int THIRD = LEN / T, STRIDE = M / LEN;
    const int idx = threadIdx.x;
    if (idx < M / T) {
        const int blk = idx / THIRD, j = idx - blk * THIRD;
        const int base = blk * LEN + j;
        u64 x[T];
#pragma unroll
        for (int k = 0; k < T; ++k) {
            const u64 v = s[base + k * THIRD];
            const int e = STRIDE * j * k;
            x[k] = e ? sf_mul_shoup(v, __ldg(iw + e), __ldg(iwp + e), q) : v;
        }
        if constexpr (T == 3) {
            ppt_dft3<true>(x[0], x[1], x[2], P);
#pragma unroll
            for (int r = 0; r < 3; ++r) s[base + r * THIRD] = x[r];
        } else {
            ppt_dft_pairs<T, true>(x, dc, q, one_p);
#pragma unroll
            for (int r = 0; r < T; ++r) s[base + r * THIRD] = x[r];
        }
    }
}

template <int T, int M, int LEN>
__device__ __forceinline__ void ppt_forward(u64 *s, const u64 *w, const u64 *wp, const u64 *dc, u64 q, u64 one_p,
                                            const SfPpMod &P)
{
    ppt_stage_fwd<T, M, LEN>(s, w, wp, dc, q, one_p, P);
    __syncthreads();
    if constexpr (LEN / T >= T) ppt_forward<T, M, LEN / T>(s, w, wp, dc, q, one_p, P);
}

// the whole forward transform with the first stage's inputs read through
// ld(index), index < M (each read once), e.g. straight from global memory
template <int T, int M, class LD>
__device__ __forceinline__ void ppt_forward_ld(u64 *s, LD ld, const u64 *w, const u64 *wp, const u64 *dc, u64 q,
                                               u64 one_p, const SfPpMod &P)
{
    ppt_stage_fwd_ld<T, M, M>(s, ld, w, wp, dc, q, one_p, P);
    __syncthreads();
    if constexpr (M / T >= T) ppt_forward<T, M, M / T>(s, w, wp, dc, q, one_p, P);
}

template <int T, int M, int LEN>
__device__ __forceinline__ void ppt_inverse(u64 *s, const u64 *iw, const u64 *iwp, const u64 *dc, u64 q, u64 one_p,
                                            const SfPpMod &P)
{
    ppt_stage_inv<T, M, LEN>(s, iw, iwp, dc, q, one_p, P);
    __syncthreads();
    if constexpr (LEN * T <= M) ppt_inverse<T, M, LEN * T>(s, iw, iwp, dc, q, one_p, P);
}

// runs the statements with constexpr T, ALPHA when (t, alpha) is one of the
// compiled rings; `done` tells whether it did
#define SF_PPT_DISPATCH(t, alpha, done, ...)                                                 \
    do {                                                                                       \
        done = true;                                                                           \
        if ((t) == 3 && (alpha) == 7) { constexpr int T = 3, ALPHA = 7; __VA_ARGS__ }          \
        else if ((t) == 3 && (alpha) == 4) { constexpr int T = 3, ALPHA = 4; __VA_ARGS__ }     \
        else if ((t) == 3 && (alpha) == 3) { constexpr int T = 3, ALPHA = 3; __VA_ARGS__ }     \
        else if ((t) == 5 && (alpha) == 5) { constexpr int T = 5, ALPHA = 5; __VA_ARGS__ }     \
        else if ((t) == 5 && (alpha) == 3) { constexpr int T = 5, ALPHA = 3; __VA_ARGS__ }     \
        else if ((t) == 5 && (alpha) == 2) { constexpr int T = 5, ALPHA = 2; __VA_ARGS__ }     \
        else if ((t) == 7 && (alpha) == 4) { constexpr int T = 7, ALPHA = 4; __VA_ARGS__ }     \
        else if ((t) == 7 && (alpha) == 2) { constexpr int T = 7, ALPHA = 2; __VA_ARGS__ }     \
        else done = false;                                                                     \
    } while (0)

// the automorphisms of the tower of Sec. 2.3: per step (h, length), the step
// maps x to sum_{k < length} tau_h^k(x)
void sf_pp_tower_steps(const SfPpRing &R, int gamma, std::vector<std::pair<int, int>> &steps);
