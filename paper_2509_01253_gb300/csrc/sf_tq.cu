// sf_tq.cu -- the paper's RLWE over the discrete torus T_q = (1/q) Z_q with
// q = 2^53 (Sec. 2.1), in the prime-power rings T_q[X] / Phi_M, with the
// gadget key switching of Sec. 2.2 and Sec. 4.2 and the homomorphic tower
// trace of Sec. 2.3.  Table 2 gives the rings and gadgets: M = 3^7 with
// (D, l) = (512, 3); 7^4 with (2^12, 3) or (2^16, 2); 5^5 with (310, 5) or
// (310, 4).
//
// A torus value x / q is the integer x in [0, 2^53), one uint64 word; input
// words are read modulo 2^53.  Ciphertexts are [count][2][N]: a, then
// b = a s + m + e.  The key for tau_h is the l encryptions
// RLWE_s(tau_h(s) / D^i): kb_i = ka_i s + e_i + round(q tau_h(s) / D^i).
// Gadget decomposition of x: xr = round(x D^l / q) mod D^l, written with
// signed base-D digits d_1 .. d_l in [-floor(D/2), D - floor(D/2)), d_1 the
// most significant, so that sum_i d_i / D^i = x / q up to 1 / (2 D^l).  The
// key switch after tau_h returns (-sum_i d_i ka_i, tau_h(b) - sum_i d_i kb_i)
// with d_i the digits of tau_h(a).
//
// Every product is a torus polynomial times a small integer polynomial (a
// digit, or the secret).  It is computed exactly over Z and then taken mod
// 2^53: modulo two NTT primes p_0, p_1 = 1 (mod M) of 50 bits -- the length-M
// radix-t transforms of sf_pp.cuh, a pointwise product, the inverse and the
// Phi_M fold per prime -- joined by Garner's CRT into the centred integer.
// Ring creation checks that every such integer is below p_0 p_1 / 2 in
// magnitude.  The paper takes these products with double-precision FFTs; the
// integer path is exact.
//
// Key switch (k_tq_ks), one block per ciphertext: tau_h(a) is formed in shared
// memory (the permutation i -> i h mod M, then the Phi_M fold) and its l digit
// polynomials are extracted once (int16 in shared memory).  Per prime each
// digit is lifted, transformed and multiplied into two register
// accumulators with the prepared key (the 2 l key polynomials transformed per
// prime, with Shoup companions).  The accumulators are transformed back and
// folded; the first prime's results stay in shared memory, and with the
// second the CRT gives the output words directly.
#include <algorithm>
#include <vector>

#include "sf_pp.cuh"

#define SF_TQ_LOGQ 53
#define SF_TQ_MASK ((1ull << SF_TQ_LOGQ) - 1)
#define SF_TQ_MAX_L 8
#define SF_TQ_MAX_D 65536
#define SF_TQ_SECRET_BOUND 65536   // |s_e| for encryption and key generation

struct SfTqGadget {
    u64 D, Dl, D_rcp;        // base, D^l, floor(2^64 / D)
    int l, half;             // depth, floor(D / 2)
    u64 crt_inv, crt_inv_p;  // p_0^-1 mod p_1 and its Shoup companion
    u64 Q_lo;                // p_0 p_1 mod 2^64
    u64 Qh_hi, Qh_lo;        // floor(p_0 p_1 / 2) as two words
};

struct sf_tq_ring {
    sf_pp_ring *pp = nullptr;    // the CRT primes p_0, p_1 and their transform tables
    SfTqGadget G;
    u64 *d_work = nullptr;       // products and trace buffers
    size_t work_words = 0;
};

// compile-time shape: T = 0 is the generic ring (runtime t, alpha).  The key
// switch of a compiled ring is bounded to two blocks per SM: at M = 3^7 and
// 5^5 that caps its registers at 40 and 48 (with a few spilled words) and was
// measured 12 and 10 % faster than one block of 72 and 94 registers; three
// blocks spill more and lose again.
template <int T, int ALPHA>
struct SfTqShape {
    static constexpr int NT = SfPpT<T, ALPHA>::THREADS, MMAX = SfPpT<T, ALPHA>::M, MINB = 2;
};
template <int ALPHA>
struct SfTqShape<0, ALPHA> {
    static constexpr int NT = SF_PP_THREADS, MMAX = SF_PP_MAX_M, MINB = 1;
};

// forward transform of the block's length-M vector modulo prime j, the first
// stage reading its inputs through ld(index), index < M (each read once)
template <int T, int ALPHA, class LD>
__device__ __forceinline__ void tq_forward_ld(u64 *s, LD ld, const SfPpRing &R, int j)
{
    if constexpr (T == 0) {
        for (int e = threadIdx.x; e < R.M; e += blockDim.x) s[e] = ld(e);
        __syncthreads();
        pp_forward(s, R, j);
    } else {
        constexpr int M = SfPpT<T, ALPHA>::M, H = (T - 1) / 2;
        const SfPpMod &P = R.mod[j];
        ppt_forward_ld<T, M>(s, ld, R.w + (size_t)j * M, R.w_p + (size_t)j * M, R.dftc + (size_t)j * H * H * 4, P.q,
                             P.one_p, P);
    }
}

// inverse transform, scaled by M^-1
template <int T, int ALPHA>
__device__ __forceinline__ void tq_inverse(u64 *s, const SfPpRing &R, int j)
{
    if constexpr (T == 0) {
        pp_inverse(s, R, j);
    } else {
        constexpr int M = SfPpT<T, ALPHA>::M, H = (T - 1) / 2, NT = SfPpT<T, ALPHA>::THREADS;
        const SfPpMod &P = R.mod[j];
        ppt_inverse<T, M, T>(s, R.iw + (size_t)j * M, R.iw_p + (size_t)j * M, R.dftc + (size_t)j * H * H * 4, P.q,
                             P.one_p, P);
        for (int e = threadIdx.x; e < M; e += NT) s[e] = sf_mul_shoup(s[e], P.minv, P.minv_p, P.q);
        __syncthreads();
    }
}

// a signed integer as a residue modulo P.q
__device__ __forceinline__ u64 tq_lift_signed(long long v, const SfPpMod &P)
{
    const u64 mag = v >= 0 ? (u64)v : (u64)0 - (u64)v;
    const u64 r = sf_reduce(mag, P.q, P.one_p);
    return (v < 0 && r) ? P.q - r : r;
}

// floor(x 2^64 / q) for x < q: 2^64 = one_p q + rm, and floor(x rm / q) by
// Shoup's product with at most one correction
__device__ __forceinline__ u64 tq_companion(u64 x, const SfPpMod &P)
{
    u64 h = sf_mulhi(x, P.rm_p);
    const u64 rem = x * P.rm - h * P.q;
    if (rem >= P.q) ++h;
    return x * P.one_p + h;
}

// round(x D^l / 2^53) mod D^l for x < 2^53 (halves rounded up)
__device__ __forceinline__ u64 tq_rounded(u64 x, const SfTqGadget &G)
{
    const u64 lo = x * G.Dl, hi = sf_mulhi(x, G.Dl);
    const u64 lo2 = lo + (1ull << (SF_TQ_LOGQ - 1));
    const u64 hi2 = hi + (lo2 < lo ? 1 : 0);
    const u64 xr = (hi2 << (64 - SF_TQ_LOGQ)) | (lo2 >> SF_TQ_LOGQ);
    return xr >= G.Dl ? xr - G.Dl : xr;
}

// the next signed digit from the low end: r = x mod D taken in
// [-half, D - half), x <- (x - r) / D.  The quotient estimate
// floor(x D_rcp / 2^64) is floor(x / D) or one less.
__device__ __forceinline__ int tq_next_digit(u64 &x, const SfTqGadget &G)
{
    u64 qd = sf_mulhi(x, G.D_rcp);
    u64 r = x - qd * G.D;
    if (r >= G.D) {
        r -= G.D;
        ++qd;
    }
    int d = (int)r;
    if (d >= (int)G.D - G.half) {
        d -= (int)G.D;
        ++qd;
    }
    x = qd;
    return d;
}

// Garner's CRT of x0 (mod p_0) and x1 (mod p_1) to the integer X in
// (-p_0 p_1 / 2, p_0 p_1 / 2), returned mod 2^53
__device__ __forceinline__ u64 tq_crt(u64 x0, u64 x1, const SfPpRing &R, const SfTqGadget &G)
{
    const SfPpMod &P1 = R.mod[1];
    const u64 x0r = sf_reduce(x0, P1.q, P1.one_p);
    const u64 v = sf_mul_shoup(sf_sub(x1, x0r, P1.q), G.crt_inv, G.crt_inv_p, P1.q);
    const u64 p0 = R.mod[0].q;
    u64 lo = p0 * v, hi = sf_mulhi(p0, v);
    const u64 lo2 = lo + x0;
    hi += lo2 < lo ? 1 : 0;
    lo = lo2;
    const bool upper = hi > G.Qh_hi || (hi == G.Qh_hi && lo > G.Qh_lo);
    return (upper ? lo - G.Q_lo : lo) & SF_TQ_MASK;
}

// coefficient i of tau_h(x) mod Phi_M read from x (length N) by gathering:
// the unreduced image has x_k at k h mod M, and position i < N receives the
// image at i minus the image at N + (i mod m); hinv = h^-1 mod M
__device__ __forceinline__ u64 tq_auto_at(const u64 *x, int i, const SfPpRing &R, int hinv)
{
    const int k0 = (int)(((long long)i * hinv) % R.M);
    const int k1 = (int)(((long long)(R.N + i % R.m) * hinv) % R.M);
    const u64 v0 = k0 < R.N ? x[k0] & SF_TQ_MASK : 0;
    const u64 v1 = k1 < R.N ? x[k1] & SF_TQ_MASK : 0;
    return (v0 - v1) & SF_TQ_MASK;
}

// ------------------------------------------------------------- kernels ----

// shared memory of the key switch: the length-M vector, the first prime's two
// result polynomials, the l int16 digit polynomials
static size_t tq_ks_smem(const SfPpRing &R, int l)
{
    return sizeof(u64) * ((size_t)R.M + 2 * (size_t)R.N) + (((size_t)2 * l * R.N + 7) & ~(size_t)7);
}

// Key switch after tau_h, one block per ciphertext.  key: [l][2][2][M]
// transformed key values (digit i, part a / b, prime j), then their Shoup
// companions in the same order.
template <int T, int ALPHA>
__global__ void __launch_bounds__(SfTqShape<T, ALPHA>::NT, SfTqShape<T, ALPHA>::MINB)
    k_tq_ks(SfPpRing R, SfTqGadget G, const u64 *ct, u64 *out, int h, int hinv, const u64 *key)
{
    constexpr int NT = SfTqShape<T, ALPHA>::NT, EPT = (SfTqShape<T, ALPHA>::MMAX + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *vec = (u64 *)smem_raw;
    u64 *res0 = vec + R.M;                      // [2][N]
    int16_t *dig = (int16_t *)(res0 + 2 * R.N);  // [l][N]
    const int M = R.M, N = R.N, m = R.m;
    const size_t c = blockIdx.x;
    const u64 *a = ct + c * 2 * N, *b = a + N;
    // tau_h(a): permute, then X^(N + e) = -sum_{k < t-1} X^(e + k m)
    for (int e = threadIdx.x; e < M; e += NT) vec[e] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < N; e += NT) vec[(int)(((long long)e * h) % M)] = a[e] & SF_TQ_MASK;
    __syncthreads();
    for (int e = threadIdx.x; e < m; e += NT) {
        const u64 v = vec[N + e];
        for (int k = 0; k < R.t - 1; ++k) vec[e + k * m] = (vec[e + k * m] - v) & SF_TQ_MASK;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N; e += NT) {
        u64 xr = tq_rounded(vec[e], G);
        for (int i = G.l - 1; i >= 0; --i) dig[(size_t)i * N + e] = (int16_t)tq_next_digit(xr, G);
    }
    __syncthreads();
    const size_t kw = (size_t)4 * G.l * M;   // companions follow the values
    for (int j = 0; j < 2; ++j) {
        const SfPpMod &P = R.mod[j];
        u64 acc_a[EPT], acc_b[EPT];
#pragma unroll
        for (int x = 0; x < EPT; ++x) acc_a[x] = acc_b[x] = 0;
        for (int i = 0; i < G.l; ++i) {
            // digit i lifted mod p_j as the first stage reads it
            const int16_t *di = dig + (size_t)i * N;
            const u64 pq = P.q;
            tq_forward_ld<T, ALPHA>(
                vec,
                [di, N, pq](int e) -> u64 {
                    const int d = e < N ? di[e] : 0;
                    return d >= 0 ? (u64)d : pq - (u64)(-d);
                },
                R, j);
            const u64 *ka = key + ((size_t)(i * 2 + 0) * 2 + j) * M;
            const u64 *kb = key + ((size_t)(i * 2 + 1) * 2 + j) * M;
#pragma unroll
            for (int x = 0; x < EPT; ++x) {
                const int e = threadIdx.x + x * NT;
                if (e < M) {
                    const u64 v = vec[e];
                    acc_a[x] += sf_mul_shoup_lazy(v, __ldg(ka + e), __ldg(ka + kw + e), P.q);
                    acc_b[x] += sf_mul_shoup_lazy(v, __ldg(kb + e), __ldg(kb + kw + e), P.q);
                }
            }
            __syncthreads();
        }
        for (int part = 0; part < 2; ++part) {
#pragma unroll
            for (int x = 0; x < EPT; ++x) {
                const int e = threadIdx.x + x * NT;
                if (e < M) vec[e] = sf_reduce(part ? acc_b[x] : acc_a[x], P.q, P.one_p);
            }
            __syncthreads();
            tq_inverse<T, ALPHA>(vec, R, j);
            for (int e = threadIdx.x; e < m; e += NT) {
                const u64 v = vec[N + e];
                for (int k = 0; k < R.t - 1; ++k) vec[e + k * m] = sf_sub(vec[e + k * m], v, P.q);
            }
            __syncthreads();
            if (j == 0) {
                for (int e = threadIdx.x; e < N; e += NT) res0[(size_t)part * N + e] = vec[e];
            } else {
                u64 *o = out + c * 2 * N + (size_t)part * N;
                for (int e = threadIdx.x; e < N; e += NT) {
                    const u64 X = tq_crt(res0[(size_t)part * N + e], vec[e], R, G);
                    o[e] = ((part ? tq_auto_at(b, e, R, hinv) : 0) - X) & SF_TQ_MASK;
                }
            }
            __syncthreads();
        }
    }
}

// out[c] = a[c] s mod 2^53: a [count] torus polynomials at stride sa words,
// s a signed polynomial (|s_e| <= SF_TQ_SECRET_BOUND); one block per polynomial
template <int T, int ALPHA>
__global__ void __launch_bounds__(SfTqShape<T, ALPHA>::NT)
    k_tq_prod(SfPpRing R, SfTqGadget G, const u64 *a, size_t sa, const int64_t *s, u64 *out)
{
    constexpr int NT = SfTqShape<T, ALPHA>::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *va = (u64 *)smem_raw, *vs = va + R.M, *res0 = vs + R.M;
    const int M = R.M, N = R.N, m = R.m;
    const u64 *x = a + blockIdx.x * sa;
    for (int j = 0; j < 2; ++j) {
        const SfPpMod &P = R.mod[j];
        tq_forward_ld<T, ALPHA>(
            va, [x, N, &P](int e) -> u64 { return e < N ? sf_reduce(x[e] & SF_TQ_MASK, P.q, P.one_p) : 0; }, R, j);
        tq_forward_ld<T, ALPHA>(vs, [s, N, &P](int e) -> u64 { return e < N ? tq_lift_signed(s[e], P) : 0; }, R, j);
        for (int e = threadIdx.x; e < M; e += NT) va[e] = pp_mulmod(va[e], vs[e], P);
        __syncthreads();
        tq_inverse<T, ALPHA>(va, R, j);
        for (int e = threadIdx.x; e < m; e += NT) {
            const u64 v = va[N + e];
            for (int k = 0; k < R.t - 1; ++k) va[e + k * m] = sf_sub(va[e + k * m], v, P.q);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < N; e += NT) {
            if (j == 0) res0[e] = va[e];
            else out[(size_t)blockIdx.x * N + e] = tq_crt(res0[e], va[e], R, G);
        }
        __syncthreads();
    }
}

// The prepared key: grid (2 primes, 2 l polynomials); polynomial p is digit
// p / 2, part p % 2 (ka, kb), each [l][N] torus words.
template <int T, int ALPHA>
__global__ void __launch_bounds__(SfTqShape<T, ALPHA>::NT)
    k_tq_key_ntt(SfPpRing R, int l, const u64 *ka, const u64 *kb, u64 *key)
{
    constexpr int NT = SfTqShape<T, ALPHA>::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *vec = (u64 *)smem_raw;
    const int j = blockIdx.x, p = blockIdx.y, i = p / 2, part = p % 2;
    const SfPpMod &P = R.mod[j];
    const u64 *x = (part ? kb : ka) + (size_t)i * R.N;
    const int N = R.N;
    tq_forward_ld<T, ALPHA>(
        vec, [x, N, &P](int e) -> u64 { return e < N ? sf_reduce(x[e] & SF_TQ_MASK, P.q, P.one_p) : 0; }, R, j);
    u64 *dst = key + ((size_t)(i * 2 + part) * 2 + j) * R.M;
    const size_t kw = (size_t)4 * l * R.M;
    for (int e = threadIdx.x; e < R.M; e += NT) {
        dst[e] = vec[e];
        dst[kw + e] = tq_companion(vec[e], P);
    }
}

// digits [count][l][N] (int32) of [count][N] torus polynomials
__global__ void k_tq_decompose(int N, SfTqGadget G, const u64 *x, int32_t *digits, size_t total)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = k / N, e = k - c * N;
        u64 xr = tq_rounded(x[k] & SF_TQ_MASK, G);
        for (int i = G.l - 1; i >= 0; --i) digits[(c * G.l + i) * N + e] = tq_next_digit(xr, G);
    }
}

// ct[c] = (a[c], prod[c] + m[c] + e[c]) mod 2^53
__global__ void k_tq_enc_finish(int N, const u64 *a, const u64 *prod, const u64 *msg, const int64_t *e, u64 *ct,
                                size_t total)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = k / N, r = k - c * N;
        ct[c * 2 * N + r] = a[k] & SF_TQ_MASK;
        ct[c * 2 * N + N + r] = (prod[k] + msg[k] + (u64)e[k]) & SF_TQ_MASK;
    }
}

// phase[c] = b[c] - prod[c] mod 2^53
__global__ void k_tq_dec_finish(int N, const u64 *ct, const u64 *prod, u64 *phase, size_t total)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = k / N, r = k - c * N;
        phase[k] = (ct[c * 2 * N + N + r] - prod[k]) & SF_TQ_MASK;
    }
}

// kb_i = prod_i + e_i + round(q ts / D^i) mod 2^53, ts = tau_h(s) (a signed
// polynomial, gathered from s as in tq_auto_at), rounding halves up
__global__ void k_tq_ksk_finish(SfPpRing R, SfTqGadget G, const int64_t *s, int hinv, const u64 *prod,
                                const int64_t *e, u64 *kb)
{
    const size_t total = (size_t)G.l * R.N;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / R.N), n = (int)(k - (size_t)i * R.N);
        const int k0 = (int)(((long long)n * hinv) % R.M);
        const int k1 = (int)(((long long)(R.N + n % R.m) * hinv) % R.M);
        const long long ts = (k0 < R.N ? s[k0] : 0) - (k1 < R.N ? s[k1] : 0);
        __int128 Di = 1;
        for (int x = 0; x <= i; ++x) Di *= (__int128)G.D;
        const __int128 num = (__int128)2 * ts * ((__int128)1 << SF_TQ_LOGQ) + Di, den = 2 * Di;
        __int128 g = num / den;
        if (num % den != 0 && num < 0) g -= 1;   // floor
        kb[k] = (prod[k] + (u64)e[k] + (u64)g) & SF_TQ_MASK;
    }
}

// acc += x mod 2^53
__global__ void k_tq_add(u64 *acc, const u64 *x, size_t total)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x)
        acc[k] = (acc[k] + x[k]) & SF_TQ_MASK;
}

// ---------------------------------------------------------------- host ----

#define SF_TQ_DISPATCH(R, ...)                               \
    do {                                                     \
        bool done_ = false;                                  \
        SF_PPT_DISPATCH((R).t, (R).alpha, done_, __VA_ARGS__); \
        if (!done_) {                                        \
            constexpr int T = 0, ALPHA = 0;                  \
            __VA_ARGS__                                      \
        }                                                    \
    } while (0)

static int tq_grid(size_t total) { return (int)std::min<size_t>((total + 255) / 256, 8192); }

static size_t tq_prod_smem(const SfPpRing &R) { return sizeof(u64) * (2 * (size_t)R.M + R.N); }

static sf_status tq_work(sf_tq_ring *r, size_t words, u64 **out)
{
    if (r->work_words < words) {
        if (r->d_work) cudaFree(r->d_work);
        r->d_work = nullptr;
        r->work_words = 0;
        SF_CUDA_TRY(cudaMalloc((void **)&r->d_work, sizeof(u64) * words));
        r->work_words = words;
    }
    *out = r->d_work;
    return SF_OK;
}

static sf_status tq_check(const sf_tq_ring *r, const void *a, const void *b, int count)
{
    if (!r || !a || !b || count < 1) return sf_set_error(SF_EINVAL, "torus ring: bad arguments");
    if (cudaSetDevice(r->pp->device) != cudaSuccess) return sf_set_error(SF_ECUDA, "cudaSetDevice failed");
    return SF_OK;
}

static int tq_unit(const SfPpRing &R, int h, int *hinv)
{
    const int hh = ((h % R.M) + R.M) % R.M;
    if (hh % R.t == 0) return -1;
    int x = 1;   // h^-1 mod M by search (M <= 4096 is composite: no Fermat inverse)
    while ((long long)hh * x % R.M != 1) ++x;
    *hinv = x;
    return hh;
}

extern "C" sf_status sf_tq_ring_create(int32_t t, int32_t alpha, int32_t D, int32_t l, int32_t device,
                                       sf_tq_ring **out)
{
    if (!out) return sf_set_error(SF_EINVAL, "sf_tq_ring_create: null output");
    *out = nullptr;
    if (D < 2 || D > SF_TQ_MAX_D || l < 1 || l > SF_TQ_MAX_L)
        return sf_set_error(SF_EINVAL, "sf_tq_ring_create: need 2 <= D <= %d and 1 <= l <= %d", SF_TQ_MAX_D,
                            SF_TQ_MAX_L);
    unsigned __int128 Dl = 1;
    for (int i = 0; i < l; ++i) Dl *= (unsigned)D;
    if (Dl > ((unsigned __int128)1 << SF_TQ_LOGQ)) return sf_set_error(SF_EINVAL, "sf_tq_ring_create: D^l exceeds 2^53");
    sf_pp_ring *pp = nullptr;
    SF_TRY(sf_pp_ring_create(t, alpha, 2, 50, device, &pp));
    const SfPpRing &R = pp->R;
    const u64 p0 = pp->q[0], p1 = pp->q[1];
    const unsigned __int128 Q = (unsigned __int128)p0 * p1;
    // |sum_i d_i k_i| <= l * 2N * ceil(D/2) * 2^53 after the Phi_M fold (every
    // output coefficient collects two cyclic coefficients of at most N terms);
    // products with the secret stay below 2N * bound * 2^53
    const unsigned __int128 two53 = (unsigned __int128)1 << SF_TQ_LOGQ;
    const unsigned __int128 ks_bound = (unsigned __int128)l * 2 * R.N * ((D + 1) / 2) * two53;
    const unsigned __int128 s_bound = (unsigned __int128)2 * R.N * SF_TQ_SECRET_BOUND * two53;
    if (2 * std::max(ks_bound, s_bound) >= Q) {
        sf_pp_ring_destroy(pp);
        return sf_set_error(SF_EINVAL, "sf_tq_ring_create: products would exceed the CRT range");
    }
    sf_tq_ring *r = new sf_tq_ring();
    r->pp = pp;
    SfTqGadget &G = r->G;
    G.D = (u64)D;
    G.Dl = (u64)Dl;
    G.D_rcp = (u64)((((unsigned __int128)1) << 64) / (u64)D);
    G.l = l;
    G.half = D / 2;
    G.crt_inv = sf_host_invmod(p0 % p1, p1);
    G.crt_inv_p = sf_shoup_companion(G.crt_inv, p1);
    G.Q_lo = (u64)Q;
    G.Qh_hi = (u64)((Q >> 1) >> 64);
    G.Qh_lo = (u64)(Q >> 1);
    // the limit is per kernel, not per ring: allow the most a block may take, so
    // that rings of other gadgets sharing the kernel keep launching
    const int mx = 227 * 1024;
    cudaError_t err = cudaSuccess;
    SF_TQ_DISPATCH(R, {
        err = cudaFuncSetAttribute(k_tq_ks<T, ALPHA>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_tq_prod<T, ALPHA>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    });
    if (err != cudaSuccess) {
        cudaGetLastError();
        sf_pp_ring_destroy(pp);
        delete r;
        return sf_set_error(SF_ECUDA, "sf_tq_ring_create: kernel attributes failed: %s", cudaGetErrorString(err));
    }
    *out = r;
    return SF_OK;
}

extern "C" void sf_tq_ring_destroy(sf_tq_ring *r)
{
    if (!r) return;
    cudaSetDevice(r->pp->device);
    if (r->d_work) cudaFree(r->d_work);
    sf_pp_ring_destroy(r->pp);
    delete r;
}

extern "C" sf_status sf_tq_ring_info(const sf_tq_ring *r, int32_t *N, int32_t *M, uint64_t *primes,
                                     int64_t *key_words)
{
    if (!r) return sf_set_error(SF_EINVAL, "sf_tq_ring_info: null ring");
    if (N) *N = r->pp->R.N;
    if (M) *M = r->pp->R.M;
    if (primes) {
        primes[0] = r->pp->q[0];
        primes[1] = r->pp->q[1];
    }
    if (key_words) *key_words = (int64_t)8 * r->G.l * r->pp->R.M;
    return SF_OK;
}

extern "C" sf_status sf_tq_decompose(sf_tq_ring *r, const uint64_t *d_in, int32_t *d_digits, int32_t count,
                                     void *stream)
{
    SF_TRY(tq_check(r, d_in, d_digits, count));
    const size_t total = (size_t)count * r->pp->R.N;
    k_tq_decompose<<<tq_grid(total), 256, 0, (cudaStream_t)stream>>>(r->pp->R.N, r->G, d_in, d_digits, total);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// out[c] = a[c] s mod 2^53 for count polynomials at stride sa
static sf_status tq_prod(sf_tq_ring *r, const u64 *a, size_t sa, const int64_t *s, u64 *out, int count,
                         cudaStream_t st)
{
    const SfPpRing &R = r->pp->R;
    SF_TQ_DISPATCH(R, {
        k_tq_prod<T, ALPHA><<<count, SfTqShape<T, ALPHA>::NT, tq_prod_smem(R), st>>>(R, r->G, a, sa, s, out);
    });
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_tq_encrypt(sf_tq_ring *r, const int64_t *d_s, const uint64_t *d_a, const uint64_t *d_m,
                                   const int64_t *d_e, uint64_t *d_ct, int32_t count, void *stream)
{
    SF_TRY(tq_check(r, d_s, d_a, count));
    if (!d_m || !d_e || !d_ct) return sf_set_error(SF_EINVAL, "sf_tq_encrypt: null buffer");
    const int N = r->pp->R.N;
    cudaStream_t st = (cudaStream_t)stream;
    u64 *prod;
    SF_TRY(tq_work(r, (size_t)count * N, &prod));
    SF_TRY(tq_prod(r, d_a, N, d_s, prod, count, st));
    const size_t total = (size_t)count * N;
    k_tq_enc_finish<<<tq_grid(total), 256, 0, st>>>(N, d_a, prod, d_m, d_e, d_ct, total);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_tq_decrypt(sf_tq_ring *r, const int64_t *d_s, const uint64_t *d_ct, uint64_t *d_phase,
                                   int32_t count, void *stream)
{
    SF_TRY(tq_check(r, d_s, d_ct, count));
    if (!d_phase) return sf_set_error(SF_EINVAL, "sf_tq_decrypt: null output");
    const int N = r->pp->R.N;
    cudaStream_t st = (cudaStream_t)stream;
    u64 *prod;
    SF_TRY(tq_work(r, (size_t)count * N, &prod));
    SF_TRY(tq_prod(r, d_ct, 2 * (size_t)N, d_s, prod, count, st));
    const size_t total = (size_t)count * N;
    k_tq_dec_finish<<<tq_grid(total), 256, 0, st>>>(N, d_ct, prod, d_phase, total);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_tq_ksk(sf_tq_ring *r, const int64_t *d_s, int32_t h, const uint64_t *d_ka, const int64_t *d_e,
                               uint64_t *d_kb, void *stream)
{
    SF_TRY(tq_check(r, d_s, d_ka, 1));
    if (!d_e || !d_kb) return sf_set_error(SF_EINVAL, "sf_tq_ksk: null buffer");
    const SfPpRing &R = r->pp->R;
    int hinv;
    if (tq_unit(R, h, &hinv) < 0) return sf_set_error(SF_EINVAL, "sf_tq_ksk: h = %d not coprime to M = %d", h, R.M);
    cudaStream_t st = (cudaStream_t)stream;
    u64 *prod;
    SF_TRY(tq_work(r, (size_t)r->G.l * R.N, &prod));
    SF_TRY(tq_prod(r, d_ka, R.N, d_s, prod, r->G.l, st));
    k_tq_ksk_finish<<<tq_grid((size_t)r->G.l * R.N), 256, 0, st>>>(R, r->G, d_s, hinv, prod, d_e, d_kb);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_tq_key_prepare(sf_tq_ring *r, const uint64_t *d_ka, const uint64_t *d_kb, uint64_t *d_key,
                                       void *stream)
{
    SF_TRY(tq_check(r, d_ka, d_kb, 1));
    if (!d_key) return sf_set_error(SF_EINVAL, "sf_tq_key_prepare: null key");
    const SfPpRing &R = r->pp->R;
    SF_TQ_DISPATCH(R, {
        k_tq_key_ntt<T, ALPHA><<<dim3(2, 2 * r->G.l), SfTqShape<T, ALPHA>::NT, sizeof(u64) * R.M, (cudaStream_t)stream>>>(
            R, r->G.l, d_ka, d_kb, d_key);
    });
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

static sf_status tq_keyswitch(sf_tq_ring *r, const u64 *in, u64 *out, int count, int h, int hinv, const u64 *key,
                              cudaStream_t st)
{
    const SfPpRing &R = r->pp->R;
    const size_t sm = tq_ks_smem(R, r->G.l);
    SF_TQ_DISPATCH(R, {
        k_tq_ks<T, ALPHA><<<count, SfTqShape<T, ALPHA>::NT, sm, st>>>(R, r->G, in, out, h, hinv, key);
    });
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_tq_keyswitch(sf_tq_ring *r, const uint64_t *d_ct, uint64_t *d_out, int32_t count, int32_t h,
                                     const uint64_t *d_key, void *stream)
{
    SF_TRY(tq_check(r, d_ct, d_out, count));
    if (!d_key || d_ct == d_out) return sf_set_error(SF_EINVAL, "sf_tq_keyswitch: null key or in place");
    int hinv;
    const int hh = tq_unit(r->pp->R, h, &hinv);
    if (hh < 0) return sf_set_error(SF_EINVAL, "sf_tq_keyswitch: h = %d not coprime to M", h);
    return tq_keyswitch(r, d_ct, d_out, count, hh, hinv, d_key, (cudaStream_t)stream);
}

extern "C" sf_status sf_tq_hom_trace(sf_tq_ring *r, const uint64_t *d_ct, uint64_t *d_out, int32_t count,
                                     int32_t gamma, int32_t n_keys, const int32_t *hs, const uint64_t *const *d_keys,
                                     int32_t *n_keyswitches, void *stream)
{
    SF_TRY(tq_check(r, d_ct, d_out, count));
    const SfPpRing &R = r->pp->R;
    if (gamma < 0 || gamma > R.alpha) return sf_set_error(SF_EINVAL, "sf_tq_hom_trace: gamma must lie in [0, alpha]");
    if (n_keys < 0 || (n_keys > 0 && (!hs || !d_keys))) return sf_set_error(SF_EINVAL, "sf_tq_hom_trace: bad key list");
    if (d_ct == d_out) return sf_set_error(SF_EINVAL, "sf_tq_hom_trace: in place is not supported");
    std::vector<std::pair<int, int>> steps;
    sf_pp_tower_steps(R, gamma, steps);
    std::vector<int> key_of(steps.size());
    for (size_t k = 0; k < steps.size(); ++k) {
        key_of[k] = -1;
        for (int x = 0; x < n_keys; ++x)
            if (((hs[x] % R.M) + R.M) % R.M == steps[k].first) key_of[k] = x;
        if (key_of[k] < 0 || !d_keys[key_of[k]])
            return sf_set_error(SF_EINVAL, "sf_tq_hom_trace: no key for tau_%d", steps[k].first);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = (size_t)count * 2 * R.N;
    u64 *cur;
    SF_TRY(tq_work(r, 2 * words, &cur));
    u64 *nxt = cur + words;
    SF_CUDA_TRY(cudaMemcpyAsync(d_out, d_ct, sizeof(u64) * words, cudaMemcpyDeviceToDevice, st));
    int ks = 0;
    for (size_t k = 0; k < steps.size(); ++k) {
        int hinv;
        const int hh = tq_unit(R, steps[k].first, &hinv);
        SF_CUDA_TRY(cudaMemcpyAsync(cur, d_out, sizeof(u64) * words, cudaMemcpyDeviceToDevice, st));
        for (int x = 1; x < steps[k].second; ++x) {
            SF_TRY(tq_keyswitch(r, cur, nxt, count, hh, hinv, d_keys[key_of[k]], st));
            std::swap(cur, nxt);
            k_tq_add<<<tq_grid(words), 256, 0, st>>>(d_out, cur, words);
            SF_CUDA_TRY(cudaGetLastError());
            ++ks;
        }
    }
    if (n_keyswitches) *n_keyswitches = ks;
    return SF_OK;
}
