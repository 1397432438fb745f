/*
 * oracle.c -- plain, slow CPU oracle for the Safhire server-side linear-layer
 * round (arXiv 2509.01253).  TEST INFRASTRUCTURE ONLY: the tests, the smoke
 * check and the bench's CPU-baseline leg are the only callers.  The product
 * (the CUDA library under paper_2509_01253_gb300/) never links, loads or runs
 * this file, and this file shares no code, header, table or constant with it.
 *
 * Everything here is the textbook definition, written out:
 *   - negacyclic products in Z_q[X]/(X^N+1) by the schoolbook double loop
 *     (Sec. 2.1: the ring is the cyclotomic Phi_M with M = 2N, t = 2),
 *   - the ring automorphism X -> X^d by index arithmetic (Sec. 2.2),
 *   - hybrid RNS key switching: digit decomposition, fast base conversion
 *     (ModUp), inner product with the key, ModDown (Sec. 2.2, Sec. 4.2),
 *   - the weight polynomial of one linear-layer output built from the
 *     extracted rows N^-1 X^-k ct (Sec. 4.4 "Partial trace extraction",
 *     "Unshuffle", "Convolution"),
 *   - SplitMix64 / Lemire / Box-Muller samplers and Fisher-Yates shuffling
 *     (Sec. 4.4 "Shuffle"), each from its published definition.
 * The recursive packing (Sec. 2.4, Sec. 4.4 "Fast Packing") and the CRT
 * decoding are orchestrated from oracle/__init__.py on top of these.
 *
 * Arithmetic: residues are uint64 in [0, q); products use unsigned __int128.
 * OpenMP only spreads independent limbs / products over host cores; it does
 * not change any arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------ */
/* scalar modular arithmetic                                            */
/* ------------------------------------------------------------------ */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a * b) % q);
}

static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a + b) % q);
}

static uint64_t submod(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a + q - b) % q);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime q (Fermat) */
static uint64_t invmod(uint64_t a, uint64_t q)
{
    return powmod(a % q, q - 2, q);
}

/* a signed integer reduced into [0, q) */
static uint64_t from_signed(int64_t v, uint64_t q)
{
    int64_t r = v % (int64_t)q;
    if (r < 0) r += (int64_t)q;
    return (uint64_t)r;
}

uint64_t or_mulmod(uint64_t a, uint64_t b, uint64_t q) { return mulmod(a, b, q); }
uint64_t or_invmod(uint64_t a, uint64_t q) { return invmod(a, q); }

/* ------------------------------------------------------------------ */
/* primes q = 1 (mod 2N)                                                */
/* ------------------------------------------------------------------ */

/* Deterministic Miller-Rabin: the bases 2..37 decide every n < 3.3e24. */
int or_is_prime(uint64_t n)
{
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* The `count` largest primes below 2^bits that are 1 mod two_n, descending. */
int or_find_primes(uint64_t two_n, int bits, int count, uint64_t *out)
{
    uint64_t top = (bits >= 64) ? UINT64_MAX : ((uint64_t)1 << bits);
    uint64_t k = (top - 2) / two_n;            /* k*two_n + 1 < top */
    int found = 0;
    while (found < count && k > 0) {
        uint64_t c = k * two_n + 1;
        if (or_is_prime(c)) out[found++] = c;
        k--;
    }
    return found;
}

/* A primitive 2N-th root of unity mod q: g^((q-1)/2N) with (.)^N = -1. */
uint64_t or_primitive_root_2n(uint64_t q, uint64_t two_n)
{
    for (uint64_t g = 2; g < q; g++) {
        uint64_t x = powmod(g, (q - 1) / two_n, q);
        if (powmod(x, two_n / 2, q) == q - 1) return x;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* seeded samplers                                                      */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood 2014): state += golden gamma, then mix. */
static uint64_t sm64_next(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Lemire (2019) unbiased bounded integer in [0, n): multiply, reject the
 * low-word values below 2^64 mod n. */
static uint64_t uniform_below(uint64_t *state, uint64_t n)
{
    u128 m = (u128)sm64_next(state) * n;
    uint64_t low = (uint64_t)m;
    if (low < n) {
        uint64_t threshold = (0 - n) % n;
        while (low < threshold) {
            m = (u128)sm64_next(state) * n;
            low = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* Rounded Gaussian N(0, sigma^2): Box-Muller (cosine branch) on two 53-bit
 * uniforms, u1 in (0, 1], u2 in [0, 1), then round half away from zero. */
static int64_t gaussian(uint64_t *state, double sigma)
{
    double u1 = (double)((sm64_next(state) >> 11) + 1) * 0x1.0p-53;
    double u2 = (double)(sm64_next(state) >> 11) * 0x1.0p-53;
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    return llround(sigma * z);
}

void or_splitmix64(uint64_t seed, int64_t count, uint64_t *out)
{
    uint64_t st = seed;
    for (int64_t i = 0; i < count; i++) out[i] = sm64_next(&st);
}

/* Secret key s(X): N coefficients uniform in {-1, 0, 1} (ternary). */
void or_sample_secret(uint64_t seed, int n, int64_t *s)
{
    uint64_t st = seed;
    for (int k = 0; k < n; k++) s[k] = (int64_t)uniform_below(&st, 3) - 1;
}

/* Encryption randomness for n_cts ciphertexts: per ciphertext, the mask a
 * (limb by limb, uniform mod q_i; uniform mod Q by CRT), then the error e. */
void or_sample_encrypt(uint64_t seed, int n, int n_limbs, const uint64_t *q,
                       int n_cts, double sigma, uint64_t *a, int64_t *e)
{
    uint64_t st = seed;
    for (int j = 0; j < n_cts; j++) {
        for (int i = 0; i < n_limbs; i++)
            for (int k = 0; k < n; k++)
                a[((size_t)j * n_limbs + i) * n + k] = uniform_below(&st, q[i]);
        for (int k = 0; k < n; k++) e[(size_t)j * n + k] = gaussian(&st, sigma);
    }
}

/* Rotation-key randomness for automorphism index d: the stream starts at
 * seed XOR d*gamma; per digit, alpha over the n_mod extended moduli, then e. */
void or_sample_rotkey(uint64_t seed, int64_t d, int n, int dnum, int n_mod,
                      const uint64_t *mods, double sigma, uint64_t *alpha, int64_t *e)
{
    uint64_t st = seed ^ ((uint64_t)d * 0x9E3779B97F4A7C15ULL);
    for (int j = 0; j < dnum; j++) {
        for (int m = 0; m < n_mod; m++)
            for (int k = 0; k < n; k++)
                alpha[((size_t)j * n_mod + m) * n + k] = uniform_below(&st, mods[m]);
        for (int k = 0; k < n; k++) e[(size_t)j * n + k] = gaussian(&st, sigma);
    }
}

/* Sec. 4.4 "Shuffle": sigma_r drawn uniformly from a seed derived from the
 * session identifier and the round number.  Fisher-Yates from the top;
 * perm[k] = sigma(k), i.e. position k holds row sigma(k). */
void or_permutation(uint64_t session_seed, uint32_t round, uint32_t n, uint32_t *perm)
{
    uint64_t st = session_seed ^ ((uint64_t)round * 0x9E3779B97F4A7C15ULL);
    for (uint32_t k = 0; k < n; k++) perm[k] = k;
    if (n < 2) return;
    for (uint32_t k = n - 1; k >= 1; k--) {
        uint32_t r = (uint32_t)uniform_below(&st, (uint64_t)k + 1);
        uint32_t t = perm[k];
        perm[k] = perm[r];
        perm[r] = t;
    }
}

/* Fixed-point encoding: round(scale * x), half away from zero. */
void or_quantize(const double *x, int64_t count, double scale, int64_t *out)
{
    for (int64_t i = 0; i < count; i++) out[i] = llround(scale * x[i]);
}

/* ------------------------------------------------------------------ */
/* ring Z_q[X]/(X^N + 1)                                                */
/* ------------------------------------------------------------------ */

/* c = a * b in Z_q[X]/(X^N+1) by the schoolbook double loop:
 * a_i b_k lands on X^(i+k), and X^(i+k) = -X^(i+k-N) when i+k >= N.
 * Positive and negative contributions are summed exactly in 128 bits
 * (N * q^2 < 2^128 for q < 2^56, N <= 2^16) and reduced once. */
void or_polymul(const uint64_t *a, const uint64_t *b, uint64_t *c, int n, uint64_t q)
{
    u128 *pos = (u128 *)calloc((size_t)n, sizeof(u128));
    u128 *neg = (u128 *)calloc((size_t)n, sizeof(u128));
    for (int i = 0; i < n; i++) {
        if (a[i] == 0) continue;            /* a zero term adds nothing */
        u128 ai = a[i];
        for (int k = 0; k < n - i; k++) pos[i + k] += ai * b[k];
        for (int k = n - i; k < n; k++) neg[i + k - n] += ai * b[k];
    }
    for (int t = 0; t < n; t++) c[t] = submod((uint64_t)(pos[t] % q), (uint64_t)(neg[t] % q), q);
    free(pos);
    free(neg);
}

/* tau_d: a(X) -> a(X^d), d odd.  Coefficient i moves to i*d mod 2N and
 * changes sign when that exponent is >= N (X^N = -1). */
void or_automorphism(const uint64_t *a, uint64_t *out, int n, int64_t d, uint64_t q)
{
    int64_t two_n = 2 * (int64_t)n;
    int64_t dd = ((d % two_n) + two_n) % two_n;
    for (int k = 0; k < n; k++) out[k] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t e = (i * dd) % two_n;
        if (e < n) out[e] = addmod(out[e], a[i], q);
        else out[e - n] = submod(out[e - n], a[i], q);
    }
}

/* X^s * a(X) for any integer s (X^(2N) = 1, X^N = -1). */
void or_monomial_mul(const uint64_t *a, uint64_t *out, int n, int64_t s, uint64_t q)
{
    int64_t two_n = 2 * (int64_t)n;
    int64_t ss = ((s % two_n) + two_n) % two_n;
    for (int64_t i = 0; i < n; i++) {
        int64_t e = (i + ss) % two_n;
        if (e < n) out[e] = a[i];
        else out[e - n] = (a[i] == 0) ? 0 : q - a[i];
    }
}

/* ------------------------------------------------------------------ */
/* RLWE encryption / decryption (Sec. 2.1; t = 2 so Omega_0^* = 1/N and the
 * dual-basis factors reduce to the coefficient embedding)              */
/* ------------------------------------------------------------------ */

/* b = a*s + m + e  (mod q_i, every limb); a is given (sampled above). */
void or_encrypt(int n, int n_limbs, const uint64_t *q, const int64_t *s,
                const int64_t *m, const uint64_t *a, const int64_t *e, uint64_t *b)
{
    #pragma omp parallel for
    for (int i = 0; i < n_limbs; i++) {
        uint64_t *sq = (uint64_t *)malloc(sizeof(uint64_t) * n);
        uint64_t *as = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int k = 0; k < n; k++) sq[k] = from_signed(s[k], q[i]);
        or_polymul(a + (size_t)i * n, sq, as, n, q[i]);
        for (int k = 0; k < n; k++)
            b[(size_t)i * n + k] = addmod(addmod(as[k], from_signed(m[k], q[i]), q[i]),
                                          from_signed(e[k], q[i]), q[i]);
        free(sq);
        free(as);
    }
}

/* plaintext residues b - a*s  (mod q_i, every limb) */
void or_decrypt(int n, int n_limbs, const uint64_t *q, const int64_t *s,
                const uint64_t *a, const uint64_t *b, uint64_t *m)
{
    #pragma omp parallel for
    for (int i = 0; i < n_limbs; i++) {
        uint64_t *sq = (uint64_t *)malloc(sizeof(uint64_t) * n);
        uint64_t *as = (uint64_t *)malloc(sizeof(uint64_t) * n);
        for (int k = 0; k < n; k++) sq[k] = from_signed(s[k], q[i]);
        or_polymul(a + (size_t)i * n, sq, as, n, q[i]);
        for (int k = 0; k < n; k++) m[(size_t)i * n + k] = submod(b[(size_t)i * n + k], as[k], q[i]);
        free(sq);
        free(as);
    }
}

/* ------------------------------------------------------------------ */
/* hybrid key switching (Sec. 2.2, Sec. 4.2)                            */
/*                                                                      */
/* Moduli: mods[0..L-1] = data primes q_i (Q = prod q_i),               */
/*         mods[L..L+K-1] = special primes p_k (P = prod p_k).          */
/* Digit j holds the data limbs D_j = [jK, min((j+1)K, L)).             */
/* ------------------------------------------------------------------ */

static int digit_lo(int j, int K) { return j * K; }
static int digit_hi(int j, int K, int L) { int h = (j + 1) * K; return h < L ? h : L; }

/* ModUp of digit j (fast base conversion, no correction):
 *   [x]_m = sum_{i in D_j} [x_i * Qhat_i^{-1}]_{q_i} * (Qhat_i mod m)  (mod m)
 * for m outside D_j; inside D_j the residue is x_m itself.
 * x: data-limb residues [L][n] (coefficient domain); out: [L+K][n]. */
void or_modup(int n, int L, int K, const uint64_t *mods, int j,
              const uint64_t *x, uint64_t *out)
{
    int lo = digit_lo(j, K), hi = digit_hi(j, K, L);
    int nm = L + K;
    #pragma omp parallel for
    for (int m = 0; m < nm; m++) {
        uint64_t qm = mods[m];
        if (m >= lo && m < hi) {
            memcpy(out + (size_t)m * n, x + (size_t)m * n, sizeof(uint64_t) * n);
            continue;
        }
        for (int k = 0; k < n; k++) {
            uint64_t acc = 0;
            for (int i = lo; i < hi; i++) {
                /* Qhat_i = prod_{i' in D_j, i' != i} q_i' */
                uint64_t qhat_mod_qi = 1, qhat_mod_m = 1;
                for (int i2 = lo; i2 < hi; i2++) {
                    if (i2 == i) continue;
                    qhat_mod_qi = mulmod(qhat_mod_qi, mods[i2] % mods[i], mods[i]);
                    qhat_mod_m = mulmod(qhat_mod_m, mods[i2] % qm, qm);
                }
                uint64_t yi = mulmod(x[(size_t)i * n + k], invmod(qhat_mod_qi, mods[i]), mods[i]);
                acc = addmod(acc, mulmod(yi % qm, qhat_mod_m, qm), qm);
            }
            out[(size_t)m * n + k] = acc;
        }
    }
}

/* ModDown (truncating): for each data limb i,
 *   conv_i = sum_k [x_{p_k} * Phat_k^{-1}]_{p_k} * (Phat_k mod q_i)  (mod q_i)
 *   out_i  = (x_i - conv_i) * P^{-1}  (mod q_i).
 * x: [L+K][n]; out: [L][n]. */
void or_moddown(int n, int L, int K, const uint64_t *mods, const uint64_t *x, uint64_t *out)
{
    #pragma omp parallel for
    for (int i = 0; i < L; i++) {
        uint64_t qi = mods[i];
        uint64_t p_mod_qi = 1;
        for (int k = 0; k < K; k++) p_mod_qi = mulmod(p_mod_qi, mods[L + k] % qi, qi);
        uint64_t p_inv = invmod(p_mod_qi, qi);
        for (int c = 0; c < n; c++) {
            uint64_t conv = 0;
            for (int k = 0; k < K; k++) {
                uint64_t pk = mods[L + k];
                uint64_t phat_mod_pk = 1, phat_mod_qi = 1;
                for (int k2 = 0; k2 < K; k2++) {
                    if (k2 == k) continue;
                    phat_mod_pk = mulmod(phat_mod_pk, mods[L + k2] % pk, pk);
                    phat_mod_qi = mulmod(phat_mod_qi, mods[L + k2] % qi, qi);
                }
                uint64_t yk = mulmod(x[(size_t)(L + k) * n + c], invmod(phat_mod_pk, pk), pk);
                conv = addmod(conv, mulmod(yk % qi, phat_mod_qi, qi), qi);
            }
            out[(size_t)i * n + c] = mulmod(submod(x[(size_t)i * n + c], conv, qi), p_inv, qi);
        }
    }
}

/* Rotation key for tau_d (Sec. 4.2: an RLWE encryption under s(X) of the
 * gadget-scaled s(X^d)).  For digit j and every extended modulus m:
 *   alpha_j           (uniform, given)
 *   b_j = alpha_j * s + e_j - [P * g_j]_m * s(X^d)   (mod m)
 * with g_j = 1 mod q_i for i in D_j and 0 mod the other data primes;
 * P = 0 mod every special prime, so that term vanishes there.
 * key layout: [dnum][2][L+K][n], part 0 = alpha, part 1 = b. */
void or_rotkey(int n, int L, int K, const uint64_t *mods, int64_t d, const int64_t *s,
               const uint64_t *alpha, const int64_t *e, uint64_t *key)
{
    int nm = L + K;
    int dnum = (L + K - 1) / K;
    int64_t *sd = (int64_t *)malloc(sizeof(int64_t) * n);
    {   /* s(X^d) over the integers: coefficients stay in {-1, 0, 1} */
        int64_t two_n = 2 * (int64_t)n;
        int64_t dd = ((d % two_n) + two_n) % two_n;
        for (int k = 0; k < n; k++) sd[k] = 0;
        for (int64_t i = 0; i < n; i++) {
            int64_t ex = (i * dd) % two_n;
            if (ex < n) sd[ex] += s[i];
            else sd[ex - n] -= s[i];
        }
    }
    #pragma omp parallel for collapse(2)
    for (int j = 0; j < dnum; j++) {
        for (int m = 0; m < nm; m++) {
            uint64_t qm = mods[m];
            const uint64_t *al = alpha + ((size_t)j * nm + m) * n;
            uint64_t *ka = key + (((size_t)j * 2 + 0) * nm + m) * n;
            uint64_t *kb = key + (((size_t)j * 2 + 1) * nm + m) * n;
            uint64_t *sq = (uint64_t *)malloc(sizeof(uint64_t) * n);
            for (int k = 0; k < n; k++) sq[k] = from_signed(s[k], qm);
            memcpy(ka, al, sizeof(uint64_t) * n);
            or_polymul(al, sq, kb, n, qm);
            uint64_t pg = 0;                          /* [P * g_j]_m */
            if (m < L && m >= digit_lo(j, K) && m < digit_hi(j, K, L)) {
                pg = 1;
                for (int k = 0; k < K; k++) pg = mulmod(pg, mods[L + k] % qm, qm);
            }
            for (int k = 0; k < n; k++) {
                uint64_t v = addmod(kb[k], from_signed(e[(size_t)j * n + k], qm), qm);
                v = submod(v, mulmod(pg, from_signed(sd[k], qm), qm), qm);
                kb[k] = v;
            }
            free(sq);
        }
    }
    free(sd);
}

/* Key switching of the mask polynomial c (an RLWE mask under s(X^d)):
 *   ext_j = ModUp_j(c);  A = sum_j ext_j * alpha_j;  B = sum_j ext_j * b_j  (mod PQ)
 *   returns (ModDown(A), ModDown(B)).
 * c: [L][n]; key: [dnum][2][L+K][n]; outA, outB: [L][n]. */
void or_keyswitch(int n, int L, int K, const uint64_t *mods, const uint64_t *key,
                  const uint64_t *c, uint64_t *outA, uint64_t *outB)
{
    int nm = L + K;
    int dnum = (L + K - 1) / K;
    size_t poly = (size_t)n;
    uint64_t *ext = (uint64_t *)malloc(sizeof(uint64_t) * dnum * nm * poly);
    uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * dnum * 2 * nm * poly);
    uint64_t *acc = (uint64_t *)malloc(sizeof(uint64_t) * 2 * nm * poly);
    for (int j = 0; j < dnum; j++) or_modup(n, L, K, mods, j, c, ext + (size_t)j * nm * poly);
    #pragma omp parallel for collapse(3)
    for (int j = 0; j < dnum; j++)
        for (int part = 0; part < 2; part++)
            for (int m = 0; m < nm; m++)
                or_polymul(ext + ((size_t)j * nm + m) * poly,
                           key + (((size_t)j * 2 + part) * nm + m) * poly,
                           prod + (((size_t)j * 2 + part) * nm + m) * poly, n, mods[m]);
    for (int part = 0; part < 2; part++)
        for (int m = 0; m < nm; m++)
            for (int k = 0; k < n; k++) {
                uint64_t s = 0;
                for (int j = 0; j < dnum; j++)
                    s = addmod(s, prod[(((size_t)j * 2 + part) * nm + m) * poly + k], mods[m]);
                acc[((size_t)part * nm + m) * poly + k] = s;
            }
    or_moddown(n, L, K, mods, acc, outA);
    or_moddown(n, L, K, mods, acc + (size_t)nm * poly, outB);
    free(ext);
    free(prod);
    free(acc);
}

/* Automorphism plus key switch: ct = (a, b) under s(X) ->
 *   (a', b') = (tau_d a, tau_d b) under s(X^d) ->
 *   (KS_A, b' + KS_B) under s(X).
 * ct, out: [2][L][n]. */
void or_rotate(int n, int L, int K, const uint64_t *mods, const uint64_t *key, int64_t d,
               const uint64_t *ct, uint64_t *out)
{
    size_t poly = (size_t)n;
    uint64_t *ta = (uint64_t *)malloc(sizeof(uint64_t) * L * poly);
    uint64_t *tb = (uint64_t *)malloc(sizeof(uint64_t) * L * poly);
    uint64_t *kb = (uint64_t *)malloc(sizeof(uint64_t) * L * poly);
    for (int i = 0; i < L; i++) {
        or_automorphism(ct + (size_t)i * poly, ta + (size_t)i * poly, n, d, mods[i]);
        or_automorphism(ct + (size_t)(L + i) * poly, tb + (size_t)i * poly, n, d, mods[i]);
    }
    or_keyswitch(n, L, K, mods, key, ta, out, kb);
    for (int i = 0; i < L; i++)
        for (int k = 0; k < n; k++)
            out[(size_t)(L + i) * poly + k] = addmod(tb[(size_t)i * poly + k], kb[(size_t)i * poly + k], mods[i]);
    free(ta);
    free(tb);
    free(kb);
}

/* ------------------------------------------------------------------ */
/* one linear-layer output (Sec. 4.4, steps 6-8, gamma = 0)             */
/*                                                                      */
/* The extracted row for stream position p = j*N + k is N^-1 X^-k ct_j  */
/* (at t = 2, Tr(m X^-k) = N m_k).  Unshuffling places input index i at */
/* position p = sigma_prev^-1(i).  The output row                       */
/*   y_o = sum_taps W[o,i] * N^-1 X^-k ct_j = sum_j w_{o,j} * ct_j      */
/* where w_{o,j} gathers the taps that fall into ciphertext j.          */
/* tap_pos[t]: unshuffled stream position of tap t; tap_w[t]: its       */
/* quantised weight.  cts: [k_in][2][L][n]; out: [2][L][n].             */
/* ------------------------------------------------------------------ */
void or_linear_output(int n, int L, const uint64_t *q, int k_in, const uint64_t *cts,
                      int n_taps, const int64_t *tap_pos, const int64_t *tap_w, uint64_t *out)
{
    size_t poly = (size_t)n;
    memset(out, 0, sizeof(uint64_t) * 2 * L * poly);
    #pragma omp parallel for
    for (int i = 0; i < L; i++) {
        uint64_t qi = q[i];
        uint64_t n_inv = invmod((uint64_t)n % qi, qi);
        uint64_t *w = (uint64_t *)malloc(sizeof(uint64_t) * poly);
        uint64_t *prod = (uint64_t *)malloc(sizeof(uint64_t) * poly);
        for (int j = 0; j < k_in; j++) {
            int any = 0;
            memset(w, 0, sizeof(uint64_t) * poly);
            for (int t = 0; t < n_taps; t++) {
                if (tap_pos[t] / n != j) continue;
                int64_t k = tap_pos[t] % n;
                uint64_t v = mulmod(from_signed(tap_w[t], qi), n_inv, qi);
                /* X^-k = -X^(N-k) for k > 0 */
                if (k == 0) w[0] = addmod(w[0], v, qi);
                else w[n - k] = submod(w[n - k], v, qi);
                any = 1;
            }
            if (!any) continue;
            for (int part = 0; part < 2; part++) {
                const uint64_t *src = cts + (((size_t)j * 2 + part) * L + i) * poly;
                or_polymul(w, src, prod, n, qi);
                uint64_t *dst = out + ((size_t)part * L + i) * poly;
                for (int c = 0; c < n; c++) dst[c] = addmod(dst[c], prod[c], qi);
            }
        }
        free(w);
        free(prod);
    }
}

/* elementwise helpers used by the packing recursion */
void or_ct_add(int n_polys, int n, const uint64_t *q_per_poly, const uint64_t *x,
               const uint64_t *y, uint64_t *out)
{
    for (int p = 0; p < n_polys; p++)
        for (int k = 0; k < n; k++)
            out[(size_t)p * n + k] = addmod(x[(size_t)p * n + k], y[(size_t)p * n + k], q_per_poly[p]);
}

void or_ct_sub(int n_polys, int n, const uint64_t *q_per_poly, const uint64_t *x,
               const uint64_t *y, uint64_t *out)
{
    for (int p = 0; p < n_polys; p++)
        for (int k = 0; k < n; k++)
            out[(size_t)p * n + k] = submod(x[(size_t)p * n + k], y[(size_t)p * n + k], q_per_poly[p]);
}
