// sf_host.cpp -- host-side parts of the library: parameters (primes, roots,
// NTT and base-conversion tables), seeded samplers, permutations, decoding,
// error reporting, scratch memory and launch instrumentation.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>

#include "sf_internal.h"

// ------------------------------------------------------------------ errors --

static thread_local sf_status t_last_status = SF_OK;
static thread_local char t_last_msg[512] = "";

sf_status sf_set_error(sf_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_last_msg, sizeof(t_last_msg), fmt, ap);
    va_end(ap);
    t_last_status = st;
    return st;
}

extern "C" sf_status sf_last_error(char *buf, size_t len)
{
    if (buf && len) {
        strncpy(buf, t_last_msg, len - 1);
        buf[len - 1] = 0;
    }
    return t_last_status;
}

extern "C" const char *sf_version(void) { return "safhire-gb300 0.1 (sm_103a)"; }

// -------------------------------------------------------- modular helpers --

typedef unsigned __int128 u128;

u64 sf_host_mulmod(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }

u64 sf_host_powmod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = sf_host_mulmod(r, a, q);
        a = sf_host_mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

u64 sf_host_invmod(u64 a, u64 q) { return sf_host_powmod(a % q, q - 2, q); }

u64 sf_shoup_companion(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

// Miller-Rabin with the first twelve prime bases (deterministic below 3.3e24).
static bool is_prime_u64(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : bases) {
        if (n == b) return true;
        if (n % b == 0) return false;
    }
    u64 d = n - 1;
    int r = 0;
    while (!(d & 1)) { d >>= 1; ++r; }
    for (u64 b : bases) {
        u64 x = sf_host_powmod(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int k = 1; k < r && comp; ++k) {
            x = sf_host_mulmod(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

int sf_find_primes(u64 two_n, int bits, int count, u64 *out)
{
    u64 top = (u64)1 << bits;
    u64 k = (top - 2) / two_n;
    int found = 0;
    while (found < count && k > 0) {
        u64 c = k * two_n + 1;
        if (is_prime_u64(c)) out[found++] = c;
        --k;
    }
    return found;
}

u64 sf_root_2n(u64 q, u64 two_n)
{
    for (u64 g = 2; g < q; ++g) {
        u64 x = sf_host_powmod(g, (q - 1) / two_n, q);
        if (sf_host_powmod(x, two_n / 2, q) == q - 1) return x;
    }
    return 0;
}

// ------------------------------------------------------------- samplers ----

u64 SfRng::next()
{
    u64 z = (state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

u64 SfRng::below(u64 n)
{
    u128 m = (u128)next() * n;
    u64 low = (u64)m;
    if (low < n) {
        u64 thr = (0 - n) % n;
        while (low < thr) {
            m = (u128)next() * n;
            low = (u64)m;
        }
    }
    return (u64)(m >> 64);
}

int64_t SfRng::gauss(double sigma)
{
    double u1 = (double)((next() >> 11) + 1) * 0x1.0p-53;
    double u2 = (double)(next() >> 11) * 0x1.0p-53;
    double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    return llround(sigma * z);
}

extern "C" sf_status sf_permutation(uint64_t session_seed, uint32_t round, uint32_t n, uint32_t *perm)
{
    if (!perm && n) return sf_set_error(SF_EINVAL, "sf_permutation: null perm");
    SfRng rng(session_seed ^ ((u64)round * 0x9E3779B97F4A7C15ULL));
    for (uint32_t k = 0; k < n; ++k) perm[k] = k;
    for (uint32_t k = n ? n - 1 : 0; k >= 1; --k) {
        uint32_t r = (uint32_t)rng.below((u64)k + 1);
        std::swap(perm[k], perm[r]);
    }
    return SF_OK;
}

extern "C" sf_status sf_encode_input(const double *x, int64_t count, double scale, int64_t *out)
{
    if (count < 0 || (count && (!x || !out))) return sf_set_error(SF_EINVAL, "sf_encode_input: bad arguments");
    for (int64_t i = 0; i < count; ++i) {
        double v = scale * x[i];
        if (!(fabs(v) < 9.2e18)) return sf_set_error(SF_ERANGE, "sf_encode_input: value %g out of int64 range", v);
        out[i] = llround(v);
    }
    return SF_OK;
}

// Sec. 4.3 "Power computations" at t = 2: m(X^d) of each N-coefficient chunk.
// For odd d, X^k -> X^(k d mod 2N) folded by X^N = -1 is a signed permutation
// of the coefficients, so every output is plus or minus one input.
extern "C" sf_status sf_client_power(const sf_params *p, const int64_t *h_msg, int32_t n_cts, int32_t d, int64_t *h_out)
{
    if (!p || !h_msg || !h_out || n_cts < 1) return sf_set_error(SF_EINVAL, "sf_client_power: bad arguments");
    if (d <= 0 || (d & 1) == 0) return sf_set_error(SF_EINVAL, "sf_client_power: d must be odd and positive");
    const int64_t n = p->n, two_n = 2 * n, dd = d % two_n;
    for (int32_t c = 0; c < n_cts; ++c) {
        const int64_t *m = h_msg + (size_t)c * n;
        int64_t *o = h_out + (size_t)c * n;
        for (int64_t k = 0; k < n; ++k) {
            if (m[k] == INT64_MIN) return sf_set_error(SF_ERANGE, "sf_client_power: coefficient out of range");
            const int64_t e = k * dd % two_n;
            if (e < n) o[e] = m[k];
            else o[e - n] = -m[k];
        }
    }
    return SF_OK;
}

// ---------------------------------------------------------------- params ----

extern "C" sf_status sf_params_create(int32_t log_n, int32_t n_data, int32_t data_bits, int32_t n_special,
                                      int32_t special_bits, double sigma, sf_params **out)
{
    if (!out) return sf_set_error(SF_EINVAL, "sf_params_create: null out");
    *out = nullptr;
    if (log_n < 10 || log_n > 16) return sf_set_error(SF_EINVAL, "log_n must be in [10, 16]");
    if (n_data < 1 || n_special < 1 || n_data + n_special > SF_MAX_MODULI)
        return sf_set_error(SF_EINVAL, "need 1 <= n_data, 1 <= n_special, n_data + n_special <= %d", SF_MAX_MODULI);
    if (n_special > 4) return sf_set_error(SF_EINVAL, "n_special must be <= 4");
    if (data_bits < 20 || data_bits > 50 || special_bits < 20 || special_bits > 50)
        return sf_set_error(SF_EINVAL, "prime sizes must be in [20, 50] bits");
    if (!(sigma > 0 && sigma < 1e6)) return sf_set_error(SF_EINVAL, "sigma out of range");
    int dnum = (n_data + n_special - 1) / n_special;
    if (dnum > SF_MAX_DIGITS) return sf_set_error(SF_EINVAL, "too many key-switch digits");
    sf_params *p = new (std::nothrow) sf_params();
    if (!p) return sf_set_error(SF_ENOMEM, "out of host memory");
    p->log_n = log_n;
    p->n = 1 << log_n;
    p->L = n_data;
    p->K = n_special;
    p->dnum = dnum;
    p->data_bits = data_bits;
    p->special_bits = special_bits;
    p->sigma = sigma;
    u64 two_n = 2 * (u64)p->n;
    std::vector<u64> pr;
    if (data_bits == special_bits) {
        pr.resize(n_data + n_special);
        if (sf_find_primes(two_n, data_bits, n_data + n_special, pr.data()) != n_data + n_special) {
            delete p;
            return sf_set_error(SF_EINVAL, "not enough NTT primes of %d bits", data_bits);
        }
        for (int i = 0; i < n_data; ++i) p->mods.push_back(pr[n_special + i]);
        for (int k = 0; k < n_special; ++k) p->mods.push_back(pr[k]);
    } else {
        std::vector<u64> sp(n_special), dp(n_data + n_special);
        if (sf_find_primes(two_n, special_bits, n_special, sp.data()) != n_special ||
            sf_find_primes(two_n, data_bits, n_data + n_special, dp.data()) != n_data + n_special) {
            delete p;
            return sf_set_error(SF_EINVAL, "not enough NTT primes");
        }
        for (u64 c : dp) {
            if ((int)p->mods.size() == n_data) break;
            if (std::find(sp.begin(), sp.end(), c) == sp.end()) p->mods.push_back(c);
        }
        for (u64 c : sp) p->mods.push_back(c);
    }
    *out = p;
    return SF_OK;
}

extern "C" void sf_params_destroy(sf_params *p) { delete p; }

extern "C" sf_status sf_params_get_info(const sf_params *p, sf_params_info *out)
{
    if (!p || !out) return sf_set_error(SF_EINVAL, "sf_params_get_info: null argument");
    memset(out, 0, sizeof(*out));
    out->log_n = p->log_n;
    out->n = p->n;
    out->n_data = p->L;
    out->n_special = p->K;
    out->dnum = p->dnum;
    out->sigma = p->sigma;
    for (size_t i = 0; i < p->mods.size(); ++i) out->moduli[i] = p->mods[i];
    return SF_OK;
}

// ------------------------------------------------------------------ decode --

// Mixed-radix (Garner) digits of the CRT value, compared against Q/2 and
// converted to a double divided by scale without cancellation.
extern "C" sf_status sf_decode(const sf_params *p, const uint64_t *res, int32_t n_cts, int32_t stride,
                               int32_t count, double scale, double *out)
{
    if (!p || !res || !out || n_cts < 0 || stride < 1 || stride > p->n || (p->n % stride) || count < 0)
        return sf_set_error(SF_EINVAL, "sf_decode: bad arguments");
    int per = p->n / stride;
    if ((int64_t)count > (int64_t)n_cts * per) return sf_set_error(SF_EINVAL, "sf_decode: count too large");
    const int L = p->L;
    const u64 *q = p->mods.data();
    // Garner constants: inv[i][k] = q_k^-1 mod q_i for k < i
    std::vector<u64> inv(L * L, 0);
    for (int i = 0; i < L; ++i)
        for (int k = 0; k < i; ++k) inv[i * L + k] = sf_host_invmod(q[k] % q[i], q[i]);
    // digits of (Q - 1) / 2 in the mixed radix (q_0, q_1, ...): Q odd, so
    // floor(Q/2) = (Q-1)/2.  Compute by halving the mixed-radix digits of Q-1.
    std::vector<u64> half(L);
    {
        // Q - 1 has digits (q_0 - 1, q_1 - 1, ..., q_{L-1} - 1)
        // halve from the most significant digit with a carried remainder
        u64 rem = 0;  // 0 or 1 carried into the next lower digit as rem * q_{i}
        for (int i = L - 1; i >= 0; --i) {
            u128 cur = (u128)(q[i] - 1) + (u128)rem * q[i];
            half[i] = (u64)(cur / 2);
            rem = (u64)(cur % 2);
        }
    }
    std::vector<u64> dig(L);
    for (int32_t v = 0; v < count; ++v) {
        int ct = v / per;
        int pos = (v % per) * stride;
        for (int i = 0; i < L; ++i) {
            u64 x = res[((size_t)ct * L + i) * p->n + pos] % q[i];
            // x_i = (r_i - (d_0 + d_1 q_0 + ...)) / (q_0 ... q_{i-1}) mod q_i
            for (int k = 0; k < i; ++k) {
                x = (x + q[i] - dig[k] % q[i]) % q[i];
                x = sf_host_mulmod(x, inv[i * L + k], q[i]);
            }
            dig[i] = x;
        }
        // compare with floor(Q/2) from the top digit
        int cmp = 0;
        for (int i = L - 1; i >= 0 && cmp == 0; --i) cmp = dig[i] > half[i] ? 1 : (dig[i] < half[i] ? -1 : 0);
        bool neg = cmp > 0;
        if (neg) {
            // Q - value: digits (q_i - 1 - d_i) plus one
            u64 carry = 1;
            for (int i = 0; i < L; ++i) {
                u128 t = (u128)(q[i] - 1 - dig[i]) + carry;
                dig[i] = (u64)(t % q[i]);
                carry = (u64)(t / q[i]);
            }
        }
        long double acc = 0.0L, radix = 1.0L;
        for (int i = 0; i < L; ++i) {
            acc += (long double)dig[i] * radix;
            radix *= (long double)q[i];
        }
        double val = (double)(acc / (long double)scale);
        out[v] = neg ? -val : val;
    }
    return SF_OK;
}

// --------------------------------------------------------- instrumentation --

static const char *k_names[SFK_COUNT] = {
    "ntt_fwd_col", "ntt_fwd_row", "ntt_inv_row", "ntt_inv_col", "elementwise",
    "ks_gather", "ks1_inv_row", "ks2_modup_col", "ks3_inner_row", "ks3_inv_row_p", "ks4_moddown_col",
    "ks5_finish_row",
    "leaf_col", "leaf_row", "shuffle", "bntt_col", "bntt_row", "leaf_prep"};

const char *sf_kernel_name(int kind) { return (kind >= 0 && kind < SFK_COUNT) ? k_names[kind] : "?"; }

void sf_launch_begin(sf_ctx *ctx, int kind, cudaStream_t st, cudaEvent_t *ev0)
{
    ctx->stats[kind].launches++;
    *ev0 = nullptr;
    if (ctx->kernel_timing) {
        if (ctx->event_pool.empty()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            ctx->event_pool.push_back(e);
        }
        *ev0 = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        cudaEventRecord(*ev0, st);
    }
}

void sf_launch_end(sf_ctx *ctx, int kind, cudaStream_t st, cudaEvent_t ev0)
{
    if (!ev0) return;
    cudaEvent_t e1;
    if (ctx->event_pool.empty()) {
        if (cudaEventCreate(&e1) != cudaSuccess) { ctx->event_pool.push_back(ev0); return; }
    } else {
        e1 = ctx->event_pool.back();
        ctx->event_pool.pop_back();
    }
    cudaEventRecord(e1, st);
    ctx->pending.push_back({kind, ev0, e1});
    if (ctx->pending.size() > 4096) sf_collect_timings(ctx);
}

sf_status sf_collect_timings(sf_ctx *ctx)
{
    for (auto &pe : ctx->pending) {
        cudaEventSynchronize(pe.b);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) ctx->stats[pe.kind].ms += ms;
        ctx->event_pool.push_back(pe.a);
        ctx->event_pool.push_back(pe.b);
    }
    ctx->pending.clear();
    return SF_OK;
}

extern "C" sf_status sf_kernel_stats(sf_ctx *ctx, const char **names, int64_t *launches, double *ms, int32_t cap,
                                     int32_t *count)
{
    if (!ctx) return sf_set_error(SF_EINVAL, "sf_kernel_stats: null ctx");
    SF_CUDA_TRY(cudaSetDevice(ctx->device));
    sf_collect_timings(ctx);
    if (count) *count = SFK_COUNT;
    for (int k = 0; k < SFK_COUNT && k < cap; ++k) {
        if (names) names[k] = ctx->stats[k].name;
        if (launches) launches[k] = ctx->stats[k].launches;
        if (ms) ms[k] = ctx->stats[k].ms;
    }
    return SF_OK;
}

extern "C" sf_status sf_kernel_stats_reset(sf_ctx *ctx)
{
    if (!ctx) return sf_set_error(SF_EINVAL, "sf_kernel_stats_reset: null ctx");
    SF_CUDA_TRY(cudaSetDevice(ctx->device));
    sf_collect_timings(ctx);
    for (auto &s : ctx->stats) {
        s.launches = 0;
        s.ms = 0.0;
    }
    return SF_OK;
}

uint64_t sf_next_generation()
{
    static std::atomic<uint64_t> g{1};
    return g.fetch_add(1);
}

void sf_graph_cache_clear(sf_ctx *ctx)
{
    for (auto &e : ctx->graphs) cudaGraphExecDestroy(e.exec);
    ctx->graphs.clear();
}

sf_status sf_scratch(sf_ctx *ctx, size_t bytes, void **out)
{
    if (bytes > ctx->scratch_bytes) {
        sf_graph_cache_clear(ctx);
        if (ctx->scratch) {
            SF_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(ctx->scratch);
            ctx->scratch = nullptr;
            ctx->scratch_bytes = 0;
        }
        size_t want = bytes + bytes / 8;
        if (cudaMalloc(&ctx->scratch, want) != cudaSuccess) {
            cudaGetLastError();
            return sf_set_error(SF_ENOMEM, "scratch allocation of %zu bytes failed", want);
        }
        ctx->scratch_bytes = want;
    }
    *out = ctx->scratch;
    return SF_OK;
}

// ---------------------------------------------------------------- context --

static unsigned brev_bits(unsigned x, int bits)
{
    unsigned r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

template <class T>
static sf_status upload(sf_ctx *ctx, const std::vector<T> &h, const T **out)
{
    void *d = nullptr;
    if (cudaMalloc(&d, sizeof(T) * std::max<size_t>(h.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        return sf_set_error(SF_ENOMEM, "table allocation failed");
    }
    ctx->owned.push_back(d);
    if (!h.empty()) SF_CUDA_TRY(cudaMemcpy(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    *out = (const T *)d;
    return SF_OK;
}

extern "C" sf_status sf_ctx_create(const sf_params *p, int32_t device, sf_ctx **out)
{
    if (!p || !out) return sf_set_error(SF_EINVAL, "sf_ctx_create: null argument");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return sf_set_error(SF_ECUDA, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) return sf_set_error(SF_EINVAL, "device %d out of range", device);
    SF_CUDA_TRY(cudaSetDevice(device));
    sf_ctx *ctx = new sf_ctx();
    ctx->prm = p;
    ctx->device = device;
    ctx->num_sms = 1;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
    ctx->io_buf = nullptr;
    ctx->io_bytes = 0;
    // merges per key-switch launch (the autotuner's pick on the benchmark rounds);
    // the scratch is ks_batch x (3L + max(L, 2K) + max(dnum (L+K), 2L)) limbs
    ctx->ks_batch = p->log_n >= 16 ? 256 : 512;
    ctx->leaf_chunk = 1 << 30;
    ctx->leaf_sparse = 0;   // the transform measured faster than the closed form on GB300
    ctx->ks3_threads = 256;
    ctx->row_radix = 0;
    ctx->mem_budget = (size_t)64 << 30;
    ctx->use_graph = 1;
    ctx->kernel_timing = 0;
    for (int k = 0; k < SFK_COUNT; ++k) ctx->stats.push_back({k_names[k], 0, 0.0});

    const int N = p->n, nm = p->L + p->K, L = p->L, K = p->K;
    SfRing &R = ctx->ring;
    memset(&R, 0, sizeof(R));
    R.log_n = p->log_n;
    R.n = N;
    // N = R x C: C = 2^ceil(log2 N / 2), except 2^16 = 128 x 512, so that the
    // column passes of the largest ring keep 128-point columns
    R.log_c = p->log_n == 16 ? 9 : (p->log_n + 1) / 2;
    R.log_r = p->log_n - R.log_c;
    R.c = 1 << R.log_c;
    R.r = 1 << R.log_r;
    R.L = L;
    R.K = K;
    R.nm = nm;
    R.dnum = p->dnum;
    R.modup_copy = 1;
    for (int a = 0; a < nm; ++a)
        for (int b = 0; b < nm; ++b)
            if (p->mods[a] / 4 >= p->mods[b]) R.modup_copy = 0;
    std::vector<u64> psi((size_t)nm * N), psi_p((size_t)nm * N), ipsi((size_t)nm * N), ipsi_p((size_t)nm * N);
    std::vector<u64> pw((size_t)nm * 2 * N), pw_p((size_t)nm * 2 * N);
    for (int m = 0; m < nm; ++m) {
        u64 q = p->mods[m];
        SfMod &M = R.m[m];
        M.q = q;
        M.two_q = 2 * q;
        // -q^-1 mod 2^64 by Newton iteration on odd q
        u64 inv = q;
        for (int it = 0; it < 6; ++it) inv *= 2 - q * inv;
        M.qinv_neg = 0 - inv;
        M.r_mod = (u64)(((u128)1 << 64) % q);
        M.r_mod_p = sf_shoup_companion(M.r_mod, q);
        M.ninv = sf_host_invmod((u64)N % q, q);
        M.ninv_p = sf_shoup_companion(M.ninv, q);
        M.one_p = sf_shoup_companion(1, q);
        u64 root = sf_root_2n(q, 2 * (u64)N);
        u64 iroot = sf_host_invmod(root, q);
        for (int k = 0; k < N; ++k) {
            unsigned e = brev_bits((unsigned)k, p->log_n);
            u64 w = sf_host_powmod(root, e, q), iw = sf_host_powmod(iroot, e, q);
            psi[(size_t)m * N + k] = w;
            psi_p[(size_t)m * N + k] = sf_shoup_companion(w, q);
            ipsi[(size_t)m * N + k] = iw;
            ipsi_p[(size_t)m * N + k] = sf_shoup_companion(iw, q);
        }
        u64 acc = 1;
        for (int k = 0; k < 2 * N; ++k) {
            pw[(size_t)m * 2 * N + k] = acc;
            pw_p[(size_t)m * 2 * N + k] = sf_shoup_companion(acc, q);
            acc = sf_host_mulmod(acc, root, q);
        }
    }
    // Staged twiddle pairs: column table k < R (global index k), and the
    // row table of each 16-row tile, entry [k][b] = global index
    // m(k) (R + r) + k - m(k) with r = 16 tile + b, m(k) = 2^floor(log2 k).
    std::vector<ulonglong2> colT_f((size_t)nm * R.r), colT_i((size_t)nm * R.r);
    std::vector<ulonglong2> rowT_f((size_t)nm * N), rowT_i((size_t)nm * N);
    for (int m = 0; m < nm; ++m) {
        const u64 *tf = psi.data() + (size_t)m * N, *tfp = psi_p.data() + (size_t)m * N;
        const u64 *ti = ipsi.data() + (size_t)m * N, *tip = ipsi_p.data() + (size_t)m * N;
        for (int k = 0; k < R.r; ++k) {
            colT_f[(size_t)m * R.r + k] = make_ulonglong2(tf[k], tfp[k]);
            colT_i[(size_t)m * R.r + k] = make_ulonglong2(ti[k], tip[k]);
        }
        // row tiles of nb rows (sf_row_nb: 16, or 8 for 256-point rows)
        const int nb = sf_row_nb(R.log_c);
        for (int tile = 0; tile < R.r / nb; ++tile)
            for (int k = 0; k < R.c; ++k)
                for (int b = 0; b < nb; ++b) {
                    size_t dst = (size_t)m * N + ((size_t)tile * R.c + k) * nb + b;
                    if (k == 0) {
                        rowT_f[dst] = rowT_i[dst] = make_ulonglong2(0, 0);
                        continue;
                    }
                    int mk = 1;
                    while (mk * 2 <= k) mk *= 2;
                    size_t gi = (size_t)mk * (R.r + nb * tile + b) + (k - mk);
                    rowT_f[dst] = make_ulonglong2(tf[gi], tfp[gi]);
                    rowT_i[dst] = make_ulonglong2(ti[gi], tip[gi]);
                }
    }
    // powers psi^(C e), e < 2R (closed-form column pass of a sparse polynomial)
    std::vector<ulonglong2> pwc((size_t)nm * 2 * R.r);
    for (int m = 0; m < nm; ++m)
        for (int e = 0; e < 2 * R.r; ++e) {
            const size_t k = (size_t)m * 2 * N + (size_t)e * R.c;
            pwc[(size_t)m * 2 * R.r + e] = make_ulonglong2(pw[k], pw_p[k]);
        }
    // ModUp constants
    int dnum = p->dnum;
    std::vector<u64> mu_inv((size_t)dnum * K, 0), mu_inv_p((size_t)dnum * K, 0);
    std::vector<u64> mu_qhat((size_t)dnum * K * nm, 0), mu_qhat_p((size_t)dnum * K * nm, 0);
    for (int j = 0; j < dnum; ++j) {
        int lo = j * K, hi = std::min((j + 1) * K, L);
        for (int i = lo; i < hi; ++i) {
            u64 qi = p->mods[i];
            u64 qhat_qi = 1;
            for (int i2 = lo; i2 < hi; ++i2)
                if (i2 != i) qhat_qi = sf_host_mulmod(qhat_qi, p->mods[i2] % qi, qi);
            // N^-1 is folded in: the column pass of the inverse NTT leaves it out
            u64 iv = sf_host_mulmod(sf_host_invmod(qhat_qi, qi), sf_host_invmod((u64)N % qi, qi), qi);
            mu_inv[j * K + (i - lo)] = iv;
            mu_inv_p[j * K + (i - lo)] = sf_shoup_companion(iv, qi);
            for (int m = 0; m < nm; ++m) {
                u64 qm = p->mods[m];
                u64 v = 1;
                for (int i2 = lo; i2 < hi; ++i2)
                    if (i2 != i) v = sf_host_mulmod(v, p->mods[i2] % qm, qm);
                mu_qhat[((size_t)j * K + (i - lo)) * nm + m] = v;
                mu_qhat_p[((size_t)j * K + (i - lo)) * nm + m] = sf_shoup_companion(v, qm);
            }
        }
    }
    // ModDown constants.  ModDown(x) = (x_Q - conv_P(x_P)) P^-1: the factor
    // P^-1 is carried by the conversion constants (Phat_k P^-1 mod q_i) and by
    // the reduction of the key products of the data limbs (times P^-1 mod
    // q_i), so the finish is one subtraction; every residue is unchanged.
    std::vector<u64> md_inv(K), md_inv_p(K), md_phat((size_t)K * L), md_phat_p((size_t)K * L), md_pinv(L), md_pinv_p(L);
    for (int i = 0; i < L; ++i) {
        u64 qi = p->mods[i];
        u64 pm = 1;
        for (int k = 0; k < K; ++k) pm = sf_host_mulmod(pm, p->mods[L + k] % qi, qi);
        md_pinv[i] = sf_host_invmod(pm, qi);
        md_pinv_p[i] = sf_shoup_companion(md_pinv[i], qi);
    }
    for (int k = 0; k < K; ++k) {
        u64 pk = p->mods[L + k];
        u64 ph = 1;
        for (int k2 = 0; k2 < K; ++k2)
            if (k2 != k) ph = sf_host_mulmod(ph, p->mods[L + k2] % pk, pk);
        md_inv[k] = sf_host_mulmod(sf_host_invmod(ph, pk), sf_host_invmod((u64)N % pk, pk), pk);
        md_inv_p[k] = sf_shoup_companion(md_inv[k], pk);
        for (int i = 0; i < L; ++i) {
            u64 qi = p->mods[i];
            u64 v = 1;
            for (int k2 = 0; k2 < K; ++k2)
                if (k2 != k) v = sf_host_mulmod(v, p->mods[L + k2] % qi, qi);
            v = sf_host_mulmod(v, md_pinv[i], qi);
            md_phat[(size_t)k * L + i] = v;
            md_phat_p[(size_t)k * L + i] = sf_shoup_companion(v, qi);
        }
    }
    sf_status st = SF_OK;
#define UP(v, f)                                      \
    if (st == SF_OK) st = upload(ctx, v, &R.f);
    UP(psi, psi) UP(psi_p, psi_p) UP(ipsi, ipsi) UP(ipsi_p, ipsi_p) UP(pw, pw) UP(pw_p, pw_p)
    UP(colT_f, colT_f) UP(colT_i, colT_i) UP(rowT_f, rowT_f) UP(rowT_i, rowT_i) UP(pwc, pwc)
    UP(mu_inv, mu_inv) UP(mu_inv_p, mu_inv_p) UP(mu_qhat, mu_qhat) UP(mu_qhat_p, mu_qhat_p)
    UP(md_inv, md_inv) UP(md_inv_p, md_inv_p) UP(md_phat, md_phat) UP(md_phat_p, md_phat_p)
    UP(md_pinv, md_pinv) UP(md_pinv_p, md_pinv_p)
#undef UP
    if (st == SF_OK) st = sf_ntt_init_attributes();
    if (st == SF_OK) st = sf_ks_init_attributes();
    if (st == SF_OK) st = sf_bntt_init_attributes();
    if (st == SF_OK) st = sf_layer_init_attributes();
    if (st == SF_OK) {
        if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            st = sf_set_error(SF_ENOMEM, "status word allocation failed");
        } else {
            ctx->owned.push_back(ctx->d_status);
            cudaMemset(ctx->d_status, 0, sizeof(int));
            R.status = ctx->d_status;
        }
    }
    if (st != SF_OK) {
        sf_ctx_destroy(ctx);
        return st;
    }
    *out = ctx;
    return SF_OK;
}

extern "C" void sf_ctx_destroy(sf_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    sf_collect_timings(ctx);
    sf_graph_cache_clear(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    for (void *d : ctx->owned) cudaFree(d);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->io_buf) cudaFree(ctx->io_buf);
    delete ctx;
}

extern "C" sf_status sf_ctx_get_option(const sf_ctx *ctx, const char *name, int64_t *value)
{
    if (!ctx || !name || !value) return sf_set_error(SF_EINVAL, "sf_ctx_get_option: null argument");
    if (!strcmp(name, "ks_batch")) *value = ctx->ks_batch;
    else if (!strcmp(name, "ks3_threads")) *value = ctx->ks3_threads;
    else if (!strcmp(name, "row_radix")) *value = ctx->row_radix;
    else if (!strcmp(name, "leaf_sparse")) *value = ctx->leaf_sparse;
    else if (!strcmp(name, "leaf_chunk")) *value = ctx->leaf_chunk;
    else if (!strcmp(name, "mem_budget")) *value = (int64_t)ctx->mem_budget;
    else if (!strcmp(name, "use_graph")) *value = ctx->use_graph;
    else if (!strcmp(name, "kernel_timing")) *value = ctx->kernel_timing;
    else return sf_set_error(SF_EINVAL, "unknown option %s", name);
    return SF_OK;
}

extern "C" sf_status sf_ctx_set_option(sf_ctx *ctx, const char *name, int64_t value)
{
    if (!ctx || !name) return sf_set_error(SF_EINVAL, "sf_ctx_set_option: null argument");
    if (!strcmp(name, "ks_batch")) {
        if (value < 1 || value > 4096) return sf_set_error(SF_EINVAL, "ks_batch must be in [1, 4096]");
        ctx->ks_batch = (int)value;
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "leaf_sparse")) {
        if (value < -1 || value > 128) return sf_set_error(SF_EINVAL, "leaf_sparse must be in [-1, 128]");
        ctx->leaf_sparse = (int)value;
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "ks3_threads")) {
        if (value != 256 && value != 512) return sf_set_error(SF_EINVAL, "ks3_threads must be 256 or 512");
        ctx->ks3_threads = (int)value;
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "row_radix")) {
        if (value < 0 || value > 2) return sf_set_error(SF_EINVAL, "row_radix must be 0, 1 or 2");
        ctx->row_radix = (int)value;
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "leaf_chunk")) {
        if (value < 1 || (value & (value - 1))) return sf_set_error(SF_EINVAL, "leaf_chunk must be a power of two");
        ctx->leaf_chunk = (int)std::min<int64_t>(value, 1 << 30);
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "mem_budget")) {
        if (value < (1 << 20)) return sf_set_error(SF_EINVAL, "mem_budget must be at least 1 MiB");
        ctx->mem_budget = (size_t)value;
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "use_graph")) {
        if (value != 0 && value != 1) return sf_set_error(SF_EINVAL, "use_graph must be 0 or 1");
        ctx->use_graph = (int)value;
    } else if (!strcmp(name, "clear_graphs")) {
        SF_CUDA_TRY(cudaSetDevice(ctx->device));
        SF_CUDA_TRY(cudaDeviceSynchronize());
        sf_graph_cache_clear(ctx);
    } else if (!strcmp(name, "kernel_timing")) {
        if (value != 0 && value != 1) return sf_set_error(SF_EINVAL, "kernel_timing must be 0 or 1");
        SF_CUDA_TRY(cudaSetDevice(ctx->device));
        if (!value) sf_collect_timings(ctx);
        ctx->kernel_timing = (int)value;
    } else {
        return sf_set_error(SF_EINVAL, "unknown option '%s'", name);
    }
    return SF_OK;
}

extern "C" sf_status sf_sync(sf_ctx *ctx, void *stream)
{
    if (!ctx) return sf_set_error(SF_EINVAL, "sf_sync: null ctx");
    SF_CUDA_TRY(cudaSetDevice(ctx->device));
    SF_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int h = 0;
    SF_CUDA_TRY(cudaMemcpy(&h, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        SF_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(int)));
        return sf_set_error((sf_status)h, "device status word reported error %d", h);
    }
    return SF_OK;
}
