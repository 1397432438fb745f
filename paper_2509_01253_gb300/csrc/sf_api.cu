// sf_api.cu -- the C ABI declared in include/safhire.h: keys, encryption,
// layers, and the server round.  Argument marshalling and workspace layout
// live here; every arithmetic step runs in the kernels of sf_ntt.cu,
// sf_ks.cu and sf_layer.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sf_internal.h"
#include "sf_ks.h"
#include "sf_layer.h"
#include "sf_round.h"

static sf_status device_buffer(void **p, size_t bytes)
{
    if (cudaMalloc(p, std::max<size_t>(bytes, 8)) != cudaSuccess) {
        cudaGetLastError();
        return sf_set_error(SF_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    return SF_OK;
}

// ----------------------------------------------------------------- keygen --

extern "C" sf_status sf_keygen(sf_ctx *ctx, uint64_t seed, sf_secret_key **out)
{
    SF_CHECK_CTX(ctx);
    if (!out) return sf_set_error(SF_EINVAL, "sf_keygen: null out");
    *out = nullptr;
    const SfRing &R = ctx->ring;
    sf_secret_key *sk = new sf_secret_key();
    sk->ctx = ctx;
    sk->s.resize(R.n);
    SfRng rng(seed);
    for (int k = 0; k < R.n; ++k) sk->s[k] = (int64_t)rng.below(3) - 1;
    sf_status st = device_buffer((void **)&sk->d_s_mont, sizeof(u64) * R.nm * R.n);
    if (st != SF_OK) {
        delete sk;
        return st;
    }
    int64_t *d_s = nullptr;
    st = device_buffer((void **)&d_s, sizeof(int64_t) * R.n);
    if (st == SF_OK && cudaMemcpy(d_s, sk->s.data(), sizeof(int64_t) * R.n, cudaMemcpyHostToDevice) != cudaSuccess)
        st = sf_set_error(SF_ECUDA, "sf_keygen: upload failed");
    if (st == SF_OK) st = sf_signed_to_residues(ctx, d_s, sk->d_s_mont, R.nm, R.nm, 0, 0);
    std::vector<SfPolyJob> jobs;
    for (int m = 0; m < R.nm; ++m) jobs.push_back({sk->d_s_mont + (size_t)m * R.n, sk->d_s_mont + (size_t)m * R.n, m});
    if (st == SF_OK) st = sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), false, 0);
    if (st == SF_OK) st = sf_to_mont(ctx, sk->d_s_mont, R.nm, R.nm, 0, 0);
    if (st == SF_OK && cudaDeviceSynchronize() != cudaSuccess) st = sf_set_error(SF_ECUDA, "sf_keygen: device error");
    if (d_s) cudaFree(d_s);
    if (st != SF_OK) {
        sf_secret_key_destroy(sk);
        return st;
    }
    *out = sk;
    return SF_OK;
}

extern "C" void sf_secret_key_destroy(sf_secret_key *sk)
{
    if (!sk) return;
    cudaSetDevice(sk->ctx->device);
    if (sk->d_s_mont) cudaFree(sk->d_s_mont);
    delete sk;
}

extern "C" sf_status sf_secret_key_export(const sf_secret_key *sk, int64_t *h_s)
{
    if (!sk || !h_s) return sf_set_error(SF_EINVAL, "sf_secret_key_export: null argument");
    memcpy(h_s, sk->s.data(), sizeof(int64_t) * sk->s.size());
    return SF_OK;
}

extern "C" sf_status sf_gen_rotation_keys(sf_ctx *ctx, const sf_secret_key *sk, const int32_t *d, int32_t nd,
                                          uint64_t seed, sf_rotkeys **out)
{
    SF_CHECK_CTX(ctx);
    if (!sk || !out || nd < 0 || (nd > 0 && !d) || sk->ctx != ctx)
        return sf_set_error(SF_EINVAL, "sf_gen_rotation_keys: bad arguments");
    *out = nullptr;
    const SfRing &R = ctx->ring;
    const sf_params *p = ctx->prm;
    std::vector<int32_t> ds;
    if (nd == 0) {
        for (int k = 1; k <= R.log_n; ++k) ds.push_back((1 << k) + 1);
    } else {
        ds.assign(d, d + nd);
    }
    for (int32_t x : ds)
        if (x <= 1 || x >= 2 * R.n || !(x & 1)) return sf_set_error(SF_EINVAL, "automorphism index %d invalid", x);
    sf_rotkeys *rk = new sf_rotkeys();
    rk->ctx = ctx;
    rk->gen = sf_next_generation();
    rk->d = ds;
    // per key: values [dnum][2][nm][N] (NTT domain), then their Shoup companions
    rk->key_words = (size_t)2 * R.dnum * 2 * R.nm * R.n;
    sf_status st = device_buffer((void **)&rk->d_keys, sizeof(u64) * rk->key_words * ds.size());
    u64 *d_alpha = nullptr, *d_e = nullptr;
    int64_t *d_ei = nullptr;
    if (st == SF_OK) st = device_buffer((void **)&d_alpha, sizeof(u64) * R.nm * R.n);
    if (st == SF_OK) st = device_buffer((void **)&d_e, sizeof(u64) * R.nm * R.n);
    if (st == SF_OK) st = device_buffer((void **)&d_ei, sizeof(int64_t) * R.n);
    std::vector<u64> h_alpha((size_t)R.nm * R.n);
    std::vector<int64_t> h_e(R.n);
    std::vector<SfPolyJob> jobs_a, jobs_e;
    for (int m = 0; m < R.nm; ++m) {
        jobs_a.push_back({d_alpha + (size_t)m * R.n, d_alpha + (size_t)m * R.n, m});
        jobs_e.push_back({d_e + (size_t)m * R.n, d_e + (size_t)m * R.n, m});
    }
    for (size_t t = 0; t < ds.size() && st == SF_OK; ++t) {
        SfRng rng(seed ^ ((u64)ds[t] * 0x9E3779B97F4A7C15ULL));
        for (int j = 0; j < R.dnum && st == SF_OK; ++j) {
            for (int m = 0; m < R.nm; ++m)
                for (int k = 0; k < R.n; ++k) h_alpha[(size_t)m * R.n + k] = rng.below(p->mods[m]);
            for (int k = 0; k < R.n; ++k) h_e[k] = rng.gauss(p->sigma);
            if (cudaMemcpy(d_alpha, h_alpha.data(), sizeof(u64) * h_alpha.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(d_ei, h_e.data(), sizeof(int64_t) * R.n, cudaMemcpyHostToDevice) != cudaSuccess) {
                st = sf_set_error(SF_ECUDA, "rotation key upload failed");
                break;
            }
            // [P g_j]_m: P mod q_m on the digit's own data limbs, else 0
            u64 pg[SF_MAX_MODULI] = {0};
            for (int m = j * R.K; m < std::min((j + 1) * R.K, R.L); ++m) {
                u64 v = 1;
                for (int k = 0; k < R.K; ++k) v = sf_host_mulmod(v, p->mods[R.L + k] % p->mods[m], p->mods[m]);
                pg[m] = v;
            }
            u64 *ka = rk->d_keys + rk->key_words * t + (size_t)(j * 2 + 0) * R.nm * R.n;
            u64 *kb = rk->d_keys + rk->key_words * t + (size_t)(j * 2 + 1) * R.nm * R.n;
            if (st == SF_OK) st = sf_signed_to_residues(ctx, d_ei, d_e, R.nm, R.nm, 0, 0);
            if (st == SF_OK) st = sf_ntt_jobs(ctx, jobs_a.data(), R.nm, false, 0);
            if (st == SF_OK) st = sf_ntt_jobs(ctx, jobs_e.data(), R.nm, false, 0);
            if (st == SF_OK) st = sf_rotkey_finish(ctx, d_alpha, d_e, sk->d_s_mont, pg, ds[t], ka, kb, rk->key_words / 2, 0);
            if (st == SF_OK && cudaDeviceSynchronize() != cudaSuccess) st = sf_set_error(SF_ECUDA, "keygen kernel failed");
        }
    }
    if (d_alpha) cudaFree(d_alpha);
    if (d_e) cudaFree(d_e);
    if (d_ei) cudaFree(d_ei);
    if (st != SF_OK) {
        sf_rotkeys_destroy(rk);
        return st;
    }
    *out = rk;
    return SF_OK;
}

extern "C" void sf_rotkeys_destroy(sf_rotkeys *rk)
{
    if (!rk) return;
    cudaSetDevice(rk->ctx->device);
    if (rk->d_keys) cudaFree(rk->d_keys);
    delete rk;
}

static int key_slot(const sf_rotkeys *rk, int d)
{
    for (size_t t = 0; t < rk->d.size(); ++t)
        if (rk->d[t] == d) return (int)t;
    return -1;
}

extern "C" sf_status sf_rotkeys_export(sf_ctx *ctx, const sf_rotkeys *rk, int32_t d, uint64_t *h_key)
{
    SF_CHECK_CTX(ctx);
    if (!rk || !h_key || rk->ctx != ctx) return sf_set_error(SF_EINVAL, "sf_rotkeys_export: bad arguments");
    int t = key_slot(rk, d);
    if (t < 0) return sf_set_error(SF_EINVAL, "no rotation key for d = %d", d);
    const SfRing &R = ctx->ring;
    const size_t vals = rk->key_words / 2;   // the values; the companions follow
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, sizeof(u64) * vals, &w));
    u64 *tmp = (u64 *)w;
    SF_CUDA_TRY(cudaMemcpy(tmp, rk->d_keys + rk->key_words * t, sizeof(u64) * vals, cudaMemcpyDeviceToDevice));
    int npol = R.dnum * 2 * R.nm;
    std::vector<SfPolyJob> jobs;
    for (int x = 0; x < npol; ++x) jobs.push_back({tmp + (size_t)x * R.n, tmp + (size_t)x * R.n, x % R.nm});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), npol, true, 0));
    SF_CUDA_TRY(cudaMemcpy(h_key, tmp, sizeof(u64) * vals, cudaMemcpyDeviceToHost));
    // the stored data limbs carry P^-1 (see the key-switch kernels): export the key itself
    const sf_params *p = ctx->prm;
    for (int x = 0; x < npol; ++x) {
        const int m = x % R.nm;
        if (m >= R.L) continue;
        u64 pm = 1;
        for (int k = 0; k < R.K; ++k) pm = sf_host_mulmod(pm, p->mods[R.L + k] % p->mods[m], p->mods[m]);
        u64 *row = h_key + (size_t)x * R.n;
        for (int k = 0; k < R.n; ++k) row[k] = sf_host_mulmod(row[k], pm, p->mods[m]);
    }
    return SF_OK;
}

// ------------------------------------------------------ encrypt / decrypt --

extern "C" sf_status sf_encrypt(sf_ctx *ctx, const sf_secret_key *sk, const int64_t *h_msg, int64_t count,
                                uint64_t seed, uint64_t *d_cts, int32_t n_cts, void *stream)
{
    SF_CHECK_CTX(ctx);
    const SfRing &R = ctx->ring;
    if (!sk || sk->ctx != ctx || !d_cts || n_cts < 1 || count < 0 || count > (int64_t)n_cts * R.n || (count && !h_msg))
        return sf_set_error(SF_EINVAL, "sf_encrypt: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const sf_params *p = ctx->prm;
    const size_t per = (size_t)R.L * R.n;
    std::vector<u64> h_a(per * n_cts);
    std::vector<int64_t> h_e((size_t)n_cts * R.n), h_m((size_t)n_cts * R.n, 0);
    SfRng rng(seed);
    for (int j = 0; j < n_cts; ++j) {
        for (int i = 0; i < R.L; ++i)
            for (int k = 0; k < R.n; ++k) h_a[j * per + (size_t)i * R.n + k] = rng.below(p->mods[i]);
        for (int k = 0; k < R.n; ++k) h_e[(size_t)j * R.n + k] = rng.gauss(p->sigma);
    }
    if (count) memcpy(h_m.data(), h_msg, sizeof(int64_t) * count);
    Carver cv;
    size_t o_a = cv.take(per * n_cts), o_p = cv.take(per * n_cts), o_m = cv.take((size_t)n_cts * R.n),
           o_e = cv.take((size_t)n_cts * R.n);
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *ws = (u64 *)w;
    u64 *d_a = ws + o_a, *d_p = ws + o_p;
    int64_t *d_m = (int64_t *)(ws + o_m), *d_e = (int64_t *)(ws + o_e);
    SF_CUDA_TRY(cudaMemcpyAsync(d_a, h_a.data(), sizeof(u64) * h_a.size(), cudaMemcpyHostToDevice, st));
    SF_CUDA_TRY(cudaMemcpyAsync(d_m, h_m.data(), sizeof(int64_t) * h_m.size(), cudaMemcpyHostToDevice, st));
    SF_CUDA_TRY(cudaMemcpyAsync(d_e, h_e.data(), sizeof(int64_t) * h_e.size(), cudaMemcpyHostToDevice, st));
    for (int j = 0; j < n_cts; ++j)
        SF_CUDA_TRY(cudaMemcpyAsync(d_cts + (size_t)j * 2 * per, d_a + j * per, sizeof(u64) * per,
                                    cudaMemcpyDeviceToDevice, st));
    std::vector<SfPolyJob> jobs;
    for (int x = 0; x < n_cts * R.L; ++x) jobs.push_back({d_a + (size_t)x * R.n, d_p + (size_t)x * R.n, x % R.L});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), false, st));
    SF_TRY(sf_mul_secret(ctx, d_p, sk->d_s_mont, d_p, n_cts * R.L, R.L, st));
    for (auto &jb : jobs) jb.src = jb.dst;
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), true, st));
    SF_TRY(sf_encrypt_finish(ctx, d_p, d_m, d_e, d_cts, n_cts, st));
    // host vectors die at return: make sure the copies from them completed
    SF_CUDA_TRY(cudaStreamSynchronize(st));
    return SF_OK;
}

extern "C" sf_status sf_decrypt(sf_ctx *ctx, const sf_secret_key *sk, const uint64_t *d_cts, int32_t n_cts,
                                uint64_t *h_residues, void *stream)
{
    SF_CHECK_CTX(ctx);
    const SfRing &R = ctx->ring;
    if (!sk || sk->ctx != ctx || !d_cts || n_cts < 1 || !h_residues) return sf_set_error(SF_EINVAL, "sf_decrypt: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)R.L * R.n;
    Carver cv;
    size_t o_p = cv.take(per * n_cts), o_r = cv.take(per * n_cts);
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *d_p = (u64 *)w + o_p, *d_r = (u64 *)w + o_r;
    std::vector<SfPolyJob> jobs;
    for (int j = 0; j < n_cts; ++j)
        for (int i = 0; i < R.L; ++i)
            jobs.push_back({d_cts + (size_t)j * 2 * per + (size_t)i * R.n, d_p + j * per + (size_t)i * R.n, i});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), false, st));
    SF_TRY(sf_mul_secret(ctx, d_p, sk->d_s_mont, d_p, n_cts * R.L, R.L, st));
    for (auto &jb : jobs) jb.src = jb.dst;
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), true, st));
    SF_TRY(sf_decrypt_finish(ctx, d_cts, d_p, d_r, n_cts, st));
    SF_CUDA_TRY(cudaMemcpyAsync(h_residues, d_r, sizeof(u64) * per * n_cts, cudaMemcpyDeviceToHost, st));
    SF_CUDA_TRY(cudaStreamSynchronize(st));
    return SF_OK;
}

// -------------------------------------------------------------- poly mul --

extern "C" sf_status sf_poly_mul(sf_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_out, int32_t n_polys,
                                 void *stream)
{
    SF_CHECK_CTX(ctx);
    const SfRing &R = ctx->ring;
    if (!d_a || !d_b || !d_out || n_polys < 1 || n_polys % R.L)
        return sf_set_error(SF_EINVAL, "sf_poly_mul: n_polys must be a positive multiple of L");
    cudaStream_t st = (cudaStream_t)stream;
    Carver cv;
    size_t o_a = cv.take((size_t)n_polys * R.n), o_b = cv.take((size_t)n_polys * R.n);
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *ta = (u64 *)w + o_a, *tb = (u64 *)w + o_b;
    std::vector<SfPolyJob> ja, jb;
    for (int x = 0; x < n_polys; ++x) {
        ja.push_back({d_a + (size_t)x * R.n, ta + (size_t)x * R.n, x % R.L});
        jb.push_back({d_b + (size_t)x * R.n, tb + (size_t)x * R.n, x % R.L});
    }
    SF_TRY(sf_ntt_jobs(ctx, ja.data(), n_polys, false, st));
    SF_TRY(sf_ntt_jobs(ctx, jb.data(), n_polys, false, st));
    SF_TRY(sf_pointwise_mul(ctx, ta, tb, ta, n_polys, R.L, 0, st));
    for (int x = 0; x < n_polys; ++x) ja[x] = {ta + (size_t)x * R.n, d_out + (size_t)x * R.n, x % R.L};
    SF_TRY(sf_ntt_jobs(ctx, ja.data(), n_polys, true, st));
    return SF_OK;
}

// ------------------------------------------------------------------ layers --

extern "C" sf_status sf_encode_weights(sf_ctx *ctx, const sf_conv_term *terms, int32_t n_terms, const double *W,
                                       const double *bias, double weight_scale, double bias_scale, sf_layer **out)
{
    SF_CHECK_CTX(ctx);
    if (!terms || !W || !out || n_terms < 1 || n_terms > 2) return sf_set_error(SF_EINVAL, "sf_encode_weights: bad arguments");
    *out = nullptr;
    int Ho = -1, Wo = -1, Co = -1, E_in = 0;
    size_t nw = 0;
    for (int t = 0; t < n_terms; ++t) {
        const sf_conv_term &T = terms[t];
        if (T.H < 1 || T.W < 1 || T.C_in < 1 || T.C_out < 1 || T.kh < 1 || T.kw < 1 || T.stride < 1 || T.pad < 0 ||
            T.in_offset < 0 || T.H + 2 * T.pad < T.kh || T.W + 2 * T.pad < T.kw)
            return sf_set_error(SF_EINVAL, "term %d: invalid geometry", t);
        int h = (T.H + 2 * T.pad - T.kh) / T.stride + 1, w = (T.W + 2 * T.pad - T.kw) / T.stride + 1;
        if (t == 0) {
            Ho = h; Wo = w; Co = T.C_out;
        } else if (h != Ho || w != Wo || T.C_out != Co) {
            return sf_set_error(SF_EINVAL, "terms disagree on the output shape");
        }
        int64_t end = (int64_t)T.in_offset + (int64_t)T.H * T.W * T.C_in;
        if (end > (1 << 30)) return sf_set_error(SF_EINVAL, "input too large");
        E_in = std::max<int>(E_in, (int)end);
        nw += (size_t)T.C_out * T.kh * T.kw * T.C_in;
    }
    if ((int64_t)Ho * Wo * Co > (1 << 30)) return sf_set_error(SF_EINVAL, "output too large");
    sf_layer *L = new sf_layer();
    L->ctx = ctx;
    L->gen = sf_next_generation();
    L->terms.assign(terms, terms + n_terms);
    L->E_in = E_in;
    L->H_out = Ho;
    L->W_out = Wo;
    L->C_out = Co;
    L->E_out = Ho * Wo * Co;
    L->wq.resize(nw);
    L->d_wq = nullptr;
    L->d_bq = nullptr;
    L->d_terms = nullptr;
    L->d_taps = nullptr;
    std::vector<int4> taps;
    L->max_taps = 0;
    for (int t = 0; t < n_terms; ++t) L->max_taps += terms[t].kh * terms[t].kw * terms[t].C_in;
    for (int t = 0; t < n_terms; ++t) {
        const sf_conv_term &T = terms[t];
        L->tap_off.push_back((int)taps.size());
        for (int dh = 0; dh < T.kh; ++dh)
            for (int dw = 0; dw < T.kw; ++dw)
                for (int ci = 0; ci < T.C_in; ++ci)
                    taps.push_back(make_int4(dh, dw, (dh * T.W + dw) * T.C_in + ci, (dh * T.kw + dw) * T.C_in + ci));
    }
    for (size_t x = 0; x < nw; ++x) {
        double v = weight_scale * W[x];
        if (!(fabs(v) < 4.6e18)) {
            delete L;
            return sf_set_error(SF_ERANGE, "quantised weight %g out of range", v);
        }
        L->wq[x] = llround(v);
    }
    if (bias) {
        L->bq.resize(Co);
        for (int c = 0; c < Co; ++c) {
            double v = bias_scale * bias[c];
            if (!(fabs(v) < 4.6e18)) {
                delete L;
                return sf_set_error(SF_ERANGE, "quantised bias %g out of range", v);
            }
            L->bq[c] = llround(v);
        }
    }
    sf_status st = device_buffer((void **)&L->d_wq, sizeof(int64_t) * nw);
    if (st == SF_OK && cudaMemcpy(L->d_wq, L->wq.data(), sizeof(int64_t) * nw, cudaMemcpyHostToDevice) != cudaSuccess)
        st = sf_set_error(SF_ECUDA, "weight upload failed");
    if (st == SF_OK) st = device_buffer((void **)&L->d_taps, sizeof(int4) * taps.size());
    if (st == SF_OK && cudaMemcpy(L->d_taps, taps.data(), sizeof(int4) * taps.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        st = sf_set_error(SF_ECUDA, "tap table upload failed");
    if (st == SF_OK && bias) {
        st = device_buffer((void **)&L->d_bq, sizeof(int64_t) * Co);
        if (st == SF_OK && cudaMemcpy(L->d_bq, L->bq.data(), sizeof(int64_t) * Co, cudaMemcpyHostToDevice) != cudaSuccess)
            st = sf_set_error(SF_ECUDA, "bias upload failed");
    }
    if (st != SF_OK) {
        sf_layer_destroy(L);
        return st;
    }
    *out = L;
    return SF_OK;
}

extern "C" void sf_layer_destroy(sf_layer *L)
{
    if (!L) return;
    cudaSetDevice(L->ctx->device);
    if (L->d_wq) cudaFree(L->d_wq);
    if (L->d_bq) cudaFree(L->d_bq);
    if (L->d_taps) cudaFree(L->d_taps);
    delete L;
}

extern "C" sf_status sf_layer_get_info(const sf_ctx *ctx, const sf_layer *L, sf_layer_info *out)
{
    if (!ctx || !L || !out) return sf_set_error(SF_EINVAL, "sf_layer_get_info: null argument");
    const SfRing &R = ctx->ring;
    out->E_in = L->E_in;
    out->E_out = L->E_out;
    out->k_in = (L->E_in + R.n - 1) / R.n;
    int n, G;
    layer_groups(R, L->E_out, &n, &G);
    out->group_size = n;
    out->n_groups = G;
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    out->ks_count = (int64_t)G * ((n - 1) + (R.log_n - lg));
    return SF_OK;
}

extern "C" sf_status sf_linear_outputs(sf_ctx *ctx, const sf_layer *L, const uint64_t *d_in, int32_t k_in,
                                       const uint32_t *h_sigma_prev, const int32_t *h_outputs, int32_t n_outputs,
                                       uint64_t *d_out, void *stream)
{
    SF_CHECK_CTX(ctx);
    const SfRing &R = ctx->ring;
    if (!L || !d_in || !d_out || !h_outputs || n_outputs < 1 || L->ctx != ctx)
        return sf_set_error(SF_EINVAL, "sf_linear_outputs: bad arguments");
    if (k_in != (L->E_in + R.n - 1) / R.n) return sf_set_error(SF_EINVAL, "wrong number of input ciphertexts");
    for (int t = 0; t < n_outputs; ++t)
        if (h_outputs[t] < 0 || h_outputs[t] >= L->E_out) return sf_set_error(SF_EINVAL, "output index out of range");
    if (h_sigma_prev) SF_TRY(check_perm(h_sigma_prev, L->E_in, "sigma_prev"));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ct = ct_words(ctx);
    const int LB = std::min(leaf_batch_slots(R, k_in, L->max_taps), n_outputs);
    Carver cv;
    size_t o_ct = cv.take((size_t)2 * k_in * ct), o_pos = cv.take(((size_t)L->E_in + 1) / 2),
           o_sig = cv.take(((size_t)n_outputs + 1) / 2), o_w1 = cv.take((size_t)LB * k_in * R.L * R.n),
           o_lv = cv.take((size_t)n_outputs * ct), o_tap = cv.take(sf_leaf_tap_words(R, k_in, L->max_taps, LB));
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *ws = (u64 *)w;
    int *d_pos = (int *)(ws + o_pos), *d_sig = (int *)(ws + o_sig);
    std::vector<int> h_pos, h_sig(h_outputs, h_outputs + n_outputs);
    if (h_sigma_prev) SF_TRY(upload_perm_inverse(h_sigma_prev, L->E_in, d_pos, h_pos, st));
    SF_CUDA_TRY(cudaMemcpyAsync(d_sig, h_sig.data(), sizeof(int) * n_outputs, cudaMemcpyHostToDevice, st));
    SF_TRY(prepare_inputs(ctx, d_in, nullptr, k_in, ws + o_ct, st));
    SfLeafParams P = leaf_params(L);
    P.k_in = k_in;
    P.pos_of = h_sigma_prev ? d_pos : nullptr;
    P.sig_out = d_sig;
    P.ct = ws + o_ct;
    P.w1 = ws + o_w1;
    sf_leaf_tap_bind(R, P, ws + o_tap, LB);
    P.n_slots_valid = n_outputs;
    P.leaf_stride = ct;
    P.s_stride = 1;
    for (int s0 = 0; s0 < n_outputs; s0 += LB) {
        SfLeafParams p = P;
        p.s0 = s0;
        p.leaves = ws + o_lv + (size_t)s0 * ct;
        SF_TRY(sf_leaves_launch(ctx, p, std::min(LB, n_outputs - s0), st));
    }
    std::vector<SfPolyJob> jobs;
    for (int x = 0; x < n_outputs * 2 * R.L; ++x)
        jobs.push_back({ws + o_lv + (size_t)x * R.n, d_out + (size_t)x * R.n, x % R.L});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), true, st));
    SF_CUDA_TRY(cudaStreamSynchronize(st));
    return SF_OK;
}

// ---------------------------------------------------------- building blocks --

extern "C" sf_status sf_rotate(sf_ctx *ctx, const sf_rotkeys *rk, int32_t d, const uint64_t *d_ct, uint64_t *d_out,
                               int32_t count, void *stream)
{
    SF_CHECK_CTX(ctx);
    const SfRing &R = ctx->ring;
    if (!rk || rk->ctx != ctx || !d_ct || !d_out || count < 1) return sf_set_error(SF_EINVAL, "sf_rotate: bad arguments");
    int t = key_slot(rk, d);
    if (t < 0) return sf_set_error(SF_EINVAL, "no rotation key for d = %d", d);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ct = ct_words(ctx);
    const int batch = std::min(ctx->ks_batch, count);
    Carver cv;
    size_t o_in = cv.take((size_t)count * ct), o_out = cv.take((size_t)count * ct),
           o_ks = cv.take(sf_ks_scratch_words(R) * batch);
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *ws = (u64 *)w;
    SF_TRY(sf_check_residues(ctx, d_ct, count * 2 * R.L, R.L, 0, st));
    std::vector<SfPolyJob> jobs;
    for (int x = 0; x < count * 2 * R.L; ++x) jobs.push_back({d_ct + (size_t)x * R.n, ws + o_in + (size_t)x * R.n, x % R.L});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), false, st));
    SfKsBatch b;
    memset(&b, 0, sizeof(b));
    b.E = ws + o_in;
    b.E_stride = ct;
    b.out = ws + o_out;
    b.out_stride = ct;
    b.inner = 1 << 30;
    b.count = count;
    b.d = d;
    b.add_v = 0;
    b.key = rk->d_keys + rk->key_words * t;
    SF_TRY(sf_ks_run(ctx, b, ws + o_ks, batch, st));
    for (int x = 0; x < count * 2 * R.L; ++x) jobs[x] = {ws + o_out + (size_t)x * R.n, d_out + (size_t)x * R.n, x % R.L};
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), true, st));
    return SF_OK;
}

static sf_status pack_impl(sf_ctx *ctx, const sf_rotkeys *rk, const uint64_t *d_leaves, int32_t n_leaves, int32_t n,
                           int32_t gamma, uint64_t *d_out, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (gamma < 0 || gamma > 2) return sf_set_error(SF_EINVAL, "sf_pack_gamma: gamma must be 0, 1 or 2");
    const SfRing &R = ctx->ring;
    if (!rk || rk->ctx != ctx || !d_leaves || !d_out || n_leaves < 1 || n < n_leaves || n > R.n / 2 || (n & (n - 1)))
        return sf_set_error(SF_EINVAL, "sf_pack: need 1 <= n_leaves <= n <= N/2, n a power of two");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ct = ct_words(ctx);
    const int batch = std::min(ctx->ks_batch, std::max(1, n / 2));   // the widest level has n/2 merges
    Carver cv;
    size_t o_A = cv.take((size_t)n * ct), o_B = cv.take((size_t)std::max(n / 2, 1) * ct),
           o_ks = cv.take(sf_ks_scratch_words(R) * batch);
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *ws = (u64 *)w;
    std::vector<SfPolyJob> jobs;
    for (int x = 0; x < n_leaves * 2 * R.L; ++x)
        jobs.push_back({d_leaves + (size_t)x * R.n, ws + o_A + (size_t)x * R.n, x % R.L});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), false, st));
    std::vector<int> valid(1, n_leaves);
    u64 *res = nullptr;
    size_t rs = 0;
    SF_TRY(sf_pack_tree(ctx, rk->d_keys, rk->d, rk->key_words, ws + o_A, ws + o_B, 1, n, 0, valid, true, ws + o_ks, batch,
                        &res, &rs, st, gamma == 2));
    jobs.clear();
    for (int x = 0; x < 2 * R.L; ++x) jobs.push_back({res + (size_t)x * R.n, d_out + (size_t)x * R.n, x % R.L});
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), true, st));
    return SF_OK;
}

extern "C" sf_status sf_pack(sf_ctx *ctx, const sf_rotkeys *rk, const uint64_t *d_leaves, int32_t n_leaves, int32_t n,
                             uint64_t *d_out, void *stream)
{
    return pack_impl(ctx, rk, d_leaves, n_leaves, n, 0, d_out, stream);
}

extern "C" sf_status sf_pack_gamma(sf_ctx *ctx, const sf_rotkeys *rk, const uint64_t *d_leaves, int32_t n_leaves,
                                   int32_t n, int32_t gamma, uint64_t *d_out, void *stream)
{
    return pack_impl(ctx, rk, d_leaves, n_leaves, n, gamma, d_out, stream);
}

extern "C" sf_status sf_extract(sf_ctx *ctx, const uint64_t *d_ct, int32_t i, int32_t gamma, const uint64_t *d_powers,
                                uint64_t *d_out, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (gamma < 0 || gamma > 2) return sf_set_error(SF_EINVAL, "sf_extract: gamma must be 0, 1 or 2");
    if (!d_ct || !d_out || i < 0 || i >= ctx->ring.n) return sf_set_error(SF_EINVAL, "sf_extract: bad arguments");
    if (gamma == 2) {
        if (!d_powers) return sf_set_error(SF_EINVAL, "sf_extract: gamma = 2 needs the client's power");
        return sf_extract2_launch(ctx, d_ct, d_powers, d_out, i, (cudaStream_t)stream);
    }
    // gamma = 1 equals gamma = 0 at t = 2 (K_1 = K_0: the power m(X^1) is m itself)
    return sf_extract_launch(ctx, d_ct, d_out, i, (cudaStream_t)stream);
}

extern "C" sf_status sf_shuffle_cts(sf_ctx *ctx, const uint32_t *h_perm, const uint64_t *d_in, uint64_t *d_out,
                                    int32_t count, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (!h_perm || !d_in || !d_out || count < 1) return sf_set_error(SF_EINVAL, "sf_shuffle_cts: bad arguments");
    SF_TRY(check_perm(h_perm, count, "perm"));
    cudaStream_t st = (cudaStream_t)stream;
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, sizeof(int) * count, &w));
    std::vector<int> h(h_perm, h_perm + count);
    SF_CUDA_TRY(cudaMemcpyAsync(w, h.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
    SF_TRY(sf_shuffle_launch(ctx, d_in, d_out, (const int *)w, count, st));
    SF_CUDA_TRY(cudaStreamSynchronize(st));
    return SF_OK;
}
