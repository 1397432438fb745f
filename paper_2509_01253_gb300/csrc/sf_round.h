// sf_round.h -- helpers shared by the layer-round entry points.
#pragma once
#include <string.h>

#include <algorithm>
#include <vector>

#include "sf_internal.h"
#include "sf_tile.cuh"
#include "sf_layer.h"

#define SF_CHECK_CTX(ctx)                                                        \
    do {                                                                         \
        if (!(ctx)) return sf_set_error(SF_EINVAL, "%s: null context", __func__); \
        SF_CUDA_TRY(cudaSetDevice((ctx)->device));                               \
    } while (0)

static inline size_t ct_words(const sf_ctx *ctx) { return (size_t)2 * ctx->ring.L * ctx->ring.n; }
static inline size_t align_words(size_t w) { return (w + 31) & ~(size_t)31; }

// Carves consecutive regions out of the context workspace.
struct Carver {
    size_t words = 0;
    size_t take(size_t w)
    {
        size_t off = words;
        words += align_words(w);
        return off;
    }
};

static inline void layer_groups(const SfRing &R, int E_out, int *n, int *G)
{
    int g = 1;
    while (g < E_out) g *= 2;
    *n = std::min(R.n / 2, g);
    *G = (E_out + *n - 1) / *n;
}

static inline sf_status check_perm(const uint32_t *perm, int n, const char *what)
{
    std::vector<char> seen(n, 0);
    for (int k = 0; k < n; ++k) {
        if (perm[k] >= (uint32_t)n || seen[perm[k]]) return sf_set_error(SF_EINVAL, "%s is not a permutation of [0, %d)", what, n);
        seen[perm[k]] = 1;
    }
    return SF_OK;
}

static inline SfLeafParams leaf_params(const sf_layer *L)
{
    SfLeafParams P;
    memset(&P, 0, sizeof(P));
    size_t off = 0;
    for (size_t t = 0; t < L->terms.size(); ++t) {
        const sf_conv_term &T = L->terms[t];
        P.t[t] = {T.in_offset, T.H, T.W, T.C_in, T.C_out, T.kh, T.kw, T.stride, T.pad, (int)off, L->tap_off[t]};
        off += (size_t)T.C_out * T.kh * T.kw * T.C_in;
    }
    P.n_terms = (int)L->terms.size();
    P.C_out = L->C_out;
    P.W_out = L->W_out;
    P.wq = L->d_wq;
    P.taps = L->d_taps;
    P.max_taps = L->max_taps;
    return P;
}

// Input ciphertexts -> NTT domain (canonical), followed by their Shoup
// companions (for the leaf products).  With the client's powers (gamma = 2,
// d_pow non-null) the k_in powers follow the k_in inputs, so the leaves see
// 2 k_in ciphertexts; ct holds twice the words of the ciphertexts it takes.
static inline sf_status prepare_inputs(sf_ctx *ctx, const u64 *d_in, const u64 *d_pow, int k_in, u64 *ct,
                                       cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    const int k_all = d_pow ? 2 * k_in : k_in;
    const size_t words = (size_t)k_in * 2 * R.L * R.n;
    SF_TRY(sf_check_residues(ctx, d_in, k_in * 2 * R.L, R.L, 0, st));
    if (d_pow) SF_TRY(sf_check_residues(ctx, d_pow, k_in * 2 * R.L, R.L, 0, st));
    std::vector<SfPolyJob> jobs;
    for (int x = 0; x < k_all * 2 * R.L; ++x) {
        const u64 *src = x < k_in * 2 * R.L ? d_in + (size_t)x * R.n : d_pow + (size_t)x * R.n - words;
        jobs.push_back({src, ct + (size_t)x * R.n, x % R.L});
    }
    SF_TRY(sf_ntt_jobs(ctx, jobs.data(), (int)jobs.size(), false, st));
    SF_TRY(sf_companions(ctx, ct, ct + (size_t)k_all * 2 * R.L * R.n, k_all * 2 * R.L, R.L, 0, st));
    return SF_OK;
}

static inline sf_status upload_perm_inverse(const uint32_t *perm, int n, int *d_dst, std::vector<int> &host, cudaStream_t st)
{
    host.assign(n, 0);
    for (int k = 0; k < n; ++k) host[perm[k]] = k;
    SF_CUDA_TRY(cudaMemcpyAsync(d_dst, host.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    return SF_OK;
}

// slots per leaf launch: the column-pass scratch and the tap buckets stay
// within 256 MiB each
static inline int leaf_batch_slots(const SfRing &R, int k_in, int max_taps)
{
    size_t per = (size_t)k_in * R.L * R.n * sizeof(u64);
    size_t slots = ((size_t)256 << 20) / per;
    slots = std::min(slots, ((size_t)256 << 20) / ((size_t)std::max(1, max_taps) * 16));
    return (int)std::max<size_t>(1, std::min<size_t>(slots, 4096));
}

// points the tap buckets of P at words (sized by sf_leaf_tap_words)
static inline void sf_leaf_tap_bind(const SfRing &R, SfLeafParams &P, u64 *words, int slots)
{
    P.n_buckets = P.k_in * (R.c / SF_NB);
    P.tap_buf = (longlong2 *)words;
    P.tap_off = (int *)(words + (size_t)slots * P.max_taps * 2);
}

