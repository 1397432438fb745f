// sf_engine.cu -- the round engine: one or many linear-layer rounds (Sec. 4.4,
// steps 6-10) evaluated together on one GPU, as one captured launch sequence.
//
// Work is cut into units.  A unit is one residue class of CH leaves of one
// packing group of one layer: leaves l = a, a + n/CH, a + 2n/CH, ... of group
// g (the leaves that the first log2 CH levels of the PackLWEs tree combine).
// Units of every layer whose groups have the same size n form a class; the
// class is processed in waves of units that fit the memory budget:
//   leaves of every unit of the wave (leaf_col / leaf_row kernels)
//   -> the first log2 CH tree levels of all units together (shared key
//      switches: one launch sequence per level for the whole wave)
//   -> one root per unit.
// Then one tree over the n/CH roots of every group of the class (levels
// log2 CH + 1 .. log2 n) followed by the field trace gives every group's
// packed ciphertext.  With CH = n a unit is a whole group and the trace runs
// in the wave.  The launch sequence depends only on pointers and shapes; it
// is captured once into a CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "sf_internal.h"
#include "sf_ks.h"
#include "sf_layer.h"
#include "sf_round.h"

namespace {

struct Job {
    const sf_layer *L;
    const sf_rotkeys *rk;
    const u64 *d_in;
    int k_in;
    const uint32_t *sp, *so;
    u64 *d_out;
    int n, G;
    // workspace
    u64 *d_ct;
    int *d_pos, *d_sig;
    // gamma = 2: the client's powers RLWE(m_j(X^3)), [k_in][2][L][N] (null at gamma = 0)
    const u64 *d_pow;
    int k_leaf() const { return d_pow ? 2 * k_in : k_in; }
    int taps() const { return d_pow ? 2 * L->max_taps : L->max_taps; }
};

struct Unit {
    int job, g, a, va;   // va = leaves of the unit holding a real output
};

struct Class {
    const sf_rotkeys *rk;
    bool gamma2;
    int n, CH, nch, log_ch;
    std::vector<Unit> units;           // ordered (job, group, a)
    std::vector<std::pair<int, int>> groups;   // (job, g) in unit order
    int U;                             // units per wave
    size_t o_roots_a, o_roots_b;       // workspace offsets (nch > 1)
};

uint64_t fnv(uint64_t h, uint64_t v)
{
    for (int k = 0; k < 8; ++k) {
        h ^= (v >> (8 * k)) & 0xff;
        h *= 0x100000001b3ULL;
    }
    return h;
}

}  // namespace

// Evaluates jobs[0..J) (validated by the callers).
static sf_status eval_jobs(sf_ctx *ctx, std::vector<Job> &jobs, cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    const size_t ct = ct_words(ctx), ct_bytes = ct * sizeof(u64);
    // leaf slots per launch, per round (its own ciphertexts and taps: a round
    // with a huge fan-in does not shrink the launches of the others); the
    // workspace holds the largest of them
    std::vector<int> lb(jobs.size());
    size_t w1_words = 0, tap_words = 0;
    for (size_t x = 0; x < jobs.size(); ++x) {
        const Job &j = jobs[x];
        lb[x] = leaf_batch_slots(R, j.k_leaf(), j.taps());
        w1_words = std::max(w1_words, (size_t)lb[x] * j.k_leaf() * R.L * R.n);
        tap_words = std::max(tap_words, sf_leaf_tap_words(R, j.k_leaf(), j.taps(), lb[x]));
    }
    const int LB = *std::max_element(lb.begin(), lb.end());
    // ---- classes and units
    std::vector<Class> classes;
    for (int x = 0; x < (int)jobs.size(); ++x) {
        Job &j = jobs[x];
        Class *c = nullptr;
        // a class shares its tree levels, so it holds rounds of one gamma only
        for (auto &cc : classes)
            if (cc.rk == j.rk && cc.n == j.n && cc.gamma2 == (j.d_pow != nullptr)) c = &cc;
        if (!c) {
            classes.push_back(Class());
            c = &classes.back();
            c->rk = j.rk;
            c->n = j.n;
            c->gamma2 = j.d_pow != nullptr;
            // CH: largest power of two <= n such that 16 units of CH leaves
            // (plus their tree buffer) fit the budget, or the leaf_chunk cap
            int ch = j.n;
            while (ch > 1 && ((size_t)16 * ch * ct_bytes * 3 / 2 > ctx->mem_budget || ch > ctx->leaf_chunk)) ch /= 2;
            c->CH = ch;
            c->nch = j.n / ch;
            c->log_ch = 0;
            while ((1 << c->log_ch) < ch) ++c->log_ch;
        }
        for (int g = 0; g < j.G; ++g) {
            c->groups.push_back({x, g});
            const int live = j.L->E_out - g * j.n;
            for (int a = 0; a < c->nch; ++a) {
                const int va = live > a ? std::min(c->CH, (live - a + c->nch - 1) / c->nch) : 0;
                c->units.push_back({x, g, a, va});
            }
        }
    }
    // ---- workspace
    Carver cv;
    std::vector<size_t> o_ct(jobs.size()), o_pos(jobs.size()), o_sig(jobs.size());
    for (size_t x = 0; x < jobs.size(); ++x) {
        o_ct[x] = cv.take((size_t)2 * jobs[x].k_leaf() * ct);
        o_pos[x] = cv.take(((size_t)jobs[x].L->E_in + 1) / 2);
        o_sig[x] = cv.take(((size_t)jobs[x].L->E_out + 1) / 2);
    }
    const size_t o_w1 = cv.take(w1_words);
    const size_t o_tap = cv.take(tap_words);
    size_t roots_bytes = 0;
    for (auto &c : classes)
        if (c.nch > 1) roots_bytes += (size_t)c.groups.size() * c.nch * ct_bytes * 3 / 2;
    int maxU = 1;
    size_t wave_words = 0;
    for (auto &c : classes) {
        const size_t per_unit = (size_t)c.CH * ct_bytes * 3 / 2;
        const size_t avail = ctx->mem_budget > roots_bytes ? ctx->mem_budget - roots_bytes : per_unit;
        c.U = (int)std::max<size_t>(1, std::min<size_t>(c.units.size(), avail / per_unit));
        maxU = std::max(maxU, c.U);
        wave_words = std::max(wave_words, (size_t)c.U * c.CH * ct);
    }
    // merges per key-switch launch: the context's batch, or fewer when no tree
    // level of this call has that many merges
    int widest = 1;
    for (auto &c : classes) {
        widest = std::max(widest, c.U * c.CH / 2);
        widest = std::max(widest, (int)c.groups.size() * std::max(1, c.nch / 2));
    }
    const int batch = std::min(ctx->ks_batch, widest);
    const size_t o_A = cv.take(wave_words);
    const size_t o_B = cv.take(wave_words / 2 + ct);
    for (auto &c : classes) {
        if (c.nch > 1) {
            c.o_roots_a = cv.take((size_t)c.groups.size() * c.nch * ct);
            c.o_roots_b = cv.take((size_t)c.groups.size() * std::max(c.nch / 2, 1) * ct);
        }
    }
    const size_t o_ks = cv.take(sf_ks_scratch_words(R) * batch);
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, cv.words * sizeof(u64), &w));
    u64 *ws = (u64 *)w;
    std::vector<std::vector<int>> h_pos(jobs.size()), h_sig(jobs.size());
    for (size_t x = 0; x < jobs.size(); ++x) {
        Job &j = jobs[x];
        j.d_ct = ws + o_ct[x];
        j.d_pos = (int *)(ws + o_pos[x]);
        j.d_sig = (int *)(ws + o_sig[x]);
        if (j.sp) SF_TRY(upload_perm_inverse(j.sp, j.L->E_in, j.d_pos, h_pos[x], st));
        if (j.so) {
            h_sig[x].assign(j.so, j.so + j.L->E_out);
            SF_CUDA_TRY(cudaMemcpyAsync(j.d_sig, h_sig[x].data(), sizeof(int) * j.L->E_out, cudaMemcpyHostToDevice, st));
        }
    }
    u64 *A = ws + o_A, *B = ws + o_B, *d_w1 = ws + o_w1, *d_ks = ws + o_ks;

    auto launch_all = [&](cudaStream_t s) -> sf_status {
        for (auto &j : jobs) SF_TRY(prepare_inputs(ctx, j.d_in, j.d_pow, j.k_in, j.d_ct, s));
        auto leaves = [&](const Job &j, int s0, int stride, int cnt, u64 *dst) -> sf_status {
            const int jb = lb[&j - jobs.data()];
            SfLeafParams P = leaf_params(j.L);
            P.k_in = j.k_leaf();
            P.k_src = j.k_in;
            P.gamma2 = j.d_pow != nullptr;
            P.max_taps = j.taps();
            P.pos_of = j.sp ? j.d_pos : nullptr;
            P.sig_out = j.so ? j.d_sig : nullptr;
            P.ct = j.d_ct;
            P.w1 = d_w1;
            sf_leaf_tap_bind(R, P, ws + o_tap, jb);
            P.n_slots_valid = j.L->E_out;
            P.leaf_stride = ct;
            for (int t0 = 0; t0 < cnt; t0 += jb) {
                SfLeafParams p = P;
                p.s0 = s0 + t0 * stride;
                p.s_stride = stride;
                p.leaves = dst + (size_t)t0 * ct;
                SF_TRY(sf_leaves_launch(ctx, p, std::min(jb, cnt - t0), s));
            }
            return SF_OK;
        };
        auto output = [&](const u64 *res, const Job &j, int g) -> sf_status {
            SfPolyJob pj[SF_MAX_MODULI * 2];
            for (int x = 0; x < 2 * R.L; ++x) pj[x] = {res + (size_t)x * R.n, j.d_out + ct * g + (size_t)x * R.n, x % R.L};
            return sf_ntt_jobs(ctx, pj, 2 * R.L, true, s);
        };
        for (auto &c : classes) {
            const std::vector<int32_t> &kd = c.rk->d;
            u64 *RA = c.nch > 1 ? ws + c.o_roots_a : nullptr;
            u64 *RB = c.nch > 1 ? ws + c.o_roots_b : nullptr;
            for (size_t u0 = 0; u0 < c.units.size(); u0 += c.U) {
                const int wn = (int)std::min<size_t>(c.U, c.units.size() - u0);
                std::vector<int> valid(wn);
                for (int u = 0; u < wn; ++u) {
                    const Unit &un = c.units[u0 + u];
                    const Job &j = jobs[un.job];
                    valid[u] = un.va;
                    if (un.va > 0) SF_TRY(leaves(j, un.g * j.n + un.a, c.nch, c.CH, A + (size_t)u * c.CH * ct));
                }
                u64 *res = nullptr;
                size_t rs = 0;
                SF_TRY(sf_pack_tree(ctx, c.rk->d_keys, kd, c.rk->key_words, A, B, wn, c.CH, 0, valid, c.nch == 1, d_ks,
                                    batch, &res, &rs, s, c.gamma2));
                if (c.nch == 1) {
                    for (int u = 0; u < wn; ++u) {
                        const Unit &un = c.units[u0 + u];
                        SF_TRY(output(res + rs * u, jobs[un.job], un.g));
                    }
                } else {
                    SF_CUDA_TRY(cudaMemcpy2DAsync(RA + u0 * ct, ct_bytes, res, rs * sizeof(u64), ct_bytes, wn,
                                                  cudaMemcpyDeviceToDevice, s));
                    for (int u = 0; u < wn; ++u)
                        if (c.units[u0 + u].va == 0) SF_CUDA_TRY(cudaMemsetAsync(RA + (u0 + u) * ct, 0, ct_bytes, s));
                }
            }
            if (c.nch > 1) {
                std::vector<int> valid(c.groups.size());
                for (size_t gi = 0; gi < c.groups.size(); ++gi) {
                    const Job &j = jobs[c.groups[gi].first];
                    valid[gi] = std::min(c.nch, std::max(0, j.L->E_out - c.groups[gi].second * j.n));
                }
                u64 *res = nullptr;
                size_t rs = 0;
                SF_TRY(sf_pack_tree(ctx, c.rk->d_keys, kd, c.rk->key_words, RA, RB, (int)c.groups.size(), c.nch, c.log_ch,
                                    valid, true, d_ks, batch, &res, &rs, s, c.gamma2));
                for (size_t gi = 0; gi < c.groups.size(); ++gi)
                    SF_TRY(output(res + rs * gi, jobs[c.groups[gi].first], c.groups[gi].second));
            }
        }
        for (auto &j : jobs)
            if (j.L->d_bq)
                SF_TRY(sf_add_bias(ctx, j.d_out, j.G, j.n, j.L->E_out, j.so ? j.d_sig : nullptr, j.L->d_bq, j.L->C_out, s,
                                   j.d_pow ? 2 : 1));
        return SF_OK;
    };

    if (!ctx->use_graph || ctx->kernel_timing) {
        SF_TRY(launch_all(st));
    } else {
        uint64_t h = 0xcbf29ce484222325ULL;
        for (auto &j : jobs) {
            h = fnv(h, j.L->gen);
            h = fnv(h, j.rk->gen);
            h = fnv(h, (uint64_t)(uintptr_t)j.d_in);
            h = fnv(h, (uint64_t)(uintptr_t)j.d_out);
            h = fnv(h, (uint64_t)j.k_in);
            h = fnv(h, (uint64_t)(j.sp != nullptr) * 2 + (j.so != nullptr));
            h = fnv(h, (uint64_t)(uintptr_t)j.d_pow);
        }
        for (auto &c : classes) {
            h = fnv(h, (uint64_t)c.CH);
            h = fnv(h, (uint64_t)c.U);
        }
        uint64_t key[12] = {h, (uint64_t)jobs.size(), (uint64_t)(uintptr_t)ws, (uint64_t)batch, (uint64_t)LB, 2, 0, 0, 0, 0, 0, 0};
        SfGraphEntry *hit = nullptr;
        for (auto &e : ctx->graphs)
            if (!memcmp(e.key, key, sizeof(key))) hit = &e;
        if (!hit) {
            std::vector<int64_t> before(SFK_COUNT);
            for (int k = 0; k < SFK_COUNT; ++k) before[k] = ctx->stats[k].launches;
            cudaStream_t cap;
            SF_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            sf_status lst = ce == cudaSuccess ? launch_all(cap) : sf_set_error(SF_ECUDA, "stream capture failed");
            cudaError_t ee = cudaStreamEndCapture(cap, &graph);
            cudaStreamDestroy(cap);
            if (lst != SF_OK) {
                if (graph) cudaGraphDestroy(graph);
                for (int k = 0; k < SFK_COUNT; ++k) ctx->stats[k].launches = before[k];
                return lst;
            }
            if (ee != cudaSuccess || !graph) return sf_set_error(SF_ECUDA, "graph capture failed: %s", cudaGetErrorString(ee));
            SfGraphEntry e;
            memcpy(e.key, key, sizeof(key));
            cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) return sf_set_error(SF_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ie));
            e.launches.resize(SFK_COUNT);
            for (int k = 0; k < SFK_COUNT; ++k) {
                e.launches[k] = ctx->stats[k].launches - before[k];
                ctx->stats[k].launches = before[k];
            }
            // bounded cache: a serving loop sees a new combination of rounds at every call
            if (ctx->graphs.size() >= 32) {
                cudaGraphExecDestroy(ctx->graphs.front().exec);
                ctx->graphs.erase(ctx->graphs.begin());
            }
            ctx->graphs.push_back(e);
            hit = &ctx->graphs.back();
        }
        SF_CUDA_TRY(cudaGraphLaunch(hit->exec, st));
        for (int k = 0; k < SFK_COUNT; ++k) ctx->stats[k].launches += hit->launches[k];
    }
    bool host_copies = false;
    for (size_t x = 0; x < jobs.size(); ++x) host_copies |= !h_pos[x].empty() || !h_sig[x].empty();
    // the permutation host copies must outlive their asynchronous uploads
    if (host_copies) SF_CUDA_TRY(cudaStreamSynchronize(st));
    return SF_OK;
}

static sf_status make_job(sf_ctx *ctx, const sf_layer *L, const sf_rotkeys *rk, const uint64_t *d_in, int32_t k_in,
                          const uint32_t *sp, const uint32_t *so, uint64_t *d_out, int32_t out_capacity, Job *j)
{
    const SfRing &R = ctx->ring;
    if (!L || !rk || !d_in || !d_out || L->ctx != ctx || rk->ctx != ctx)
        return sf_set_error(SF_EINVAL, "layer round: null or foreign argument");
    const int need_k = (L->E_in + R.n - 1) / R.n;
    if (k_in != need_k) return sf_set_error(SF_EINVAL, "layer needs %d input ciphertexts, got %d", need_k, k_in);
    int n, G;
    layer_groups(R, L->E_out, &n, &G);
    if (out_capacity < G) return sf_set_error(SF_EINVAL, "output capacity %d < %d packed ciphertexts", out_capacity, G);
    if (sp) SF_TRY(check_perm(sp, L->E_in, "sigma_prev"));
    if (so) SF_TRY(check_perm(so, L->E_out, "sigma_out"));
    *j = Job{L, rk, d_in, k_in, sp, so, d_out, n, G, nullptr, nullptr, nullptr, nullptr};
    return SF_OK;
}

extern "C" sf_status sf_eval_linear_layer_gamma(sf_ctx *ctx, const sf_layer *L, const sf_rotkeys *rk, int32_t gamma,
                                                const uint64_t *d_in, const uint64_t *d_powers, int32_t k_in,
                                                const uint32_t *h_sigma_prev, const uint32_t *h_sigma_out,
                                                uint64_t *d_out, int32_t out_capacity, int32_t *n_out, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (gamma < 0 || gamma > 2) return sf_set_error(SF_EINVAL, "gamma must be 0, 1 or 2");
    if (gamma == 2 && !d_powers) return sf_set_error(SF_EINVAL, "gamma = 2 needs the client's powers");
    if (gamma < 2 && d_powers) return sf_set_error(SF_EINVAL, "powers are only read at gamma = 2");
    std::vector<Job> jobs(1);
    SF_TRY(make_job(ctx, L, rk, d_in, k_in, h_sigma_prev, h_sigma_out, d_out, out_capacity, &jobs[0]));
    if (gamma == 2 && 2 * k_in * (ctx->ring.c / SF_NB) > 4096)
        return sf_set_error(SF_EINVAL, "too many input ciphertexts for one round at gamma = 2");
    jobs[0].d_pow = gamma == 2 ? d_powers : nullptr;
    SF_TRY(eval_jobs(ctx, jobs, (cudaStream_t)stream));
    if (n_out) *n_out = jobs[0].G;
    return SF_OK;
}

extern "C" sf_status sf_eval_linear_layer(sf_ctx *ctx, const sf_layer *L, const sf_rotkeys *rk, const uint64_t *d_in,
                                          int32_t k_in, const uint32_t *h_sigma_prev, const uint32_t *h_sigma_out,
                                          uint64_t *d_out, int32_t out_capacity, int32_t *n_out, void *stream)
{
    SF_CHECK_CTX(ctx);
    std::vector<Job> jobs(1);
    SF_TRY(make_job(ctx, L, rk, d_in, k_in, h_sigma_prev, h_sigma_out, d_out, out_capacity, &jobs[0]));
    SF_TRY(eval_jobs(ctx, jobs, (cudaStream_t)stream));
    if (n_out) *n_out = jobs[0].G;
    return SF_OK;
}

extern "C" sf_status sf_eval_layers(sf_ctx *ctx, int32_t n_layers, const sf_layer *const *layers,
                                    const sf_rotkeys *const *rks, const uint64_t *const *d_ins, const int32_t *k_ins,
                                    const uint32_t *const *h_sigma_prevs, const uint32_t *const *h_sigma_outs,
                                    uint64_t *const *d_outs, const int32_t *out_capacities, int32_t *n_outs, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (n_layers < 1 || !layers || !rks || !d_ins || !k_ins || !d_outs || !out_capacities)
        return sf_set_error(SF_EINVAL, "sf_eval_layers: bad arguments");
    std::vector<Job> jobs(n_layers);
    for (int x = 0; x < n_layers; ++x)
        SF_TRY(make_job(ctx, layers[x], rks[x], d_ins[x], k_ins[x], h_sigma_prevs ? h_sigma_prevs[x] : nullptr,
                        h_sigma_outs ? h_sigma_outs[x] : nullptr, d_outs[x], out_capacities[x], &jobs[x]));
    SF_TRY(eval_jobs(ctx, jobs, (cudaStream_t)stream));
    if (n_outs)
        for (int x = 0; x < n_layers; ++x) n_outs[x] = jobs[x].G;
    return SF_OK;
}

extern "C" sf_status sf_eval_layers_gamma(sf_ctx *ctx, int32_t n_layers, const sf_layer *const *layers,
                                          const sf_rotkeys *const *rks, const uint64_t *const *d_ins,
                                          const uint64_t *const *d_powers, const int32_t *k_ins,
                                          const uint32_t *const *h_sigma_prevs, const uint32_t *const *h_sigma_outs,
                                          uint64_t *const *d_outs, const int32_t *out_capacities, int32_t *n_outs,
                                          void *stream)
{
    SF_CHECK_CTX(ctx);
    if (n_layers < 1 || !layers || !rks || !d_ins || !k_ins || !d_outs || !out_capacities)
        return sf_set_error(SF_EINVAL, "sf_eval_layers_gamma: bad arguments");
    std::vector<Job> jobs(n_layers);
    for (int x = 0; x < n_layers; ++x) {
        SF_TRY(make_job(ctx, layers[x], rks[x], d_ins[x], k_ins[x], h_sigma_prevs ? h_sigma_prevs[x] : nullptr,
                        h_sigma_outs ? h_sigma_outs[x] : nullptr, d_outs[x], out_capacities[x], &jobs[x]));
        jobs[x].d_pow = d_powers ? d_powers[x] : nullptr;
        if (jobs[x].d_pow && 2 * k_ins[x] * (ctx->ring.c / SF_NB) > 4096)
            return sf_set_error(SF_EINVAL, "too many input ciphertexts for one round at gamma = 2");
    }
    SF_TRY(eval_jobs(ctx, jobs, (cudaStream_t)stream));
    if (n_outs)
        for (int x = 0; x < n_layers; ++x) n_outs[x] = jobs[x].G;
    return SF_OK;
}

#define SF_AUTOTUNE_KS_SCRATCH ((size_t)16 << 30)

extern "C" sf_status sf_autotune_layers(sf_ctx *ctx, int32_t n_layers, const sf_layer *const *layers,
                                        const sf_rotkeys *const *rks, const uint64_t *const *d_ins, const int32_t *k_ins,
                                        const uint32_t *const *h_sigma_prevs, const uint32_t *const *h_sigma_outs,
                                        uint64_t *const *d_outs, const int32_t *out_capacities, int32_t repeats,
                                        int32_t *best_ks_batch, double *best_ms, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (repeats < 1) return sf_set_error(SF_EINVAL, "sf_autotune_layers: repeats must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    const int saved_timing = ctx->kernel_timing;
    ctx->kernel_timing = 0;
    cudaEvent_t e0, e1;
    SF_CUDA_TRY(cudaEventCreate(&e0));
    SF_CUDA_TRY(cudaEventCreate(&e1));
    sf_status status = SF_OK;
    // times the batch under the current options: one warm-up (also captures the graph), best of `repeats`
    auto measure = [&](double *out_ms) -> sf_status {
        sf_graph_cache_clear(ctx);
        SF_TRY(sf_eval_layers(ctx, n_layers, layers, rks, d_ins, k_ins, h_sigma_prevs, h_sigma_outs, d_outs,
                              out_capacities, nullptr, stream));
        double tmin = 1e30;
        for (int r = 0; r < repeats; ++r) {
            cudaEventRecord(e0, st);
            SF_TRY(sf_eval_layers(ctx, n_layers, layers, rks, d_ins, k_ins, h_sigma_prevs, h_sigma_outs, d_outs,
                                  out_capacities, nullptr, stream));
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            tmin = std::min(tmin, (double)ms);
        }
        *out_ms = tmin;
        return SF_OK;
    };
    // 1) merges per key-switch launch; larger batches amortise each kernel's
    // twiddle staging and tail over more merges, at ks_scratch x batch bytes of
    // workspace, which is capped at SF_AUTOTUNE_KS_SCRATCH
    static const int cand[] = {32, 64, 128, 256, 512, 1024, 2048, 4096};
    int best = ctx->ks_batch;
    double best_t = 1e30;
    for (int c : cand) {
        if (c > 512 && sf_ks_scratch_words(ctx->ring) * sizeof(u64) * c > SF_AUTOTUNE_KS_SCRATCH) continue;
        ctx->ks_batch = c;
        double t = 0;
        if ((status = measure(&t)) != SF_OK) break;
        if (t < best_t) {
            best_t = t;
            best = c;
        }
    }
    ctx->ks_batch = best;
    // 2) leaf column pass of sparse tiles: closed form (default rule) or always the transform
    if (status == SF_OK) {
        const int saved_sparse = ctx->leaf_sparse;
        int best_sparse = saved_sparse;
        for (int sp : {-1, 0}) {
            if (sp == saved_sparse) continue;
            ctx->leaf_sparse = sp;
            double t = 0;
            if ((status = measure(&t)) != SF_OK) break;
            if (t < best_t) {
                best_t = t;
                best_sparse = sp;
            }
        }
        ctx->leaf_sparse = best_sparse;
    }
    // 3) block shape of the key-switch inner product for 128-point rows:
    //    256 threads x 8 elements or 512 threads x 4 elements
    if (status == SF_OK && ctx->ring.log_c == 7) {
        const int saved = ctx->ks3_threads;
        int best_nt = saved;
        for (int nt : {256, 512}) {
            if (nt == saved) continue;
            ctx->ks3_threads = nt;
            double t = 0;
            if ((status = measure(&t)) != SF_OK) break;
            if (t < best_t) {
                best_t = t;
                best_nt = nt;
            }
        }
        ctx->ks3_threads = best_nt;
    }
    // 4) NTT radix of the row passes (key-switch rows, inner product, ModDown
    //    finish, leaf rows): radix-8 sweeps (three per row pass), radix-4
    //    sweeps only, which hold half the values per unit, or radix 8 with two
    //    sweeps of 256- and 512-point rows fused by warp-shuffle exchanges
    if (status == SF_OK) {
        const int saved = ctx->row_radix;
        int best_rad = saved;
        for (int rad : {0, 1, 2}) {
            if (rad == saved) continue;
            ctx->row_radix = rad;
            double t = 0;
            if ((status = measure(&t)) != SF_OK) break;
            if (t < best_t) {
                best_t = t;
                best_rad = rad;
            }
        }
        ctx->row_radix = best_rad;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sf_graph_cache_clear(ctx);
    ctx->kernel_timing = saved_timing;
    if (status != SF_OK) return status;
    if (best_ks_batch) *best_ks_batch = best;
    if (best_ms) *best_ms = best_t;
    return SF_OK;
}

extern "C" sf_status sf_eval_linear_layer_host(sf_ctx *ctx, const sf_layer *L, const sf_rotkeys *rk, const uint64_t *h_in,
                                               int32_t k_in, const uint32_t *h_sigma_prev, const uint32_t *h_sigma_out,
                                               uint64_t *h_out, int32_t out_capacity, int32_t *n_out, void *stream)
{
    SF_CHECK_CTX(ctx);
    if (!h_in || !h_out || k_in < 1 || out_capacity < 1) return sf_set_error(SF_EINVAL, "sf_eval_linear_layer_host: bad arguments");
    const size_t ct = ct_words(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t need = sizeof(u64) * ct * ((size_t)k_in + out_capacity);
    if (need > ctx->io_bytes) {
        if (ctx->io_buf) {
            SF_CUDA_TRY(cudaDeviceSynchronize());
            cudaFree(ctx->io_buf);
            ctx->io_buf = nullptr;
            ctx->io_bytes = 0;
        }
        if (cudaMalloc(&ctx->io_buf, need) != cudaSuccess) {
            cudaGetLastError();
            return sf_set_error(SF_ENOMEM, "device staging of %zu bytes failed", need);
        }
        ctx->io_bytes = need;
        sf_graph_cache_clear(ctx);
    }
    u64 *d_in = (u64 *)ctx->io_buf, *d_out = d_in + ct * k_in;
    SF_CUDA_TRY(cudaMemcpyAsync(d_in, h_in, sizeof(u64) * ct * k_in, cudaMemcpyHostToDevice, st));
    int32_t got = 0;
    SF_TRY(sf_eval_linear_layer(ctx, L, rk, d_in, k_in, h_sigma_prev, h_sigma_out, d_out, out_capacity, &got, stream));
    SF_CUDA_TRY(cudaMemcpyAsync(h_out, d_out, sizeof(u64) * ct * got, cudaMemcpyDeviceToHost, st));
    SF_CUDA_TRY(cudaStreamSynchronize(st));
    if (n_out) *n_out = got;
    return SF_OK;
}
