// sf_bntt.cu -- batched negacyclic NTT over every RNS limb of a batch of
// polynomials, and register-resident probes of the modular arithmetic.
//
// The batch is [count][L][N]: limb i of polynomial p is reduced modulo q_i.
// A transform is the two tiled passes of sf_tile.cuh (forward: column pass,
// then row pass; inverse: row pass, then column pass with the factor N^-1).
// Each pass is one persistent launch of one resident wave over the units
// (group, polynomial), a group being a column or row tile position and a limb:
// a block takes an equal range of units (sf_block_units), stages a group's
// twiddles when its range enters the group, and prefetches the next unit's
// tile with cp.async while it transforms the current one.
#include <algorithm>

#include "sf_async.cuh"
#include "sf_internal.h"
#include "sf_kernels.cuh"
#include "sf_round.h"

template <bool INV, int LR, int LC, int RAD = 0>
__global__ void __launch_bounds__(SfRow<LC>::NT, 3)
    k_bntt_row(SfRing R, const u64 *src, u64 *dst, int count, int ng)
{
    constexpr int NT = SfRow<LC>::NT, NB = SfRow<LC>::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const SfUnits U = sf_block_units(ng * count);
    constexpr bool DB = sf_rows_double_buffered(LC);
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *buf0 = (u64 *)(tw + NB * g.c);
    u64 *buf1 = DB ? buf0 + SfRow<LC>::WORDS : buf0;
    const size_t per = (size_t)R.L << (LR + LC);
    // unit u: group u / count = (row tile, limb i), item u % count = polynomial
    auto unit_off = [&](int u) -> size_t {
        const int gg = u / count;
        return per * (u % count) + ((size_t)(gg % R.L) << (LR + LC)) + (size_t)(gg / R.L) * NB * g.c;
    };
    if (DB && U.u0 < U.u1) issue_row_tile_t<LC, NT>(buf0, src + unit_off(U.u0));
    sf_cp_commit();
    int staged = -1;
    u64 q = 0, one_p = 0;
    for (int k = 0, u = U.u0; u < U.u1; ++k, ++u) {
        const int grp = u / count;
        if (grp != staged) {
            // the previous unit ended at a barrier: nothing reads tw now
            const int i = grp % R.L;
            load_row_tw_t<LR, LC, NT>(tw, INV ? R.rowT_i : R.rowT_f, i, (grp / R.L) * NB);
            q = R.m[i].q;
            one_p = R.m[i].one_p;
            staged = grp;
        }
        u64 *cur = (k & 1) ? buf1 : buf0, *nxt = (k & 1) ? buf0 : buf1;
        if (DB) {
            if (u + 1 < U.u1) issue_row_tile_t<LC, NT>(nxt, src + unit_off(u + 1));
            sf_cp_commit();
            sf_cp_wait<1>();
        } else {
            issue_row_tile_t<LC, NT>(cur, src + unit_off(u));
            sf_cp_commit();
            sf_cp_wait<0>();
        }
        __syncthreads();
        // forward: the last pass, canonical output; inverse: lazy in [0, 4q), the column pass follows
        if (INV) {
            u64 *gd = dst + unit_off(u);
            row_inverse_out<LC, NT, RAD>(cur, tw, q, [&](int k, int b, u64 v) { gd[(b << LC) + k] = v; });
        } else {
            row_forward_t<LC, NT, RAD>(cur, tw, q);
            store_row_tile_t<LC, NT>(dst + unit_off(u), cur, [&](u64 v) { return sf_reduce(v, q, one_p); });
        }
        __syncthreads();
    }
}

template <bool INV, int LR, int LC>
__global__ void __launch_bounds__(SfThreads<LR>::value, LR >= 8 ? 2 : 3)
    k_bntt_col(SfRing R, const u64 *src, u64 *dst, int count, int ng)
{
    constexpr int NT = SfThreads<LR>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const SfUnits U = sf_block_units(ng * count);
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *buf0 = (u64 *)(tw + g.r);
    u64 *buf1 = buf0 + tile_words(g.log_r);
    const size_t per = (size_t)R.L << (LR + LC);
    // unit u: group u / count = (column tile, limb i), item u % count = polynomial
    auto unit_off = [&](int u) -> size_t { return per * (u % count) + ((size_t)((u / count) % R.L) << (LR + LC)); };
    auto unit_c0 = [&](int u) -> int { return ((u / count) / R.L) * SF_NB; };
    if (U.u0 < U.u1) issue_col_tile_t<LR, LC, NT>(buf0, src + unit_off(U.u0), unit_c0(U.u0));
    sf_cp_commit();
    int staged = -1;
    u64 q = 0, ninv = 0, ninv_p = 0;
    for (int k = 0, u = U.u0; u < U.u1; ++k, ++u) {
        const int grp = u / count;
        if (grp != staged) {
            // the previous unit ended at a barrier: nothing reads tw now
            const int i = grp % R.L;
            load_col_tw_t<LR, NT>(tw, INV ? R.colT_i : R.colT_f, i);
            q = R.m[i].q;
            ninv = R.m[i].ninv;
            ninv_p = R.m[i].ninv_p;
            staged = grp;
        }
        u64 *cur = (k & 1) ? buf1 : buf0, *nxt = (k & 1) ? buf0 : buf1;
        if (u + 1 < U.u1) issue_col_tile_t<LR, LC, NT>(nxt, src + unit_off(u + 1), unit_c0(u + 1));
        sf_cp_commit();
        sf_cp_wait<1>();
        __syncthreads();
        // inverse: the last pass, times N^-1, canonical; forward: lazy, the row
        // pass follows.  The last sweep writes the tile to global memory itself.
        u64 *gd = dst + unit_off(u) + unit_c0(u);
        auto out = [&](int k, int b, u64 v) { gd[((size_t)k << LC) + b] = INV ? sf_mul_shoup(v, ninv, ninv_p, q) : v; };
        if (INV) col_inverse_st<LR, NT>(cur, tw, q, out);
        else col_forward_io<LR, NT>(cur, tw, q, [&](int k, int b) { return cur[tile_slot<SF_NB>(k, b)]; }, out);
        __syncthreads();
    }
}

template <class K>
static int bntt_occupancy(K kernel, int threads, size_t smem)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return std::max(1, b);
}

// one resident wave (SMs x occupancy blocks), at most one block per unit
static int bntt_blocks(const sf_ctx *ctx, int occ, int n_units)
{
    return std::max(1, std::min(ctx->num_sms * occ, n_units));
}

static size_t bntt_smem_row(const SfRing &R)
{
    return sizeof(sf_tw) * sf_row_nb(R.log_c) * R.c + sizeof(u64) * row_tile_words(R.log_c) * (sf_rows_double_buffered(R.log_c) ? 2 : 1);
}
static size_t bntt_smem_col(const SfRing &R) { return sizeof(sf_tw) * R.r + sizeof(u64) * tile_words(R.log_r) * 2; }

extern "C" sf_status sf_ntt_batch(sf_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t inverse,
                                  void *stream)
{
    SF_CHECK_CTX(ctx);
    if (!d_in || !d_out || count < 1 || (inverse != 0 && inverse != 1))
        return sf_set_error(SF_EINVAL, "sf_ntt_batch: bad arguments");
    const SfRing &R = ctx->ring;
    cudaStream_t st = (cudaStream_t)stream;
    const int rg = (R.r / sf_row_nb(R.log_c)) * R.L, cg = (R.c / SF_NB) * R.L;
    if ((long long)count * std::max(rg, cg) > INT32_MAX)
        return sf_set_error(SF_EINVAL, "sf_ntt_batch: count too large");
    const size_t smr = bntt_smem_row(R), smc = bntt_smem_col(R);
    cudaEvent_t ev;
    SF_GEO_DISPATCH(R.log_n, {
        constexpr int NTR = SfRow<LC>::NT, NTC = SfThreads<LR>::value;
        if (!inverse) {
            const int bc = bntt_blocks(ctx, bntt_occupancy(k_bntt_col<false, LR, LC>, NTC, smc), cg * count);
            sf_launch_begin(ctx, SFK_BNTT_COL, st, &ev);
            k_bntt_col<false, LR, LC><<<bc, NTC, smc, st>>>(R, d_in, d_out, count, cg);
            sf_launch_end(ctx, SFK_BNTT_COL, st, ev);
            sf_launch_begin(ctx, SFK_BNTT_ROW, st, &ev);
            SF_RAD_DISPATCH(ctx->row_radix, {
                const int br = bntt_blocks(ctx, bntt_occupancy(k_bntt_row<false, LR, LC, RAD>, NTR, smr), rg * count);
                k_bntt_row<false, LR, LC, RAD><<<br, NTR, smr, st>>>(R, d_out, d_out, count, rg);
            });
            sf_launch_end(ctx, SFK_BNTT_ROW, st, ev);
        } else {
            sf_launch_begin(ctx, SFK_BNTT_ROW, st, &ev);
            SF_RAD_DISPATCH(ctx->row_radix, {
                const int br = bntt_blocks(ctx, bntt_occupancy(k_bntt_row<true, LR, LC, RAD>, NTR, smr), rg * count);
                k_bntt_row<true, LR, LC, RAD><<<br, NTR, smr, st>>>(R, d_in, d_out, count, rg);
            });
            sf_launch_end(ctx, SFK_BNTT_ROW, st, ev);
            const int bc = bntt_blocks(ctx, bntt_occupancy(k_bntt_col<true, LR, LC>, NTC, smc), cg * count);
            sf_launch_begin(ctx, SFK_BNTT_COL, st, &ev);
            k_bntt_col<true, LR, LC><<<bc, NTC, smc, st>>>(R, d_out, d_out, count, cg);
            sf_launch_end(ctx, SFK_BNTT_COL, st, ev);
        }
    });
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

sf_status sf_bntt_init_attributes()
{
    const int mx = 227 * 1024;
#define SF_BNTT_ATTR(K) SF_CUDA_TRY(cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
#define SF_BNTT_ATTRS(LR, LC)                                                                                     \
    SF_BNTT_ATTR((k_bntt_row<false, LR, LC>)) SF_BNTT_ATTR((k_bntt_row<true, LR, LC>))                             \
    SF_BNTT_ATTR((k_bntt_row<false, LR, LC, 1>)) SF_BNTT_ATTR((k_bntt_row<true, LR, LC, 1>))                       \
    SF_BNTT_ATTR((k_bntt_row<false, LR, LC, 2>)) SF_BNTT_ATTR((k_bntt_row<true, LR, LC, 2>))                       \
    SF_BNTT_ATTR((k_bntt_col<false, LR, LC>)) SF_BNTT_ATTR((k_bntt_col<true, LR, LC>))
    SF_BNTT_ATTRS(5, 5) SF_BNTT_ATTRS(5, 6) SF_BNTT_ATTRS(6, 6) SF_BNTT_ATTRS(6, 7) SF_BNTT_ATTRS(7, 7)
    SF_BNTT_ATTRS(7, 8) SF_BNTT_ATTRS(7, 9)
#undef SF_BNTT_ATTRS
#undef SF_BNTT_ATTR
    return SF_OK;
}

// ---------------------------------------------------------------- probes ----
// Each thread keeps 8 residues in registers and applies PROBE_ITERS rounds of
// 12 operations to them (a radix-8 unit: 3 stages of 4 butterflies, or 12
// multiply-accumulates), then stores them.  Nothing else is read or written,
// so the rate is the arithmetic ceiling of these operations on this GPU.
#define PROBE_ITERS 1024
#define PROBE_OPS (12 * PROBE_ITERS)

template <int KIND>
__global__ void __launch_bounds__(256, 2) k_probe(u64 *buf, u64 q, ulonglong2 t0, ulonglong2 t1, ulonglong2 t2,
                                                 ulonglong2 t3)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[8], acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        x[i] = buf[i * stride + t];
        acc[i] = 0;
    }
    const u64 two_q = 2 * q;
    for (int it = 0; it < PROBE_ITERS; ++it) {
        if (KIND == 0) {
#pragma unroll
            for (int i = 0; i < 4; ++i) sf_bfly_ct(x[i], x[i + 4], t0.x, t0.y, q, two_q);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                sf_bfly_ct(x[i], x[i + 2], t1.x, t1.y, q, two_q);
                sf_bfly_ct(x[i + 4], x[i + 6], t2.x, t2.y, q, two_q);
            }
#pragma unroll
            for (int i = 0; i < 8; i += 2) sf_bfly_ct(x[i], x[i + 1], t3.x, t3.y, q, two_q);
        } else if (KIND == 1) {
#pragma unroll
            for (int i = 0; i < 8; i += 2) sf_bfly_gs(x[i], x[i + 1], t3.x, t3.y, q, two_q);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                sf_bfly_gs(x[i], x[i + 2], t1.x, t1.y, q, two_q);
                sf_bfly_gs(x[i + 4], x[i + 6], t2.x, t2.y, q, two_q);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) sf_bfly_gs(x[i], x[i + 4], t0.x, t0.y, q, two_q);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const ulonglong2 w = (i & 3) == 0 ? t0 : (i & 3) == 1 ? t1 : (i & 3) == 2 ? t2 : t3;
                acc[i] += sf_mul_shoup_lazy4(x[i], w.x, w.y, q);
                x[i] ^= acc[i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const ulonglong2 w = i == 0 ? t0 : i == 1 ? t1 : i == 2 ? t2 : t3;
                acc[i] += sf_mul_shoup_lazy4(x[i + 4], w.x, w.y, q);
                x[i] += acc[i + 4];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) buf[i * stride + t] = x[i] + acc[i];
}

extern "C" sf_status sf_modmul_probe(sf_ctx *ctx, int32_t kind, double *gmodmul_per_s)
{
    SF_CHECK_CTX(ctx);
    if (!gmodmul_per_s || kind < 0 || kind > 2) return sf_set_error(SF_EINVAL, "sf_modmul_probe: bad arguments");
    const SfMod &M = ctx->ring.m[0];
    int occ = 1;
    switch (kind) {
    case 0: occ = bntt_occupancy(k_probe<0>, 256, 0); break;
    case 1: occ = bntt_occupancy(k_probe<1>, 256, 0); break;
    default: occ = bntt_occupancy(k_probe<2>, 256, 0); break;
    }
    const int grid = ctx->num_sms * occ;
    const size_t words = (size_t)8 * grid * 256;
    SF_CUDA_TRY(cudaDeviceSynchronize());
    void *w = nullptr;
    SF_TRY(sf_scratch(ctx, words * sizeof(u64), &w));
    u64 *buf = (u64 *)w;
    SF_CUDA_TRY(cudaMemset(buf, 0x5a, words * sizeof(u64)));
    // four fixed twiddle pairs (w, floor(w 2^64 / q)) modulo q_0
    ulonglong2 tw[4];
    for (int i = 0; i < 4; ++i) {
        const u64 v = (M.q / 3 + 7919 * (u64)i) % M.q;
        tw[i] = make_ulonglong2(v, sf_shoup_companion(v, M.q));
    }
    auto launch = [&]() {
        switch (kind) {
        case 0: k_probe<0><<<grid, 256>>>(buf, M.q, tw[0], tw[1], tw[2], tw[3]); break;
        case 1: k_probe<1><<<grid, 256>>>(buf, M.q, tw[0], tw[1], tw[2], tw[3]); break;
        default: k_probe<2><<<grid, 256>>>(buf, M.q, tw[0], tw[1], tw[2], tw[3]); break;
        }
    };
    cudaEvent_t a = nullptr, b = nullptr;
    SF_CUDA_TRY(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return sf_set_error(SF_ECUDA, "sf_modmul_probe: event creation failed");
    }
    const int reps = 5;
    for (int r = 0; r < 2; ++r) launch();
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return sf_set_error(SF_ECUDA, "sf_modmul_probe: %s", cudaGetErrorString(e));
    SF_CUDA_TRY(cudaGetLastError());
    const double ops = (double)PROBE_OPS * grid * 256 * reps;
    *gmodmul_per_s = ms > 0.f ? ops / (ms * 1e-3) / 1e9 : 0.0;
    return SF_OK;
}
