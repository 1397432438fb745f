// sf_layer.cu -- the linear-layer round (Sec. 4.4, steps 6-10) on the GPU.
//
// Steps 6-8 (extraction at gamma = 0, unshuffle, linear layer): the row
// extracted for stream position p = jN + k is N^-1 X^-k ct_j, so output o is
//     y_o = sum_j w_{o,j}(X) * ct_j,   w_{o,j} = N^-1 sum_{taps i in ct j} Wq[o,i] X^-k(i)
// with k(i) the in-ciphertext position of input i after unshuffling
// (p = sigma_prev^-1(i)).  Three kernels per batch of outputs:
//   leaf_prep: walks each output's receptive field once and buckets its taps
//              by (input ciphertext, 16-column tile),
//   leaf_col : builds the sparse w_{o,j} column tile in shared memory from its
//              bucket and runs the forward column pass (or its closed form),
//   leaf_row : forward row pass, then the product with every input ciphertext
//              (NTT domain, Shoup companions stored beside it), lazy sums -> leaf.
// Step 9 (shuffle) is the slot -> output map sigma_out; step 10 (packing) is
// the PackLWEs tree plus field trace driven by sf_pack_tree below.
#include "sf_internal.h"
#include "sf_kernels.cuh"
#include "sf_ks.h"
#include "sf_layer.h"

__device__ __forceinline__ int leaf_output(const SfLeafParams &P, int slot)
{
    if (slot >= P.n_slots_valid) return -1;
    return P.sig_out ? P.sig_out[slot] : slot;
}

// Taps of one column tile kept for the closed-form column pass.  A tile
// with few taps skips the sweep: the column pass maps column c of a
// polynomial to its values at the R roots of Y^R = -1, z_k =
// phi^(2 brev(k) + 1) with phi = psi^C, so a single tap v at row r
// contributes v * psi^(C r (2 brev(k) + 1) mod 2N) to row k -- R products per
// tap instead of (R/2) log2 R butterflies per column.
#define SF_LEAF_TAPS 128

size_t sf_smem_leaf_col(const SfRing &R) { return sf_smem_col(R, 1) + sizeof(sf_tw) * 2 * R.r; }

// Calls f(j, row, column, signed Wq) for every tap of output o: input
// ciphertext j, and the coefficient N - k (or 0) of w_{o,j} it lands on as
// (row, column) of the R x C split; the sign carries the X^-k = -X^(N-k) of
// the extraction.  Threads split the taps.
template <class F>
__device__ __forceinline__ void leaf_taps_all(const SfRing &R, const SfGeo &g, const SfLeafParams &P, int o, F f)
{
    const int co = o % P.C_out, hw = o / P.C_out;
    const int ho = hw / P.W_out, wo = hw % P.W_out;
    for (int ti = 0; ti < P.n_terms; ++ti) {
        const SfTermDev &T = P.t[ti];
        const int ntap = T.kh * T.kw * T.C_in;
        const int h0 = ho * T.stride - T.pad, w0 = wo * T.stride - T.pad;
        const int base = T.in_offset + (h0 * T.W + w0) * T.C_in;
        const int64_t *wrow = P.wq + T.w_off + (size_t)co * ntap;
        for (int tt = threadIdx.x; tt < ntap; tt += blockDim.x) {
            const int4 tp = P.taps[T.tap_off + tt];
            const int h = h0 + tp.x, w = w0 + tp.y;
            if (h < 0 || h >= T.H || w < 0 || w >= T.W) continue;
            const int idx = base + tp.z;
            const int p = P.pos_of ? P.pos_of[idx] : idx;
            const int k = p & (R.n - 1);
            const int cidx = k ? R.n - k : 0;
            const int64_t wq = P.gamma2 ? 2 * wrow[tp.w] : wrow[tp.w];
            f(p >> R.log_n, cidx >> g.log_c, cidx & (g.c - 1), k ? -wq : wq);
            if (P.gamma2) {
                // gamma = 2 (Lemma 1 at t = 2): the row is (N/2)^-1 (X^-k ct_j + X^-3k ct3_j), so
                // the tap also lands at X^-3k of the power ct3_j.  With e = 3k mod 2N,
                // X^-e = 1 (e = 0), -X^(N - e) (0 < e <= N), X^(2N - e) (N < e < 2N).
                const int e = (3 * k) & (2 * R.n - 1);
                const int c3 = e == 0 ? 0 : (e <= R.n ? R.n - e : 2 * R.n - e);
                const bool neg = e != 0 && e <= R.n;
                f(P.k_src + (p >> R.log_n), c3 >> g.log_c, c3 & (g.c - 1), neg ? -wq : wq);
            }
        }
    }
}

size_t sf_leaf_tap_words(const SfRing &R, int k_in, int max_taps, int slots)
{
    const size_t nb = (size_t)k_in * (R.c / SF_NB) + 1;
    return (size_t)slots * max_taps * 2 + (slots * nb + 1) / 2;
}

// leaf_prep: grid (slots).  Buckets the taps of each slot's output by
// (input ciphertext, column tile) with a counting sort, so that a column
// block reads its own taps instead of scanning the whole receptive field.
#define SF_MAX_BUCKETS 4096
__global__ void __launch_bounds__(256) k_leaf_prep(SfRing R, SfLeafParams P)
{
    __shared__ int cnt[SF_MAX_BUCKETS + 1];
    const SfGeo g = ring_geo(R);
    const int z = blockIdx.x;
    const int o = leaf_output(P, P.s0 + z * P.s_stride);
    if (o < 0) return;   // leaf_col skips this slot as well
    const int nb = P.n_buckets, tiles = g.c / SF_NB;
    int *off = P.tap_off + (size_t)z * (nb + 1);
    for (int b = threadIdx.x; b <= nb; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    leaf_taps_all(R, g, P, o, [&](int j, int row, int col, int64_t) { atomicAdd(&cnt[j * tiles + (col >> 4)], 1); });
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < nb; ++b) {
            const int c = cnt[b];
            cnt[b] = acc;
            off[b] = acc;
            acc += c;
        }
        off[nb] = acc;
    }
    __syncthreads();
    longlong2 *dst = P.tap_buf + (size_t)z * P.max_taps;
    leaf_taps_all(R, g, P, o, [&](int j, int row, int col, int64_t wq) {
        const int pos = atomicAdd(&cnt[j * tiles + (col >> 4)], 1);
        dst[pos] = make_longlong2((row << 4) | (col & 15), wq);
    });
}

// N^-1 * wq mod q, canonical (|wq| < 2^63)
__device__ __forceinline__ u64 leaf_coeff(const SfMod &M, int64_t wq)
{
    const u64 a = sf_reduce((u64)(wq < 0 ? -wq : wq), M.q, M.one_p);
    const u64 v = sf_mul_shoup(a, M.ninv, M.ninv_p, M.q);
    return (wq < 0 && v) ? M.q - v : v;
}

// leaf_col: grid (C/16 column tiles, k_in * L, slots).  smem: column
// twiddles + 1 tile + the powers psi^(C e), e < 2R.
template <int LR, int LC>
__global__ void __launch_bounds__(SfThreads<LR>::value, SfThreads<LR>::value >= 512 ? 2 : 4) k_leaf_col(SfRing R, SfLeafParams P)
{
    constexpr int NT = SfThreads<LR>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ u64 tap_v[SF_LEAF_TAPS];
    __shared__ int tap_rc[SF_LEAF_TAPS];
    // sparse form: taps sorted by column (start[b] .. start[b+1])
    __shared__ int col_start[SF_NB + 1];
    __shared__ int col_fill[SF_NB];
    __shared__ int srt_t[SF_LEAF_TAPS];
    constexpr SfGeoT<LR, LC> g{};
    const int c0 = blockIdx.x * SF_NB;
    const int j = blockIdx.y / R.L, i = blockIdx.y % R.L;
    const int slot = P.s0 + blockIdx.z * P.s_stride;
    const int o = leaf_output(P, slot);
    if (o < 0) return;
    const SfMod &M = R.m[i];
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *sm = (u64 *)(tw + g.r);
    sf_tw *pwc = (sf_tw *)(sm + tile_words(g.log_r));
    constexpr int ne = SF_NB << LR;
    u64 *dst = P.w1 + (((size_t)blockIdx.z * P.k_in + j) * R.L + i) * (size_t)(1 << (LR + LC));
    // this block's bucket of taps (built by leaf_prep)
    const int *off = P.tap_off + (size_t)blockIdx.z * (P.n_buckets + 1);
    const int bk = j * (g.c / SF_NB) + blockIdx.x;
    const int t0 = off[bk], nt = off[bk + 1] - t0;
    const longlong2 *src = P.tap_buf + (size_t)blockIdx.z * P.max_taps + t0;
    if (threadIdx.x < SF_NB) col_fill[threadIdx.x] = 0;
    if (nt <= P.sparse_max) {
        // stage the powers for the closed form while the taps load
        const sf_tw *pw = R.pwc + (size_t)i * 2 * g.r;
        for (int e = threadIdx.x; e < 2 * g.r; e += NT) pwc[e] = pw[e];
    }
    __syncthreads();
    if (nt <= SF_LEAF_TAPS) {
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const longlong2 e = src[t];
            tap_v[t] = leaf_coeff(M, e.y);
            tap_rc[t] = (int)e.x;
            atomicAdd(&col_fill[e.x & 15], 1);
        }
    }
    __syncthreads();
    if (nt <= P.sparse_max) {
        // counting sort by column; the order inside a column does not matter (exact sums)
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int b = 0; b < SF_NB; ++b) {
                col_start[b] = acc;
                acc += col_fill[b];
                col_fill[b] = col_start[b];
            }
            col_start[SF_NB] = acc;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nt; t += blockDim.x) srt_t[atomicAdd(&col_fill[tap_rc[t] & 15], 1)] = t;
        __syncthreads();
        const unsigned emask = 2u * g.r - 1;
        for (int e = threadIdx.x; e < ne; e += NT) {
            const int k = e >> 4, b = e & 15;
            const unsigned br2 = 2u * (__brev((unsigned)k) >> (32 - g.log_r)) + 1u;
            u64 acc = 0;
            for (int t = col_start[b]; t < col_start[b + 1]; ++t) {
                const int tt = srt_t[t];
                const sf_tw z = pwc[(((unsigned)tap_rc[tt] >> 4) * br2) & emask];
                acc += sf_mul_shoup_lazy(tap_v[tt], z.x, z.y, M.q);
            }
            dst[col_gidx_t<LC>(c0, e)] = sf_reduce(acc, M.q, M.one_p);
        }
        return;
    }
    for (int e = threadIdx.x; e < tile_words(g.log_r); e += blockDim.x) sm[e] = 0;
    load_col_tw_t<LR, NT>(tw, R.colT_f, i);
    __syncthreads();
    if (nt <= SF_LEAF_TAPS) {
        for (int t = threadIdx.x; t < nt; t += blockDim.x) sm[(tap_rc[t] >> 4) * SF_PAD + (tap_rc[t] & 15)] = tap_v[t];
    } else {
        for (int t = threadIdx.x; t < nt; t += blockDim.x) {
            const longlong2 e = src[t];
            sm[(e.x >> 4) * SF_PAD + (e.x & 15)] = leaf_coeff(M, e.y);
        }
    }
    __syncthreads();
    // forward column pass; its last sweep writes the tile to global memory
    u64 *gd = dst + c0;
    col_forward_io<LR, NT>(sm, tw, M.q, [&](int k, int b) { return sm[tile_slot<SF_NB>(k, b)]; },
                           [&](int k, int b, u64 v) { gd[((size_t)k << LC) + b] = v; });
}

// leaf_row: grid (R/16 row tiles, L, slots).  smem: forward row twiddles + 1 tile.
template <int LR, int LC, int RAD = 0>
__global__ void __launch_bounds__(SfRow<LC>::NT, 3) k_leaf_row(SfRing R, SfLeafParams P)
{
    constexpr int NT = SfRow<LC>::NT, NB = SfRow<LC>::NB, EPT = SfRow<LC>::ELEMS / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const int r0 = blockIdx.x * NB, i = blockIdx.y;
    const int slot = P.s0 + blockIdx.z * P.s_stride;
    const int o = leaf_output(P, slot);
    const size_t tile_off = (size_t)r0 * g.c;
    u64 *leaf = P.leaves + P.leaf_stride * blockIdx.z;
    u64 *da = leaf + ((size_t)i << (LR + LC)) + tile_off;
    u64 *db = leaf + ((size_t)(R.L + i) << (LR + LC)) + tile_off;
    if (o < 0) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = threadIdx.x + k * NT;
            da[e] = 0;
            db[e] = 0;
        }
        return;
    }
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *sm = (u64 *)(tw + NB * g.c);
    const SfMod M = R.m[i];
    load_row_tw_t<LR, LC, NT>(tw, R.rowT_f, i, r0);
    // per input ciphertext w * ct (w < 68q lazy, ct < q with its Shoup
    // companion) lands in [0, 4q) and is summed: below 4 q k_in < 2^63 for k_in < 1024
    u64 acc_a[EPT], acc_b[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) acc_a[k] = acc_b[k] = 0;
    for (int j = 0; j < P.k_in; ++j) {
        const u64 *src = P.w1 + (((size_t)blockIdx.z * P.k_in + j) * R.L + i) * (size_t)(1 << (LR + LC)) + tile_off;
#pragma unroll
        for (int x = 0; x < EPT; ++x) {
            const int e = threadIdx.x + x * NT;
            sm[row_slot_t<LC>(e)] = src[e];
        }
        __syncthreads();
        row_forward_t<LC, NT, RAD>(sm, tw, M.q);
        const size_t comp = (size_t)P.k_in * 2 * R.L << (LR + LC);
        const u64 *ca = P.ct + (((size_t)j * 2 + 0) * R.L + i) * (size_t)(1 << (LR + LC)) + tile_off;
        const u64 *cb = P.ct + (((size_t)j * 2 + 1) * R.L + i) * (size_t)(1 << (LR + LC)) + tile_off;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = threadIdx.x + k * NT;
            const u64 w = sm[row_slot_t<LC>(e)];
            acc_a[k] += sf_mul_shoup_lazy4(w, __ldg(ca + e), __ldg(ca + comp + e), M.q);
            acc_b[k] += sf_mul_shoup_lazy4(w, __ldg(cb + e), __ldg(cb + comp + e), M.q);
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = threadIdx.x + k * NT;
        da[e] = sf_reduce(acc_a[k], M.q, M.one_p);
        db[e] = sf_reduce(acc_b[k], M.q, M.one_p);
    }
}

sf_status sf_leaves_launch(sf_ctx *ctx, const SfLeafParams &P, int cnt, cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    if (cnt <= 0) return SF_OK;
    const size_t smem_c = sf_smem_leaf_col(R), smem_r = sf_smem_row(R, 1);
    // closed form while nt R products cost less than the tile's 16 (R/2) log2 R butterflies
    const int sparse_max = std::min(SF_LEAF_TAPS, ctx->leaf_sparse >= 0 ? ctx->leaf_sparse : SF_NB * R.log_r / 2);
    cudaEvent_t ev;
    for (int off = 0; off < cnt; off += 65535) {
        SfLeafParams p = P;
        p.sparse_max = sparse_max;
        const int c = std::min(65535, cnt - off);
        p.s0 = P.s0 + off * P.s_stride;
        p.w1 = P.w1;    // w1 holds `cnt` slots; reuse from its start for each sub-launch
        p.leaves = P.leaves + P.leaf_stride * off;
        if (P.n_buckets > SF_MAX_BUCKETS) return sf_set_error(SF_EINVAL, "too many input ciphertexts for one round");
        sf_launch_begin(ctx, SFK_LEAF_PREP, st, &ev);
        k_leaf_prep<<<c, 256, 0, st>>>(R, p);
        sf_launch_end(ctx, SFK_LEAF_PREP, st, ev);
        sf_launch_begin(ctx, SFK_LEAF_COL, st, &ev);
        SF_GEO_DISPATCH(R.log_n, k_leaf_col<LR, LC><<<dim3(R.c / SF_NB, P.k_in * R.L, c), SfThreads<LR>::value, smem_c, st>>>(R, p););
        sf_launch_end(ctx, SFK_LEAF_COL, st, ev);
        sf_launch_begin(ctx, SFK_LEAF_ROW, st, &ev);
        const dim3 gr(R.r / sf_row_nb(R.log_c), R.L, c);
        SF_GEO_DISPATCH(R.log_n, SF_RAD_DISPATCH(ctx->row_radix, k_leaf_row<LR, LC, RAD><<<gr, SfRow<LC>::NT, smem_r, st>>>(R, p);););
        sf_launch_end(ctx, SFK_LEAF_ROW, st, ev);
    }
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// ------------------------------------------------------------ pack tree --

// Level-1 merge at gamma = 2, NTT domain: out = E + X^s O (out = E without O).
// grid (N / (256 SF_EW), L, merges), SfKsBatch indexing as in the key switch.
#define SF_EW2 8
__global__ void __launch_bounds__(256) k_merge_plain(SfRing R, SfKsBatch B)
{
    const int b = blockIdx.z, i = blockIdx.y;
    int g = (B.first + b) / B.inner, t = (B.first + b) - g * B.inner;
    const u64 *E = B.E + B.E_outer * g + B.E_stride * t;
    const u64 *O = B.O ? B.O + B.O_outer * g + B.O_stride * t : nullptr;
    u64 *out = B.out + B.out_outer * g + B.out_stride * t;
    const SfMod &M = R.m[i];
    const size_t pb = (size_t)i << (R.log_n + 1);
    const int j0 = blockIdx.x * (256 * SF_EW2) + threadIdx.x;
#pragma unroll
    for (int x = 0; x < SF_EW2; ++x) {
        const int j = j0 + x * 256;
        if (j >= R.n) break;
        for (int part = 0; part < 2; ++part) {
            const size_t off = ((size_t)(part * R.L + i) << R.log_n) + j;
            u64 v = E[off];
            if (O) {
                const unsigned kk = mono_index(j, B.s, R.log_n);
                v = sf_add(v, sf_mul_shoup(O[off], R.pw[pb + kk], R.pw_p[pb + kk], M.q), M.q);
            }
            out[off] = v;
        }
    }
}

static sf_status merge_plain_run(sf_ctx *ctx, const SfKsBatch &B, cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    cudaEvent_t ev;
    for (int off = 0; off < B.count; off += 32768) {
        SfKsBatch b = B;
        b.count = std::min(32768, B.count - off);
        b.first = B.first + off;
        sf_launch_begin(ctx, SFK_ELEMWISE, st, &ev);
        k_merge_plain<<<dim3((R.n + 256 * SF_EW2 - 1) / (256 * SF_EW2), R.L, b.count), 256, 0, st>>>(R, b);
        sf_launch_end(ctx, SFK_ELEMWISE, st, ev);
    }
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// Pack-tree levels level0+1 .. level1 (see sf_layer.h).  Node i of a level
// is zero iff i >= valid[g]; a merge whose O-node is zero runs without O
// (identical result, X^s * 0 = 0), and merges producing zero nodes are
// skipped.  Level lvl merges node t with node t + n_lvl/2 (n_lvl = nodes at
// level lvl-1) using s = N / 2^lvl and d = 2^lvl + 1.
sf_status sf_pack_tree(sf_ctx *ctx, const u64 *keys_base, const std::vector<int32_t> &key_d, size_t key_words,
                       u64 *A, u64 *B, int G, int n_nodes, int level0, const std::vector<int> &valid, bool trace,
                       u64 *ks_scratch, int batch, u64 **res, size_t *res_stride, cudaStream_t st, bool tau3_done)
{
    const SfRing &R = ctx->ring;
    const size_t ct = (size_t)2 * R.L * R.n;
    auto key_for = [&](int d, const u64 **k) -> sf_status {
        for (size_t t = 0; t < key_d.size(); ++t)
            if (key_d[t] == d) {
                *k = keys_base + key_words * t;
                return SF_OK;
            }
        return sf_set_error(SF_EINVAL, "no rotation key for d = %d", d);
    };
    int levels = 0;
    while ((1 << levels) < n_nodes) ++levels;
    const int level1 = level0 + levels;
    u64 *cur = A, *nxt = B;
    size_t cur_gs = (size_t)n_nodes * ct, nxt_gs = (size_t)(n_nodes / 2 > 0 ? n_nodes / 2 : 1) * ct;
    for (int lvl = level0 + 1; lvl <= level1; ++lvl) {
        const int half = n_nodes >> (lvl - level0);
        const int d = (1 << lvl) + 1;
        // gamma = 2: the tau_3 level is a plain merge (no key, no key switch)
        const bool plain = tau3_done && lvl == 1;
        auto run = [&](const SfKsBatch &b) -> sf_status {
            return plain ? merge_plain_run(ctx, b, st) : sf_ks_run(ctx, b, ks_scratch, batch, st);
        };
        const u64 *key = nullptr;
        if (!plain) SF_TRY(key_for(d, &key));
        SfKsBatch kb;
        memset(&kb, 0, sizeof(kb));
        kb.E_stride = ct;
        kb.O_stride = ct;
        kb.out_stride = ct;
        kb.E_outer = cur_gs;
        kb.O_outer = cur_gs;
        kb.out_outer = nxt_gs;
        kb.d = d;
        kb.s = (unsigned)(R.n >> lvl);
        kb.add_v = 1;
        kb.key = key;
        int gi = 0;
        while (gi < G) {
            if (valid[gi] >= n_nodes) {
                // a run of full groups: one batch with (group, merge) indexing
                int g1 = gi;
                while (g1 < G && valid[g1] >= n_nodes) ++g1;
                SfKsBatch b = kb;
                b.E = cur + gi * cur_gs;
                b.O = b.E + (size_t)half * ct;
                b.out = nxt + gi * nxt_gs;
                b.inner = half;
                b.count = (g1 - gi) * half;
                SF_TRY(run(b));
                gi = g1;
                continue;
            }
            const int V = std::min(valid[gi], 2 * half);
            const int active = std::min(V, half);
            const int with_o = std::max(0, std::min(active, V - half));
            SfKsBatch b = kb;
            b.E = cur + gi * cur_gs;
            b.out = nxt + gi * nxt_gs;
            b.inner = 1 << 30;
            if (with_o > 0) {
                SfKsBatch b1 = b;
                b1.O = b.E + (size_t)half * ct;
                b1.count = with_o;
                SF_TRY(run(b1));
            }
            if (active > with_o) {
                SfKsBatch b2 = b;
                b2.O = nullptr;
                b2.first = with_o;
                b2.count = active - with_o;
                SF_TRY(run(b2));
            }
            ++gi;
        }
        std::swap(cur, nxt);
        std::swap(cur_gs, nxt_gs);
    }
    // field trace: for k = level1+1 .. log2(N): ct <- ct + tau_{2^k+1}(ct)
    // (from k = 2 at gamma = 2: the client's power supplied the tau_3 term)
    for (int k = std::max(level1 + 1, tau3_done ? 2 : 1); trace && k <= R.log_n; ++k) {
        const int d = (1 << k) + 1;
        const u64 *key;
        SF_TRY(key_for(d, &key));
        SfKsBatch b;
        memset(&b, 0, sizeof(b));
        b.E = cur;
        b.E_stride = cur_gs;
        b.out = nxt;
        b.out_stride = nxt_gs;
        b.inner = 1 << 30;
        b.count = G;
        b.d = d;
        b.add_v = 1;
        b.key = key;
        SF_TRY(sf_ks_run(ctx, b, ks_scratch, batch, st));
        std::swap(cur, nxt);
        std::swap(cur_gs, nxt_gs);
    }
    *res = cur;
    *res_stride = cur_gs;
    return SF_OK;
}

// ------------------------------------------------------------- small ops --

// Bias (the affine part b of f(x) = Ax + b): b-part coefficient l*N/n of
// group g gets bq[channel(sigma_out(g n + l))].
__global__ void k_add_bias(SfRing R, u64 *out, int G, int n, int E_out, const int *sig_out, const int64_t *bq,
                           int C_out, int scale)
{
    const size_t ct = (size_t)2 * R.L * R.n;
    const int stride = R.n / n;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < G * n; x += gridDim.x * blockDim.x) {
        if (x >= E_out) continue;
        int g = x / n, l = x % n;
        int o = sig_out ? sig_out[x] : x;
        int64_t v = bq[o % C_out];
        for (int i = 0; i < R.L; ++i) {
            int64_t q = (int64_t)R.m[i].q;
            int64_t r = v % q;
            if (r < 0) r += q;
            const u64 r1 = (u64)r;
            for (int k = 1; k < scale; ++k) r = (int64_t)sf_add((u64)r, r1, (u64)q);
            u64 *p = out + g * ct + ((size_t)(R.L + i) << R.log_n) + (size_t)l * stride;
            *p = sf_add(*p, (u64)r, (u64)q);
        }
    }
}

sf_status sf_add_bias(sf_ctx *ctx, u64 *out, int G, int n, int E_out, const int *d_sig_out, const int64_t *d_bq,
                      int C_out, cudaStream_t st, int scale)
{
    cudaEvent_t ev;
    sf_launch_begin(ctx, SFK_ELEMWISE, st, &ev);
    int total = G * n;
    k_add_bias<<<std::max(1, std::min((total + 255) / 256, 1024)), 256, 0, st>>>(ctx->ring, out, G, n, E_out, d_sig_out,
                                                                                 d_bq, C_out, scale);
    sf_launch_end(ctx, SFK_ELEMWISE, st, ev);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// Whole-ciphertext gather: out[k] = in[perm[k]].
__global__ void k_shuffle_cts(const u64 *in, u64 *out, const int *perm, int count, size_t ct_words)
{
    size_t total = (size_t)count * ct_words;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        size_t k = x / ct_words, w = x % ct_words;
        out[x] = in[(size_t)perm[k] * ct_words + w];
    }
}

sf_status sf_shuffle_launch(sf_ctx *ctx, const u64 *in, u64 *out, const int *d_perm, int count, cudaStream_t st)
{
    const size_t ct = (size_t)2 * ctx->ring.L * ctx->ring.n;
    cudaEvent_t ev;
    sf_launch_begin(ctx, SFK_SHUFFLE, st, &ev);
    size_t total = (size_t)count * ct;
    k_shuffle_cts<<<(int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 32), 256, 0, st>>>(in, out, d_perm, count, ct);
    sf_launch_end(ctx, SFK_SHUFFLE, st, ev);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// Extraction at gamma = 0 (Lemma 1 with t = 2): out = N^-1 X^-i ct, coefficient domain.
__global__ void k_extract(SfRing R, const u64 *ct, u64 *out, int i)
{
    const size_t total = (size_t)2 * R.L * R.n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        int limb = (int)((x >> R.log_n) % R.L);
        int k = (int)(x & (R.n - 1));
        size_t base = x - k;
        const SfMod &M = R.m[limb];
        // coefficient k of X^-i a = coefficient k + i of a, negated when k + i >= N
        int src = k + i;
        u64 v = ct[base + (src & (R.n - 1))];
        if (src >= R.n && v) v = M.q - v;
        out[x] = sf_mul_shoup(v, M.ninv, M.ninv_p, M.q);
    }
}

// Extraction at gamma = 2 (Lemma 1 at t = 2, scaled by [K_2 : K_0] = 2):
// out = (N/2)^-1 (X^-i ct + X^-3i ct3), coefficient domain.
__global__ void k_extract2(SfRing R, const u64 *ct, const u64 *ct3, u64 *out, int i)
{
    const size_t total = (size_t)2 * R.L * R.n;
    const int two_n = 2 * R.n;
    for (size_t x = blockIdx.x * (size_t)blockDim.x + threadIdx.x; x < total; x += (size_t)gridDim.x * blockDim.x) {
        int limb = (int)((x >> R.log_n) % R.L);
        int k = (int)(x & (R.n - 1));
        size_t base = x - k;
        const SfMod &M = R.m[limb];
        // coefficient k of X^-e a is a[(k + e) mod 2N] folded by X^N = -1
        auto coef = [&](const u64 *a, int e) -> u64 {
            const int src = (k + e) % two_n;
            u64 v = a[base + (src & (R.n - 1))];
            return (src >= R.n && v) ? M.q - v : v;
        };
        const u64 v = sf_add(coef(ct, i), coef(ct3, (3 * i) % two_n), M.q);
        // (N/2)^-1 = 2 N^-1
        out[x] = sf_add(sf_mul_shoup(v, M.ninv, M.ninv_p, M.q), sf_mul_shoup(v, M.ninv, M.ninv_p, M.q), M.q);
    }
}

sf_status sf_extract2_launch(sf_ctx *ctx, const u64 *ct, const u64 *ct3, u64 *out, int i, cudaStream_t st)
{
    cudaEvent_t ev;
    sf_launch_begin(ctx, SFK_ELEMWISE, st, &ev);
    size_t total = (size_t)2 * ctx->ring.L * ctx->ring.n;
    k_extract2<<<(int)((total + 255) / 256), 256, 0, st>>>(ctx->ring, ct, ct3, out, i);
    sf_launch_end(ctx, SFK_ELEMWISE, st, ev);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

sf_status sf_extract_launch(sf_ctx *ctx, const u64 *ct, u64 *out, int i, cudaStream_t st)
{
    cudaEvent_t ev;
    sf_launch_begin(ctx, SFK_ELEMWISE, st, &ev);
    size_t total = (size_t)2 * ctx->ring.L * ctx->ring.n;
    k_extract<<<(int)((total + 255) / 256), 256, 0, st>>>(ctx->ring, ct, out, i);
    sf_launch_end(ctx, SFK_ELEMWISE, st, ev);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

sf_status sf_layer_init_attributes()
{
    const int mx = 227 * 1024;
#define SF_LEAF_ATTRS(LR, LC)                                                                               \
    {                                                                                                        \
        /* the tap list is static shared memory: the dynamic part gets the rest */                          \
        cudaFuncAttributes fa;                                                                               \
        SF_CUDA_TRY(cudaFuncGetAttributes(&fa, k_leaf_col<LR, LC>));                                         \
        SF_CUDA_TRY(cudaFuncSetAttribute(k_leaf_col<LR, LC>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                         mx - (int)fa.sharedSizeBytes));                                     \
    }
    SF_LEAF_ATTRS(5, 5) SF_LEAF_ATTRS(5, 6) SF_LEAF_ATTRS(6, 6) SF_LEAF_ATTRS(6, 7) SF_LEAF_ATTRS(7, 7)
    SF_LEAF_ATTRS(7, 8) SF_LEAF_ATTRS(7, 9)
#undef SF_LEAF_ATTRS
#define SF_LEAF_ROW_ATTR(LR, LC) \
    SF_CUDA_TRY(cudaFuncSetAttribute((k_leaf_row<LR, LC>), cudaFuncAttributeMaxDynamicSharedMemorySize, mx)); \
    SF_CUDA_TRY(cudaFuncSetAttribute((k_leaf_row<LR, LC, 1>), cudaFuncAttributeMaxDynamicSharedMemorySize, mx)); \
    SF_CUDA_TRY(cudaFuncSetAttribute((k_leaf_row<LR, LC, 2>), cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_LEAF_ROW_ATTR(5, 5) SF_LEAF_ROW_ATTR(5, 6) SF_LEAF_ROW_ATTR(6, 6) SF_LEAF_ROW_ATTR(6, 7) SF_LEAF_ROW_ATTR(7, 7)
    SF_LEAF_ROW_ATTR(7, 8) SF_LEAF_ROW_ATTR(7, 9)
#undef SF_LEAF_ROW_ATTR
    return SF_OK;
}
