// sf_ks.cu -- automorphism + hybrid key switching for batches of "merges".
//
// A merge (Sec. 2.4 packing step, Sec. 2.2 key switching) takes E, O (NTT
// domain, [2][L][N]), a shift s and an automorphism index d:
//     u = E - X^s O,  v = E + X^s O
//     (A', B') = KS(tau_d(u.a))        (hybrid: ModUp, <., ksk_d>, ModDown)
//     out = (v.a + A',  v.b + tau_d(u.b) + B')          [add_v = 1]
//     out = (A',        tau_d(u.b) + B')                [add_v = 0: plain rotate]
// Without O, u = v = E (the trace step ct + tau_d(ct), or a rotation).
//
// Five kernels per batch of merges that share d (and so the key), with the
// NTT split into a row pass and a column pass (see sf_tile.cuh):
//   K1 rows : gather tau_d(u.a) (a permutation of NTT slots) -> TA, inverse row pass
//   K2 cols : inverse column pass, times N^-1 -> coefficients; ModUp of each
//             digit to the other moduli (fast base conversion); forward column pass
//   K3 rows : forward row pass of each digit's extension, inner product with
//             the key over all digits (128-bit accumulation, one Montgomery
//             reduction); P-limbs continue with the inverse row pass
//   K4 cols : inverse column pass of the P-limbs, times N^-1 -> coefficients;
//             base conversion P -> each q_i; forward column pass
//   K5 rows : forward row pass; (acc_Q - conv) * P^-1; add v and tau_d(u.b); store
#include "sf_internal.h"
#include "sf_kernels.cuh"
#include "sf_ks.h"

// scratch words per merge: TA[L] | X1/ACC_P[max(L, 2K)] | X2/X3[dnum*nm] | ACC_Q[2L]
size_t sf_ks_scratch_words(const SfRing &R)
{
    int x1 = R.L > 2 * R.K ? R.L : 2 * R.K;
    int x2 = R.dnum * R.nm > 2 * R.L ? R.dnum * R.nm : 2 * R.L;
    return (size_t)(R.L + x1 + x2 + 2 * R.L) << R.log_n;
}

struct KsLayout {
    u64 *ta, *x1, *x2, *accq;
};

__device__ __forceinline__ KsLayout ks_layout(const SfRing &R, const SfKsBatch &B, int b)
{
    int x1 = R.L > 2 * R.K ? R.L : 2 * R.K;
    int x2 = R.dnum * R.nm > 2 * R.L ? R.dnum * R.nm : 2 * R.L;
    size_t per = (size_t)(R.L + x1 + x2 + 2 * R.L) << R.log_n;
    u64 *base = B.scratch + per * b;
    KsLayout Lo;
    Lo.ta = base;
    Lo.x1 = base + ((size_t)R.L << R.log_n);
    Lo.x2 = Lo.x1 + ((size_t)x1 << R.log_n);
    Lo.accq = Lo.x2 + ((size_t)x2 << R.log_n);
    return Lo;
}

__device__ __forceinline__ void merge_gt(const SfKsBatch &B, int b, int &g, int &t)
{
    int x = B.first + b;
    g = x / B.inner;
    t = x - g * B.inner;
}
__device__ __forceinline__ const u64 *merge_E(const SfKsBatch &B, int b)
{
    int g, t;
    merge_gt(B, b, g, t);
    return B.E + B.E_outer * g + B.E_stride * t;
}
__device__ __forceinline__ const u64 *merge_O(const SfKsBatch &B, int b)
{
    if (!B.O) return nullptr;
    int g, t;
    merge_gt(B, b, g, t);
    return B.O + B.O_outer * g + B.O_stride * t;
}
__device__ __forceinline__ u64 *merge_out(const SfKsBatch &B, int b)
{
    int g, t;
    merge_gt(B, b, g, t);
    return B.out + B.out_outer * g + B.out_stride * t;
}

// u at NTT slot js of limb i, part p: E - psi^(s e) O  (canonical)
__device__ __forceinline__ u64 merge_u(const SfRing &R, const SfKsBatch &B, const u64 *E, const u64 *O, int p, int i,
                                       int js)
{
    size_t off = (((size_t)p * R.L + i) << R.log_n) + js;
    u64 e = E[off];
    if (!O) return e;
    const SfMod &M = R.m[i];
    unsigned k = mono_index(js, B.s, R.log_n);
    size_t pk = ((size_t)i << (R.log_n + 1)) + k;
    u64 xo = sf_mul_shoup(O[off], R.pw[pk], R.pw_p[pk], M.q);
    return sf_sub(e, xo, M.q);
}

__device__ __forceinline__ u64 merge_v(const SfRing &R, const SfKsBatch &B, const u64 *E, const u64 *O, int p, int i,
                                       int j)
{
    size_t off = (((size_t)p * R.L + i) << R.log_n) + j;
    u64 e = E[off];
    if (!O) return e;
    const SfMod &M = R.m[i];
    unsigned k = mono_index(j, B.s, R.log_n);
    size_t pk = ((size_t)i << (R.log_n + 1)) + k;
    u64 xo = sf_mul_shoup(O[off], R.pw[pk], R.pw_p[pk], M.q);
    return sf_add(e, xo, M.q);
}

// K1: grid (R/16 row tiles, L limbs, merges).  smem: inverse row twiddles + 1 tile.
__global__ void __launch_bounds__(SF_THREADS) k_ks1(SfRing R, SfKsBatch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SfGeo g = ring_geo(R);
    const int r0 = blockIdx.x * SF_NB, i = blockIdx.y, b = blockIdx.z;
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *s = (u64 *)(tw + SF_NB * g.c);
    const u64 *E = merge_E(B, b), *O = merge_O(B, b);
    KsLayout Lo = ks_layout(R, B, b);
    const int ne = row_elems(g);
    const size_t gbase = ((size_t)i << R.log_n) + (size_t)r0 * g.c;
    load_row_tw(tw, R.rowT_i, g, i, r0);
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const int j = r0 * g.c + e;
        const u64 u = merge_u(R, B, E, O, 0, i, auto_src(j, B.d, R.log_n));
        s[row_slot(g, e)] = u;
        Lo.ta[gbase + e] = u;
    }
    __syncthreads();
    row_inverse(s, tw, g.log_c, R.m[i].q);
    for (int e = threadIdx.x; e < ne; e += blockDim.x) Lo.x1[gbase + e] = s[row_slot(g, e)];
}

// K2: grid (C/16 column tiles, dnum digits, merges).
// smem: column twiddles + K source tiles + 1 work tile.
__global__ void __launch_bounds__(SF_THREADS) k_ks2(SfRing R, SfKsBatch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SfGeo g = ring_geo(R);
    const int c0 = blockIdx.x * SF_NB, j = blockIdx.y, b = blockIdx.z;
    KsLayout Lo = ks_layout(R, B, b);
    const int ne = col_elems(g), tw_words = tile_words(g.log_r);
    const int lo = j * R.K, hi = min((j + 1) * R.K, R.L), nd = hi - lo;
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *src_t = (u64 *)(tw + g.r);
    u64 *work = src_t + (size_t)nd * tw_words;
    // inverse column pass of the digit's limbs, then y_i = x_i N^-1 Qhat_i^-1 mod q_i
    for (int t = 0; t < nd; ++t) {
        const int i = lo + t;
        u64 *st = src_t + (size_t)t * tw_words;
        const u64 *src = Lo.x1 + ((size_t)i << R.log_n);
        load_col_tw(tw, R.colT_i, g, i);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) st[col_slot(e)] = src[col_gidx(g, c0, e)];
        __syncthreads();
        col_inverse(st, tw, g.log_r, R.m[i].q);
        const u64 w = R.mu_inv[j * R.K + t], wp = R.mu_inv_p[j * R.K + t];
        for (int e = threadIdx.x; e < ne; e += blockDim.x) st[col_slot(e)] = sf_mul_shoup(st[col_slot(e)], w, wp, R.m[i].q);
        __syncthreads();
    }
    // ModUp to every modulus outside the digit, then the forward column pass
    for (int m = 0; m < R.nm; ++m) {
        if (m >= lo && m < hi) continue;
        const SfMod &M = R.m[m];
        load_col_tw(tw, R.colT_f, g, m);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int sl = col_slot(e);
            u64 acc = 0;
            for (int t = 0; t < nd; ++t) {
                const size_t ci = ((size_t)(j * R.K + t)) * R.nm + m;
                acc = sf_add(acc, sf_mul_shoup(src_t[(size_t)t * tw_words + sl], R.mu_qhat[ci], R.mu_qhat_p[ci], M.q), M.q);
            }
            work[sl] = acc;
        }
        __syncthreads();
        col_forward(work, tw, g.log_r, M.q);
        u64 *dst = Lo.x2 + ((size_t)(j * R.nm + m) << R.log_n);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) dst[col_gidx(g, c0, e)] = work[col_slot(e)];
        __syncthreads();
    }
}

// K3: grid (R/16 row tiles, nm moduli, merges).  EPT = tile elements per thread.
// smem: row twiddles (forward, then inverse for special moduli) + 1 tile.
template <int EPT>
__global__ void __launch_bounds__(SF_THREADS, EPT >= 16 ? 1 : 3) k_ks3(SfRing R, SfKsBatch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SfGeo g = ring_geo(R);
    const int r0 = blockIdx.x * SF_NB, m = blockIdx.y, b = blockIdx.z;
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *s = (u64 *)(tw + SF_NB * g.c);
    KsLayout Lo = ks_layout(R, B, b);
    const int ne = row_elems(g);
    const SfMod M = R.m[m];
    const size_t tile_off = (size_t)r0 * g.c;
    load_row_tw(tw, R.rowT_f, g, m, r0);
    // per digit c * key (c < 36q lazy, key < q) is Montgomery-reduced into
    // [0, 2q) and summed: the sums stay below 2 q dnum < 2^55
    u64 acc_a[EPT], acc_b[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) acc_a[k] = acc_b[k] = 0;
    for (int j = 0; j < R.dnum; ++j) {
        const int lo = j * R.K, hi = min((j + 1) * R.K, R.L);
        const bool own = (m >= lo && m < hi);
        const u64 *src = (own ? Lo.ta + ((size_t)m << R.log_n) : Lo.x2 + ((size_t)(j * R.nm + m) << R.log_n)) + tile_off;
        for (int e = threadIdx.x; e < ne; e += blockDim.x) s[row_slot(g, e)] = src[e];
        __syncthreads();
        if (!own) row_forward(s, tw, g.log_c, M.q);
        const u64 *ka = B.key + ((((size_t)j * 2 + 0) * R.nm + m) << R.log_n) + tile_off;
        const u64 *kb = B.key + ((((size_t)j * 2 + 1) * R.nm + m) << R.log_n) + tile_off;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = threadIdx.x + k * SF_THREADS;
            const u64 c = s[row_slot(g, e)];
            const u64 xa = __ldg(ka + e), xb = __ldg(kb + e);
            acc_a[k] += sf_redc_lazy(sf_mulhi(c, xa), c * xa, M.q, M.qinv_neg);
            acc_b[k] += sf_redc_lazy(sf_mulhi(c, xb), c * xb, M.q, M.qinv_neg);
        }
        __syncthreads();
    }
    if (m < R.L) {
        u64 *da = Lo.accq + ((size_t)m << R.log_n) + tile_off;
        u64 *db = Lo.accq + ((size_t)(R.L + m) << R.log_n) + tile_off;
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int e = threadIdx.x + k * SF_THREADS;
            da[e] = sf_reduce(acc_a[k], M.q, M.one_p);
            db[e] = sf_reduce(acc_b[k], M.q, M.one_p);
        }
    } else {
        // special prime: inverse row pass of both parts, into ACC_P (x1 region)
        const int kk = m - R.L;
        load_row_tw(tw, R.rowT_i, g, m, r0);
        for (int p = 0; p < 2; ++p) {
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                const int e = threadIdx.x + k * SF_THREADS;
                s[row_slot(g, e)] = sf_reduce(p == 0 ? acc_a[k] : acc_b[k], M.q, M.one_p);
            }
            __syncthreads();
            row_inverse(s, tw, g.log_c, M.q);
            u64 *dst = Lo.x1 + ((size_t)(p * R.K + kk) << R.log_n) + tile_off;
            for (int e = threadIdx.x; e < ne; e += blockDim.x) dst[e] = s[row_slot(g, e)];
            __syncthreads();
        }
    }
}

// K4: grid (C/16 column tiles, 2 parts, merges).
// smem: column twiddles + K source tiles + 1 work tile.
__global__ void __launch_bounds__(SF_THREADS) k_ks4(SfRing R, SfKsBatch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SfGeo g = ring_geo(R);
    const int c0 = blockIdx.x * SF_NB, p = blockIdx.y, b = blockIdx.z;
    KsLayout Lo = ks_layout(R, B, b);
    const int ne = col_elems(g), tw_words = tile_words(g.log_r);
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *src_t = (u64 *)(tw + g.r);
    u64 *work = src_t + (size_t)R.K * tw_words;
    for (int k = 0; k < R.K; ++k) {
        const int m = R.L + k;
        u64 *st = src_t + (size_t)k * tw_words;
        const u64 *src = Lo.x1 + ((size_t)(p * R.K + k) << R.log_n);
        load_col_tw(tw, R.colT_i, g, m);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) st[col_slot(e)] = src[col_gidx(g, c0, e)];
        __syncthreads();
        col_inverse(st, tw, g.log_r, R.m[m].q);
        const u64 w = R.md_inv[k], wp = R.md_inv_p[k];
        for (int e = threadIdx.x; e < ne; e += blockDim.x) st[col_slot(e)] = sf_mul_shoup(st[col_slot(e)], w, wp, R.m[m].q);
        __syncthreads();
    }
    for (int i = 0; i < R.L; ++i) {
        const SfMod &M = R.m[i];
        load_col_tw(tw, R.colT_f, g, i);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            const int sl = col_slot(e);
            u64 acc = 0;
            for (int k = 0; k < R.K; ++k) {
                const size_t ci = (size_t)k * R.L + i;
                acc = sf_add(acc, sf_mul_shoup(src_t[(size_t)k * tw_words + sl], R.md_phat[ci], R.md_phat_p[ci], M.q), M.q);
            }
            work[sl] = acc;
        }
        __syncthreads();
        col_forward(work, tw, g.log_r, M.q);
        u64 *dst = Lo.x2 + ((size_t)(p * R.L + i) << R.log_n);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) dst[col_gidx(g, c0, e)] = work[col_slot(e)];
        __syncthreads();
    }
}

// K5: grid (R/16 row tiles, L limbs, 2 * merges).  smem: forward row twiddles + 1 tile.
__global__ void __launch_bounds__(SF_THREADS) k_ks5(SfRing R, SfKsBatch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SfGeo g = ring_geo(R);
    const int r0 = blockIdx.x * SF_NB, i = blockIdx.y, p = blockIdx.z & 1, b = blockIdx.z >> 1;
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *s = (u64 *)(tw + SF_NB * g.c);
    KsLayout Lo = ks_layout(R, B, b);
    const u64 *E = merge_E(B, b), *O = merge_O(B, b);
    u64 *out = merge_out(B, b);
    const int ne = row_elems(g);
    const SfMod M = R.m[i];
    const size_t tile_off = (size_t)r0 * g.c;
    const u64 *src = Lo.x2 + ((size_t)(p * R.L + i) << R.log_n) + tile_off;
    load_row_tw(tw, R.rowT_f, g, i, r0);
    for (int e = threadIdx.x; e < ne; e += blockDim.x) s[row_slot(g, e)] = src[e];
    __syncthreads();
    row_forward(s, tw, g.log_c, M.q);
    const u64 *acc = Lo.accq + ((size_t)(p * R.L + i) << R.log_n) + tile_off;
    u64 *dst = out + (((size_t)p * R.L + i) << R.log_n) + tile_off;
    const u64 pinv = R.md_pinv[i], pinv_p = R.md_pinv_p[i];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const u64 conv = sf_reduce(s[row_slot(g, e)], M.q, M.one_p);
        u64 res = sf_mul_shoup(sf_sub(acc[e], conv, M.q), pinv, pinv_p, M.q);
        const int j = r0 * g.c + e;
        if (B.add_v) res = sf_add(res, merge_v(R, B, E, O, p, i, j), M.q);
        if (p == 1) res = sf_add(res, merge_u(R, B, E, O, 1, i, auto_src(j, B.d, R.log_n)), M.q);
        dst[e] = res;
    }
}

sf_status sf_ks_launch(sf_ctx *ctx, const SfKsBatch &B, cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    if (B.count <= 0) return SF_OK;
    const int maxd = std::min(R.K, R.L);
    const size_t smem1 = sf_smem_row(R, 1), smem2 = sf_smem_col(R, maxd + 1), smem3 = sf_smem_row(R, 1),
                 smem4 = sf_smem_col(R, R.K + 1), smem5 = sf_smem_row(R, 1);
    cudaEvent_t ev;
    for (int off = 0; off < B.count; off += 16384) {
        SfKsBatch b = B;
        b.count = std::min(16384, B.count - off);
        b.first = B.first + off;
        b.scratch += sf_ks_scratch_words(R) * off;

        sf_launch_begin(ctx, SFK_KS1_GATHER_INV_ROW, st, &ev);
        k_ks1<<<dim3(R.r / SF_NB, R.L, b.count), SF_THREADS, smem1, st>>>(R, b);
        sf_launch_end(ctx, SFK_KS1_GATHER_INV_ROW, st, ev);

        sf_launch_begin(ctx, SFK_KS2_MODUP_COL, st, &ev);
        k_ks2<<<dim3(R.c / SF_NB, R.dnum, b.count), SF_THREADS, smem2, st>>>(R, b);
        sf_launch_end(ctx, SFK_KS2_MODUP_COL, st, ev);

        sf_launch_begin(ctx, SFK_KS3_INNER_ROW, st, &ev);
        int ept = (R.c * SF_NB) / SF_THREADS;
        dim3 g3(R.r / SF_NB, R.nm, b.count);
        switch (ept) {
        case 2: k_ks3<2><<<g3, SF_THREADS, smem3, st>>>(R, b); break;
        case 4: k_ks3<4><<<g3, SF_THREADS, smem3, st>>>(R, b); break;
        case 8: k_ks3<8><<<g3, SF_THREADS, smem3, st>>>(R, b); break;
        case 16: k_ks3<16><<<g3, SF_THREADS, smem3, st>>>(R, b); break;
        default: return sf_set_error(SF_EINVAL, "unsupported ring split");
        }
        sf_launch_end(ctx, SFK_KS3_INNER_ROW, st, ev);

        sf_launch_begin(ctx, SFK_KS4_MODDOWN_COL, st, &ev);
        k_ks4<<<dim3(R.c / SF_NB, 2, b.count), SF_THREADS, smem4, st>>>(R, b);
        sf_launch_end(ctx, SFK_KS4_MODDOWN_COL, st, ev);

        sf_launch_begin(ctx, SFK_KS5_FINISH_ROW, st, &ev);
        k_ks5<<<dim3(R.r / SF_NB, R.L, 2 * b.count), SF_THREADS, smem5, st>>>(R, b);
        sf_launch_end(ctx, SFK_KS5_FINISH_ROW, st, ev);
    }
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// Runs `count` merges sharing (d, s, add_v, key) in launch batches.
sf_status sf_ks_run(sf_ctx *ctx, SfKsBatch B, u64 *scratch, int batch, cudaStream_t st)
{
    batch = std::max(1, batch);
    const int total = B.count;
    for (int off = 0; off < total; off += batch) {
        SfKsBatch b = B;
        b.count = std::min(batch, total - off);
        b.first = B.first + off;
        b.scratch = scratch;
        SF_TRY(sf_ks_launch(ctx, b, st));
    }
    return SF_OK;
}

// Opt every kernel of this unit into the full shared-memory carve-out (large
// rings need more than the default 48 KB for K2/K4 tiles).
sf_status sf_ks_init_attributes()
{
    const int mx = 227 * 1024;
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks1, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks2, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks3<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks3<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks3<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks3<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks4, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ks5, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    return SF_OK;
}
