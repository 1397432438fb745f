// sf_ntt.cu -- batched negacyclic NTT passes over job lists, plus the
// elementwise kernels used around them (Montgomery conversion, pointwise
// products, encryption and decryption finishing, key generation).
#include "sf_internal.h"
#include "sf_kernels.cuh"

// One pass of a batched transform.  blockIdx.y selects the job, blockIdx.x
// the tile.  Forward = column pass (reads job.src) then row pass (reduces to
// [0, q)); inverse = row pass (reads job.src) then column pass (multiplies by
// N^-1 and reduces).  Later passes work in place on job.dst.
template <bool INV, bool COLS, int NT>
__global__ void __launch_bounds__(NT) k_ntt_pass(SfRing R, SfJobList jobs)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SfPolyJob jb = jobs.j[blockIdx.y];
    const SfGeo g = ring_geo(R);
    const SfMod M = R.m[jb.mod];
    const bool first = (INV != COLS);   // forward starts with columns, inverse with rows
    const u64 *src = first ? jb.src : jb.dst;
    sf_tw *tw = (sf_tw *)smem_raw;
    if (COLS) {
        u64 *s = (u64 *)(tw + g.r);
        const int c0 = blockIdx.x * SF_NB;
        load_col_tw(tw, INV ? R.colT_i : R.colT_f, g, jb.mod);
        for (int e = threadIdx.x; e < col_elems(g); e += blockDim.x) s[col_slot(e)] = src[col_gidx(g, c0, e)];
        __syncthreads();
        if (INV) col_inverse<NT>(s, tw, g.log_r, M.q);
        else col_forward<NT>(s, tw, g.log_r, M.q);
        for (int e = threadIdx.x; e < col_elems(g); e += blockDim.x) {
            u64 v = s[col_slot(e)];
            if (INV) v = sf_csub(sf_mul_shoup_lazy(v, M.ninv, M.ninv_p, M.q), M.q);
            jb.dst[col_gidx(g, c0, e)] = v;
        }
    } else {
        u64 *s = (u64 *)(tw + sf_row_nb(g.log_c) * g.c);
        const int r0 = blockIdx.x * sf_row_nb(g.log_c);
        load_row_tw(tw, INV ? R.rowT_i : R.rowT_f, g, jb.mod, r0);
        const u64 *s0 = src + (size_t)r0 * g.c;
        for (int e = threadIdx.x; e < row_elems(g); e += blockDim.x) s[row_slot(g, e)] = s0[e];
        __syncthreads();
        if (INV) row_inverse<NT>(s, tw, g.log_c, M.q);
        else row_forward<NT>(s, tw, g.log_c, M.q);
        u64 *d0 = jb.dst + (size_t)r0 * g.c;
        for (int e = threadIdx.x; e < row_elems(g); e += blockDim.x) {
            u64 v = s[row_slot(g, e)];
            if (!INV) v = sf_reduce(v, M.q, M.one_p);
            d0[e] = v;
        }
    }
}

// dynamic shared memory of the pass kernels
size_t sf_smem_col(const SfRing &R, int tiles) { return sizeof(sf_tw) * R.r + sizeof(u64) * tile_words(R.log_r) * tiles; }
size_t sf_smem_row(const SfRing &R, int tiles)
{
    return sizeof(sf_tw) * sf_row_nb(R.log_c) * R.c + sizeof(u64) * row_tile_words(R.log_c) * tiles;
}

sf_status sf_ntt_jobs(sf_ctx *ctx, const SfPolyJob *h_jobs, int n_jobs, bool inverse, cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    const size_t smem_col = sf_smem_col(R, 1), smem_row = sf_smem_row(R, 1);
    for (int off = 0; off < n_jobs; off += SF_MAX_JOBS) {
        int cnt = std::min(SF_MAX_JOBS, n_jobs - off);
        SfJobList jl;
        for (int i = 0; i < cnt; ++i) jl.j[i] = h_jobs[off + i];
        dim3 gc(R.c / SF_TC, cnt), gr(R.r / sf_row_nb(R.log_c), cnt);
        cudaEvent_t ev;
        const int ntc = sf_tile_threads(R.log_r), ntr = SF_THREADS;   // row tiles: 256 threads
        if (!inverse) {
            sf_launch_begin(ctx, SFK_NTT_FWD_COL, st, &ev);
            SF_NT_DISPATCH(ntc, k_ntt_pass<false, true, NT><<<gc, NT, smem_col, st>>>(R, jl););
            sf_launch_end(ctx, SFK_NTT_FWD_COL, st, ev);
            sf_launch_begin(ctx, SFK_NTT_FWD_ROW, st, &ev);
            SF_NT_DISPATCH(ntr, k_ntt_pass<false, false, NT><<<gr, NT, smem_row, st>>>(R, jl););
            sf_launch_end(ctx, SFK_NTT_FWD_ROW, st, ev);
        } else {
            sf_launch_begin(ctx, SFK_NTT_INV_ROW, st, &ev);
            SF_NT_DISPATCH(ntr, k_ntt_pass<true, false, NT><<<gr, NT, smem_row, st>>>(R, jl););
            sf_launch_end(ctx, SFK_NTT_INV_ROW, st, ev);
            sf_launch_begin(ctx, SFK_NTT_INV_COL, st, &ev);
            SF_NT_DISPATCH(ntc, k_ntt_pass<true, true, NT><<<gc, NT, smem_col, st>>>(R, jl););
            sf_launch_end(ctx, SFK_NTT_INV_COL, st, ev);
        }
    }
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// ----------------------------------------------------------- elementwise --
//
// Polynomial t of an elementwise launch uses modulus offset + (t % period).

#define SF_GRID_STRIDE(i, total) \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (total); i += (size_t)gridDim.x * blockDim.x)

// x -> x * 2^64 mod q (Montgomery form), in place.
__global__ void k_to_mont(SfRing R, u64 *d, int n_polys, int period, int offset)
{
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        const SfMod &M = R.m[offset + (int)((i >> R.log_n) % period)];
        d[i] = sf_mul_shoup(d[i], M.r_mod, M.r_mod_p, M.q);
    }
}

// Montgomery form -> normal form, in place (x * 2^-64 mod q).
__global__ void k_from_mont(SfRing R, u64 *d, int n_polys, int period, int offset)
{
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        const SfMod &M = R.m[offset + (int)((i >> R.log_n) % period)];
        d[i] = sf_redc(0, d[i], M.q, M.qinv_neg);
    }
}

// out = a * b mod q for NTT-domain polynomials (REDC, then times 2^64 mod q).
__global__ void k_pointwise_mul(SfRing R, const u64 *a, const u64 *b, u64 *out, int n_polys, int period, int offset)
{
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        const SfMod &M = R.m[offset + (int)((i >> R.log_n) % period)];
        u64 t = sf_redc(sf_mulhi(a[i], b[i]), a[i] * b[i], M.q, M.qinv_neg);
        out[i] = sf_mul_shoup(t, M.r_mod, M.r_mod_p, M.q);
    }
}

// out[t] = a[t] * s_mont[t % period] (s in Montgomery form), moduli 0..period-1.
__global__ void k_mul_secret(SfRing R, const u64 *a, const u64 *s_mont, u64 *out, int n_polys, int period)
{
    size_t per = (size_t)period << R.log_n;
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        size_t w = i % per;
        const SfMod &M = R.m[(int)(w >> R.log_n)];
        out[i] = sf_mul_mont(a[i], s_mont[w], M.q, M.qinv_neg);
    }
}

// b = p + m + e  (mod q_i), m and e signed; p: [n_cts][L][N]; cts: [n_cts][2][L][N].
__global__ void k_encrypt_finish(SfRing R, const u64 *p, const int64_t *m, const int64_t *e, u64 *cts, int n_cts)
{
    size_t per = (size_t)R.L * R.n;
    SF_GRID_STRIDE(i, per * n_cts)
    {
        size_t ct = i / per, w = i % per;
        int limb = (int)(w >> R.log_n);
        int k = (int)(w & (R.n - 1));
        int64_t q = (int64_t)R.m[limb].q;
        int64_t r = (m[ct * R.n + k] % q + e[ct * R.n + k] % q) % q;
        if (r < 0) r += q;
        cts[ct * 2 * per + per + w] = sf_add(p[i], (u64)r, (u64)q);
    }
}

// out = b - p (mod q_i) for a batch of ciphertexts (decryption).
__global__ void k_decrypt_finish(SfRing R, const u64 *cts, const u64 *p, u64 *out, int n_cts)
{
    size_t per = (size_t)R.L * R.n;
    SF_GRID_STRIDE(i, per * n_cts)
    {
        size_t ct = i / per, w = i % per;
        int limb = (int)(w >> R.log_n);
        out[i] = sf_sub(cts[ct * 2 * per + per + w], p[i], R.m[limb].q);
    }
}

// Signed integer polynomials -> residues: out poly t = v[t / period] mod q_{offset + t % period}.
__global__ void k_signed_to_residues(SfRing R, const int64_t *v, u64 *out, int n_polys, int period, int offset)
{
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        size_t t = i >> R.log_n;
        int k = (int)(i & (R.n - 1));
        int64_t q = (int64_t)R.m[offset + (int)(t % period)].q;
        int64_t x = v[(t / period) * R.n + k] % q;
        out[i] = (u64)(x < 0 ? x + q : x);
    }
}

// Rotation key, NTT domain, for one digit over all nm moduli:
//   a = alpha^,  b = alpha^ s + e^ - [P g_j]_m s^(tau_d),  both to Montgomery form.
// alpha, e: [nm][N] NTT domain, canonical; s_mont: [nm][N]; pg[m] = [P g_j]_m.
struct SfPg {
    u64 v[SF_MAX_MODULI];
};
__global__ void k_rotkey_finish(SfRing R, const u64 *alpha, const u64 *e, const u64 *s_mont, SfPg pg, int d,
                                u64 *key_a, u64 *key_b, size_t comp)
{
    SF_GRID_STRIDE(i, (size_t)R.nm * R.n)
    {
        int m = (int)(i >> R.log_n);
        int j = (int)(i & (R.n - 1));
        const SfMod &M = R.m[m];
        u64 as = sf_mul_mont(alpha[i], s_mont[i], M.q, M.qinv_neg);
        int js = auto_src(j, d, R.log_n);
        u64 sd = sf_mul_mont(pg.v[m], s_mont[((size_t)m << R.log_n) + js], M.q, M.qinv_neg);
        u64 b = sf_sub(sf_add(as, e[i], M.q), sd, M.q);
        u64 a = alpha[i];
        // The data limbs are stored times P^-1 mod q_m: the inner product
        // then yields ACC_Q P^-1, the term ModDown needs, with no product of
        // its own (sf_rotkeys_export multiplies the factor back out).
        if (m < R.L) {
            a = sf_mul_shoup(a, R.md_pinv[m], R.md_pinv_p[m], M.q);
            b = sf_mul_shoup(b, R.md_pinv[m], R.md_pinv_p[m], M.q);
        }
        // plain values, then their Shoup companions `comp` words later
        key_a[i] = a;
        key_b[i] = b;
        key_a[i + comp] = sf_shoup_companion_dev(a, M);
        key_b[i + comp] = sf_shoup_companion_dev(b, M);
    }
}

// grid-stride launches: at most 16 resident 256-thread blocks per SM
static int grid_for(const sf_ctx *ctx, size_t total)
{
    return (int)std::min<size_t>((total + 255) / 256, (size_t)ctx->num_sms * 16);
}

#define SF_ELEM_LAUNCH(kernel, total, ...)                                           \
    do {                                                                             \
        cudaEvent_t ev__;                                                            \
        sf_launch_begin(ctx, SFK_ELEMWISE, st, &ev__);                               \
        kernel<<<grid_for(ctx, total), 256, 0, st>>>(ctx->ring, __VA_ARGS__);             \
        sf_launch_end(ctx, SFK_ELEMWISE, st, ev__);                                  \
        SF_CUDA_TRY(cudaGetLastError());                                             \
    } while (0)

sf_status sf_to_mont(sf_ctx *ctx, u64 *d, int n_polys, int period, int offset, cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_to_mont, (size_t)n_polys * ctx->ring.n, d, n_polys, period, offset);
    return SF_OK;
}

sf_status sf_from_mont(sf_ctx *ctx, u64 *d, int n_polys, int period, int offset, cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_from_mont, (size_t)n_polys * ctx->ring.n, d, n_polys, period, offset);
    return SF_OK;
}

sf_status sf_pointwise_mul(sf_ctx *ctx, const u64 *a, const u64 *b, u64 *out, int n_polys, int period, int offset,
                           cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_pointwise_mul, (size_t)n_polys * ctx->ring.n, a, b, out, n_polys, period, offset);
    return SF_OK;
}

sf_status sf_mul_secret(sf_ctx *ctx, const u64 *a, const u64 *s_mont, u64 *out, int n_polys, int period, cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_mul_secret, (size_t)n_polys * ctx->ring.n, a, s_mont, out, n_polys, period);
    return SF_OK;
}

sf_status sf_encrypt_finish(sf_ctx *ctx, const u64 *p, const int64_t *m, const int64_t *e, u64 *cts, int n_cts,
                            cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_encrypt_finish, (size_t)n_cts * ctx->ring.L * ctx->ring.n, p, m, e, cts, n_cts);
    return SF_OK;
}

sf_status sf_decrypt_finish(sf_ctx *ctx, const u64 *cts, const u64 *p, u64 *out, int n_cts, cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_decrypt_finish, (size_t)n_cts * ctx->ring.L * ctx->ring.n, cts, p, out, n_cts);
    return SF_OK;
}

sf_status sf_signed_to_residues(sf_ctx *ctx, const int64_t *v, u64 *out, int n_polys, int period, int offset,
                                cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_signed_to_residues, (size_t)n_polys * ctx->ring.n, v, out, n_polys, period, offset);
    return SF_OK;
}

sf_status sf_rotkey_finish(sf_ctx *ctx, const u64 *alpha, const u64 *e, const u64 *s_mont, const u64 *pg, int d,
                           u64 *key_a, u64 *key_b, size_t comp, cudaStream_t st)
{
    SfPg p;
    for (int m = 0; m < SF_MAX_MODULI; ++m) p.v[m] = m < ctx->ring.nm ? pg[m] : 0;
    SF_ELEM_LAUNCH(k_rotkey_finish, (size_t)ctx->ring.nm * ctx->ring.n, alpha, e, s_mont, p, d, key_a, key_b, comp);
    return SF_OK;
}

// Shoup companions of NTT-domain residues, in place into dst: dst[i] = floor(x[i] 2^64 / q)
__global__ void k_shoup_companions(SfRing R, const u64 *x, u64 *dst, int n_polys, int period, int offset)
{
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        const SfMod &M = R.m[offset + (int)((i >> R.log_n) % period)];
        dst[i] = sf_shoup_companion_dev(x[i], M);
    }
}

// Latches SF_ERANGE in the device status word when a residue of the caller's
// input is not below its modulus (the words are read, never written).
__global__ void k_check_residues(SfRing R, const u64 *x, int n_polys, int period, int offset)
{
    bool bad = false;
    SF_GRID_STRIDE(i, (size_t)n_polys * R.n)
    {
        bad |= x[i] >= R.m[offset + (int)((i >> R.log_n) % period)].q;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0 && R.status) atomicCAS(R.status, 0, SF_ERANGE);
}

sf_status sf_check_residues(sf_ctx *ctx, const u64 *x, int n_polys, int period, int offset, cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_check_residues, (size_t)n_polys * ctx->ring.n, x, n_polys, period, offset);
    return SF_OK;
}

sf_status sf_companions(sf_ctx *ctx, const u64 *x, u64 *dst, int n_polys, int period, int offset, cudaStream_t st)
{
    SF_ELEM_LAUNCH(k_shoup_companions, (size_t)n_polys * ctx->ring.n, x, dst, n_polys, period, offset);
    return SF_OK;
}

sf_status sf_ntt_init_attributes()
{
    const int mx = 227 * 1024;
#define SF_NTT_ATTR(NT)                                                                                             \
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ntt_pass<false, true, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));  \
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ntt_pass<false, false, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx)); \
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ntt_pass<true, true, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));   \
    SF_CUDA_TRY(cudaFuncSetAttribute(k_ntt_pass<true, false, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    SF_NTT_ATTR(256)
    SF_NTT_ATTR(512)
#undef SF_NTT_ATTR
    return SF_OK;
}
