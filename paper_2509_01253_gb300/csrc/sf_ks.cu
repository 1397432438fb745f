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
// Kernels per batch of merges that share d (and so the key), with the NTT
// split into a row pass and a column pass (see sf_tile.cuh):
//   gather  : TA = tau_d(u.a) (a permutation of NTT slots); out = v, plus tau_d(u.b) on b
//   K1 rows : inverse row pass of TA
//   K2 cols : inverse column pass, times N^-1 -> coefficients; ModUp of each
//             digit to the other moduli (fast base conversion); forward column pass
//   K3 rows : forward row pass of each digit's extension, inner product with
//             the key over all digits (Shoup products with the key's stored
//             companions, lazy sums, one reduction; the key's data limbs
//             carry the ModDown factor P^-1); the P-limbs' inverse row pass
//             follows in a second row kernel
//   K4 cols : inverse column pass of the P-limbs, times N^-1 -> coefficients;
//             base conversion P -> each q_i (constants Phat_k P^-1 mod q_i);
//             forward column pass
//   K5 rows : forward row pass; out += acc_Q P^-1 - conv P^-1
#include "sf_async.cuh"
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

__device__ __forceinline__ size_t sf_ks_scratch_words_dev(const SfRing &R)
{
    const int x1 = R.L > 2 * R.K ? R.L : 2 * R.K;
    const int x2 = R.dnum * R.nm > 2 * R.L ? R.dnum * R.nm : 2 * R.L;
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

// ---------------------------------------------------------------------------
// Persistent transform kernels.  Work units are (group, item) pairs: a group is
// a tile position and a modulus or digit, an item a merge of the launch batch.
// One resident wave of blocks splits the units group-major into equal ranges
// (sf_block_units); a block stages a group's twiddles when its range enters
// the group and prefetches the next unit's tiles with cp.async while it
// transforms the current one.
// ---------------------------------------------------------------------------


// Elementwise, one pass over E and O per merge (a slot permutation and
// monomial products in the NTT domain):
//   TA[b][i][j] = tau_d(u.a)[j],  u = E - X^s O
//   out.a[j]    = v.a[j]                      (0 for a plain rotation)
//   out.b[j]    = v.b[j] + tau_d(u.b)[j],     v = E + X^s O
// The ModDown finish (k_ks5) then adds the key-switch result into out.
// grid (N / (256 SF_EW), L, merges): each thread does SF_EW slots, so the
// per-merge pointers are set up once per thread.
#define SF_EW 8
__global__ void __launch_bounds__(256) k_ks_gather(SfRing R, SfKsBatch B)
{
    const int b = blockIdx.z, i = blockIdx.y;
    const u64 *E = merge_E(B, b), *O = merge_O(B, b);
    u64 *ta = ks_layout(R, B, b).ta + ((size_t)i << R.log_n);
    u64 *out = merge_out(B, b);
    u64 *oa = out + ((size_t)i << R.log_n), *ob = out + ((size_t)(R.L + i) << R.log_n);
    const u64 q = R.m[i].q;
    const int j0 = blockIdx.x * (256 * SF_EW) + threadIdx.x;
    const SfMod &M = R.m[i];
    const size_t ea = (size_t)i << R.log_n, eb = (size_t)(R.L + i) << R.log_n;
    const size_t pb = (size_t)i << (R.log_n + 1);
#pragma unroll
    for (int x = 0; x < SF_EW; ++x) {
        const int j = j0 + x * 256;
        if (j >= R.n) break;   // rings smaller than one block's 256 SF_EW slots
        const int src = auto_src(j, B.d, R.log_n);
        // every load before any store (the stores could alias nothing, but the
        // compiler cannot know): 4 coalesced, 4 gathered, 2 monomial pairs
        u64 Eaj = E[ea + j], Ebj = E[eb + j], Eas = E[ea + src], Ebs = E[eb + src];
        if (O) {
            const unsigned kj = mono_index(j, B.s, R.log_n), ks = mono_index(src, B.s, R.log_n);
            const u64 wj = R.pw[pb + kj], wjp = R.pw_p[pb + kj], ws = R.pw[pb + ks], wsp = R.pw_p[pb + ks];
            const u64 Oaj = O[ea + j], Obj = O[eb + j], Oas = O[ea + src], Obs = O[eb + src];
            const u64 xaj = sf_mul_shoup(Oaj, wj, wjp, M.q), xbj = sf_mul_shoup(Obj, wj, wjp, M.q);
            const u64 xas = sf_mul_shoup(Oas, ws, wsp, M.q), xbs = sf_mul_shoup(Obs, ws, wsp, M.q);
            ta[j] = sf_sub(Eas, xas, M.q);
            const u64 ub = sf_sub(Ebs, xbs, M.q);
            oa[j] = B.add_v ? sf_add(Eaj, xaj, M.q) : 0;
            ob[j] = B.add_v ? sf_add(sf_add(Ebj, xbj, M.q), ub, q) : ub;
        } else {
            ta[j] = Eas;
            oa[j] = B.add_v ? Eaj : 0;
            ob[j] = B.add_v ? sf_add(Ebj, Ebs, q) : Ebs;
        }
    }
}

// Generic row pass over a per-merge set of npoly polynomials in the scratch:
// poly t reads scratch + src_off + t N, writes scratch + dst_off + t N, with
// modulus mod_base + t % mod_period.  Groups: (row tile, t); items: merges.
struct SfRowSet {
    size_t src_off, dst_off;
    int npoly, mod_base, mod_period;
};

template <bool INV, int LR, int LC, int RAD = 0>
__global__ void __launch_bounds__(SfRow<LC>::NT, 3) k_rows(SfRing R, SfKsBatch B, SfRowSet S, int ng)
{
    constexpr int NT = SfRow<LC>::NT, NB = SfRow<LC>::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const size_t per = sf_ks_scratch_words_dev(R);
    const SfUnits U = sf_block_units(ng * B.count);
    constexpr bool DB = sf_rows_double_buffered(LC);
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *buf0 = (u64 *)(tw + NB * g.c);
    u64 *buf1 = DB ? buf0 + SfRow<LC>::WORDS : buf0;
    // unit u: group u / count = (row tile, poly t), item u % count = merge
    auto unit_off = [&](int u, size_t base) -> size_t {
        const int grp = u / B.count, t = grp % S.npoly, r0 = (grp / S.npoly) * NB;
        return per * (u % B.count) + base + ((size_t)t << (LR + LC)) + (size_t)r0 * g.c;
    };
    if (DB && U.u0 < U.u1) issue_row_tile_t<LC, NT>(buf0, B.scratch + unit_off(U.u0, S.src_off));
    sf_cp_commit();
    int staged = -1;
    u64 q = 0;
    for (int k = 0, u = U.u0; u < U.u1; ++k, ++u) {
        const int grp = u / B.count;
        if (grp != staged) {
            // the previous unit ended at a barrier: nothing reads tw now
            const int mod = S.mod_base + (grp % S.npoly) % S.mod_period;
            load_row_tw_t<LR, LC, NT>(tw, INV ? R.rowT_i : R.rowT_f, mod, (grp / S.npoly) * NB);
            q = R.m[mod].q;
            staged = grp;
        }
        u64 *cur = (k & 1) ? buf1 : buf0, *nxt = (k & 1) ? buf0 : buf1;
        if (DB) {
            if (u + 1 < U.u1) issue_row_tile_t<LC, NT>(nxt, B.scratch + unit_off(u + 1, S.src_off));
            sf_cp_commit();
            sf_cp_wait<1>();
        } else {
            issue_row_tile_t<LC, NT>(cur, B.scratch + unit_off(u, S.src_off));
            sf_cp_commit();
            sf_cp_wait<0>();
        }
        __syncthreads();
        u64 *dst = B.scratch + unit_off(u, S.dst_off);
        if (INV) {
            row_inverse_out<LC, NT, RAD>(cur, tw, q, [&](int kk, int bb, u64 v) { dst[(bb << LC) + kk] = v; });
        } else {
            row_forward_t<LC, NT, RAD>(cur, tw, q);
            #pragma unroll
            for (int e = threadIdx.x; e < SfRow<LC>::ELEMS; e += NT) dst[e] = cur[row_slot_t<LC>(e)];
        }
        __syncthreads();
    }
}

// ModUp.  Groups: (column tile, digit j); items: merges.  smem: inverse and
// the inverse column tables of the digit's limbs and the forward tables of the
// other moduli (nm tables in all), the nd source tiles (two buffers when db),
// one work tile.
template <int LR, int LC>
__global__ void __launch_bounds__(SfThreads<LR>::value, SfThreads<LR>::value >= 512 ? 1 : 3)
    k_ks2(SfRing R, SfKsBatch B, int ng, int db)
{
    constexpr int NT = SfThreads<LR>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const int maxd = min(R.K, R.L);
    const int tw_words = tile_words(g.log_r);
    const SfUnits U = sf_block_units(ng * B.count);
    sf_tw *twi = (sf_tw *)smem_raw;                 // [nd][R] inverse, the digit's limbs
    sf_tw *twf = twi;                               // [nm - nd][R] forward, slot m (m < lo) or m - nd (m >= hi)
    u64 *bufs = (u64 *)(twi + (size_t)R.nm * g.r);  // (db ? 2 : 1) x maxd tiles
    u64 *work = bufs + (size_t)(db ? 2 : 1) * maxd * tw_words;
    // unit u: group u / count = (column tile, digit j), item u % count = merge
    auto issue = [&](u64 *dst, int u) {
        const int grp = u / B.count, jj = grp % R.dnum, cc = (grp / R.dnum) * SF_NB;
        const int l0 = jj * R.K, n0 = min((jj + 1) * R.K, R.L) - l0;
        const KsLayout Ls = ks_layout(R, B, u % B.count);
        for (int t = 0; t < n0; ++t) issue_col_tile_t<LR, LC, NT>(dst + (size_t)t * tw_words, Ls.x1 + ((size_t)(l0 + t) << (LR + LC)), cc);
    };
    if (db && U.u0 < U.u1) issue(bufs, U.u0);
    sf_cp_commit();
    int staged = -1, j = 0, c0 = 0, lo = 0, hi = 0, nd = 0;
    for (int k = 0, u = U.u0; u < U.u1; ++k, ++u) {
        const int grp = u / B.count, b = u % B.count;
        if (grp != staged) {
            // the previous unit ended at a barrier: nothing reads the tables now
            j = grp % R.dnum;
            c0 = (grp / R.dnum) * SF_NB;
            lo = j * R.K;
            hi = min((j + 1) * R.K, R.L);
            nd = hi - lo;
            twf = twi + (size_t)nd * g.r;
            for (int t = 0; t < nd; ++t) load_col_tw_t<LR, NT>(twi + (size_t)t * g.r, R.colT_i, lo + t);
            for (int m = 0; m < R.nm; ++m)
                if (m < lo || m >= hi) load_col_tw_t<LR, NT>(twf + (size_t)(m < lo ? m : m - nd) * g.r, R.colT_f, m);
            staged = grp;
        }
        u64 *cur = bufs + (size_t)(db ? (k & 1) : 0) * maxd * tw_words, *nxt = bufs + (size_t)((k + 1) & 1) * maxd * tw_words;
        if (db) {
            if (u + 1 < U.u1) issue(nxt, u + 1);
            sf_cp_commit();
            sf_cp_wait<1>();
        } else {
            issue(cur, u);
            sf_cp_commit();
            sf_cp_wait<0>();
        }
        __syncthreads();
        // inverse column pass of the digit's limbs, then y_i = x_i N^-1 Qhat_i^-1 mod q_i
        // (the scaling rides on the last inverse sweep)
        for (int t = 0; t < nd; ++t) {
            const int i = lo + t;
            u64 *sti = cur + (size_t)t * tw_words;
            const u64 w = R.mu_inv[j * R.K + t], wp = R.mu_inv_p[j * R.K + t], qi = R.m[i].q;
            col_inverse_st<LR, NT>(sti, twi + (size_t)t * g.r, qi, [&](int k, int bb, u64 v) {
                sti[tile_slot<SF_NB>(k, bb)] = sf_mul_shoup(v, w, wp, qi);
            });
        }
        __syncthreads();
        const KsLayout Lo = ks_layout(R, B, b);
        for (int m = 0; m < R.nm; ++m) {
            if (m >= lo && m < hi) continue;
            const SfMod &M = R.m[m];
            const sf_tw *twm = twf + (size_t)(m < lo ? m : m - nd) * g.r;
            u64 *dst = Lo.x2 + ((size_t)(j * R.nm + m) << (LR + LC)) + c0;
            // the forward column pass reads the conversion and writes x2 directly
            auto out = [&](int k, int bb, u64 v) { dst[((size_t)k << LC) + bb] = v; };
            if (nd == 1 && R.modup_copy) {
                // one-limb digit: Qhat = 1, so the conversion is the canonical
                // residue itself, below 4 q_m and taken as it is by the transform
                col_forward_io<LR, NT>(work, twm, M.q, [&](int k, int bb) { return cur[tile_slot<SF_NB>(k, bb)]; }, out);
            } else {
                // base conversion, lazy: each term in [0, 2q), the sum below 2q * nd
                // (digits hold at most 4 limbs: K <= 4)
                u64 qh[4], qhp[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const size_t ci = ((size_t)(j * R.K + t)) * R.nm + m;
                    qh[t] = t < nd ? R.mu_qhat[ci] : 0;
                    qhp[t] = t < nd ? R.mu_qhat_p[ci] : 0;
                }
                col_forward_io<LR, NT>(work, twm, M.q, [&](int k, int bb) {
                    const int sl = tile_slot<SF_NB>(k, bb);
                    u64 acc = 0;
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (t < nd) acc += sf_mul_shoup_lazy(cur[(size_t)t * tw_words + sl], qh[t], qhp[t], M.q);
                    return acc;
                }, out);
            }
            __syncthreads();
        }
    }
}

// Inner product with the key.  Groups: (row tile, modulus m); items: merges,
// each taking dnum steps (one per digit) whose tiles are double-buffered.
// Output: ACC (data moduli, NTT domain) or, for the special moduli, their NTT
// values in the x1 region (the inverse row pass runs in k_rows<true>).
// NT: 256 (8 elements per thread, three blocks per SM) or, for 128-point
// rows when the context asks for it, 512 (4 elements per thread, half the
// accumulator registers, two 16-warp blocks per SM).
template <int LR, int LC, int NT, int RAD = 0>
__global__ void __launch_bounds__(NT, NT >= 512 ? 2 : 3) k_ks3(SfRing R, SfKsBatch B, int ng)
{
    constexpr int NB = SfRow<LC>::NB, EPT = SfRow<LC>::ELEMS / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const SfUnits U = sf_block_units(ng * B.count);
    constexpr bool DB = true;
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *buf0 = (u64 *)(tw + NB * g.c);
    u64 *buf1 = DB ? buf0 + SfRow<LC>::WORDS : buf0;
    const int steps = (U.u1 - U.u0) * R.dnum;
    // step k -> unit U.u0 + k / dnum (group (row tile, modulus m), item a
    // merge), digit k % dnum; its tile is TA's limb m when m is one of digit
    // j's own limbs, else the digit's extension
    auto step_src = [&](int kk) -> const u64 * {
        const int uu = U.u0 + kk / R.dnum, jj = kk % R.dnum;
        const int gg = uu / B.count, ms = gg % R.nm;
        const KsLayout Ls = ks_layout(R, B, uu % B.count);
        const bool own_s = (ms >= jj * R.K && ms < min((jj + 1) * R.K, R.L));
        return (own_s ? Ls.ta + ((size_t)ms << (LR + LC)) : Ls.x2 + ((size_t)(jj * R.nm + ms) << (LR + LC))) +
               (size_t)(gg / R.nm) * NB * g.c;
    };
    if (DB && steps > 0) issue_row_tile_t<LC, NT>(buf0, step_src(0));
    sf_cp_commit();
    u64 acc_a[EPT], acc_b[EPT];
#pragma unroll
    for (int x = 0; x < EPT; ++x) acc_a[x] = acc_b[x] = 0;
    int staged = -1, m = 0;
    size_t tile_off = 0;
    u64 q = 0, one_p = 0;
    for (int k = 0; k < steps; ++k) {
        const int u = U.u0 + k / R.dnum, j = k % R.dnum;
        const int grp = u / B.count, b = u % B.count;
        if (grp != staged) {
            // a new group starts at digit 0, after the previous unit's last barrier
            m = grp % R.nm;
            const int r0 = (grp / R.nm) * NB;
            tile_off = (size_t)r0 * g.c;
            load_row_tw_t<LR, LC, NT>(tw, R.rowT_f, m, r0);
            q = R.m[m].q;
            one_p = R.m[m].one_p;
            staged = grp;
        }
        u64 *cur = (k & 1) ? buf1 : buf0, *nxt = (k & 1) ? buf0 : buf1;
        if (DB) {
            if (k + 1 < steps) issue_row_tile_t<LC, NT>(nxt, step_src(k + 1));
            sf_cp_commit();
            sf_cp_wait<1>();
        } else {
            issue_row_tile_t<LC, NT>(cur, step_src(k));
            sf_cp_commit();
            sf_cp_wait<0>();
        }
        __syncthreads();
        const bool own = (m >= j * R.K && m < min((j + 1) * R.K, R.L));
        if (!own) tile_forward_t<LC, true, NT, NB, RAD>(cur, tw, q);
        const size_t comp = (size_t)R.dnum * 2 * R.nm << (LR + LC);   // companions follow the key values
        const u64 *ka = B.key + ((((size_t)j * 2 + 0) * R.nm + m) << (LR + LC)) + tile_off;
        const u64 *kb = B.key + ((((size_t)j * 2 + 1) * R.nm + m) << (LR + LC)) + tile_off;
        // per digit c * key (c lazy < 68q, key < q with its Shoup companion) lands in [0, 4q) and is summed
#pragma unroll
        for (int x = 0; x < EPT; ++x) {
            const int e = threadIdx.x + x * NT;
            const u64 c = cur[row_slot_t<LC>(e)];
            acc_a[x] += sf_mul_shoup_lazy4(c, __ldg(ka + e), __ldg(ka + comp + e), q);
            acc_b[x] += sf_mul_shoup_lazy4(c, __ldg(kb + e), __ldg(kb + comp + e), q);
        }
        if (j == R.dnum - 1) {
            const KsLayout Lo = ks_layout(R, B, b);
            u64 *da, *db;
            if (m < R.L) {
                da = Lo.accq + ((size_t)m << (LR + LC)) + tile_off;
                db = Lo.accq + ((size_t)(R.L + m) << (LR + LC)) + tile_off;
            } else {
                da = Lo.x1 + ((size_t)(m - R.L) << (LR + LC)) + tile_off;
                db = Lo.x1 + ((size_t)(R.K + m - R.L) << (LR + LC)) + tile_off;
            }
#pragma unroll
            for (int x = 0; x < EPT; ++x) {
                const int e = threadIdx.x + x * NT;
                da[e] = sf_reduce(acc_a[x], q, one_p);
                db[e] = sf_reduce(acc_b[x], q, one_p);
                acc_a[x] = acc_b[x] = 0;
            }
        }
        __syncthreads();
    }
}

// ModDown conversion.  Groups: (column tile, part p); items: merges.  smem: K
// inverse (special) + L forward (data) column tables, K source tiles (two
// buffers when db), one work tile.
template <int LR, int LC>
__global__ void __launch_bounds__(SfThreads<LR>::value, SfThreads<LR>::value >= 512 ? 1 : 3)
    k_ks4(SfRing R, SfKsBatch B, int ng, int db)
{
    constexpr int NT = SfThreads<LR>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const SfUnits U = sf_block_units(ng * B.count);
    const int tw_words = tile_words(g.log_r);
    sf_tw *twi = (sf_tw *)smem_raw;                 // [K][R] inverse, special moduli
    sf_tw *twf = twi + (size_t)R.K * g.r;           // [L][R] forward, data moduli
    u64 *bufs = (u64 *)(twf + (size_t)R.L * g.r);   // (db ? 2 : 1) x K tiles
    u64 *work = bufs + (size_t)(db ? 2 : 1) * R.K * tw_words;
    for (int k = 0; k < R.K; ++k) load_col_tw_t<LR, NT>(twi + (size_t)k * g.r, R.colT_i, R.L + k);
    for (int i = 0; i < R.L; ++i) load_col_tw_t<LR, NT>(twf + (size_t)i * g.r, R.colT_f, i);
    // unit u: group u / count = (column tile, part p), item u % count = merge;
    // the staged tables are the same for every group
    auto issue = [&](u64 *dst, int u) {
        const int gg = u / B.count, pp = gg % 2, cc = (gg / 2) * SF_NB;
        const KsLayout Ls = ks_layout(R, B, u % B.count);
        for (int k = 0; k < R.K; ++k)
            issue_col_tile_t<LR, LC, NT>(dst + (size_t)k * tw_words, Ls.x1 + ((size_t)(pp * R.K + k) << (LR + LC)), cc);
    };
    if (db && U.u0 < U.u1) issue(bufs, U.u0);
    sf_cp_commit();
    for (int kk = 0, u = U.u0; u < U.u1; ++kk, ++u) {
        const int grp = u / B.count, b = u % B.count;
        const int p = grp % 2, c0 = (grp / 2) * SF_NB;
        u64 *cur = bufs + (size_t)(db ? (kk & 1) : 0) * R.K * tw_words, *nxt = bufs + (size_t)((kk + 1) & 1) * R.K * tw_words;
        if (db) {
            if (u + 1 < U.u1) issue(nxt, u + 1);
            sf_cp_commit();
            sf_cp_wait<1>();
        } else {
            issue(cur, u);
            sf_cp_commit();
            sf_cp_wait<0>();
        }
        __syncthreads();
        // inverse column pass of the special limbs, scaled by the ModDown
        // constants on the last inverse sweep
        for (int k = 0; k < R.K; ++k) {
            const int m = R.L + k;
            u64 *stk = cur + (size_t)k * tw_words;
            const u64 w = R.md_inv[k], wp = R.md_inv_p[k], qm = R.m[m].q;
            col_inverse_st<LR, NT>(stk, twi + (size_t)k * g.r, qm, [&](int kk2, int bb, u64 v) {
                stk[tile_slot<SF_NB>(kk2, bb)] = sf_mul_shoup(v, w, wp, qm);
            });
        }
        __syncthreads();
        const KsLayout Lo = ks_layout(R, B, b);
        for (int i = 0; i < R.L; ++i) {
            const SfMod &M = R.m[i];
            // base conversion, lazy: each term in [0, 2q), the sum below 2q * K,
            // read by the forward column pass, which writes x2 directly
            u64 ph[4], php[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ph[k] = k < R.K ? R.md_phat[(size_t)k * R.L + i] : 0;
                php[k] = k < R.K ? R.md_phat_p[(size_t)k * R.L + i] : 0;
            }
            u64 *dst = Lo.x2 + ((size_t)(p * R.L + i) << (LR + LC)) + c0;
            col_forward_io<LR, NT>(work, twf + (size_t)i * g.r, M.q, [&](int kk2, int bb) {
                const int sl = tile_slot<SF_NB>(kk2, bb);
                u64 acc = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < R.K) acc += sf_mul_shoup_lazy(cur[(size_t)k * tw_words + sl], ph[k], php[k], M.q);
                return acc;
            }, [&](int kk2, int bb, u64 v) { dst[((size_t)kk2 << LC) + bb] = v; });
            __syncthreads();
        }
    }
}

// ModDown finish.  Groups: (row tile, limb i); items: (merge b, part p).
// out += ACC - conv, both already multiplied by P^-1.  smem: forward row twiddles and two conversion
// tiles (double-buffered); ACC and out are read elementwise from global into
// registers before the row pass.
template <int LR, int LC, int RAD = 0>
__global__ void __launch_bounds__(SfRow<LC>::NT, 3) k_ks5(SfRing R, SfKsBatch B, int ng)
{
    constexpr int NT = SfRow<LC>::NT, NB = SfRow<LC>::NB, EPT = SfRow<LC>::ELEMS / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr SfGeoT<LR, LC> g{};
    const int n_items = 2 * B.count;
    const SfUnits U = sf_block_units(ng * n_items);
    const int tw_words = SfRow<LC>::WORDS;
    constexpr bool DB = true;
    sf_tw *tw = (sf_tw *)smem_raw;
    u64 *bufs = (u64 *)(tw + NB * g.c);             // 2 conversion tiles
    // unit u: group u / n_items = (row tile, limb i), item u % n_items = (merge, part)
    auto unit_src = [&](int uu) -> const u64 * {
        const int gg = uu / n_items, it2 = uu % n_items;
        const KsLayout Ls = ks_layout(R, B, it2 >> 1);
        return Ls.x2 + ((size_t)((it2 & 1) * R.L + gg % R.L) << (LR + LC)) + (size_t)(gg / R.L) * NB * g.c;
    };
    if (DB && U.u0 < U.u1) issue_row_tile_t<LC, NT>(bufs, unit_src(U.u0));
    sf_cp_commit();
    int staged = -1, i = 0;
    size_t tile_off = 0;
    u64 q = 0, one_p = 0, conv_off = 0;
    for (int k = 0, u = U.u0; u < U.u1; ++k, ++u) {
        const int grp = u / n_items, it = u % n_items;
        if (grp != staged) {
            // the previous unit ended at a barrier: nothing reads tw now
            i = grp % R.L;
            const int r0 = (grp / R.L) * NB;
            tile_off = (size_t)r0 * g.c;
            load_row_tw_t<LR, LC, NT>(tw, R.rowT_f, i, r0);
            q = R.m[i].q;
            one_p = R.m[i].one_p;
            // conv leaves the lazy forward transform below 72 q (inputs below 2 K q <= 8 q,
            // at most 16 stages adding 4 q each); 128 q keeps the sum positive
            conv_off = 128 * q;
            staged = grp;
        }
        u64 *cur = bufs + (DB ? (size_t)(k & 1) * tw_words : 0), *nxt = bufs + (DB ? (size_t)((k + 1) & 1) * tw_words : 0);
        if (DB) {
            if (u + 1 < U.u1) issue_row_tile_t<LC, NT>(nxt, unit_src(u + 1));
            sf_cp_commit();
            sf_cp_wait<1>();
        } else {
            issue_row_tile_t<LC, NT>(cur, unit_src(u));
            sf_cp_commit();
            sf_cp_wait<0>();
        }
        const int b = it >> 1, p = it & 1;
        const size_t off = ((size_t)(p * R.L + i) << (LR + LC)) + tile_off;
        const u64 *acc = ks_layout(R, B, b).accq + off;
        u64 *out = merge_out(B, b) + off;   // holds v (+ tau_d(u.b)) from k_ks_gather
        // this thread's accumulator and output words, loaded into registers
        // before the row pass so that the loads are in flight while it runs
        u64 va[EPT], vo[EPT];
#pragma unroll
        for (int x = 0; x < EPT; ++x) {
            va[x] = acc[threadIdx.x + x * NT];
            vo[x] = out[threadIdx.x + x * NT];
        }
        __syncthreads();
        row_forward_t<LC, NT, RAD>(cur, tw, q);
        // acc and conv both carry P^-1 already: out += acc - conv, one reduction
#pragma unroll
        for (int x = 0; x < EPT; ++x) {
            const int e = threadIdx.x + x * NT;
            out[e] = sf_reduce(vo[x] + va[x] + conv_off - cur[row_slot_t<LC>(e)], q, one_p);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launching ----

static size_t smem_rows(const SfRing &R, int tiles)
{
    return sizeof(sf_tw) * sf_row_nb(R.log_c) * R.c + sizeof(u64) * row_tile_words(R.log_c) * tiles;
}

template <class K>
static int occupancy(K kernel, int threads, size_t smem)
{
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        b = 1;
    }
    return std::max(1, b);
}

// blocks of a persistent launch over n_units (group, item) units: one
// resident wave (num_sms x occupancy blocks), at most one block per unit.
// The kernels split the units evenly (sf_block_units), so no block slot idles
// when the group count does not divide the wave.
static int wave_blocks(const sf_ctx *ctx, int occ, int n_units)
{
    return std::max(1, std::min(ctx->num_sms * occ, n_units));
}

// The 512-thread inner product (128-point rows only, when the context asks
// for it); false when the default block shape is to run.  A template, so
// that the discarded branch instantiates nothing for the other ring splits.
template <int LR, int LC>
static bool ks3_launch_wide(sf_ctx *ctx, const SfKsBatch &b, size_t sm3, int ng, cudaStream_t st)
{
    if constexpr (LC == 7) {
        if (ctx->ks3_threads != 512) return false;
        const int nb = wave_blocks(ctx, occupancy(k_ks3<LR, LC, 512>, 512, sm3), ng * b.count);
        k_ks3<LR, LC, 512><<<nb, 512, sm3, st>>>(ctx->ring, b, ng);
        return true;
    } else {
        return false;
    }
}

sf_status sf_ks_launch(sf_ctx *ctx, const SfKsBatch &B0, cudaStream_t st)
{
    const SfRing &R = ctx->ring;
    if (B0.count <= 0) return SF_OK;
    const int maxd = std::min(R.K, R.L);
    const int rtiles = R.r / sf_row_nb(R.log_c), ctiles = R.c / SF_NB;
    const int row_bufs = sf_rows_double_buffered(R.log_c) ? 2 : 1;
    const size_t sm_rows = smem_rows(R, row_bufs);
    // ks2 / ks4 shared memory with two buffers of source tiles (db) or one
    const size_t tw_bytes = sizeof(u64) * tile_words(R.log_r);
    const size_t sm2[2] = {sizeof(sf_tw) * R.nm * R.r + tw_bytes * (maxd + 1),
                           sizeof(sf_tw) * R.nm * R.r + tw_bytes * (2 * maxd + 1)};
    const size_t sm3 = smem_rows(R, 2);
    const size_t sm4[2] = {sizeof(sf_tw) * (R.K + R.L) * R.r + tw_bytes * (R.K + 1),
                           sizeof(sf_tw) * (R.K + R.L) * R.r + tw_bytes * (2 * R.K + 1)};
    const size_t sm5 = smem_rows(R, 2);
    cudaEvent_t ev;
    for (int off = 0; off < B0.count; off += 32768) {
        SfKsBatch b = B0;
        b.count = std::min(32768, B0.count - off);
        b.first = B0.first + off;
        b.scratch += sf_ks_scratch_words(R) * off;
        const int ew_blocks = (R.n + 256 * SF_EW - 1) / (256 * SF_EW);
        const dim3 eg(ew_blocks, R.L, b.count);
        SF_GEO_DISPATCH(R.log_n, {
            constexpr int NTR = SfRow<LC>::NT, NTC = SfThreads<LR>::value;
            sf_launch_begin(ctx, SFK_KS_GATHER, st, &ev);
            k_ks_gather<<<eg, 256, 0, st>>>(R, b);
            sf_launch_end(ctx, SFK_KS_GATHER, st, ev);

            sf_launch_begin(ctx, SFK_KS1_INV_ROW, st, &ev);
            {
                const SfRowSet S{0, (size_t)R.L << R.log_n, R.L, 0, R.L};   // TA -> X1
                const int ng = rtiles * S.npoly;
                SF_RAD_DISPATCH(ctx->row_radix, {
                    const int nb = wave_blocks(ctx, occupancy(k_rows<true, LR, LC, RAD>, NTR, sm_rows), ng * b.count);
                    k_rows<true, LR, LC, RAD><<<nb, NTR, sm_rows, st>>>(R, b, S, ng);
                });
            }
            sf_launch_end(ctx, SFK_KS1_INV_ROW, st, ev);

            sf_launch_begin(ctx, SFK_KS2_MODUP_COL, st, &ev);
            {
                const int ng = ctiles * R.dnum;
                const int o1 = occupancy(k_ks2<LR, LC>, NTC, sm2[0]), o2 = occupancy(k_ks2<LR, LC>, NTC, sm2[1]);
                const int db = o2 >= o1;   // double-buffer unless one buffer fits more blocks
                const int nb = wave_blocks(ctx, db ? o2 : o1, ng * b.count);
                k_ks2<LR, LC><<<nb, NTC, sm2[db], st>>>(R, b, ng, db);
            }
            sf_launch_end(ctx, SFK_KS2_MODUP_COL, st, ev);

            sf_launch_begin(ctx, SFK_KS3_INNER_ROW, st, &ev);
            {
                const int ng = rtiles * R.nm;
                if (!ks3_launch_wide<LR, LC>(ctx, b, sm3, ng, st)) {
                    SF_RAD_DISPATCH(ctx->row_radix, {
                        const int nb = wave_blocks(ctx, occupancy(k_ks3<LR, LC, NTR, RAD>, NTR, sm3), ng * b.count);
                        k_ks3<LR, LC, NTR, RAD><<<nb, NTR, sm3, st>>>(R, b, ng);
                    });
                }
            }
            sf_launch_end(ctx, SFK_KS3_INNER_ROW, st, ev);
            sf_launch_begin(ctx, SFK_KS3_INV_ROW_P, st, &ev);
            {
                // inverse row pass of the special limbs' accumulators, in place in x1
                const SfRowSet S{(size_t)R.L << R.log_n, (size_t)R.L << R.log_n, 2 * R.K, R.L, R.K};
                const int ng2 = rtiles * S.npoly;
                SF_RAD_DISPATCH(ctx->row_radix, {
                    const int nb2 = wave_blocks(ctx, occupancy(k_rows<true, LR, LC, RAD>, NTR, sm_rows), ng2 * b.count);
                    k_rows<true, LR, LC, RAD><<<nb2, NTR, sm_rows, st>>>(R, b, S, ng2);
                });
            }
            sf_launch_end(ctx, SFK_KS3_INV_ROW_P, st, ev);

            sf_launch_begin(ctx, SFK_KS4_MODDOWN_COL, st, &ev);
            {
                const int ng = ctiles * 2;
                const int o1 = occupancy(k_ks4<LR, LC>, NTC, sm4[0]), o2 = occupancy(k_ks4<LR, LC>, NTC, sm4[1]);
                const int db = o2 >= o1;
                const int nb = wave_blocks(ctx, db ? o2 : o1, ng * b.count);
                k_ks4<LR, LC><<<nb, NTC, sm4[db], st>>>(R, b, ng, db);
            }
            sf_launch_end(ctx, SFK_KS4_MODDOWN_COL, st, ev);

            sf_launch_begin(ctx, SFK_KS5_FINISH_ROW, st, &ev);
            {
                const int ng = rtiles * R.L;
                SF_RAD_DISPATCH(ctx->row_radix, {
                    const int nb = wave_blocks(ctx, occupancy(k_ks5<LR, LC, RAD>, NTR, sm5), ng * 2 * b.count);
                    k_ks5<LR, LC, RAD><<<nb, NTR, sm5, st>>>(R, b, ng);
                });
            }
            sf_launch_end(ctx, SFK_KS5_FINISH_ROW, st, ev);
        });
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
#define SF_KS_ATTR(K) SF_CUDA_TRY(cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
#define SF_KS_ATTRS(LR, LC)                                                                                  \
    SF_KS_ATTR((k_rows<true, LR, LC>)) SF_KS_ATTR((k_ks2<LR, LC>)) SF_KS_ATTR((k_ks3<LR, LC, SfRow<LC>::NT>)) \
    SF_KS_ATTR((k_ks4<LR, LC>)) SF_KS_ATTR((k_ks5<LR, LC>)) SF_KS_ATTR((k_rows<true, LR, LC, 1>))               \
    SF_KS_ATTR((k_ks3<LR, LC, SfRow<LC>::NT, 1>)) SF_KS_ATTR((k_ks5<LR, LC, 1>)) SF_KS_ATTR((k_rows<true, LR, LC, 2>))  \
    SF_KS_ATTR((k_ks3<LR, LC, SfRow<LC>::NT, 2>)) SF_KS_ATTR((k_ks5<LR, LC, 2>))
    SF_KS_ATTRS(5, 5) SF_KS_ATTRS(5, 6) SF_KS_ATTRS(6, 6) SF_KS_ATTRS(6, 7) SF_KS_ATTRS(7, 7) SF_KS_ATTRS(7, 8)
    SF_KS_ATTRS(7, 9)
    SF_KS_ATTR((k_ks3<6, 7, 512>)) SF_KS_ATTR((k_ks3<7, 7, 512>))
#undef SF_KS_ATTRS
#undef SF_KS_ATTR
    return SF_OK;
}
