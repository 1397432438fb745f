// sf_pp.cu -- arithmetic in the paper's prime-power cyclotomic rings
// K = Q[X] / Phi_M(X), M = t^alpha with t an odd prime (Sec. 2.1-2.3; Table 2
// lists M = 3^7, 7^4, 5^5), modulo RNS primes q_i = 1 (mod M).
//
// Phi_M(X) = sum_{k < t} X^(k m), m = M / t, N = phi(M) = (t - 1) m.  Products
// in Z_q[X] / Phi_M are taken as cyclic products of length M (Phi_M divides
// X^M - 1) followed by the reduction X^(N + e) = -sum_{k < t-1} X^(e + k m),
// e < m.  The cyclic product uses a length-M radix-t number-theoretic
// transform over Z_q with omega a primitive M-th root of unity: decimation in
// frequency (Gentleman-Sande) forward, natural input and base-t digit-reversed
// output, and the mirror decimation in time inverse with the factor M^-1.
// Automorphisms tau_d: X -> X^d permute the length-M coefficients (i -> i d
// mod M) before the same reduction; traces are sums of automorphisms taken
// along the tower of Sec. 2.3.
//
// One block per (polynomial, limb) holds its length-M vector in shared memory
// (at most 3125 words for Table 2's rings).  Each radix-t butterfly runs the
// t-point DFT with t - 1 products per output, summed lazily below 2 t q, then
// one reduction; the compiled rings pair conjugate terms instead ((t-1)^2 / 2
// products, ppt_dft_pairs; two at t = 3, ppt_dft3);
// twiddles and t-th roots come from a per-limb table of omega^e.  Table 2's
// rings and the small test rings are compiled with t and alpha as constants
// (k_ppt_ntt); other rings run the generic kernel (k_pp_ntt).
#include <algorithm>
#include <vector>

#include "sf_pp.cuh"

template <int T, int ALPHA>
__global__ void __launch_bounds__(SfPpT<T, ALPHA>::THREADS) k_ppt_ntt(SfPpRing R, const u64 *in, u64 *out, int inverse)
{
    constexpr int M = SfPpT<T, ALPHA>::M, NT = SfPpT<T, ALPHA>::THREADS;
    __shared__ u64 s[M];
    const int i = blockIdx.x;
    const SfPpMod &P = R.mod[i];
    const size_t off = ((size_t)blockIdx.y * R.L + i) * M;
    if (inverse) {
        for (int e = threadIdx.x; e < M; e += NT) s[e] = in[off + e];
        __syncthreads();
        constexpr int H = (T - 1) / 2;
        ppt_inverse<T, M, T>(s, R.iw + (size_t)i * M, R.iw_p + (size_t)i * M, R.dftc + (size_t)i * H * H * 4, P.q,
                             P.one_p, P);
        for (int e = threadIdx.x; e < M; e += NT) out[off + e] = sf_mul_shoup(s[e], P.minv, P.minv_p, P.q);
    } else {
        constexpr int H = (T - 1) / 2;
        // the first stage reads the input straight from global memory
        const u64 *src = in + off;
        ppt_forward_ld<T, M>(s, [src](int e) { return src[e]; }, R.w + (size_t)i * M, R.w_p + (size_t)i * M,
                             R.dftc + (size_t)i * H * H * 4, P.q, P.one_p, P);
        for (int e = threadIdx.x; e < M; e += NT) out[off + e] = s[e];
    }
}

// Batched length-M transform: grid (L, count); [count][L][M] in and out.
__global__ void __launch_bounds__(SF_PP_THREADS) k_pp_ntt(SfPpRing R, const u64 *in, u64 *out, int inverse)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *s = (u64 *)smem_raw;
    const int i = blockIdx.x;
    const size_t off = ((size_t)blockIdx.y * R.L + i) * R.M;
    for (int e = threadIdx.x; e < R.M; e += blockDim.x) s[e] = in[off + e];
    __syncthreads();
    if (inverse) pp_inverse(s, R, i);
    else pp_forward(s, R, i);
    for (int e = threadIdx.x; e < R.M; e += blockDim.x) out[off + e] = s[e];
}

// Products in Z_q[X] / Phi_M: grid (L, count); a, b, out [count][L][N], canonical.
// b_polys: b holds that many polynomials, polynomial y of a pairs with y mod b_polys
__global__ void __launch_bounds__(SF_PP_THREADS) k_pp_mul(SfPpRing R, const u64 *a, const u64 *b, u64 *out, int b_polys)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *sa = (u64 *)smem_raw, *sb = sa + R.M;
    const int i = blockIdx.x;
    const size_t off = ((size_t)blockIdx.y * R.L + i) * R.N;
    const size_t offb = ((size_t)(blockIdx.y % b_polys) * R.L + i) * R.N;
    for (int e = threadIdx.x; e < R.M; e += blockDim.x) {
        sa[e] = e < R.N ? a[off + e] : 0;
        sb[e] = e < R.N ? b[offb + e] : 0;
    }
    __syncthreads();
    pp_forward(sa, R, i);
    pp_forward(sb, R, i);
    for (int e = threadIdx.x; e < R.M; e += blockDim.x) sa[e] = pp_mulmod(sa[e], sb[e], R.mod[i]);
    __syncthreads();
    pp_inverse(sa, R, i);
    pp_reduce_phi(sa, R, i);
    for (int e = threadIdx.x; e < R.N; e += blockDim.x) out[off + e] = sa[e];
}

// tau_d: X -> X^d, gcd(d, M) = 1: coefficient i moves to i d mod M (distinct
// targets), then the Phi_M reduction.  grid (L, count); [count][L][N].
__global__ void __launch_bounds__(SF_PP_THREADS) k_pp_auto(SfPpRing R, const u64 *in, u64 *out, int d)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    u64 *s = (u64 *)smem_raw;
    const int i = blockIdx.x;
    const size_t off = ((size_t)blockIdx.y * R.L + i) * R.N;
    for (int e = threadIdx.x; e < R.M; e += blockDim.x) s[e] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < R.N; e += blockDim.x) s[(int)(((long long)e * d) % R.M)] = in[off + e];
    __syncthreads();
    pp_reduce_phi(s, R, i);
    for (int e = threadIdx.x; e < R.N; e += blockDim.x) out[off + e] = s[e];
}

// acc += x, limb-wise modulo q_i; [count][L][N]
__global__ void k_pp_add(SfPpRing R, u64 *acc, const u64 *x, size_t total)
{
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)((k / R.N) % R.L);
        acc[k] = sf_add(acc[k], x[k], R.mod[i].q);
    }
}

// ------------------------------------------------------------------ host ----

static u64 pp_powmod(u64 a, u64 e, u64 q) { return sf_host_powmod(a, e, q); }

// element of exact multiplicative order M = t^alpha modulo q (q = 1 mod M)
static u64 pp_root(u64 q, int M, int t)
{
    for (u64 g = 2; g < q; ++g) {
        const u64 x = pp_powmod(g, (q - 1) / (u64)M, q);
        if (pp_powmod(x, (u64)(M / t), q) != 1) return x;
    }
    return 0;
}

static bool pp_is_odd_prime(int t)
{
    if (t < 3 || !(t & 1)) return false;
    for (int d = 3; d * d <= t; d += 2)
        if (t % d == 0) return false;
    return true;
}

extern "C" sf_status sf_pp_ring_create(int32_t t, int32_t alpha, int32_t L, int32_t bits, int32_t device,
                                       sf_pp_ring **out)
{
    if (!out) return sf_set_error(SF_EINVAL, "sf_pp_ring_create: null output");
    *out = nullptr;
    if (!pp_is_odd_prime(t) || t > SF_PP_MAX_T || alpha < 1 || L < 1 || L > SF_MAX_MODULI || bits < 20 || bits > 61)
        return sf_set_error(SF_EINVAL, "sf_pp_ring_create: t must be an odd prime <= 7, 1 <= L <= %d, 20 <= bits <= 61",
                            SF_MAX_MODULI);
    long long M = 1;
    for (int k = 0; k < alpha; ++k) M *= t;
    if (M < t * t || M > SF_PP_MAX_M) return sf_set_error(SF_EINVAL, "sf_pp_ring_create: M = t^alpha must lie in [t^2, %d]", SF_PP_MAX_M);
    sf_pp_ring *r = new sf_pp_ring();
    r->device = device;
    SfPpRing &R = r->R;
    R.t = t;
    R.alpha = alpha;
    R.M = (int)M;
    R.m = (int)(M / t);
    R.N = (t - 1) * R.m;
    R.L = L;
    r->q.resize(L);
    if (sf_find_primes((u64)M, bits, L, r->q.data()) != L) {
        delete r;
        return sf_set_error(SF_EINVAL, "sf_pp_ring_create: not enough primes = 1 mod %lld below 2^%d", M, bits);
    }
    const int H = (t - 1) / 2;
    const size_t o_qhat = (size_t)4 * L * R.M, o_dftc = o_qhat + (size_t)2 * L * L;
    std::vector<u64> tab(o_dftc + (size_t)4 * L * H * H);
    for (int i = 0; i < L; ++i) {
        const u64 q = r->q[i];
        const u64 w = pp_root(q, R.M, t), iw = sf_host_invmod(w, q);
        u64 a = 1, b = 1;
        for (int e = 0; e < R.M; ++e) {
            tab[(size_t)0 * L * R.M + (size_t)i * R.M + e] = a;
            tab[(size_t)1 * L * R.M + (size_t)i * R.M + e] = sf_shoup_companion(a, q);
            tab[(size_t)2 * L * R.M + (size_t)i * R.M + e] = b;
            tab[(size_t)3 * L * R.M + (size_t)i * R.M + e] = sf_shoup_companion(b, q);
            a = sf_host_mulmod(a, w, q);
            b = sf_host_mulmod(b, iw, q);
        }
        SfPpMod &P = R.mod[i];
        P.q = q;
        P.one_p = sf_shoup_companion(1, q);
        u64 inv = 1;   // q^-1 mod 2^64 by Newton iteration
        for (int k = 0; k < 6; ++k) inv *= 2 - q * inv;
        P.qinv_neg = (u64)0 - inv;
        const u64 r1 = (u64)(((unsigned __int128)1 << 64) % q);
        P.r2 = sf_host_mulmod(r1, r1, q);
        P.rm = r1;
        P.rm_p = sf_shoup_companion(r1, q);
        P.minv = sf_host_invmod((u64)R.M % q, q);
        P.minv_p = sf_shoup_companion(P.minv, q);
        P.h2 = sf_host_invmod(2, q);
        P.h2_p = sf_shoup_companion(P.h2, q);
        // zeta = omega^(M/3): c = (zeta - zeta^2) / 2 (used at t = 3 only)
        const u64 z = sf_host_powmod(w, (u64)(R.M / t), q), z2 = sf_host_mulmod(z, z, q);
        P.c3 = sf_host_mulmod((z + q - z2) % q, P.h2, q);
        P.c3_p = sf_shoup_companion(P.c3, q);
        // paired t-point DFT: C_rk = (z^(rk) + z^(-rk)) / 2, S_rk = (z^(rk) - z^(-rk)) / 2
        for (int rr = 1; rr <= H; ++rr)
            for (int kk = 1; kk <= H; ++kk) {
                const int e = (rr * kk) % t;
                const u64 zp = sf_host_powmod(z, (u64)e, q), zm = sf_host_powmod(z, (u64)(t - e), q);
                const u64 C = sf_host_mulmod((zp + zm) % q, P.h2, q), S = sf_host_mulmod((zp + q - zm) % q, P.h2, q);
                u64 *d = &tab[o_dftc + 4 * (((size_t)i * H + (rr - 1)) * H + (kk - 1))];
                d[0] = C;
                d[1] = sf_shoup_companion(C, q);
                d[2] = S;
                d[3] = sf_shoup_companion(S, q);
            }
    }
    // RNS digits: (Q / q_i) mod q_j and (Q / q_i)^-1 mod q_i
    for (int i = 0; i < L; ++i) {
        for (int j = 0; j < L; ++j) {
            u64 v = 1;
            for (int k = 0; k < L; ++k)
                if (k != i) v = sf_host_mulmod(v, r->q[k] % r->q[j], r->q[j]);
            tab[o_qhat + 2 * ((size_t)i * L + j)] = v;
            tab[o_qhat + 2 * ((size_t)i * L + j) + 1] = sf_shoup_companion(v, r->q[j]);
            if (j == i) {
                R.mod[i].qh_inv = sf_host_invmod(v, r->q[i]);
                R.mod[i].qh_inv_p = sf_shoup_companion(R.mod[i].qh_inv, r->q[i]);
            }
        }
    }
    // the product kernel holds two length-M vectors (up to 64 KB of shared memory)
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaFuncSetAttribute(k_pp_mul, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * sizeof(u64) * SF_PP_MAX_M)) != cudaSuccess ||
        cudaMalloc((void **)&r->d_tables, sizeof(u64) * tab.size()) != cudaSuccess ||
        cudaMemcpy(r->d_tables, tab.data(), sizeof(u64) * tab.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (r->d_tables) cudaFree(r->d_tables);
        delete r;
        return sf_set_error(SF_ECUDA, "sf_pp_ring_create: table upload failed");
    }
    R.w = r->d_tables;
    R.w_p = R.w + (size_t)L * R.M;
    R.iw = R.w_p + (size_t)L * R.M;
    R.iw_p = R.iw + (size_t)L * R.M;
    R.qhat = R.iw_p + (size_t)L * R.M;
    R.dftc = R.qhat + (size_t)2 * L * L;
    *out = r;
    return SF_OK;
}

extern "C" void sf_pp_ring_destroy(sf_pp_ring *r)
{
    if (!r) return;
    cudaSetDevice(r->device);
    if (r->d_tables) cudaFree(r->d_tables);
    if (r->d_scratch) cudaFree(r->d_scratch);
    if (r->d_ks) cudaFree(r->d_ks);
    delete r;
}

extern "C" sf_status sf_pp_ring_info(const sf_pp_ring *r, int32_t *N, int32_t *M, uint64_t *moduli)
{
    if (!r) return sf_set_error(SF_EINVAL, "sf_pp_ring_info: null ring");
    if (N) *N = r->R.N;
    if (M) *M = r->R.M;
    if (moduli)
        for (int i = 0; i < r->R.L; ++i) moduli[i] = r->q[i];
    return SF_OK;
}

static sf_status pp_check(const sf_pp_ring *r, const void *a, const void *b, int count)
{
    if (!r || !a || !b || count < 1) return sf_set_error(SF_EINVAL, "prime-power ring: bad arguments");
    if (count > 65535) return sf_set_error(SF_EINVAL, "prime-power ring: at most 65535 polynomials per call");
    if (cudaSetDevice(r->device) != cudaSuccess) return sf_set_error(SF_ECUDA, "cudaSetDevice failed");
    return SF_OK;
}

extern "C" sf_status sf_pp_ntt(sf_pp_ring *r, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t inverse,
                               void *stream)
{
    SF_TRY(pp_check(r, d_in, d_out, count));
    if (inverse != 0 && inverse != 1) return sf_set_error(SF_EINVAL, "sf_pp_ntt: inverse must be 0 or 1");
    const SfPpRing &R = r->R;
    bool done = false;
    SF_PPT_DISPATCH(R.t, R.alpha, done, {
        k_ppt_ntt<T, ALPHA><<<dim3(R.L, count), SfPpT<T, ALPHA>::THREADS, 0, (cudaStream_t)stream>>>(R, d_in, d_out,
                                                                                                    inverse);
    });
    if (!done)
        k_pp_ntt<<<dim3(R.L, count), SF_PP_THREADS, sizeof(u64) * R.M, (cudaStream_t)stream>>>(R, d_in, d_out, inverse);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_pp_mul(sf_pp_ring *r, const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_out,
                               int32_t count, void *stream)
{
    SF_TRY(pp_check(r, d_a, d_b, count));
    if (!d_out) return sf_set_error(SF_EINVAL, "sf_pp_mul: null output");
    const SfPpRing &R = r->R;
    k_pp_mul<<<dim3(R.L, count), SF_PP_THREADS, 2 * sizeof(u64) * R.M, (cudaStream_t)stream>>>(R, d_a, d_b, d_out,
                                                                                                count);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

static sf_status pp_auto(sf_pp_ring *r, const u64 *in, u64 *out, int count, int d, cudaStream_t st)
{
    const SfPpRing &R = r->R;
    const int dd = ((d % R.M) + R.M) % R.M;
    if (dd % R.t == 0) return sf_set_error(SF_EINVAL, "automorphism index %d not coprime to M = %d", d, R.M);
    k_pp_auto<<<dim3(R.L, count), SF_PP_THREADS, sizeof(u64) * R.M, st>>>(R, in, out, dd);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_pp_automorphism(sf_pp_ring *r, const uint64_t *d_in, uint64_t *d_out, int32_t count,
                                        int32_t d, void *stream)
{
    SF_TRY(pp_check(r, d_in, d_out, count));
    if (d_in == d_out) return sf_set_error(SF_EINVAL, "sf_pp_automorphism: in place is not supported");
    return pp_auto(r, d_in, d_out, count, d, (cudaStream_t)stream);
}

static void pp_prime_factors(int x, std::vector<int> &out)
{
    for (int d = 2; d * d <= x; ++d)
        while (x % d == 0) {
            out.push_back(d);
            x /= d;
        }
    if (x > 1) out.push_back(x);
}

void sf_pp_tower_steps(const SfPpRing &R, int gamma, std::vector<std::pair<int, int>> &steps)
{
    long long tp = 1;
    for (int k = 0; k < R.alpha - 1; ++k) tp *= R.t;     // t^(alpha-1)
    // Tr_{K_(i+1) / K_i} for i = alpha - 1 .. max(gamma, 1): generator 1 + t^i, order t
    for (int i = R.alpha - 1; i >= std::max(gamma, 1); --i, tp /= R.t) steps.push_back({(int)((1 + tp) % R.M), R.t});
    if (gamma >= 1) return;
    // Tr_{K_1 / K_0}: the cyclic group (Z/MZ)^* / (1 + tZ) of order t - 1, one
    // prime factor l at a time, with a primitive root g mod M
    std::vector<int> fac;
    pp_prime_factors(R.N, fac);
    std::sort(fac.begin(), fac.end());
    fac.erase(std::unique(fac.begin(), fac.end()), fac.end());
    int g = 2;
    for (; g < R.M; ++g) {
        if (g % R.t == 0) continue;
        bool ok = true;
        for (int f : fac) ok = ok && sf_host_powmod((u64)g, (u64)(R.N / f), (u64)R.M) != 1;
        if (ok) break;
    }
    std::vector<int> lf;
    pp_prime_factors(R.t - 1, lf);
    int rest = R.t - 1;
    for (int l : lf) {
        rest /= l;
        steps.push_back({(int)sf_host_powmod((u64)g, (u64)rest, (u64)R.M), l});
    }
}

extern "C" sf_status sf_pp_trace(sf_pp_ring *r, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t gamma,
                                 int32_t *n_automorphisms, void *stream)
{
    SF_TRY(pp_check(r, d_in, d_out, count));
    const SfPpRing &R = r->R;
    if (gamma < 0 || gamma > R.alpha) return sf_set_error(SF_EINVAL, "sf_pp_trace: gamma must lie in [0, alpha]");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t words = (size_t)count * R.L * R.N;
    if (r->scratch_words < 2 * words) {
        if (r->d_scratch) cudaFree(r->d_scratch);
        r->d_scratch = nullptr;
        r->scratch_words = 0;
        SF_CUDA_TRY(cudaMalloc((void **)&r->d_scratch, sizeof(u64) * 2 * words));
        r->scratch_words = 2 * words;
    }
    u64 *cur = r->d_scratch, *nxt = cur + words;
    std::vector<std::pair<int, int>> steps;
    sf_pp_tower_steps(R, gamma, steps);
    // acc (in d_out) starts as the input; each step: acc <- sum_k tau_h^k(acc)
    SF_CUDA_TRY(cudaMemcpyAsync(d_out, d_in, sizeof(u64) * words, cudaMemcpyDeviceToDevice, st));
    int autos = 0;
    const int grid = (int)std::min<size_t>((words + 255) / 256, 4096);
    for (const auto &s : steps) {
        SF_CUDA_TRY(cudaMemcpyAsync(cur, d_out, sizeof(u64) * words, cudaMemcpyDeviceToDevice, st));
        for (int k = 1; k < s.second; ++k) {
            SF_TRY(pp_auto(r, cur, nxt, count, s.first, st));
            std::swap(cur, nxt);
            k_pp_add<<<grid, 256, 0, st>>>(R, d_out, cur, words);
            SF_CUDA_TRY(cudaGetLastError());
            ++autos;
        }
    }
    if (n_automorphisms) *n_automorphisms = autos;
    return SF_OK;
}

// ------------------------------------------------------ RLWE over Phi_M ----
// Ciphertexts uint64[count][2][L][N]: part 0 = a, part 1 = b = a s + m + e.

// signed integer polynomials [polys][N] -> residues [polys][L][N]
__global__ void k_pp_signed(SfPpRing R, const int64_t *v, u64 *out, int polys)
{
    const size_t total = (size_t)polys * R.L * R.N;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(k % R.N), j = (int)((k / R.N) % R.L);
        const size_t p = k / ((size_t)R.N * R.L);
        const long long x = v[p * R.N + e];
        const u64 q = R.mod[j].q;
        const long long r = x % (long long)q;
        out[k] = r < 0 ? (u64)(r + (long long)q) : (u64)r;
    }
}

// ct[c] = (a[c], prod[c] + m[c] + e[c]); m, e already residues [count][L][N]
__global__ void k_pp_enc_finish(SfPpRing R, const u64 *a, const u64 *prod, const u64 *m, const u64 *e, u64 *ct,
                                int count)
{
    const size_t per = (size_t)R.L * R.N, total = (size_t)count * per;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = k / per, r = k - c * per;
        const u64 q = R.mod[(int)(r / R.N)].q;
        ct[c * 2 * per + r] = a[k];
        ct[c * 2 * per + per + r] = sf_add(sf_add(prod[k], m[k], q), e[k], q);
    }
}

// out = x - y limb-wise; [count][L][N] with x, y at strides sx, sy (words per polynomial)
__global__ void k_pp_sub(SfPpRing R, const u64 *x, size_t sx, const u64 *y, size_t sy, u64 *out, int count)
{
    const size_t per = (size_t)R.L * R.N, total = (size_t)count * per;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const size_t c = k / per, r = k - c * per;
        out[k] = sf_sub(x[c * sx + r], y[c * sy + r], R.mod[(int)(r / R.N)].q);
    }
}

// key for tau_h: kb[i][j] = prod[i][j] + e_i + (Q / q_i mod q_j) ts[j] (mod q_j)
__global__ void k_pp_ksk_finish(SfPpRing R, const u64 *prod, const u64 *e_res, const u64 *ts, u64 *kb)
{
    const size_t per = (size_t)R.L * R.N, total = (size_t)R.L * per;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / per);
        const size_t r = k - (size_t)i * per;
        const int j = (int)(r / R.N);
        const u64 q = R.mod[j].q;
        const u64 *qh = R.qhat + 2 * ((size_t)i * R.L + j);
        kb[k] = sf_add(sf_add(prod[k], e_res[k], q), sf_mul_shoup(ts[r], qh[0], qh[1], q), q);
    }
}

// RNS digits of ta = tau_h(a): d_i = [ta_i (Q/q_i)^-1]_{q_i} (an integer below
// q_i), written as residues modulo every q_j: D[i][j][e]
__global__ void k_pp_digits(SfPpRing R, const u64 *ta, u64 *D)
{
    const size_t per = (size_t)R.L * R.N, total = (size_t)R.L * per;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k / per);
        const size_t r = k - (size_t)i * per;
        const int j = (int)(r / R.N), e = (int)(r % R.N);
        const SfPpMod &Pi = R.mod[i];
        const u64 d = sf_mul_shoup(ta[(size_t)i * R.N + e], Pi.qh_inv, Pi.qh_inv_p, Pi.q);
        D[k] = j == i ? d : sf_reduce(d, R.mod[j].q, R.mod[j].one_p);
    }
}

// out = (-sum_i PA[i], tb - sum_i PB[i]) for one ciphertext
__global__ void k_pp_ks_combine(SfPpRing R, const u64 *PA, const u64 *PB, const u64 *tb, u64 *out)
{
    const size_t per = (size_t)R.L * R.N;
    for (size_t r = (size_t)blockIdx.x * blockDim.x + threadIdx.x; r < per; r += (size_t)gridDim.x * blockDim.x) {
        const u64 q = R.mod[(int)(r / R.N)].q;
        u64 a = 0, b = tb[r];
        for (int i = 0; i < R.L; ++i) {
            a = sf_sub(a, PA[(size_t)i * per + r], q);
            b = sf_sub(b, PB[(size_t)i * per + r], q);
        }
        out[r] = a;
        out[per + r] = b;
    }
}

static int pp_grid(size_t total) { return (int)std::min<size_t>((total + 255) / 256, 8192); }

static sf_status pp_ks_buffer(sf_pp_ring *r, size_t words, u64 **out)
{
    if (r->ks_words < words) {
        if (r->d_ks) cudaFree(r->d_ks);
        r->d_ks = nullptr;
        r->ks_words = 0;
        SF_CUDA_TRY(cudaMalloc((void **)&r->d_ks, sizeof(u64) * words));
        r->ks_words = words;
    }
    *out = r->d_ks;
    return SF_OK;
}

extern "C" sf_status sf_pp_encrypt(sf_pp_ring *r, const int64_t *d_s, const uint64_t *d_a, const int64_t *d_m,
                                   const int64_t *d_e, uint64_t *d_ct, int32_t count, void *stream)
{
    SF_TRY(pp_check(r, d_s, d_a, count));
    if (!d_m || !d_e || !d_ct) return sf_set_error(SF_EINVAL, "sf_pp_encrypt: null buffer");
    const SfPpRing &R = r->R;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)R.L * R.N;
    u64 *buf;
    SF_TRY(pp_ks_buffer(r, per * (1 + 3 * (size_t)count), &buf));
    u64 *S = buf, *prod = S + per, *mr = prod + per * count, *er = mr + per * count;
    k_pp_signed<<<pp_grid(per), 256, 0, st>>>(R, d_s, S, 1);
    k_pp_signed<<<pp_grid(per * count), 256, 0, st>>>(R, d_m, mr, count);
    k_pp_signed<<<pp_grid(per * count), 256, 0, st>>>(R, d_e, er, count);
    k_pp_mul<<<dim3(R.L, count), SF_PP_THREADS, 2 * sizeof(u64) * R.M, st>>>(R, d_a, S, prod, 1);
    k_pp_enc_finish<<<pp_grid(per * count), 256, 0, st>>>(R, d_a, prod, mr, er, d_ct, count);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_pp_decrypt(sf_pp_ring *r, const int64_t *d_s, const uint64_t *d_ct, uint64_t *d_out,
                                   int32_t count, void *stream)
{
    SF_TRY(pp_check(r, d_s, d_ct, count));
    if (!d_out) return sf_set_error(SF_EINVAL, "sf_pp_decrypt: null output");
    const SfPpRing &R = r->R;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)R.L * R.N;
    u64 *buf;
    SF_TRY(pp_ks_buffer(r, per * (1 + 2 * (size_t)count), &buf));
    u64 *S = buf, *a = S + per, *prod = a + per * count;
    k_pp_signed<<<pp_grid(per), 256, 0, st>>>(R, d_s, S, 1);
    // gather the a parts, multiply by s, subtract from the b parts
    for (int c = 0; c < count; ++c)
        SF_CUDA_TRY(cudaMemcpyAsync(a + per * c, d_ct + 2 * per * c, sizeof(u64) * per, cudaMemcpyDeviceToDevice, st));
    k_pp_mul<<<dim3(R.L, count), SF_PP_THREADS, 2 * sizeof(u64) * R.M, st>>>(R, a, S, prod, 1);
    k_pp_sub<<<pp_grid(per * count), 256, 0, st>>>(R, d_ct + per, 2 * per, prod, per, d_out, count);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_pp_ksk(sf_pp_ring *r, const int64_t *d_s, int32_t h, const uint64_t *d_ka, const int64_t *d_e,
                               uint64_t *d_kb, void *stream)
{
    SF_TRY(pp_check(r, d_s, d_ka, 1));
    if (!d_e || !d_kb) return sf_set_error(SF_EINVAL, "sf_pp_ksk: null buffer");
    const SfPpRing &R = r->R;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t per = (size_t)R.L * R.N;
    u64 *buf;
    SF_TRY(pp_ks_buffer(r, per * (2 + 2 * (size_t)R.L), &buf));
    u64 *S = buf, *TS = S + per, *er = TS + per, *prod = er + per * R.L;
    k_pp_signed<<<pp_grid(per), 256, 0, st>>>(R, d_s, S, 1);
    SF_TRY(pp_auto(r, S, TS, 1, h, st));
    k_pp_signed<<<pp_grid(per * R.L), 256, 0, st>>>(R, d_e, er, R.L);
    k_pp_mul<<<dim3(R.L, R.L), SF_PP_THREADS, 2 * sizeof(u64) * R.M, st>>>(R, d_ka, S, prod, 1);
    k_pp_ksk_finish<<<pp_grid(per * R.L), 256, 0, st>>>(R, prod, er, TS, d_kb);
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

// tau_h then the key switch back to s, one ciphertext at a time; `in` and
// `out` may not alias; work: 2 + 3 L polynomials of L limbs
static sf_status pp_keyswitch(sf_pp_ring *r, const u64 *in, u64 *out, int count, int h, const u64 *ka, const u64 *kb,
                              u64 *work, cudaStream_t st)
{
    const SfPpRing &R = r->R;
    const size_t per = (size_t)R.L * R.N;
    u64 *T = work, *D = T + 2 * per, *PA = D + per * R.L, *PB = PA + per * R.L;
    for (int c = 0; c < count; ++c) {
        SF_TRY(pp_auto(r, in + 2 * per * c, T, 2, h, st));
        k_pp_digits<<<pp_grid(per * R.L), 256, 0, st>>>(R, T, D);
        k_pp_mul<<<dim3(R.L, R.L), SF_PP_THREADS, 2 * sizeof(u64) * R.M, st>>>(R, D, ka, PA, R.L);
        k_pp_mul<<<dim3(R.L, R.L), SF_PP_THREADS, 2 * sizeof(u64) * R.M, st>>>(R, D, kb, PB, R.L);
        k_pp_ks_combine<<<pp_grid(per), 256, 0, st>>>(R, PA, PB, T + per, out + 2 * per * c);
    }
    SF_CUDA_TRY(cudaGetLastError());
    return SF_OK;
}

extern "C" sf_status sf_pp_keyswitch(sf_pp_ring *r, const uint64_t *d_ct, uint64_t *d_out, int32_t count, int32_t h,
                                     const uint64_t *d_ka, const uint64_t *d_kb, void *stream)
{
    SF_TRY(pp_check(r, d_ct, d_out, count));
    if (!d_ka || !d_kb || d_ct == d_out) return sf_set_error(SF_EINVAL, "sf_pp_keyswitch: bad key or aliasing");
    const SfPpRing &R = r->R;
    u64 *work;
    SF_TRY(pp_ks_buffer(r, (size_t)R.L * R.N * (2 + 3 * (size_t)R.L), &work));
    return pp_keyswitch(r, d_ct, d_out, count, h, d_ka, d_kb, work, (cudaStream_t)stream);
}

extern "C" sf_status sf_pp_hom_trace(sf_pp_ring *r, const uint64_t *d_ct, uint64_t *d_out, int32_t count,
                                     int32_t gamma, int32_t n_keys, const int32_t *hs, const uint64_t *const *d_kas,
                                     const uint64_t *const *d_kbs, int32_t *n_keyswitches, void *stream)
{
    SF_TRY(pp_check(r, d_ct, d_out, count));
    const SfPpRing &R = r->R;
    if (gamma < 0 || gamma > R.alpha) return sf_set_error(SF_EINVAL, "sf_pp_hom_trace: gamma must lie in [0, alpha]");
    if (n_keys < 0 || (n_keys > 0 && (!hs || !d_kas || !d_kbs)))
        return sf_set_error(SF_EINVAL, "sf_pp_hom_trace: bad key list");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<std::pair<int, int>> steps;
    sf_pp_tower_steps(R, gamma, steps);
    std::vector<int> key_of(steps.size());
    for (size_t k = 0; k < steps.size(); ++k) {
        key_of[k] = -1;
        for (int x = 0; x < n_keys; ++x)
            if (((hs[x] % R.M) + R.M) % R.M == steps[k].first) key_of[k] = x;
        if (key_of[k] < 0) return sf_set_error(SF_EINVAL, "sf_pp_hom_trace: no key for tau_%d", steps[k].first);
    }
    const size_t words = (size_t)count * 2 * R.L * R.N;
    if (r->scratch_words < 2 * words) {
        if (r->d_scratch) cudaFree(r->d_scratch);
        r->d_scratch = nullptr;
        r->scratch_words = 0;
        SF_CUDA_TRY(cudaMalloc((void **)&r->d_scratch, sizeof(u64) * 2 * words));
        r->scratch_words = 2 * words;
    }
    u64 *work;
    SF_TRY(pp_ks_buffer(r, (size_t)R.L * R.N * (2 + 3 * (size_t)R.L), &work));
    u64 *cur = r->d_scratch, *nxt = cur + words;
    SF_CUDA_TRY(cudaMemcpyAsync(d_out, d_ct, sizeof(u64) * words, cudaMemcpyDeviceToDevice, st));
    int ks = 0;
    const int grid = pp_grid(words);
    for (size_t k = 0; k < steps.size(); ++k) {
        SF_CUDA_TRY(cudaMemcpyAsync(cur, d_out, sizeof(u64) * words, cudaMemcpyDeviceToDevice, st));
        for (int x = 1; x < steps[k].second; ++x) {
            SF_TRY(pp_keyswitch(r, cur, nxt, count, steps[k].first, d_kas[key_of[k]], d_kbs[key_of[k]], work, st));
            std::swap(cur, nxt);
            k_pp_add<<<grid, 256, 0, st>>>(R, d_out, cur, words);
            SF_CUDA_TRY(cudaGetLastError());
            ++ks;
        }
    }
    if (n_keyswitches) *n_keyswitches = ks;
    return SF_OK;
}
