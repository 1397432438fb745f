// sf_internal.h -- library-internal types shared by the host and device code.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/safhire.h"
#include "sf_arith.cuh"

#define SF_MAX_DIGITS 8

// Rows per row tile of the two-pass NTT: 16, 8 for 256-point rows, 4 for
// 512-point rows, so a row tile holds at most 2048 residues (8 per thread of
// a 256-thread block).
SF_HD int sf_row_nb(int log_c) { return log_c >= 9 ? 4 : (log_c >= 8 ? 8 : 16); }

// Per-modulus constants, passed to kernels by value (kernel parameter space).
struct SfMod {
    u64 q, two_q;
    u64 qinv_neg;      // -q^-1 mod 2^64 (Montgomery)
    u64 r_mod;         // 2^64 mod q (to Montgomery form via Shoup)
    u64 r_mod_p;
    u64 ninv, ninv_p;  // N^-1 mod q (Shoup)
    u64 one_p;         // floor(2^64 / q): Shoup companion of 1 (full reduction)
};

// Everything a kernel needs about the ring, by value.
struct SfRing {
    int log_n, n, log_r, r, log_c, c;
    int L, K, nm, dnum;
    // every modulus is below 4x every other one: a one-limb digit's ModUp
    // (its residue itself, Qhat = 1) is a valid lazy input of the forward NTT
    // modulo any other modulus, with no reduction
    int modup_copy;
    SfMod m[SF_MAX_MODULI];
    // twiddle tables, [nm][N] each (index 0 unused)
    const u64 *psi, *psi_p, *ipsi, *ipsi_p;
    // staged twiddle pairs (w, w'): column tables [nm][R] (k < R) and row
    // tables [nm][R/16][C][16] reordered per 16-row tile (see sf_tile.cuh)
    const ulonglong2 *colT_f, *colT_i, *rowT_f, *rowT_i;
    // powers psi^k, k in [0, 2N), [nm][2N] (monomials in the NTT domain)
    const u64 *pw, *pw_p;
    // pairs (psi^(C e), companion), e < 2R, [nm][2R] (sparse column pass)
    const ulonglong2 *pwc;
    // ModUp: for digit j, limb i in the digit: N^-1 (Qhat_i mod q_i)^-1 with
    //        Shoup (N^-1 finishes the inverse NTT); Qhat_i mod m for every m.
    const u64 *mu_inv, *mu_inv_p;   // [dnum][K]
    const u64 *mu_qhat, *mu_qhat_p; // [dnum][K][nm]
    // ModDown: N^-1 (Phat_k mod p_k)^-1; Phat_k P^-1 mod q_i (the conversion
    // carries the final factor P^-1); P^-1 mod q_i (all Shoup)
    const u64 *md_inv, *md_inv_p;   // [K]
    const u64 *md_phat, *md_phat_p; // [K][L]
    const u64 *md_pinv, *md_pinv_p; // [L]
    int *status;                    // device status word (first latched error)
};

struct sf_params {
    int log_n, n, L, K, dnum;
    int data_bits, special_bits;
    double sigma;
    std::vector<u64> mods;  // q_0..q_{L-1}, p_0..p_{K-1}
};

struct KernelStat {
    const char *name;
    int64_t launches;
    double ms;
};

struct PendingEvent {
    int kind;
    cudaEvent_t a, b;
};

// A captured launch sequence of one layer round, replayed with one launch.
struct SfGraphEntry {
    uint64_t key[12];
    cudaGraphExec_t exec;
    std::vector<int64_t> launches;   // per kernel family, for the counters
};

struct sf_ctx {
    const sf_params *prm;
    int device;
    int num_sms;
    SfRing ring;
    // owned device allocations for the tables
    std::vector<void *> owned;
    // scratch pool
    void *scratch;
    size_t scratch_bytes;
    // device staging for the host-buffer round
    void *io_buf;
    size_t io_bytes;
    // options
    int ks_batch;
    int leaf_chunk;
    int leaf_sparse;          // taps per column tile up to which the leaf column pass uses the closed form (-1: default rule)
    int ks3_threads;          // block size of the key-switch inner product for 128-point rows (256 or 512)
    int row_radix;            // row-pass sweep schedule of the key-switch and leaf row kernels: 0 radix-8, 1 radix-4, 2 radix-8 with warp-shuffle exchanges
    size_t mem_budget;        // bytes of leaf + tree buffers a round may use
    int use_graph;
    int kernel_timing;
    // instrumentation
    std::vector<KernelStat> stats;
    std::vector<PendingEvent> pending;
    std::vector<cudaEvent_t> event_pool;
    int *d_status;
    std::vector<SfGraphEntry> graphs;
};

void sf_graph_cache_clear(sf_ctx *ctx);
uint64_t sf_next_generation();

struct sf_secret_key {
    sf_ctx *ctx;
    std::vector<int64_t> s;   // host copy of s(X)
    u64 *d_s_mont;            // [nm][N] NTT domain, Montgomery form
};

struct sf_rotkeys {
    sf_ctx *ctx;
    uint64_t gen;             // unique per handle (graph cache key)
    std::vector<int32_t> d;   // automorphism indices
    u64 *d_keys;              // per key: [dnum][2][nm][N] NTT-domain values, then their Shoup companions
    size_t key_words;         // words per key
};

struct sf_layer {
    sf_ctx *ctx;
    uint64_t gen;             // unique per handle (graph cache key)
    std::vector<sf_conv_term> terms;
    int E_in, E_out, H_out, W_out, C_out;
    int max_taps;             // upper bound of taps per output
    std::vector<int64_t> wq;  // host copy, concatenated per term [C_out][kh][kw][C_in]
    std::vector<int64_t> bq;  // quantised bias per output channel (empty = none)
    int64_t *d_wq;            // device copy of the quantised weights
    int64_t *d_bq;            // device copy of the bias (or null)
    sf_conv_term *d_terms;
    // per term, per tap t = (dh kw + dw) C_in + ci: {dh, dw, (dh W + dw) C_in + ci, t}
    int4 *d_taps;
    std::vector<int> tap_off; // first tap of each term in d_taps
};

// ------------------------------------------------------------------ errors --

sf_status sf_set_error(sf_status st, const char *fmt, ...);

#define SF_CUDA_TRY(call)                                                                 \
    do {                                                                                  \
        cudaError_t err__ = (call);                                                       \
        if (err__ != cudaSuccess)                                                         \
            return sf_set_error(SF_ECUDA, "%s failed: %s (%s:%d)", #call,                \
                                cudaGetErrorString(err__), __FILE__, __LINE__);           \
    } while (0)

#define SF_TRY(expr)                       \
    do {                                   \
        sf_status st__ = (expr);           \
        if (st__ != SF_OK) return st__;    \
    } while (0)

// --------------------------------------------------------- host utilities --

u64 sf_host_powmod(u64 a, u64 e, u64 q);
u64 sf_host_invmod(u64 a, u64 q);
u64 sf_host_mulmod(u64 a, u64 b, u64 q);
u64 sf_shoup_companion(u64 w, u64 q);
int sf_find_primes(u64 two_n, int bits, int count, u64 *out);
u64 sf_root_2n(u64 q, u64 two_n);

// SplitMix64 stream with Lemire bounded draws and a rounded Box-Muller Gaussian.
struct SfRng {
    u64 state;
    explicit SfRng(u64 seed) : state(seed) {}
    u64 next();
    u64 below(u64 n);
    int64_t gauss(double sigma);
};

// ------------------------------------------------------ kernel launchers --

enum SfKernelKind {
    SFK_NTT_FWD_COL = 0,
    SFK_NTT_FWD_ROW,
    SFK_NTT_INV_ROW,
    SFK_NTT_INV_COL,
    SFK_ELEMWISE,
    SFK_KS_GATHER,
    SFK_KS1_INV_ROW,
    SFK_KS2_MODUP_COL,
    SFK_KS3_INNER_ROW,
    SFK_KS3_INV_ROW_P,
    SFK_KS4_MODDOWN_COL,
    SFK_KS5_FINISH_ROW,
    SFK_LEAF_COL,
    SFK_LEAF_ROW,
    SFK_SHUFFLE,
    SFK_BNTT_COL,
    SFK_BNTT_ROW,
    SFK_LEAF_PREP,
    SFK_COUNT
};

const char *sf_kernel_name(int kind);

// Bracket a launch with events when timing is on; always counts the launch.
void sf_launch_begin(sf_ctx *ctx, int kind, cudaStream_t st, cudaEvent_t *ev0);
void sf_launch_end(sf_ctx *ctx, int kind, cudaStream_t st, cudaEvent_t ev0);
sf_status sf_collect_timings(sf_ctx *ctx);

sf_status sf_scratch(sf_ctx *ctx, size_t bytes, void **out);

// Batched full transforms over a list of polynomials (non-hot-path uses).
struct SfPolyJob {
    const u64 *src;
    u64 *dst;
    int mod;
};
sf_status sf_ntt_jobs(sf_ctx *ctx, const SfPolyJob *h_jobs, int n_jobs, bool inverse, cudaStream_t st);
// dynamic shared memory: staged twiddles + `tiles` data tiles (sf_tile.cuh)
size_t sf_smem_col(const SfRing &R, int tiles);
size_t sf_smem_row(const SfRing &R, int tiles);

// Elementwise helpers (sf_ntt.cu).  Polynomial t uses modulus offset + t % period.
sf_status sf_to_mont(sf_ctx *ctx, u64 *d, int n_polys, int period, int offset, cudaStream_t st);
sf_status sf_from_mont(sf_ctx *ctx, u64 *d, int n_polys, int period, int offset, cudaStream_t st);
sf_status sf_pointwise_mul(sf_ctx *ctx, const u64 *a, const u64 *b, u64 *out, int n_polys, int period, int offset,
                           cudaStream_t st);
sf_status sf_mul_secret(sf_ctx *ctx, const u64 *a, const u64 *s_mont, u64 *out, int n_polys, int period,
                        cudaStream_t st);
sf_status sf_encrypt_finish(sf_ctx *ctx, const u64 *p, const int64_t *m, const int64_t *e, u64 *cts, int n_cts,
                            cudaStream_t st);
sf_status sf_decrypt_finish(sf_ctx *ctx, const u64 *cts, const u64 *p, u64 *out, int n_cts, cudaStream_t st);
sf_status sf_signed_to_residues(sf_ctx *ctx, const int64_t *v, u64 *out, int n_polys, int period, int offset,
                                cudaStream_t st);
sf_status sf_rotkey_finish(sf_ctx *ctx, const u64 *alpha, const u64 *e, const u64 *s_mont, const u64 *pg, int d,
                           u64 *key_a, u64 *key_b, size_t comp, cudaStream_t st);
// device-side range check of caller input: latches SF_ERANGE in the status
// word (reported by sf_sync) if a residue of poly t is >= modulus offset + t % period
sf_status sf_check_residues(sf_ctx *ctx, const u64 *x, int n_polys, int period, int offset, cudaStream_t st);
// Shoup companions floor(x 2^64 / q) of residues x (poly t uses modulus offset + t % period)
sf_status sf_companions(sf_ctx *ctx, const u64 *x, u64 *dst, int n_polys, int period, int offset, cudaStream_t st);

// Raise the dynamic shared-memory limit of every kernel (once per device).
sf_status sf_ntt_init_attributes();
sf_status sf_bntt_init_attributes();
sf_status sf_ks_init_attributes();
sf_status sf_layer_init_attributes();
