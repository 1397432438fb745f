/*
 * safhire.h -- C ABI of the GB300 (sm_103a) implementation of the server side
 * of one Safhire round (arXiv 2509.01253): a network's linear layer evaluated
 * as plaintext-weight x RLWE-ciphertext products on RNS ciphertexts, followed
 * by the secret output shuffle and fast packing, with no bootstrapping.
 *
 * Conventions (every entry point):
 *  - Returns sf_status (SF_OK = 0).  On failure a human-readable message is
 *    kept per thread; read it with sf_last_error().  No exception crosses the ABI.
 *  - Handles (sf_params, sf_ctx, sf_secret_key, sf_rotkeys, sf_layer) are
 *    owned by the library; free them with the matching *_destroy.
 *  - Buffers named d_* are CALLER-owned device pointers, h_* are caller-owned
 *    host pointers.  The library never frees them and keeps no reference
 *    after the call returns (device work it enqueued may still read them until
 *    the stream reaches that point).
 *  - Residues are uint64 words in [0, q) for every modulus (30- and 50-bit
 *    primes alike).  A ciphertext is uint64[2][L][N]: part 0 is the mask a,
 *    part 1 is b = a*s + m + e (Sec. 2.1 sign convention), limb-major, natural
 *    coefficient order.  Arrays of ciphertexts are uint64[count][2][L][N].
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device work is enqueued on it and may still be running when a
 *    call returns, unless the call writes a host buffer (then it synchronises
 *    the stream before returning).  Errors detected on the device are latched
 *    in a device status word that sf_sync() reports.
 *  - Nothing here falls back to the CPU: without a usable CUDA device every
 *    device entry point fails with SF_ECUDA.
 *
 * Parameters: t = 2 instance of the paper's prime-power cyclotomic ring
 * (M = 2N, N = phi(M) a power of two, Sec. 2.1), RNS modulus Q = prod q_i of
 * L data primes plus P = prod p_k of K special primes for hybrid key
 * switching; all primes are 1 mod 2N.  Key-switch digits are consecutive
 * groups of K data limbs, dnum = ceil(L / K).  The sf_pp_* calls at the end
 * work over the prime-power rings M = t^alpha with t an odd prime.
 */
#ifndef SAFHIRE_H
#define SAFHIRE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------ */
/* status                                                                    */
/* ------------------------------------------------------------------------ */

typedef int32_t sf_status;

#define SF_OK 0
#define SF_EINVAL 1   /* invalid argument: null pointer, size or index out of range, unknown key */
#define SF_ENOMEM 2   /* host or device allocation failed, or a memory budget was exceeded */
#define SF_ECUDA 3    /* a CUDA runtime call failed, or no usable device */
#define SF_ERANGE 6   /* a value does not fit the requested representation, or (latched on the
                         device, see sf_sync) an input residue is not below its modulus */
#define SF_ENOTSUP 8  /* valid request that this library does not implement */
/* (codes 4, 5 and 7 are not used) */

/* Copies the calling thread's last error message into buf (always
 * NUL-terminated when len > 0) and returns the status that set it. */
sf_status sf_last_error(char *buf, size_t len);

/* Library version string (static storage). */
const char *sf_version(void);

/* ------------------------------------------------------------------------ */
/* parameters (host only)                                                    */
/* ------------------------------------------------------------------------ */

typedef struct sf_params sf_params;

/* Sec. 2.1, Table 2 (parameter roles).  Ring degree N = 2^log_n with
 * 10 <= log_n <= 16.  n_data (1..8) data primes of data_bits bits and
 * n_special (1..4) special primes of special_bits bits, 20 <= bits <= 50.
 * Primes: the largest primes below 2^bits that are 1 mod 2N, in descending
 * order; when data_bits == special_bits the first n_special found are the
 * special primes and the next n_data the data primes.  sigma: standard
 * deviation of the rounded Gaussian noise.  Errors: SF_EINVAL for values
 * out of range, SF_ENOMEM. */
sf_status sf_params_create(int32_t log_n, int32_t n_data, int32_t data_bits, int32_t n_special,
                           int32_t special_bits, double sigma, sf_params **out);
void sf_params_destroy(sf_params *p);

#define SF_MAX_MODULI 12
typedef struct {
    int32_t log_n;
    int32_t n;          /* N */
    int32_t n_data;     /* L */
    int32_t n_special;  /* K */
    int32_t dnum;       /* key-switch digits, ceil(L / K) */
    double sigma;
    uint64_t moduli[SF_MAX_MODULI]; /* q_0..q_{L-1}, then p_0..p_{K-1} */
} sf_params_info;

sf_status sf_params_get_info(const sf_params *p, sf_params_info *out);

/* ------------------------------------------------------------------------ */
/* context: one per (params, device)                                         */
/* ------------------------------------------------------------------------ */

typedef struct sf_ctx sf_ctx;

/* Uploads the NTT, base-conversion and automorphism tables to `device` and
 * makes that device current for every later call on this context.  The
 * params handle must outlive the context.  Errors: SF_EINVAL, SF_ECUDA,
 * SF_ENOMEM. */
sf_status sf_ctx_create(const sf_params *p, int32_t device, sf_ctx **out);
void sf_ctx_destroy(sf_ctx *ctx);

/* Tuning and instrumentation knobs (name, value):
 *   "ks_batch"      merges per key-switch batch (1..4096; default chosen per N)
 *   "leaf_sparse"   taps per 16-column tile up to which the leaf column pass
 *                   evaluates the sparse weight polynomial in closed form
 *                   instead of running the transform (-1: 8 log2 R, where the
 *                   closed form has fewer multiplications; 0: always the
 *                   transform, the default; at most 128)
 *   "ks3_threads"   threads per block of the key-switch inner product when
 *                   the NTT's rows have 128 points (N = 2^13, 2^14): 256
 *                   (8 residues per thread, the default) or 512 (4 per
 *                   thread, radix-4 row sweeps)
 *   "row_radix"     sweep schedule of the row passes of the key-switch and
 *                   leaf kernels: 0 radix-8 sweeps (the default), 1 radix-4
 *                   sweeps, 2 radix-8 sweeps with the two sweeps nearest
 *                   the rows' short butterflies of 256- and 512-point rows
 *                   run back to back in registers, the lanes of a warp
 *                   trading values by shuffles in between (other row
 *                   lengths as 0); every schedule gives identical residues
 *   "leaf_chunk"    cap on the leaves per packing unit (power of two): a group
 *                   of n leaves is packed as n/CH residue classes of CH leaves
 *                   reduced to roots, then the roots finish the tree
 *   "mem_budget"    bytes of leaf and pack-tree buffers one round may hold
 *                   (default 64 GiB); larger layers are packed group by group,
 *                   and groups larger than the budget in chunks of leaves
 *   "use_graph"     1 = capture a layer's launch sequence in a CUDA graph and
 *                   replay it (default 1), 0 = launch directly
 *   "kernel_timing" 1 = bracket every launch with CUDA events on its stream
 *                   and accumulate per-kernel times (read with sf_kernel_stats)
 * Errors: SF_EINVAL for an unknown name or value. */
sf_status sf_ctx_set_option(sf_ctx *ctx, const char *name, int64_t value);

/* Reads the current value of one of the options above that holds a value
 * ("ks_batch", "ks3_threads", "leaf_sparse", "row_radix", "leaf_chunk",
 * "mem_budget", "use_graph", "kernel_timing"), e.g. after sf_autotune_layers.  Errors:
 * SF_EINVAL for a null argument or an unknown name. */
sf_status sf_ctx_get_option(const sf_ctx *ctx, const char *name, int64_t *value);

/* Waits for `stream`, then reports (and clears) the context's device status
 * word: SF_OK, or the first error a kernel latched since the last sf_sync.
 * The one device-side check: sf_eval_linear_layer(_host), sf_eval_layers,
 * sf_autotune_layers, sf_linear_outputs and sf_rotate read the caller's input
 * ciphertexts once more to check that every residue is below its modulus;
 * if one is not, SF_ERANGE is latched (the call itself returned SF_OK, and
 * the outputs it wrote are unspecified). */
sf_status sf_sync(sf_ctx *ctx, void *stream);

/* Per-kernel counters since the last reset: for each kernel family, the
 * number of launches and (when kernel_timing is on) the summed device time.
 * names/launches/ms are arrays of `cap` entries; *count receives the number
 * of families (at most cap are written).  Names are static strings. */
sf_status sf_kernel_stats(sf_ctx *ctx, const char **names, int64_t *launches, double *ms,
                          int32_t cap, int32_t *count);
sf_status sf_kernel_stats_reset(sf_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* keys, encryption, decryption (client side; used by tests and the bench)  */
/* ------------------------------------------------------------------------ */

typedef struct sf_secret_key sf_secret_key;
typedef struct sf_rotkeys sf_rotkeys;

/* Sec. 2.1 / Sec. 4.2: secret key s(X) with N coefficients uniform in
 * {-1, 0, 1}, drawn from SplitMix64(seed) with Lemire's bounded draw.  The
 * key stays resident on the context's device.  Errors: SF_ECUDA, SF_ENOMEM. */
sf_status sf_keygen(sf_ctx *ctx, uint64_t seed, sf_secret_key **out);
void sf_secret_key_destroy(sf_secret_key *sk);
/* Copies s(X) to h_s (int64[N]). */
sf_status sf_secret_key_export(const sf_secret_key *sk, int64_t *h_s);

/* Sec. 4.2: key-switching keys for the automorphisms X -> X^d, one per entry
 * of d[0..nd-1] (odd, 1 < d < 2N); d = NULL / nd = 0 selects the set the
 * packing needs, {2^k + 1 : 1 <= k <= log2 N}.  Key for d, digit j:
 * (alpha_j, alpha_j*s + e_j - P*g_j*s(X^d)) mod PQ, g_j the CRT gadget of
 * digit j.  Randomness: SplitMix64 stream seeded with seed XOR d*0x9E3779B97F4A7C15;
 * per digit alpha over the L+K moduli then e.  Keys stay resident on the
 * device until destroyed.  Errors: SF_EINVAL (bad d), SF_ECUDA, SF_ENOMEM. */
sf_status sf_gen_rotation_keys(sf_ctx *ctx, const sf_secret_key *sk, const int32_t *d, int32_t nd,
                               uint64_t seed, sf_rotkeys **out);
void sf_rotkeys_destroy(sf_rotkeys *rk);
/* Copies the key for d to h_key, uint64[dnum][2][L+K][N], coefficient
 * domain (tests compare it with an independent implementation). */
sf_status sf_rotkeys_export(sf_ctx *ctx, const sf_rotkeys *rk, int32_t d, uint64_t *h_key);

/* Fixed-point encoding of inputs: out[i] = round(scale * x[i]), half away
 * from zero.  Errors: SF_ERANGE if a result does not fit int64. */
sf_status sf_encode_input(const double *x, int64_t count, double scale, int64_t *out);

/* Client side, Sec. 4.3 "Power computations" at t = 2: for each of n_cts
 * chunks of N integer message coefficients (h_msg: int64[n_cts][N]) writes
 * m(X^d) mod X^N + 1 to h_out (same shape; d odd and positive, so every
 * output coefficient is plus or minus one input coefficient).  d = 3 gives
 * the power the client encrypts for gamma = 2.  Errors: SF_EINVAL (bad
 * arguments, even d), SF_ERANGE (a coefficient equal to INT64_MIN). */
sf_status sf_client_power(const sf_params *p, const int64_t *h_msg, int32_t n_cts, int32_t d, int64_t *h_out);

/* Sec. 4.3 "Flatten and chunk" + Sec. 2.1: encrypts h_msg[0..count) (int64,
 * count <= n_cts * N, zero-padded) into n_cts ciphertexts at d_cts
 * (uint64[n_cts][2][L][N]).  Randomness: one SplitMix64(seed) stream, per
 * ciphertext the mask a limb by limb (Lemire draw mod q_i) then the error
 * (rounded Box-Muller Gaussian, sigma).  Errors: SF_EINVAL, SF_ECUDA. */
sf_status sf_encrypt(sf_ctx *ctx, const sf_secret_key *sk, const int64_t *h_msg, int64_t count,
                     uint64_t seed, uint64_t *d_cts, int32_t n_cts, void *stream);

/* Sec. 2.1 decryption without the final projection: h_residues receives
 * b - a*s mod q_i, uint64[n_cts][L][N].  Synchronises `stream`. */
sf_status sf_decrypt(sf_ctx *ctx, const sf_secret_key *sk, const uint64_t *d_cts, int32_t n_cts,
                     uint64_t *h_residues, void *stream);

/* Sec. 4.5 client read-out: CRT of the residues (uint64[n_cts][L][N]) to the
 * centred integer in (-Q/2, Q/2], divided by scale.  Value v is read from
 * ciphertext v / (N/stride) at coefficient (v mod (N/stride)) * stride, for
 * v < count.  Errors: SF_EINVAL if count exceeds n_cts * N / stride. */
sf_status sf_decode(const sf_params *p, const uint64_t *h_residues, int32_t n_cts, int32_t stride,
                    int32_t count, double scale, double *out);

/* ------------------------------------------------------------------------ */
/* linear layers                                                             */
/* ------------------------------------------------------------------------ */

/* One linear term of a layer (Sec. 4.4 "Convolution"; Sec. 5 f(x) = Ax + b):
 * a convolution over the input segment of H x W x C_in values (row-major,
 * channels last, Sec. 4.3) that starts at flat index in_offset of the layer
 * input.  Output H' x W' x C_out with H' = (H + 2 pad - kh) / stride + 1.
 * A fully connected layer is H = W = kh = kw = 1; global-average-pooled FC is
 * a kernel as large as its input; a residual shortcut is a second term over
 * its own input segment (all terms must agree on H', W', C_out). */
typedef struct {
    int32_t in_offset;
    int32_t H, W, C_in;
    int32_t C_out;
    int32_t kh, kw;
    int32_t stride, pad;
} sf_conv_term;

typedef struct sf_layer sf_layer;

/* Quantises and uploads the weights: Wq = round(weight_scale * W) for every
 * term (W: float64, per term [C_out][kh][kw][C_in], terms concatenated), and
 * the optional bias (float64[C_out], NULL = none) as round(bias_scale * b).
 * The quantised integers stay resident on the device.  Errors: SF_EINVAL
 * (geometry), SF_ERANGE (|Wq| >= 2^62), SF_ENOMEM, SF_ECUDA. */
sf_status sf_encode_weights(sf_ctx *ctx, const sf_conv_term *terms, int32_t n_terms, const double *W,
                            const double *bias, double weight_scale, double bias_scale,
                            sf_layer **out);
void sf_layer_destroy(sf_layer *layer);

typedef struct {
    int32_t E_in;        /* flattened input values */
    int32_t E_out;       /* outputs E' */
    int32_t k_in;        /* input ciphertexts ceil(E_in / N) */
    int32_t group_size;  /* n = min(N/2, next power of two >= E') values per packed ciphertext */
    int32_t n_groups;    /* packed output ciphertexts ceil(E' / n) */
    int64_t ks_count;    /* key switches of the paper's algorithm: groups * ((n-1) + log2(N/n)) */
} sf_layer_info;

sf_status sf_layer_get_info(const sf_ctx *ctx, const sf_layer *layer, sf_layer_info *out);

/* The server round for one linear layer (Sec. 4.4, steps 6-10, gamma = 0):
 *   6 extraction: the row of stream position p = jN + k is N^-1 X^-k ct_j;
 *   7 unshuffle: input index i sits at position sigma_prev^-1(i)
 *     (h_sigma_prev: uint32[E_in], position -> index; NULL = identity, the
 *     first round);
 *   8 linear layer: y_o = sum_i Wq[o,i] * row(i), evaluated exactly as
 *     sum_j w_{o,j}(X) * ct_j with the weight polynomial w_{o,j};
 *   9 shuffle: leaf l of group g is y_{sigma_out(g n + l)} (h_sigma_out:
 *     uint32[E_out]; NULL = no shuffle, the last layer, Sec. 5);
 *  10 fast packing: PackLWEs tree over the n leaves of each group (padding
 *     leaves are zero), then the field trace; packed value l sits at
 *     coefficient l*N/n of output ciphertext g, times Wq*x scale; the bias
 *     (if any) is added there.
 * d_in: uint64[k_in][2][L][N]; d_out: uint64[out_capacity][2][L][N].
 * *n_out receives the number of packed ciphertexts written.  The result is
 * bit-identical to the paper's algorithm evaluated literally.
 * Errors: SF_EINVAL (k_in mismatch, capacity too small, missing key, bad
 * permutation), SF_ENOMEM, SF_ECUDA. */
sf_status sf_eval_linear_layer(sf_ctx *ctx, const sf_layer *layer, const sf_rotkeys *rk,
                               const uint64_t *d_in, int32_t k_in, const uint32_t *h_sigma_prev,
                               const uint32_t *h_sigma_out, uint64_t *d_out, int32_t out_capacity,
                               int32_t *n_out, void *stream);

/* The same round at partial trace extraction level gamma (Sec. 4.3, 4.4,
 * Lemma 1 at t = 2, where K_1 = K_0).  gamma 0 or 1: identical to
 * sf_eval_linear_layer (d_powers must be NULL).  gamma 2: d_powers holds the
 * client's powers, uint64[k_in][2][L][N], chunk j an encryption under the same
 * secret of m_j(X^3) (sf_client_power with d = 3); the row of position
 * p = jN + k is (N/2)^-1 (X^-k ct_j + X^-3k ct3_j), Lemma 1's sum over the
 * automorphisms {1, 3} scaled by [K_2 : K_0] = 2, and the packing skips the
 * tau_3 level: the bottom level of every tree merges E + X^(N/2) O with no key
 * switch (the field trace starts at k = 2 when a group holds one value), so a
 * group of n values costs n/2 - 1 + log2(N/n) key switches instead of
 * n - 1 + log2(N/n).  The packed values (and the bias added there) carry the
 * factor 2 = [K_2 : K_0]: the client halves them after decryption (output
 * scale 2 S).  Leaves read 2 k_in ciphertexts, so the linear step costs twice
 * its gamma = 0 work.  Errors: those of sf_eval_linear_layer, and SF_EINVAL for
 * gamma outside [0, 2], missing powers at gamma = 2 or powers at gamma < 2. */
sf_status sf_eval_linear_layer_gamma(sf_ctx *ctx, const sf_layer *layer, const sf_rotkeys *rk, int32_t gamma,
                                     const uint64_t *d_in, const uint64_t *d_powers, int32_t k_in,
                                     const uint32_t *h_sigma_prev, const uint32_t *h_sigma_out, uint64_t *d_out,
                                     int32_t out_capacity, int32_t *n_out, void *stream);

/* Same round with HOST buffers: copies h_in to the device, evaluates, and
 * copies the packed ciphertexts back to h_out (uint64[out_capacity][2][L][N]).
 * Synchronises `stream`.  Pinned host memory gives the fastest copies. */
sf_status sf_eval_linear_layer_host(sf_ctx *ctx, const sf_layer *layer, const sf_rotkeys *rk,
                                    const uint64_t *h_in, int32_t k_in, const uint32_t *h_sigma_prev,
                                    const uint32_t *h_sigma_out, uint64_t *h_out, int32_t out_capacity,
                                    int32_t *n_out, void *stream);

/* Several rounds at once (batching of uneven layers): round x evaluates
 * layers[x] with rks[x] on d_ins[x] (k_ins[x] ciphertexts) into d_outs[x],
 * exactly as sf_eval_linear_layer would, each result bit-identical to the
 * single call.  The layers' packing groups of equal size share their
 * key-switch launches (one batch per tree level across all layers), and the
 * whole launch sequence is captured once into one CUDA graph and replayed.
 * h_sigma_prevs / h_sigma_outs may be NULL (no shuffles at all) or hold NULL
 * entries.  n_outs[x] (may be NULL) receives the packed ciphertexts of round x.
 * Errors: as sf_eval_linear_layer, for the first offending round. */
sf_status sf_eval_layers(sf_ctx *ctx, int32_t n_layers, const sf_layer *const *layers, const sf_rotkeys *const *rks,
                         const uint64_t *const *d_ins, const int32_t *k_ins, const uint32_t *const *h_sigma_prevs,
                         const uint32_t *const *h_sigma_outs, uint64_t *const *d_outs, const int32_t *out_capacities,
                         int32_t *n_outs, void *stream);

/* sf_eval_layers with partial trace extraction per round (Sec. 4.3, 4.4):
 * d_powers NULL evaluates every round at gamma = 0 (exactly sf_eval_layers);
 * otherwise round x runs at gamma = 2 when d_powers[x] is non-NULL (the
 * client's powers RLWE(m_j(X^3)), uint64[k_ins[x]][2][L][N], as in
 * sf_eval_linear_layer_gamma) and at gamma = 0 when it is NULL.  Rounds of the
 * two kinds never share tree levels (the gamma = 2 bottom level has no key
 * switch).  Each result is bit-identical to the single-round call.
 * Errors: those of sf_eval_layers. */
sf_status sf_eval_layers_gamma(sf_ctx *ctx, int32_t n_layers, const sf_layer *const *layers,
                               const sf_rotkeys *const *rks, const uint64_t *const *d_ins,
                               const uint64_t *const *d_powers, const int32_t *k_ins,
                               const uint32_t *const *h_sigma_prevs, const uint32_t *const *h_sigma_outs,
                               uint64_t *const *d_outs, const int32_t *out_capacities, int32_t *n_outs, void *stream);

/* Autotuner: times sf_eval_layers on the given rounds (which it evaluates,
 * results valid), `repeats` timed runs per candidate after a warm-up:
 * first each key-switch launch batch (32 ... 4096 merges; those above 512
 * only while their key-switch workspace stays within 16 GiB), then, with the
 * best batch, the leaf column pass of sparse tiles in closed form or as a
 * transform ("leaf_sparse" -1 or 0), then, for rings with 128-point rows,
 * the block shape of the key-switch inner product ("ks3_threads" 256 or
 * 512), then the row-pass schedule ("row_radix" 0, 1, 2).  Keeps the
 * fastest choices in the context and reports the batch with the best time
 * in milliseconds.
 * Synchronises `stream`. */
sf_status sf_autotune_layers(sf_ctx *ctx, int32_t n_layers, const sf_layer *const *layers, const sf_rotkeys *const *rks,
                             const uint64_t *const *d_ins, const int32_t *k_ins, const uint32_t *const *h_sigma_prevs,
                             const uint32_t *const *h_sigma_outs, uint64_t *const *d_outs, const int32_t *out_capacities,
                             int32_t repeats, int32_t *best_ks_batch, double *best_ms, void *stream);

/* Steps 6-8 only, for selected outputs: d_out[t] = y_{outputs[t]} (the RLWE
 * row of that output before shuffling and packing), coefficient domain,
 * uint64[n_outputs][2][L][N].  Errors: SF_EINVAL for an output index out of
 * range. */
sf_status sf_linear_outputs(sf_ctx *ctx, const sf_layer *layer, const uint64_t *d_in, int32_t k_in,
                            const uint32_t *h_sigma_prev, const int32_t *h_outputs, int32_t n_outputs,
                            uint64_t *d_out, void *stream);

/* ------------------------------------------------------------------------ */
/* building blocks                                                           */
/* ------------------------------------------------------------------------ */

/* Sec. 2.2: for each of `count` ciphertexts, apply X -> X^d to a and b
 * (RLWE under s(X^d)) and key-switch back to s(X) with the hybrid gadget:
 * out = (ModDown(sum_j c_j alpha_j), tau_d(b) + ModDown(sum_j c_j b_j)),
 * c_j = ModUp of digit j of tau_d(a).  d_ct, d_out: uint64[count][2][L][N]
 * (may not overlap).  Errors: SF_EINVAL if rk holds no key for d. */
sf_status sf_rotate(sf_ctx *ctx, const sf_rotkeys *rk, int32_t d, const uint64_t *d_ct, uint64_t *d_out,
                    int32_t count, void *stream);

/* Sec. 2.4 / Sec. 4.4 "Fast Packing" at t = 2: packs n_leaves ciphertexts
 * (zero-padded to n, a power of two with n_leaves <= n <= N/2) into one
 * ciphertext whose coefficient l*N/n is N times coefficient 0 of leaf l; all
 * other coefficients are cleared by the field trace.  Uses (n - 1) + log2(N/n)
 * key switches.  d_leaves: uint64[n_leaves][2][L][N]; d_out: uint64[2][L][N]. */
sf_status sf_pack(sf_ctx *ctx, const sf_rotkeys *rk, const uint64_t *d_leaves, int32_t n_leaves, int32_t n,
                  uint64_t *d_out, void *stream);

/* sf_pack at partial trace extraction level gamma (Sec. 4.4 "Fast Packing"):
 * gamma 0 and 1 are sf_pack; gamma 2 expects leaves that encrypt
 * y + tau_3(y) (rows extracted at gamma = 2) and merges the tau_3 level with
 * no key switch (n/2 fewer key switches, one fewer when n = 1); coefficient
 * l*N/n of the result then holds N times coefficient 0 of y_l.
 * Errors: those of sf_pack, SF_EINVAL for gamma outside [0, 2]. */
sf_status sf_pack_gamma(sf_ctx *ctx, const sf_rotkeys *rk, const uint64_t *d_leaves, int32_t n_leaves, int32_t n,
                        int32_t gamma, uint64_t *d_out, void *stream);

/* Sec. 4.4 "Partial trace extraction" (Lemma 1) at t = 2: the RLWE row for
 * coefficient i.  gamma 0 (and 1, identical at t = 2): N^-1 X^-i ct, whose
 * trace is an encryption of coefficient i.  gamma 2: (N/2)^-1 (X^-i ct +
 * X^-3i ct3) with d_powers = ct3 an encryption of m(X^3) (Lemma 1's sum
 * scaled by [K_2 : K_0] = 2; its trace over K / K_2, sf_pack_gamma with
 * gamma = 2, holds 2 times coefficient i).  d_ct, d_powers, d_out:
 * uint64[2][L][N], coefficient domain.  Errors: SF_EINVAL (gamma outside
 * [0, 2], i out of range, missing power at gamma = 2). */
sf_status sf_extract(sf_ctx *ctx, const uint64_t *d_ct, int32_t i, int32_t gamma, const uint64_t *d_powers,
                     uint64_t *d_out, void *stream);

/* Sec. 4.4 "Shuffle": sigma_r drawn uniformly from a seed derived from the
 * session id and the round: Fisher-Yates from the top driven by
 * SplitMix64(session_seed XOR round*0x9E3779B97F4A7C15) with Lemire draws;
 * perm[k] = sigma(k) (position k holds row sigma(k)).  Host only. */
sf_status sf_permutation(uint64_t session_seed, uint32_t round, uint32_t n, uint32_t *perm);

/* Gathers whole ciphertexts: d_out[k] = d_in[h_perm[k]] for k < count
 * (h_perm must be a permutation of [0, count)).  Errors: SF_EINVAL. */
sf_status sf_shuffle_cts(sf_ctx *ctx, const uint32_t *h_perm, const uint64_t *d_in, uint64_t *d_out,
                         int32_t count, void *stream);

/* Same operation as sf_rotate, for callers that cannot allocate device
 * memory: code running under a fixed device-memory budget owned by another
 * allocator (a framework's caching allocator, a serving process that reserves
 * the whole GPU up front), or latency-critical paths where an allocation, or
 * the device-wide synchronisation of freeing a grown workspace, would stall.
 * This call allocates nothing: its scratch is a fixed 32 MiB array compiled
 * into the library, reserved on every GPU that loads the library and held
 * until the process exits.  The paper has no counterpart; this is an
 * integration variant only.
 *  - Limit: 2 * count ciphertexts plus min(count, ks_batch) key-switch
 *    workspaces (ks_batch: the context option, as in sf_rotate) must fit in
 *    32 MiB: up to 7 ciphertexts at N = 2^14 with 3 data + 1 special primes
 *    (768 KiB each, 3 MiB of workspace per key switch) at the default
 *    ks_batch; larger requests fail with SF_EINVAL and a message giving the
 *    sizes, before anything is enqueued.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture on the device.
 *  - Every call uses the same array: calls whose work overlaps on the GPU
 *    (different streams, or other threads) race and corrupt each other's
 *    results; issue them on one stream or wait in between.  Each call writes
 *    every scratch word before reading it, so nothing needs to start at zero.
 * Arguments, layout and results are those of sf_rotate (bit-identical). */
sf_status sf_rotate_noalloc(sf_ctx *ctx, const sf_rotkeys *rk, int32_t d, const uint64_t *d_ct, uint64_t *d_out,
                            int32_t count, void *stream);

/* Batched negacyclic NTT over every RNS limb (the transform that stands in
 * for the paper's FFT, Sec. 6.1; used by every step of the round).  d_in and
 * d_out hold `count` polynomials [count][L][N] of uint64 residues, limb i
 * modulo q_i (device memory, caller-owned; d_out may equal d_in).
 * inverse = 0: coefficients (each residue below 4 q_i) -> NTT domain,
 * canonical, slot j holding the evaluation at psi^(2 brev(j) + 1) with psi a
 * primitive 2N-th root modulo q_i; inverse = 1: NTT-domain values (below
 * 4 q_i) -> canonical coefficients.  Two persistent launches on `stream`;
 * the row pass follows the context's "row_radix" schedule (same output).
 * Errors: SF_EINVAL for null buffers, count < 1, inverse not 0/1, or a batch
 * whose count x L x (tiles per limb) exceeds 2^31 - 1 (larger than any
 * device memory). */
sf_status sf_ntt_batch(sf_ctx *ctx, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t inverse,
                       void *stream);

/* Measurement utility with no counterpart in the paper: the arithmetic
 * ceiling of this library's modular operations on the context's GPU.  A
 * register-resident kernel (no memory traffic besides one load and one store
 * per value) applies 12 x 1024 operations to 8 residues per thread modulo q_0
 * on one full wave of blocks, and *gmodmul_per_s receives the measured rate
 * in 10^9 modular multiplications per second.  kind 0: forward (Cooley-Tukey)
 * butterflies, 1: inverse (Gentleman-Sande) butterflies, 2: multiply-
 * accumulates with a stored Shoup companion.  Synchronizes the device first
 * and uses the context's workspace; not for use while other work of the
 * context is in flight.  Errors: SF_EINVAL, SF_ECUDA. */
sf_status sf_modmul_probe(sf_ctx *ctx, int32_t kind, double *gmodmul_per_s);

/* Negacyclic product per limb (via the NTT): d_out[t] = d_a[t] * d_b[t] in
 * Z_{q_i}[X]/(X^N+1), arrays uint64[n_polys][L][N].  A test hook for the
 * transform kernels. */
sf_status sf_poly_mul(sf_ctx *ctx, const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_out, int32_t n_polys,
                      void *stream);

/* ---- prime-power cyclotomic rings (Sec. 2.1-2.3; Table 2's M = 3^7, 7^4, 5^5)
 *
 * K = Q[X]/Phi_M(X) with M = t^alpha, t an odd prime, N = phi(M) = (t-1) t^(alpha-1),
 * Phi_M(X) = sum_{k<t} X^(k M/t), reduced modulo L RNS primes q_i = 1 (mod M).
 * Polynomials are uint64[count][L][N] coefficient arrays, canonical residues,
 * device memory owned by the caller; count <= 65535 per call.  Every call is
 * asynchronous on `stream`. */
typedef struct sf_pp_ring sf_pp_ring;

/* The ring for (t, alpha) with the L largest primes q = 1 (mod M) below 2^bits
 * and, per prime, a primitive M-th root of unity omega and its power tables
 * (uploaded to `device`).  Errors: SF_EINVAL (t not an odd prime <= 7, M = t^alpha
 * outside [t^2, 4096], 1 <= L <= SF_MAX_MODULI and 20 <= bits <= 61 violated, or too few
 * primes), SF_ECUDA. */
sf_status sf_pp_ring_create(int32_t t, int32_t alpha, int32_t L, int32_t bits, int32_t device, sf_pp_ring **out);
void sf_pp_ring_destroy(sf_pp_ring *ring);
/* N, M and the L moduli (each output may be NULL). */
sf_status sf_pp_ring_info(const sf_pp_ring *ring, int32_t *N, int32_t *M, uint64_t *moduli);

/* Length-M cyclic transform over Z_{q_i} of uint64[count][L][M] (d_out may
 * equal d_in).  inverse = 0: natural order in, out[j] = sum_k in[k] omega^(k rev(j)),
 * rev(j) reversing the alpha base-t digits of j; inverse = 1: the exact
 * inverse (digit-reversed in, natural out, times M^-1).  The transform that
 * stands in for the paper's length-M FFT (Sec. 6.1).  Errors: SF_EINVAL, SF_ECUDA. */
sf_status sf_pp_ntt(sf_pp_ring *ring, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t inverse,
                    void *stream);

/* d_out[x] = d_a[x] * d_b[x] in Z_{q_i}[X]/Phi_M (length-M cyclic product by
 * the transform, then the reduction modulo Phi_M).  Errors: SF_EINVAL, SF_ECUDA. */
sf_status sf_pp_mul(sf_pp_ring *ring, const uint64_t *d_a, const uint64_t *d_b, uint64_t *d_out, int32_t count,
                    void *stream);

/* d_out[x] = tau_d(d_in[x]) = d_in[x](X^d) mod Phi_M for gcd(d, M) = 1 (Sec. 2.2);
 * d_out must not alias d_in.  Errors: SF_EINVAL (d a multiple of t), SF_ECUDA. */
sf_status sf_pp_automorphism(sf_pp_ring *ring, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t d,
                             void *stream);

/* The trace along the tower of Sec. 2.3: gamma = 0 the full trace Tr_{K/Q}
 * (Tr_{K_(i+1)/K_i} for i = alpha-1 .. 1 by powers of tau_(1+t^i), then
 * Tr_{K_1/K_0} one prime factor of t - 1 at a time), gamma >= 1 the partial
 * trace Tr_{K/K_gamma} only.  *n_automorphisms (may be NULL) receives the
 * automorphisms applied: (alpha - max(gamma,1))(t-1), plus sum (l - 1) over the
 * prime factors l of t - 1 at gamma = 0.  Uses a grow-only scratch of the ring
 * (2 x count x L x N words).  Errors: SF_EINVAL (gamma outside [0, alpha]), SF_ECUDA. */
sf_status sf_pp_trace(sf_pp_ring *ring, const uint64_t *d_in, uint64_t *d_out, int32_t count, int32_t gamma,
                      int32_t *n_automorphisms, void *stream);

/* RLWE over the same ring modulo Q = prod q_i (Sec. 2.1 at general t).  A
 * ciphertext is uint64[2][L][N] residues (a, b = a s + m + e), arrays of them
 * uint64[count][2][L][N].  The secret s, messages m and noise e are int64
 * coefficient arrays (s: [N], m and e: [count][N]); the uniform masks are
 * inputs too (drawn by the caller).  These calls use a grow-only work buffer
 * of the ring.  Errors: SF_EINVAL for null or aliasing buffers, SF_ECUDA. */
sf_status sf_pp_encrypt(sf_pp_ring *ring, const int64_t *d_s, const uint64_t *d_a, const int64_t *d_m,
                        const int64_t *d_e, uint64_t *d_ct, int32_t count, void *stream);
/* d_out = residues of b - a s, uint64[count][L][N]. */
sf_status sf_pp_decrypt(sf_pp_ring *ring, const int64_t *d_s, const uint64_t *d_ct, uint64_t *d_out, int32_t count,
                        void *stream);

/* Key switching after tau_h (Sec. 2.2) by the RNS limbs of tau_h(a): digit i
 * is d_i = [tau_h(a)_i (Q/q_i)^-1]_{q_i}, so tau_h(a) = sum_i d_i Q/q_i (mod Q).
 * sf_pp_ksk: from the uniform d_ka uint64[L digits][L limbs][N] and the noise
 * d_e int64[L][N], d_kb[i] = ka_i s + e_i + (Q/q_i) tau_h(s) (mod Q).
 * sf_pp_keyswitch: d_out[c] = (-sum_i d_i ka_i, tau_h(b) - sum_i d_i kb_i),
 * which decrypts under s to tau_h(m + e) - sum_i d_i e_i; d_out must not
 * alias d_ct. */
sf_status sf_pp_ksk(sf_pp_ring *ring, const int64_t *d_s, int32_t h, const uint64_t *d_ka, const int64_t *d_e,
                    uint64_t *d_kb, void *stream);
sf_status sf_pp_keyswitch(sf_pp_ring *ring, const uint64_t *d_ct, uint64_t *d_out, int32_t count, int32_t h,
                          const uint64_t *d_ka, const uint64_t *d_kb, void *stream);

/* The trace of sf_pp_trace on ciphertexts: the same tower steps, every
 * automorphism followed by its key switch, with keys (hs[x], d_kas[x],
 * d_kbs[x]) for x < n_keys (host arrays of device pointers).  *n_keyswitches
 * (may be NULL) receives the key switches run.  Errors: SF_EINVAL (gamma
 * outside [0, alpha], or no key for an automorphism of the tower), SF_ECUDA. */
sf_status sf_pp_hom_trace(sf_pp_ring *ring, const uint64_t *d_ct, uint64_t *d_out, int32_t count, int32_t gamma,
                          int32_t n_keys, const int32_t *hs, const uint64_t *const *d_kas,
                          const uint64_t *const *d_kbs, int32_t *n_keyswitches, void *stream);

/* ---- the paper's torus scheme: RLWE over T_q = (1/q) Z_q, q = 2^53 (Sec. 2.1),
 * in the prime-power rings above, with the gadget key switching of Sec. 2.2 and
 * Sec. 4.2 (base D, depth l; Table 2: M = 3^7 with (512, 3), 7^4 with (2^12, 3)
 * or (2^16, 2), 5^5 with (310, 5) or (310, 4)).
 *
 * A torus value x / q is the integer x in [0, 2^53) in one uint64 word; input
 * words are read modulo 2^53.  Polynomials are uint64[count][N], ciphertexts
 * uint64[count][2][N] (a, then b = a s + m + e mod 2^53).  The secret s
 * (int64[N], |s_e| <= 65536) and the noise (int64) are inputs, as are the
 * uniform masks a and ka.  Products are exact: computed over Z through two NTT
 * primes p_0, p_1 = 1 (mod M) of 50 bits and the CRT, then taken mod 2^53.  All
 * buffers are device memory owned by the caller; every call is asynchronous on
 * `stream` and uses a grow-only work buffer of the ring, so calls on one ring
 * must not overlap in time (growing the buffer synchronizes the device). */
typedef struct sf_tq_ring sf_tq_ring;

/* The ring for (t, alpha) with the gadget (D, l).  Errors: SF_EINVAL (the
 * limits of sf_pp_ring_create on t and alpha, 2 <= D <= 65536, 1 <= l <= 8,
 * D^l <= 2^53, or products that could leave the CRT range), SF_ECUDA. */
sf_status sf_tq_ring_create(int32_t t, int32_t alpha, int32_t D, int32_t l, int32_t device, sf_tq_ring **out);
void sf_tq_ring_destroy(sf_tq_ring *ring);
/* N, M, the two CRT primes (uint64[2]) and the words of a prepared key,
 * 8 l M (each output may be NULL). */
sf_status sf_tq_ring_info(const sf_tq_ring *ring, int32_t *N, int32_t *M, uint64_t *primes, int64_t *key_words);

/* Gadget decomposition of uint64[count][N] torus polynomials into
 * int32[count][l][N] signed digits: with xr = round(x D^l / q) mod D^l (halves
 * up), d_1 .. d_l (d_1 most significant) in [-floor(D/2), D - floor(D/2)) and
 * sum_i d_i D^(l-i) = xr (mod D^l), so sum_i d_i / D^i = x / q up to 1 / (2 D^l).
 * Errors: SF_EINVAL, SF_ECUDA. */
sf_status sf_tq_decompose(sf_tq_ring *ring, const uint64_t *d_in, int32_t *d_digits, int32_t count, void *stream);

/* d_ct[c] = (a[c], a[c] s + m[c] + e[c]): d_a and d_m uint64[count][N] torus
 * words (the message already scaled, mu q / p), d_e int64[count][N]. */
sf_status sf_tq_encrypt(sf_tq_ring *ring, const int64_t *d_s, const uint64_t *d_a, const uint64_t *d_m,
                        const int64_t *d_e, uint64_t *d_ct, int32_t count, void *stream);
/* d_phase[c] = b - a s mod 2^53 (m + noise), uint64[count][N]; decoding is
 * round(p x / q) mod p (Sec. 2.1). */
sf_status sf_tq_decrypt(sf_tq_ring *ring, const int64_t *d_s, const uint64_t *d_ct, uint64_t *d_phase, int32_t count,
                        void *stream);

/* The key for tau_h (Sec. 4.2): l encryptions of tau_h(s) / D^i, i = 1 .. l:
 * d_kb[i-1] = ka_i s + e_i + round(q tau_h(s) / D^i) mod 2^53 (halves up),
 * from the uniform d_ka uint64[l][N] and the noise d_e int64[l][N].  Errors:
 * SF_EINVAL (h a multiple of t, null buffers), SF_ECUDA. */
sf_status sf_tq_ksk(sf_tq_ring *ring, const int64_t *d_s, int32_t h, const uint64_t *d_ka, const int64_t *d_e,
                    uint64_t *d_kb, void *stream);
/* The key in the form the key switch reads: the 2 l polynomials ka_i, kb_i
 * transformed modulo each CRT prime, with Shoup companions; d_key holds
 * key_words (sf_tq_ring_info) words. */
sf_status sf_tq_key_prepare(sf_tq_ring *ring, const uint64_t *d_ka, const uint64_t *d_kb, uint64_t *d_key,
                            void *stream);

/* Key switch after tau_h (Sec. 2.2): with d_i the gadget digits of tau_h(a),
 * d_out[c] = (-sum_i d_i ka_i, tau_h(b) - sum_i d_i kb_i) mod 2^53, which
 * decrypts to tau_h(m + e) - sum_i d_i e_i up to the gadget's rounding.  One
 * fused kernel per call.  d_key: the prepared key of tau_h.  Errors: SF_EINVAL
 * (h a multiple of t, null key, d_out == d_ct), SF_ECUDA. */
sf_status sf_tq_keyswitch(sf_tq_ring *ring, const uint64_t *d_ct, uint64_t *d_out, int32_t count, int32_t h,
                          const uint64_t *d_key, void *stream);

/* The homomorphic tower trace of sf_pp_hom_trace over the torus: every
 * automorphism followed by its gadget key switch, keys (hs[x], d_keys[x])
 * prepared by sf_tq_key_prepare.  Errors: SF_EINVAL (gamma outside [0, alpha],
 * no key for an automorphism of the tower, d_out == d_ct), SF_ECUDA. */
sf_status sf_tq_hom_trace(sf_tq_ring *ring, const uint64_t *d_ct, uint64_t *d_out, int32_t count, int32_t gamma,
                          int32_t n_keys, const int32_t *hs, const uint64_t *const *d_keys, int32_t *n_keyswitches,
                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SAFHIRE_H */
