// sf_layer.h -- linear-layer leaves, pack tree and small ciphertext ops.
#pragma once
#include "sf_internal.h"

struct SfTermDev {
    int in_offset, H, W, C_in, C_out, kh, kw, stride, pad;
    int w_off;  // offset of this term's weights in the concatenated array
    int tap_off; // first entry of this term in the tap table
};

// Launch slot z computes slot s = s0 + z * s_stride, i.e. output sig_out[s]
// (or s when sig_out is null); slots >= n_slots_valid are zero padding leaves.
struct SfLeafParams {
    SfTermDev t[2];
    int n_terms;
    int C_out, W_out;
    int k_in;               // input ciphertexts the leaves read (2 k_src with the client's powers)
    int k_src;              // input ciphertexts of the round (chunks of the layer input)
    int gamma2;             // gamma = 2: ciphertexts k_src .. 2 k_src - 1 are the powers RLWE(m_j(X^3))
    int s0;
    int s_stride;
    int n_slots_valid;
    const int64_t *wq;      // quantised weights (device)
    const int4 *taps;       // tap geometry table (see sf_layer)
    const int *pos_of;      // input index -> stream position (null = identity)
    const int *sig_out;     // slot -> output index (null = identity)
    const u64 *ct;          // [k_in][2][L][N] NTT domain, then the same shape of Shoup companions
    u64 *w1;                // [slots][k_in][L][N] column-pass scratch
    // taps of each slot's output bucketed by (input ciphertext j, column tile):
    // bucket j (C/16) + tile holds entries (row << 4 | column in tile, signed Wq)
    longlong2 *tap_buf;     // [slots][max_taps]
    int *tap_off;           // [slots][n_buckets + 1] bucket starts
    int max_taps, n_buckets;
    int sparse_max;         // closed-form column pass for tiles with at most this many taps
    u64 *leaves;            // leaf of slot s0 + z at leaves + z * leaf_stride
    size_t leaf_stride;
};

sf_status sf_leaves_launch(sf_ctx *ctx, const SfLeafParams &P, int cnt, cudaStream_t st);
// scratch words of the tap buckets for `slots` slots
size_t sf_leaf_tap_words(const SfRing &R, int k_in, int max_taps, int slots);
// Pack-tree levels level0+1 .. level1 over G groups.  A holds, per group,
// the n_nodes = 2^(level1 - level0) nodes of level `level0` (level 0 = leaves)
// at group stride a_gs; B has room for half as many.  valid[g] = non-zero
// nodes of group g.  With trace, the field-trace steps k = level1+1 .. log2 N
// follow.  Result (G ciphertexts, NTT domain) at *res, group stride *res_stride.
// tau3_done (gamma = 2): the leaves already hold y + tau_3(y), so level 1
// merges are E + X^(N/2) O with no key switch and the trace starts at k = 2.
sf_status sf_pack_tree(sf_ctx *ctx, const u64 *keys_base, const std::vector<int32_t> &key_d, size_t key_words,
                       u64 *A, u64 *B, int G, int n_nodes, int level0, const std::vector<int> &valid, bool trace,
                       u64 *ks_scratch, int batch, u64 **res, size_t *res_stride, cudaStream_t st,
                       bool tau3_done = false);
// bias times `scale` (2 at gamma = 2, where packed values carry [K_2 : K_0] = 2)
sf_status sf_add_bias(sf_ctx *ctx, u64 *out, int G, int n, int E_out, const int *d_sig_out, const int64_t *d_bq,
                      int C_out, cudaStream_t st, int scale = 1);
// gamma = 2 extraction: out = (N/2)^-1 (X^-i ct + X^-3i ct3), coefficient domain
sf_status sf_extract2_launch(sf_ctx *ctx, const u64 *ct, const u64 *ct3, u64 *out, int i, cudaStream_t st);
sf_status sf_shuffle_launch(sf_ctx *ctx, const u64 *in, u64 *out, const int *d_perm, int count, cudaStream_t st);
sf_status sf_extract_launch(sf_ctx *ctx, const u64 *ct, u64 *out, int i, cudaStream_t st);
