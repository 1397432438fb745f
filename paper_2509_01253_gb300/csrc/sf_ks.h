// sf_ks.h -- batched automorphism + key switching (see sf_ks.cu).
#pragma once
#include "sf_internal.h"

// `count` merges sharing d, s, add_v and the key.  Merge number
// x = first + i (i < count) splits into (g, t) = (x / inner, x % inner):
//   E_x = E + g*E_outer + t*E_stride, likewise O_x (O may be null) and out_x;
// every operand [2][L][N] in the NTT domain.  out must not alias E or O.
struct SfKsBatch {
    const u64 *E;
    size_t E_stride, E_outer;
    const u64 *O;
    size_t O_stride, O_outer;
    u64 *out;
    size_t out_stride, out_outer;
    int first;
    int inner;
    int count;
    int d;          // automorphism X -> X^d
    unsigned s;     // O is multiplied by X^s
    int add_v;      // 1: out = v + KS(...), 0: plain rotation
    const u64 *key; // [dnum][2][nm][N] NTT-domain values, then the same shape of Shoup companions
    u64 *scratch;   // sf_ks_scratch_words(R) words per merge of one launch batch
};

size_t sf_ks_scratch_words(const SfRing &R);
// One launch sequence (K1..K5) for B.count merges, scratch for all of them.
sf_status sf_ks_launch(sf_ctx *ctx, const SfKsBatch &B, cudaStream_t st);
// Splits B into launch batches of `batch` merges reusing `scratch`
// (batch * sf_ks_scratch_words words).
sf_status sf_ks_run(sf_ctx *ctx, SfKsBatch B, u64 *scratch, int batch, cudaStream_t st);
