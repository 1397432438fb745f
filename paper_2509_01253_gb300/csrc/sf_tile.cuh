// sf_tile.cuh -- negacyclic NTT over Z_q[X]/(X^N+1) as two tiled passes.
//
// Transform (Longa-Naehrig 2016 merged form): forward Cooley-Tukey with the
// table psi_brev[k] = psi^brev(k) (psi a primitive 2N-th root), natural-order
// input, bit-reversed output: out[j] = a(psi^(2 brev(j) + 1)).  Inverse:
// Gentleman-Sande with psi^-brev(k), then a factor N^-1.
//
// Index j = r*C + c with N = R*C.  The forward stages with butterfly
// distance >= C only mix elements of one column ("column pass"); the stages
// with distance < C stay inside one row ("row pass").  Forward = column pass
// then row pass; inverse = row pass then column pass.  A column tile is
// R rows x SF_TC columns, a row tile SF_TR rows x C columns, both staged in
// shared memory; each sweep fuses two stages (radix 4) per shared-memory
// round trip.
//
// Within a tile, sub-transform b (a column or a row) of size S has element k
// at s[b*bs + k*es].  The global twiddle index of local stage with m groups,
// group g, is m*base(b) + g with base = 1 for every column and base = R + r
// for row r (r the global row).
#pragma once
#include "sf_arith.cuh"

#define SF_TC 16
#define SF_TR 16
#define SF_THREADS 256

struct SfGeo {
    int log_n, n, log_r, r, log_c, c;
};

struct TileDesc {
    int nb;      // sub-transforms in the tile
    int bs, es;  // strides (elements) between sub-transforms / elements
    int log_s;   // log2 sub-transform size
    int base0, bstep;
    bool b_fast; // thread mapping: consecutive threads on consecutive sub-transforms
};

__device__ __forceinline__ TileDesc col_tile_desc(const SfGeo &g)
{
    TileDesc t;
    t.nb = SF_TC; t.bs = 1; t.es = SF_TC; t.log_s = g.log_r; t.base0 = 1; t.bstep = 0; t.b_fast = true;
    return t;
}

__device__ __forceinline__ TileDesc row_tile_desc(const SfGeo &g, int r0)
{
    TileDesc t;
    t.nb = SF_TR; t.bs = g.c; t.es = 1; t.log_s = g.log_c; t.base0 = g.r + r0; t.bstep = 1; t.b_fast = false;
    return t;
}

// decompose a unit index into (sub-transform b, unit-in-transform u)
__device__ __forceinline__ void unit_split(const TileDesc &t, int idx, int log_units, int &b, int &u)
{
    if (t.b_fast) {
        b = idx % t.nb;          // nb is a power of two
        u = idx / t.nb;
    } else {
        u = idx & ((1 << log_units) - 1);
        b = idx >> log_units;
    }
}

// Forward (CT) stages of every sub-transform in the tile.  Values in [0, 4q).
static __device__ __forceinline__ void tile_forward(u64 *s, const TileDesc &t, const u64 *__restrict__ tw,
                             const u64 *__restrict__ twp, u64 q)
{
    const u64 two_q = 2 * q;
    int log_s = t.log_s;
    int S = 1 << log_s;
    int h = S >> 1;  // current butterfly half-distance (local)
    if (log_s & 1) {
        // one radix-2 stage first (half S/2, a single group)
        int units = S >> 1;
        for (int idx = threadIdx.x; idx < t.nb * units; idx += blockDim.x) {
            int b, u;
            unit_split(t, idx, log_s - 1, b, u);
            int base = t.base0 + b * t.bstep;
            u64 *p = s + b * t.bs;
            int i1 = base;  // m = 1, g = 0
            u64 w = __ldg(tw + i1), wp = __ldg(twp + i1);
            u64 x = p[u * t.es], y = p[(u + h) * t.es];
            sf_bfly_ct(x, y, w, wp, q, two_q);
            p[u * t.es] = x;
            p[(u + h) * t.es] = y;
        }
        __syncthreads();
        h >>= 1;
    }
    for (; h >= 2; h >>= 2) {
        // radix-4: stages with half h and h/2; m = S / (2h) groups in the first
        int m = S / (2 * h);
        int hh = h >> 1;
        int log_hh = __ffs(hh) - 1;
        int units = S >> 2;
        for (int idx = threadIdx.x; idx < t.nb * units; idx += blockDim.x) {
            int b, u;
            unit_split(t, idx, log_s - 2, b, u);
            int g = u >> log_hh, o = u & (hh - 1);
            int k0 = 2 * h * g + o;
            int base = t.base0 + b * t.bstep;
            u64 *p = s + b * t.bs;
            u64 x0 = p[k0 * t.es], x1 = p[(k0 + hh) * t.es];
            u64 x2 = p[(k0 + h) * t.es], x3 = p[(k0 + h + hh) * t.es];
            int i1 = m * base + g;
            u64 w1 = __ldg(tw + i1), w1p = __ldg(twp + i1);
            sf_bfly_ct(x0, x2, w1, w1p, q, two_q);
            sf_bfly_ct(x1, x3, w1, w1p, q, two_q);
            int i2 = 2 * m * base + 2 * g;
            u64 wa = __ldg(tw + i2), wap = __ldg(twp + i2);
            u64 wb = __ldg(tw + i2 + 1), wbp = __ldg(twp + i2 + 1);
            sf_bfly_ct(x0, x1, wa, wap, q, two_q);
            sf_bfly_ct(x2, x3, wb, wbp, q, two_q);
            p[k0 * t.es] = x0;
            p[(k0 + hh) * t.es] = x1;
            p[(k0 + h) * t.es] = x2;
            p[(k0 + h + hh) * t.es] = x3;
        }
        __syncthreads();
    }
}

// Inverse (GS) stages of every sub-transform in the tile.  Values in [0, 2q).
static __device__ __forceinline__ void tile_inverse(u64 *s, const TileDesc &t, const u64 *__restrict__ tw,
                             const u64 *__restrict__ twp, u64 q)
{
    const u64 two_q = 2 * q;
    int log_s = t.log_s;
    int S = 1 << log_s;
    int h = 1;
    for (; 4 * h <= S; h <<= 2) {
        // radix-4: halves h then 2h; m = S / (2h) groups in the first
        int m = S / (2 * h);
        int log_h = __ffs(h) - 1;
        int units = S >> 2;
        for (int idx = threadIdx.x; idx < t.nb * units; idx += blockDim.x) {
            int b, u;
            unit_split(t, idx, log_s - 2, b, u);
            int g = u >> log_h, o = u & (h - 1);
            int k0 = 4 * h * g + o;
            int base = t.base0 + b * t.bstep;
            u64 *p = s + b * t.bs;
            u64 x0 = p[k0 * t.es], x1 = p[(k0 + h) * t.es];
            u64 x2 = p[(k0 + 2 * h) * t.es], x3 = p[(k0 + 3 * h) * t.es];
            int i1 = m * base + 2 * g;
            u64 wa = __ldg(tw + i1), wap = __ldg(twp + i1);
            u64 wb = __ldg(tw + i1 + 1), wbp = __ldg(twp + i1 + 1);
            sf_bfly_gs(x0, x1, wa, wap, q, two_q);
            sf_bfly_gs(x2, x3, wb, wbp, q, two_q);
            int i2 = (m >> 1) * base + g;
            u64 w2 = __ldg(tw + i2), w2p = __ldg(twp + i2);
            sf_bfly_gs(x0, x2, w2, w2p, q, two_q);
            sf_bfly_gs(x1, x3, w2, w2p, q, two_q);
            p[k0 * t.es] = x0;
            p[(k0 + h) * t.es] = x1;
            p[(k0 + 2 * h) * t.es] = x2;
            p[(k0 + 3 * h) * t.es] = x3;
        }
        __syncthreads();
    }
    if (h < S) {
        // one radix-2 stage last (half S/2, a single group)
        int units = S >> 1;
        for (int idx = threadIdx.x; idx < t.nb * units; idx += blockDim.x) {
            int b, u;
            unit_split(t, idx, log_s - 1, b, u);
            int base = t.base0 + b * t.bstep;
            u64 *p = s + b * t.bs;
            u64 w = __ldg(tw + base), wp = __ldg(twp + base);
            u64 x = p[u * t.es], y = p[(u + h) * t.es];
            sf_bfly_gs(x, y, w, wp, q, two_q);
            p[u * t.es] = x;
            p[(u + h) * t.es] = y;
        }
        __syncthreads();
    }
}

// Column tile c0..c0+SF_TC-1 of a polynomial stored as N contiguous words:
// tile element (r, cc) sits at smem[r*SF_TC + cc].
__device__ __forceinline__ int col_tile_elems(const SfGeo &g) { return g.r * SF_TC; }
__device__ __forceinline__ int col_tile_gidx(const SfGeo &g, int c0, int e)
{
    return (e / SF_TC) * g.c + c0 + (e % SF_TC);
}
// Row tile r0..r0+SF_TR-1: tile element e sits at global r0*C + e.
__device__ __forceinline__ int row_tile_elems(const SfGeo &g) { return SF_TR * g.c; }
