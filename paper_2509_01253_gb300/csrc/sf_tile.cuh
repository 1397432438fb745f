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
// then row pass; inverse = row pass then column pass.
//
// A tile holds NB sub-transforms (16 columns of R elements, or NB rows of C
// elements: NB = 16, 8 for 256-point rows, 4 for 512-point rows) in shared
// memory as [k][b] (tile_slot): a 17-word pitch for 16-wide tiles, XOR-swizzled
// rows of NB words otherwise, so that the coalesced copies and nearly every
// butterfly sweep are free of bank conflicts.
//
// Twiddles are staged in shared memory as (w, w') pairs, w' = floor(w 2^64/q)
// (Shoup).  Local stage with m groups, group g, uses local index k = m + g:
//  * column pass: the global index is m + g for every column, so the tile
//    reads colT[k] (k < R), one table shared by all 16 columns;
//  * row pass: the global index is m*(R + r) + g for row r, so the host
//    stores, per NB-row tile, rowT[tile][k][b] = psi_brev[m(k)(R + NB tile + b)
//    + k - m(k)] (m(k) the largest power of two <= k); the tile's NB*C pairs
//    are one contiguous chunk copied straight into shared memory.
// Each sweep runs 2 or 3 stages (radix 4 / radix 8) on register-resident
// units with lazy Harvey butterflies; in 256- and 512-point rows two sweeps can
// run back to back in registers, the lanes of a warp trading values by
// shuffles in between (schedule RAD = 2).
#pragma once
#include "sf_arith.cuh"
#include "sf_async.cuh"

#define SF_NB 16
#define SF_PAD 17
#define SF_TC SF_NB
#define SF_TR SF_NB
#define SF_THREADS 256
// threads per block of a kernel whose column tiles (16 columns) hold
// sub-transforms of 2^log_s points: 256 (8 warps) up to 128 points, 512 for
// 256 points, so that every thread holds 8 elements; row tiles always run
// 256 threads (their width halves instead, see SfRow)
__host__ __device__ __forceinline__ int sf_tile_threads(int log_s) { return log_s >= 8 ? 512 : SF_THREADS; }
// Row passes double-buffer their tiles with cp.async: a row tile (at most
// 2048 residues) and its staged twiddles leave room for three blocks per SM.
__host__ __device__ constexpr bool sf_rows_double_buffered(int) { return true; }

// runs the statements with the compile-time block size NT = nt (256 or 512)
#define SF_NT_DISPATCH(nt, ...)          \
    do {                                 \
        if ((nt) == 512) {               \
            constexpr int NT = 512;      \
            __VA_ARGS__                  \
        } else {                         \
            constexpr int NT = SF_THREADS; \
            __VA_ARGS__                  \
        }                                \
    } while (0)

struct SfGeo {
    int log_n, n, log_r, r, log_c, c;
};

typedef ulonglong2 sf_tw;   // (w, w')

// Shared-memory word of element k of sub-transform b in a tile of NB
// sub-transforms.  NB = 16: a padded row of 17 words per k (conflict-free for
// the sweeps and the coalesced copies).  NB = 8 (4): rows of 8 (4) words with
// the sub-transform index XOR-swizzled by bits 1..3 (2..3) of k, so that 16
// consecutive k of one b (a coalesced copy) hit 16 distinct bank pairs, and so
// do the units of a half-warp in every sweep whose units start consecutively.
// The sweep of the shortest butterflies (units 4 or 8 elements apart) keeps a
// 2-way (4-way at NB = 4) conflict: a layout that also permutes k inside
// 16-word segments removes it, but its extra index arithmetic cost the
// integer-bound inner product more than the conflicts did.
template <int NB>
__device__ __forceinline__ int tile_slot(int k, int b)
{
    if constexpr (NB == 8) return (k << 3) + (b ^ ((k >> 1) & 7));
    else if constexpr (NB == 4) return (k << 2) + (b ^ ((k >> 2) & 3));
    else return k * (NB + 1) + b;
}

// elements of a tile buffer in shared memory (S rows of SF_PAD words)
__host__ __device__ __forceinline__ int tile_words(int log_s) { return (1 << log_s) * SF_PAD; }
// words of a row tile buffer (2^log_c rows of sf_row_nb(log_c) + 1 words)
__host__ __device__ __forceinline__ int row_tile_words(int log_c)
{
    return (1 << log_c) * (sf_row_nb(log_c) < 16 ? sf_row_nb(log_c) : sf_row_nb(log_c) + 1);
}

// The R_ST stages of one sweep on one register-resident unit x[0 .. 2^R_ST)
// of sub-transform b; blk is the unit's block (its group index base).
// Forward: halves H0, H0/2, ..., H0 >> (R_ST-1).  Inverse: halves H0, ..., H0 << (R_ST-1).
template <int LOG_S, int LOG_H0, int R_ST, bool INV, bool ROWTW, int NB>
__device__ __forceinline__ void unit_stages(u64 *x, int blk, int b, const sf_tw *tw, u64 q, u64 two_q)
{
    constexpr int S = 1 << LOG_S;
    constexpr int U = 1 << R_ST;
#pragma unroll
    for (int sg = 0; sg < R_ST; ++sg) {
        const int d = INV ? (1 << sg) : (1 << (R_ST - 1 - sg));
        const int m = INV ? (S >> (LOG_H0 + 1 + sg)) : ((S >> (LOG_H0 + 1)) << sg);
#pragma unroll
        for (int t = 0; t < U; ++t) {
            if (t & d) continue;
            const int g = INV ? ((blk << (R_ST - sg - 1)) + (t >> (sg + 1))) : ((blk << sg) + (t >> (R_ST - sg)));
            const sf_tw w = ROWTW ? tw[(m + g) * NB + b] : tw[m + g];
            if (INV) sf_bfly_gs(x[t], x[t + d], w.x, w.y, q, two_q);
            else sf_bfly_ct(x[t], x[t + d], w.x, w.y, q, two_q);
        }
    }
}

// One sweep of R_ST consecutive stages over every unit of the tile, element
// (k, b) read through ld(k, b) and written through st(k, b, v); no barrier.
template <int LOG_S, int LOG_H0, int R_ST, bool INV, bool ROWTW, int NT, int NB, class LD, class ST>
__device__ __forceinline__ void tile_sweep_io(const sf_tw *tw, u64 q, LD ld, ST st)
{
    constexpr int S = 1 << LOG_S;
    constexpr int U = 1 << R_ST;
    constexpr int UNITS = NB * S / U;
    constexpr int LOG_NB = NB == 4 ? 2 : (NB == 8 ? 3 : 4);
    constexpr int ITER = (UNITS + NT - 1) / NT;
    constexpr int LOG_STEP = INV ? LOG_H0 : (LOG_H0 - (R_ST - 1));
    constexpr int LOG_BLK = INV ? (LOG_H0 + R_ST) : (LOG_H0 + 1);
    const u64 two_q = 2 * q;
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int idx = threadIdx.x + it * NT;
        if ((UNITS % NT) != 0 && idx >= UNITS) break;
        const int b = idx & (NB - 1);
        const int u = idx >> LOG_NB;
        const int o = u & ((1 << LOG_STEP) - 1);
        const int blk = u >> LOG_STEP;
        const int first = (blk << LOG_BLK) + o;
        u64 x[U];
#pragma unroll
        for (int t = 0; t < U; ++t) x[t] = ld(first + (t << LOG_STEP), b);
        unit_stages<LOG_S, LOG_H0, R_ST, INV, ROWTW, NB>(x, blk, b, tw, q, two_q);
#pragma unroll
        for (int t = 0; t < U; ++t) st(first + (t << LOG_STEP), b, x[t]);
    }
}

// One sweep of R_ST consecutive stages over every unit of the tile, in place
// in shared memory, then a block barrier.
template <int LOG_S, int LOG_H0, int R_ST, bool INV, bool ROWTW, int NT, int NB = SF_NB>
__device__ __forceinline__ void tile_sweep(u64 *s, const sf_tw *tw, u64 q)
{
    tile_sweep_io<LOG_S, LOG_H0, R_ST, INV, ROWTW, NT, NB>(
        tw, q, [&](int k, int b) { return s[tile_slot<NB>(k, b)]; },
        [&](int k, int b, u64 v) { s[tile_slot<NB>(k, b)] = v; });
    __syncthreads();
}

// ---- warp-shuffle exchanges ----------------------------------------------
// Two consecutive sweeps of a row pass fused through registers: the units of
// the first sweep that touch one block of 32 or 64 consecutive elements per row
// are held by the lanes of one warp, which exchange values with __shfl_xor_sync so that every lane then
// holds its unit of the second sweep.  This drops one shared-memory round trip
// and one block barrier per transform.  A lane exchange swaps one bit of the
// lane index (mask LM) with one bit of the register index (mask RM): values
// whose two bits differ move to the partner lane, the others stay.
template <int RM>
__device__ __forceinline__ void lane_exchange(u64 *x, int lm)
{
    const bool hi = (threadIdx.x & lm) != 0;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        if (t & RM) continue;
        const u64 send = hi ? x[t] : x[t | RM];
        const u64 recv = __shfl_xor_sync(0xffffffffu, send, lm);
        if (hi) x[t] = recv;
        else x[t | RM] = recv;
    }
}

// Forward, the last two sweeps of a 512-point row pass (4-row tiles): the
// radix-8 sweep over halves 32, 16, 8 and the one over halves 4, 2, 1.  Lane
// bits 2..4 (o) and the register index (t) swap: lane o of a 64-element block
// first holds elements 8t + o, then 8o + t.
template <bool ROWTW, int NT>
__device__ __forceinline__ void row_pair_fwd9(u64 *s, const sf_tw *tw, u64 q)
{
    static_assert(4 * 512 / 8 == NT, "one unit per thread");
    const u64 two_q = 2 * q;
    const int idx = threadIdx.x, b = idx & 3, o = (idx >> 2) & 7, blk = idx >> 5;
    u64 x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = s[tile_slot<4>((blk << 6) + o + (t << 3), b)];
    unit_stages<9, 5, 3, false, ROWTW, 4>(x, blk, b, tw, q, two_q);
    lane_exchange<1>(x, 4);
    lane_exchange<2>(x, 8);
    lane_exchange<4>(x, 16);
    const int blk3 = (blk << 3) + o;
    unit_stages<9, 2, 3, false, ROWTW, 4>(x, blk3, b, tw, q, two_q);
    __syncwarp();   // every lane's loads of this block are done before any store
#pragma unroll
    for (int t = 0; t < 8; ++t) s[tile_slot<4>((blk3 << 3) + t, b)] = x[t];
    __syncthreads();
}

// Inverse, the first two sweeps of a 512-point row pass: halves 1, 2, 4, then
// 8, 16, 32 (the same lane / register swap, in the other direction).
template <bool ROWTW, int NT>
__device__ __forceinline__ void row_pair_inv9(u64 *s, const sf_tw *tw, u64 q)
{
    static_assert(4 * 512 / 8 == NT, "one unit per thread");
    const u64 two_q = 2 * q;
    const int idx = threadIdx.x, b = idx & 3, o = (idx >> 2) & 7, k = idx >> 5;
    u64 x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = s[tile_slot<4>((k << 6) + (o << 3) + t, b)];
    unit_stages<9, 0, 3, true, ROWTW, 4>(x, (k << 3) + o, b, tw, q, two_q);
    lane_exchange<1>(x, 4);
    lane_exchange<2>(x, 8);
    lane_exchange<4>(x, 16);
    unit_stages<9, 3, 3, true, ROWTW, 4>(x, k, b, tw, q, two_q);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 8; ++t) s[tile_slot<4>((k << 6) + o + (t << 3), b)] = x[t];
    __syncthreads();
}

// Forward, the last two sweeps of a 256-point row pass (8-row tiles): radix 8
// over halves 16, 8, 4, then two radix-4 units over halves 2, 1.  Lane bits
// 3..4 (o) of a 32-element block: lane o first holds elements 4t + o, then
// 8o + t (two exchanges and a fixed renaming of the registers).
template <bool ROWTW, int NT>
__device__ __forceinline__ void row_pair_fwd8(u64 *s, const sf_tw *tw, u64 q)
{
    static_assert(8 * 256 / 8 == NT, "one unit per thread");
    const u64 two_q = 2 * q;
    const int idx = threadIdx.x, b = idx & 7, o = (idx >> 3) & 3, blk = idx >> 5;
    u64 x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = s[tile_slot<8>((blk << 5) + o + (t << 2), b)];
    unit_stages<8, 4, 3, false, ROWTW, 8>(x, blk, b, tw, q, two_q);
    lane_exchange<2>(x, 8);
    lane_exchange<4>(x, 16);
    // register r now holds element bits (E2, E0, E1); y[t] the element 8o + t
    u64 y[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) y[t] = x[((t >> 2) & 1) | ((t & 1) << 1) | (((t >> 1) & 1) << 2)];
    const int blk3 = (blk << 3) + (o << 1);
    unit_stages<8, 1, 2, false, ROWTW, 8>(y, blk3, b, tw, q, two_q);
    unit_stages<8, 1, 2, false, ROWTW, 8>(y + 4, blk3 + 1, b, tw, q, two_q);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 8; ++t) s[tile_slot<8>((blk << 5) + (o << 3) + t, b)] = y[t];
    __syncthreads();
}

// Inverse, the first two sweeps of a 256-point row pass: two radix-4 units
// over halves 1, 2, then radix 8 over halves 4, 8, 16.
template <bool ROWTW, int NT>
__device__ __forceinline__ void row_pair_inv8(u64 *s, const sf_tw *tw, u64 q)
{
    static_assert(8 * 256 / 8 == NT, "one unit per thread");
    const u64 two_q = 2 * q;
    const int idx = threadIdx.x, b = idx & 7, o = (idx >> 3) & 3, k = idx >> 5;
    u64 x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = s[tile_slot<8>((k << 5) + (o << 3) + t, b)];
    unit_stages<8, 0, 2, true, ROWTW, 8>(x, (k << 3) + (o << 1), b, tw, q, two_q);
    unit_stages<8, 0, 2, true, ROWTW, 8>(x + 4, (k << 3) + (o << 1) + 1, b, tw, q, two_q);
    // undo the renaming of the forward pair, then its exchanges in reverse order
    u64 z[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) z[r] = x[((r >> 1) & 1) | (((r >> 2) & 1) << 1) | ((r & 1) << 2)];
    lane_exchange<4>(z, 16);
    lane_exchange<2>(z, 8);
    unit_stages<8, 2, 3, true, ROWTW, 8>(z, k, b, tw, q, two_q);
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 8; ++t) s[tile_slot<8>((k << 5) + o + (t << 2), b)] = z[t];
    __syncthreads();
}

// Forward stages of all NB sub-transforms of size 2^LOG_S; values in [0, 4q).
// 128-point sub-transforms in 512-thread blocks (4 elements per thread) run
// radix-4 sweeps so that every thread holds one unit.
template <int LOG_S, bool ROWTW, int NT, int NB = SF_NB, int RAD = 0>
__device__ __forceinline__ void tile_forward_t(u64 *s, const sf_tw *tw, u64 q)
{
    if constexpr (RAD == 2 && LOG_S == 9 && NB == 4 && NT == 256) {
        // radix 8, the last two sweeps fused by warp-shuffle exchanges
        tile_sweep<9, 8, 3, false, ROWTW, NT, NB>(s, tw, q);
        row_pair_fwd9<ROWTW, NT>(s, tw, q);
    } else if constexpr (RAD == 2 && LOG_S == 8 && NB == 8 && NT == 256) {
        tile_sweep<8, 7, 3, false, ROWTW, NT, NB>(s, tw, q);
        row_pair_fwd8<ROWTW, NT>(s, tw, q);
    } else if constexpr (RAD == 1) {
        // radix-4 sweeps only (two stages per sweep, a radix-2 sweep last for an odd count)
        tile_sweep<LOG_S, LOG_S - 1, 2, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<LOG_S, LOG_S - 3, 2, false, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S >= 6) tile_sweep<LOG_S, LOG_S - 5, 2, false, ROWTW, NT, NB>(s, tw, q);
        else tile_sweep<LOG_S, 0, 1, false, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S == 7) tile_sweep<LOG_S, 0, 1, false, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S >= 8) tile_sweep<LOG_S, LOG_S - 7, 2, false, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S == 9) tile_sweep<LOG_S, 0, 1, false, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 7 && NT == 512) {
        tile_sweep<7, 6, 2, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 4, 2, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 2, 2, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 0, 1, false, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 5) {
        tile_sweep<5, 4, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<5, 1, 2, false, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 6) {
        tile_sweep<6, 5, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<6, 2, 3, false, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 7) {
        tile_sweep<7, 6, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 3, 2, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 1, 2, false, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 8) {
        tile_sweep<8, 7, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<8, 4, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<8, 1, 2, false, ROWTW, NT, NB>(s, tw, q);
    } else {
        tile_sweep<9, 8, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<9, 5, 3, false, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<9, 2, 3, false, ROWTW, NT, NB>(s, tw, q);
    }
}

// Inverse stages (no N^-1 factor); inputs and values in [0, 4q).
template <int LOG_S, bool ROWTW, int NT, int NB = SF_NB, int RAD = 0>
__device__ __forceinline__ void tile_inverse_t(u64 *s, const sf_tw *tw, u64 q)
{
    if constexpr (RAD == 2 && LOG_S == 9 && NB == 4 && NT == 256) {
        // radix 8, the first two sweeps fused by warp-shuffle exchanges
        row_pair_inv9<ROWTW, NT>(s, tw, q);
        tile_sweep<9, 6, 3, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (RAD == 2 && LOG_S == 8 && NB == 8 && NT == 256) {
        row_pair_inv8<ROWTW, NT>(s, tw, q);
        tile_sweep<8, 5, 3, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (RAD == 1) {
        tile_sweep<LOG_S, 0, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<LOG_S, 2, 2, true, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S == 5) tile_sweep<LOG_S, 4, 1, true, ROWTW, NT, NB>(s, tw, q);
        else tile_sweep<LOG_S, 4, 2, true, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S == 7) tile_sweep<LOG_S, 6, 1, true, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S >= 8) tile_sweep<LOG_S, 6, 2, true, ROWTW, NT, NB>(s, tw, q);
        if constexpr (LOG_S == 9) tile_sweep<LOG_S, 8, 1, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 7 && NT == 512) {
        tile_sweep<7, 0, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 2, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 4, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 6, 1, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 5) {
        tile_sweep<5, 0, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<5, 2, 3, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 6) {
        tile_sweep<6, 0, 3, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<6, 3, 3, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 7) {
        tile_sweep<7, 0, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 2, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<7, 4, 3, true, ROWTW, NT, NB>(s, tw, q);
    } else if constexpr (LOG_S == 8) {
        tile_sweep<8, 0, 2, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<8, 2, 3, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<8, 5, 3, true, ROWTW, NT, NB>(s, tw, q);
    } else {
        tile_sweep<9, 0, 3, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<9, 3, 3, true, ROWTW, NT, NB>(s, tw, q);
        tile_sweep<9, 6, 3, true, ROWTW, NT, NB>(s, tw, q);
    }
}

// Forward column transform of a 16-column tile whose input is produced by
// ld(k, b) (element k of column b) and whose output is consumed by
// st(k, b, v), staged in s in between.  For 128-point columns the first sweep
// reads through ld and the last writes through st, so the producer (a base
// conversion) and the consumer (the store to global memory: 16 consecutive
// columns of one row per half-warp, 128 contiguous bytes) need no shared-
// memory round trip and no barrier of their own.  No barrier at the end: the
// caller syncs before it reuses s.
template <int LOG_S, int NT, class LD, class ST>
__device__ __forceinline__ void col_forward_io(u64 *s, const sf_tw *tw, u64 q, LD ld, ST st)
{
    auto s_ld = [&](int k, int b) { return s[tile_slot<SF_NB>(k, b)]; };
    auto s_st = [&](int k, int b, u64 v) { s[tile_slot<SF_NB>(k, b)] = v; };
    if constexpr (LOG_S == 7 && NT == 256) {
        // the schedule of tile_forward_t<7>: radix 8, radix 4, radix 4
        tile_sweep_io<7, 6, 3, false, false, NT, SF_NB>(tw, q, ld, s_st);
        __syncthreads();
        tile_sweep<7, 3, 2, false, false, NT, SF_NB>(s, tw, q);
        tile_sweep_io<7, 1, 2, false, false, NT, SF_NB>(tw, q, s_ld, st);
    } else {
        for (int e = threadIdx.x; e < (SF_NB << LOG_S); e += NT) s_st(e >> 4, e & 15, ld(e >> 4, e & 15));
        __syncthreads();
        tile_forward_t<LOG_S, false, NT>(s, tw, q);
        for (int e = threadIdx.x; e < (SF_NB << LOG_S); e += NT) st(e >> 4, e & 15, s_ld(e >> 4, e & 15));
    }
}

// Inverse column transform of the tile in s whose output goes through
// st(k, b, v) (a scaling written back in place): for 128-point columns the
// last sweep writes through st directly.  No barrier at the end.
template <int LOG_S, int NT, class ST>
__device__ __forceinline__ void col_inverse_st(u64 *s, const sf_tw *tw, u64 q, ST st)
{
    auto s_ld = [&](int k, int b) { return s[tile_slot<SF_NB>(k, b)]; };
    if constexpr (LOG_S == 7 && NT == 256) {
        // the schedule of tile_inverse_t<7>: radix 4, radix 4, radix 8
        tile_sweep<7, 0, 2, true, false, NT, SF_NB>(s, tw, q);
        tile_sweep<7, 2, 2, true, false, NT, SF_NB>(s, tw, q);
        tile_sweep_io<7, 4, 3, true, false, NT, SF_NB>(tw, q, s_ld, st);
    } else {
        tile_inverse_t<LOG_S, false, NT>(s, tw, q);
        for (int e = threadIdx.x; e < (SF_NB << LOG_S); e += NT) st(e >> 4, e & 15, s_ld(e >> 4, e & 15));
    }
}

// Runtime dispatch on the sub-transform size (R for columns, C for rows).
template <int NT = SF_THREADS>
__device__ __forceinline__ void col_forward(u64 *s, const sf_tw *tw, int log_r, u64 q)
{
    switch (log_r) {
    case 5: tile_forward_t<5, false, NT>(s, tw, q); break;
    case 6: tile_forward_t<6, false, NT>(s, tw, q); break;
    case 7: tile_forward_t<7, false, NT>(s, tw, q); break;
    default: tile_forward_t<8, false, NT>(s, tw, q); break;
    }
}
template <int NT = SF_THREADS>
__device__ __forceinline__ void col_inverse(u64 *s, const sf_tw *tw, int log_r, u64 q)
{
    switch (log_r) {
    case 5: tile_inverse_t<5, false, NT>(s, tw, q); break;
    case 6: tile_inverse_t<6, false, NT>(s, tw, q); break;
    case 7: tile_inverse_t<7, false, NT>(s, tw, q); break;
    default: tile_inverse_t<8, false, NT>(s, tw, q); break;
    }
}
template <int NT = SF_THREADS>
__device__ __forceinline__ void row_forward(u64 *s, const sf_tw *tw, int log_c, u64 q)
{
    switch (log_c) {
    case 5: tile_forward_t<5, true, NT>(s, tw, q); break;
    case 6: tile_forward_t<6, true, NT>(s, tw, q); break;
    case 7: tile_forward_t<7, true, NT>(s, tw, q); break;
    case 8: tile_forward_t<8, true, NT, 8>(s, tw, q); break;
    default: tile_forward_t<9, true, NT, 4>(s, tw, q); break;
    }
}
template <int NT = SF_THREADS>
__device__ __forceinline__ void row_inverse(u64 *s, const sf_tw *tw, int log_c, u64 q)
{
    switch (log_c) {
    case 5: tile_inverse_t<5, true, NT>(s, tw, q); break;
    case 6: tile_inverse_t<6, true, NT>(s, tw, q); break;
    case 7: tile_inverse_t<7, true, NT>(s, tw, q); break;
    case 8: tile_inverse_t<8, true, NT, 8>(s, tw, q); break;
    default: tile_inverse_t<9, true, NT, 4>(s, tw, q); break;
    }
}

// ---- tile <-> global ------------------------------------------------------
// Thread-iteration index e enumerates a tile in global (coalesced) order;
// these map it to the global offset and to the shared-memory slot.

// column tile c0..c0+15: global r*C + c0 + b, e = r*16 + b
__device__ __forceinline__ int col_elems(const SfGeo &g) { return g.r * SF_NB; }
__device__ __forceinline__ int col_gidx(const SfGeo &g, int c0, int e) { return (e >> 4) * g.c + c0 + (e & 15); }
__device__ __forceinline__ int col_slot(int e) { return (e >> 4) * SF_PAD + (e & 15); }
// row tile r0..r0+NB-1: global (r0 + b)*C + k, e = b*C + k
__device__ __forceinline__ int row_elems(const SfGeo &g) { return sf_row_nb(g.log_c) * g.c; }
__device__ __forceinline__ int row_slot(const SfGeo &g, int e)
{
    const int nb = sf_row_nb(g.log_c);
    return nb == 4 ? tile_slot<4>(e & (g.c - 1), e >> g.log_c)
                   : (nb == 8 ? tile_slot<8>(e & (g.c - 1), e >> g.log_c) : tile_slot<16>(e & (g.c - 1), e >> g.log_c));
}

// Stage twiddles: column table (R pairs) or the row table of tile r0/NB
// (NB*C pairs), for modulus `mod`; tables are [nm][...] in global memory.
__device__ __forceinline__ void load_col_tw(sf_tw *dst, const sf_tw *__restrict__ table, const SfGeo &g, int mod)
{
    const sf_tw *src = table + (size_t)mod * g.r;
    for (int k = threadIdx.x; k < g.r; k += blockDim.x) dst[k] = src[k];
}
__device__ __forceinline__ void load_row_tw(sf_tw *dst, const sf_tw *__restrict__ table, const SfGeo &g, int mod, int r0)
{
    const sf_tw *src = table + ((size_t)mod << g.log_n) + (size_t)r0 * g.c;
    for (int k = threadIdx.x; k < sf_row_nb(g.log_c) * g.c; k += blockDim.x) dst[k] = src[k];
}

// ---- balanced persistent partition ----------------------------------------
// A persistent launch of gridDim.x blocks over n_units work units numbered
// group-major (u = group * n_items + item, where a group is a tile position
// and modulus whose twiddles a block stages, and an item a merge or a
// polynomial) gives block x the units [x n / grid, (x + 1) n / grid): every
// block the floor or the ceiling of the mean, whatever the group count, and
// a block restages twiddles only where its range crosses into a new group.
struct SfUnits {
    int u0, u1;
};
__device__ __forceinline__ SfUnits sf_block_units(int n_units)
{
    return {(int)((long long)blockIdx.x * n_units / gridDim.x),
            (int)(((long long)blockIdx.x + 1) * n_units / gridDim.x)};
}

// ---- compile-time geometry -------------------------------------------------
// The same helpers with the R x C split as template parameters, for kernels
// instantiated per ring size: loops unroll and slot arithmetic folds into
// constants.  LR = log2 R, LC = log2 C, NT = threads per block.

template <int LR, int LC>
struct SfGeoT {
    static constexpr int log_r = LR, r = 1 << LR, log_c = LC, c = 1 << LC, log_n = LR + LC, n = 1 << (LR + LC);
};

// threads per block for tiles of 2^log_s-point sub-transforms (constexpr twin of sf_tile_threads)
template <int LOG_S>
struct SfThreads {
    static constexpr int value = LOG_S >= 8 ? 512 : SF_THREADS;
};

// Row tiles: NB rows of 2^LC points (NB = 16, 8 for 256-point, 4 for 512-point rows),
// always processed by 256-thread blocks (NB 2^LC / 256 residues per thread).
template <int LC>
struct SfRow {
    static constexpr int NB = LC >= 9 ? 4 : (LC >= 8 ? 8 : 16);
    static constexpr int NT = SF_THREADS;
    static constexpr int ELEMS = NB << LC;
    static constexpr int WORDS = (1 << LC) * (NB < 16 ? NB : NB + 1);   // words of one tile buffer (see tile_slot)
};

template <int LC>
__device__ __forceinline__ int row_slot_t(int e) { return tile_slot<SfRow<LC>::NB>(e & ((1 << LC) - 1), e >> LC); }
template <int LC>
__device__ __forceinline__ int col_gidx_t(int c0, int e) { return ((e >> 4) << LC) + c0 + (e & 15); }

// row tile (NB rows of C) global -> shared via 8-byte cp.async
template <int LC, int NT>
__device__ __forceinline__ void issue_row_tile_t(u64 *dst, const u64 *src)
{
    constexpr int E = SfRow<LC>::ELEMS / NT;
#pragma unroll
    for (int x = 0; x < E; ++x) {
        const int e = threadIdx.x + x * NT;
        sf_cp8(dst + row_slot_t<LC>(e), src + e);
    }
}

// column tile (R rows of 16 columns from c0) global -> shared via 8-byte cp.async
template <int LR, int LC, int NT>
__device__ __forceinline__ void issue_col_tile_t(u64 *dst, const u64 *src, int c0)
{
    constexpr int E = (SF_NB << LR) / NT;
    const u64 *s0 = src + c0 + (threadIdx.x & 15) + (size_t)(threadIdx.x >> 4) * (1 << LC);
    u64 *d0 = dst + (threadIdx.x >> 4) * SF_PAD + (threadIdx.x & 15);
#pragma unroll
    for (int x = 0; x < E; ++x) sf_cp8(d0 + x * (NT / 16) * SF_PAD, s0 + (size_t)x * (NT / 16) * (1 << LC));
}

// shared row tile -> global (NB rows of C), with an optional per-value map
template <int LC, int NT, class F>
__device__ __forceinline__ void store_row_tile_t(u64 *dst, const u64 *src, F f)
{
    constexpr int E = SfRow<LC>::ELEMS / NT;
#pragma unroll
    for (int x = 0; x < E; ++x) {
        const int e = threadIdx.x + x * NT;
        dst[e] = f(src[row_slot_t<LC>(e)]);
    }
}

// twiddles of the row tile starting at row r0 for modulus mod ([nm][R/NB][C][NB] table)
template <int LR, int LC, int NT>
__device__ __forceinline__ void load_row_tw_t(sf_tw *dst, const sf_tw *__restrict__ table, int mod, int r0)
{
    constexpr int E = SfRow<LC>::ELEMS / NT;
    const sf_tw *src = table + ((size_t)mod << (LR + LC)) + ((size_t)r0 << LC);
#pragma unroll
    for (int x = 0; x < E; ++x) dst[threadIdx.x + x * NT] = src[threadIdx.x + x * NT];
}

// forward / inverse row pass of a row tile (its width from the row length)
// RAD: 0 radix-8 sweeps (the default schedule), 1 radix-4 sweeps only; the
// autotuner times both (context option row_radix)
template <int LC, int NT, int RAD = 0>
__device__ __forceinline__ void row_forward_t(u64 *s, const sf_tw *tw, u64 q)
{
    tile_forward_t<LC, true, NT, SfRow<LC>::NB, RAD>(s, tw, q);
}
template <int LC, int NT, int RAD = 0>
__device__ __forceinline__ void row_inverse_t(u64 *s, const sf_tw *tw, u64 q)
{
    tile_inverse_t<LC, true, NT, SfRow<LC>::NB, RAD>(s, tw, q);
}

// Inverse row pass whose output goes to st(k, b, v) (element k of row b).  In
// 256- and 512-point rows under the radix-8 schedule the last sweep writes
// through st itself: its units hold elements 32 or 64 apart, so a warp stores
// 4 or 8 consecutive elements of each of its rows (whole 32-byte sectors).
// Otherwise the pass runs in shared memory and a copy loop calls st in row
// order.  No barrier at the end.
template <int LC, int NT, int RAD, class ST>
__device__ __forceinline__ void row_inverse_out(u64 *s, const sf_tw *tw, u64 q, ST st)
{
    constexpr int NB = SfRow<LC>::NB;
    auto s_ld = [&](int k, int b) { return s[tile_slot<NB>(k, b)]; };
    if constexpr (RAD == 0 && NT == 256 && LC == 9 && NB == 4) {
        tile_sweep<9, 0, 3, true, true, NT, NB>(s, tw, q);
        tile_sweep<9, 3, 3, true, true, NT, NB>(s, tw, q);
        tile_sweep_io<9, 6, 3, true, true, NT, NB>(tw, q, s_ld, st);
    } else if constexpr (RAD == 0 && NT == 256 && LC == 8 && NB == 8) {
        tile_sweep<8, 0, 2, true, true, NT, NB>(s, tw, q);
        tile_sweep<8, 2, 3, true, true, NT, NB>(s, tw, q);
        tile_sweep_io<8, 5, 3, true, true, NT, NB>(tw, q, s_ld, st);
    } else {
        row_inverse_t<LC, NT, RAD>(s, tw, q);
#pragma unroll
        for (int e = threadIdx.x; e < SfRow<LC>::ELEMS; e += NT) st(e & ((1 << LC) - 1), e >> LC, s_ld(e & ((1 << LC) - 1), e >> LC));
    }
}

// column twiddles (R pairs) of modulus mod
template <int LR, int NT>
__device__ __forceinline__ void load_col_tw_t(sf_tw *dst, const sf_tw *__restrict__ table, int mod)
{
    const sf_tw *src = table + ((size_t)mod << LR);
    for (int k = threadIdx.x; k < (1 << LR); k += NT) dst[k] = src[k];
}

// runs the statements with the row-pass sweep schedule RAD (0: radix-8
// sweeps, 1: radix-4 sweeps, 2: radix-8 with two sweeps of 256- and
// 512-point rows fused by warp-shuffle exchanges) as a compile-time constant
#define SF_RAD_DISPATCH(rad, ...)           \
    do {                                    \
        if ((rad) == 2) {                   \
            constexpr int RAD = 2;          \
            __VA_ARGS__                     \
        } else if ((rad) == 1) {            \
            constexpr int RAD = 1;          \
            __VA_ARGS__                     \
        } else {                            \
            constexpr int RAD = 0;          \
            __VA_ARGS__                     \
        }                                   \
    } while (0)

// runs the statements with constexpr LR, LC for the ring size log_n (10..16)
#define SF_GEO_DISPATCH(log_n, ...)                       \
    do {                                                  \
        switch (log_n) {                                  \
        case 10: { constexpr int LR = 5, LC = 5; __VA_ARGS__ } break; \
        case 11: { constexpr int LR = 5, LC = 6; __VA_ARGS__ } break; \
        case 12: { constexpr int LR = 6, LC = 6; __VA_ARGS__ } break; \
        case 13: { constexpr int LR = 6, LC = 7; __VA_ARGS__ } break; \
        case 14: { constexpr int LR = 7, LC = 7; __VA_ARGS__ } break; \
        case 15: { constexpr int LR = 7, LC = 8; __VA_ARGS__ } break; \
        default: { constexpr int LR = 7, LC = 9; __VA_ARGS__ } break; \
        }                                                 \
    } while (0)
