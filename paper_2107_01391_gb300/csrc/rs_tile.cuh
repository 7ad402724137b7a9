// rs_tile.cuh -- one CTA ranks one tile of keys by one 8-bit digit group.
//
// The tile's keys sit in registers, warp-striped: warp w, item i, lane l holds
// tile position w*32*IPT + i*32 + l, so (warp, item, lane) order is input
// order.  rank_scatter() counts the tile's keys per cell (the hashing cycle
// on one digit group, §3.1), turns the counts into raster-order starts (the
// extraction cycle's cursor, §3.2), and writes every key (and value) to its
// stable position in shared memory.  Used by the segmented sort's CTA tiers,
// where a CTA owns a whole segment and needs no look-back between tiles.
#pragma once

#include "rs_kernels.cuh"  // ValTraits, rs_device.cuh

namespace rs {

struct TileShared {
    uint32_t wh[WARPS][RADIX];  // per-warp counts, then per-warp next positions
    uint32_t count[RADIX];      // keys of each cell in the tile
    uint32_t excl[RADIX];       // tile-local start of each cell
    uint32_t warp_sum[WARPS];
};

// Positions [0, n_valid) of the tile hold keys; the rest are ignored.
// `rows` (1 .. IPT): item rows per warp, so warp w holds positions
// [w*32*rows, (w+1)*32*rows) in items 0 .. rows-1; a tile shorter than
// BLOCK * IPT is spread over every warp with rows = ceil(n / BLOCK) instead of
// filling the first warps, so its rank costs rows, not IPT, rounds per warp.
// With kFull, rows is a multiple of ROWS_Q (or IPT).
// Returns with `stage` holding the tile in (cell, input) order and
// ts.count / ts.excl filled.  Every thread of the CTA must call it.
// s_run (optional): running per-cell output offsets of a sweep over several
// tiles; the previous tile's ts.count is added to them once every thread is
// past its write-out (the first barrier below), so the sweep itself needs
// no barrier between tiles.
// kLut: the table match (match_digit_lut) in place of match_digit, for
// shapes whose register budget holds its five lane constants.  kFull: every
// item of the first `rows` holds a key (n_valid == BLOCK * rows), so no
// position is tested.
constexpr uint32_t ROWS_Q = 4;  // granularity of a padded tile's item rows

template <typename Cell, typename VS, int IPT, bool kPairs, bool kLut = false,
          bool kFull = false, int STILE>
__device__ __forceinline__ void rank_scatter(const Cell (&k)[IPT], const VS (&v)[IPT],
                                             uint32_t n_valid, uint32_t shift, TileShared& ts,
                                             const Stage<Cell, VS, kPairs, STILE>& stage,
                                             uint32_t* s_run = nullptr, uint32_t rows = IPT) {
    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    const uint32_t wbase = warp * 32 * rows;
    for (uint32_t d = lane; d < RADIX; d += 32) ts.wh[warp][d] = 0;
    __syncwarp();
    const uint32_t warp_items =
        kFull ? 32u * rows : (wbase < n_valid ? min(n_valid - wbase, 32u * rows) : 0u);
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (kFull && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;  // block-uniform
        if (kFull || (uint32_t)i * 32 + lane < warp_items)
            atomicAdd(&ts.wh[warp][digit_of(k[i], shift)], 1u);
    }
    __syncthreads();

    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < WARPS; w++) {
        const uint32_t x = ts.wh[w][t];
        ts.wh[w][t] = run;
        run += x;
    }
    uint32_t total;
    const uint32_t excl = block_exclusive_scan(run, ts.warp_sum, &total);
#pragma unroll
    for (int w = 0; w < WARPS; w++) ts.wh[w][t] += excl;
    if (s_run) s_run[t] += ts.count[t];  // thread t owns cell t in both
    ts.count[t] = run;
    ts.excl[t] = excl;
    __syncthreads();

    const uint32_t lt = lanemask_lt(), gt = lanemask_gt();
    const LaneBits lbits = lane_bits();
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (kFull ? i % ROWS_Q == 0 && (uint32_t)i >= rows
                  : (uint32_t)i * 32 >= warp_items)
            break;  // warp-uniform
        const bool valid = kFull || (uint32_t)i * 32 + lane < warp_items;
        const uint32_t vmask = kFull ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
        const uint32_t d = digit_of(k[i], shift);
        const uint32_t peers = peer_mask<kLut>(d, lbits) & vmask;
        uint32_t* slot = &ts.wh[warp][d];
        const uint32_t at = valid ? *slot : 0u;
        const uint32_t below = __popc(peers & lt);
        __syncwarp();
        if (valid) {
            if ((peers & gt) == 0) *slot = at + below + 1;
            stage.put(at + below, k[i], v[i]);
        }
        __syncwarp();
    }
    __syncthreads();
}


// ----------------------------------------------------------------------------
// Whole sorts of equal rows of at most BLOCK * IPT keys, one row per CTA at a
// time (a grid-stride loop over rows): the row's keys (and values) are loaded
// once into registers, ranked through shared memory once per non-trivial
// 8-bit digit group, and written once.  Every input is in registers before
// the first store, so the sort may be in place.  A group in which every key
// of the row has the same digit is an identity permutation and is skipped
// (one block-wide AND).  One row of at most SMALL_TILE keys is how every
// small sort runs; equal segments of up to ROW_TILE keys use the same kernel.

constexpr int SMALL_IPT = 16;
constexpr uint32_t SMALL_TILE = BLOCK * SMALL_IPT;
constexpr int ROW_IPT = 32;
constexpr uint32_t ROW_TILE = BLOCK * ROW_IPT;

struct RowsArgs {
    const void* keys_in;
    void* keys_out;
    const void* vals_in;   // NULL with iota: values are the key's index in its row
    void* vals_out;
    uint64_t rows;
    uint32_t len;          // keys per row, 1 .. BLOCK * IPT
    uint32_t iota;
    uint32_t passes;       // digit groups of the cell
    CodecParams prm;
    uint32_t* status;
    DevInfo* info;         // nullable: the plan report of a single sort
    const uint32_t* skip;  // nullable; non-zero at run time: the sort is a no-op
};

// One row of n keys starting at key `base`: load, one rank per non-trivial
// digit group, write.  kCheckIO: loads and stores test the position (n may
// be below BLOCK * IPT), and the row is spread over every warp in `rows`
// item rows, ceil(n / BLOCK) rounded up to a multiple of ROWS_Q.
// kCheckRank: the ranks test it too; without it a short row is ranked as
// BLOCK * rows keys whose positions from n on hold padding keys of the
// largest cell, which start after every real key and so stay in the last
// positions through every stable group (the trivial-group test looks at the
// real keys only).
template <class C, typename V, int IPT, typename VR, bool kCheckIO, bool kCheckRank>
__device__ __forceinline__ uint32_t sort_row(const RowsArgs& a, uint64_t base, uint32_t n,
                                             TileShared& ts,
                                             typename C::Cell& s_ref,
                                             const Stage<typename C::Cell,
                                                         typename std::conditional<
                                                             ValTraits<V>::kPairs, VR,
                                                             uint32_t>::type,
                                                         ValTraits<V>::kPairs,
                                                         BLOCK * IPT>& stage) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    using Out = typename C::Out;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    using VS = typename std::conditional<kPairs, VR, uint32_t>::type;
    using VM = typename std::conditional<kPairs, V, uint32_t>::type;
    // the table match where the 32-key rows leave room for its constants
    constexpr bool kLut = IPT == ROW_IPT && sizeof(Cell) == 4 && sizeof(VS) == 4;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    static_assert(IPT % ROWS_Q == 0, "item rows are skipped ROWS_Q at a time");
    const uint32_t rows =
        kCheckIO ? min((uint32_t)IPT, (n + BLOCK * ROWS_Q - 1) / (BLOCK * ROWS_Q) * ROWS_Q)
                 : (uint32_t)IPT;
    const uint32_t w0 = warp * 32 * rows + lane;  // warp-striped: input order
    Cell k[IPT];
    VS v[IPT];
    bool ok = true;
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        const uint32_t j = w0 + i * 32;
        k[i] = ~Cell(0);
        v[i] = VS(0);
        if (kCheckIO && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;  // block-uniform
        if (!kCheckIO || j < n) {
            k[i] = C::decode(static_cast<const In*>(a.keys_in)[base + j], a.prm, ok);
            if constexpr (kPairs)
                v[i] = a.iota ? (VS)j : (VS) static_cast<const VM*>(a.vals_in)[base + j];
        }
    }
    if (!ok) atomicOr(a.status, STATUS_RANGE);
    if (threadIdx.x == 0) s_ref = k[0];  // the row's first key
    __syncthreads();
    const Cell ref = s_ref;
    uint32_t moved = 0;
    for (uint32_t p = 0; p < a.passes; p++) {
        const uint32_t shift = p * RADIX_BITS;
        bool same = true;
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            if (kCheckIO && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;
            if (!kCheckIO || w0 + i * 32 < n) same &= digit_of(k[i], shift) == digit_of(ref, shift);
        }
        if (__syncthreads_and(same)) continue;  // every key in one cell
        moved++;
        rank_scatter<Cell, VS, IPT, kPairs, kLut, !kCheckRank>(
            k, v, kCheckRank ? n : BLOCK * rows, shift, ts, stage, nullptr, rows);
#pragma unroll
        for (int i = 0; i < IPT; i++) {
            if (kCheckIO && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;
            const uint32_t j = w0 + i * 32;
            if (!kCheckRank || j < n) stage.get(j, k[i], v[i]);
        }
        __syncthreads();  // the staged tile is rewritten by the next group
    }
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (kCheckIO && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;
        const uint32_t j = w0 + i * 32;
        if (!kCheckIO || j < n) {
            static_cast<Out*>(a.keys_out)[base + j] = C::encode(k[i], a.prm);
            if constexpr (kPairs) static_cast<VM*>(a.vals_out)[base + j] = (VM)v[i];
        }
    }
    return moved;
}

// VR: the type a value is carried in through the passes (registers and
// shared memory); V is its type in memory.  An argsort's indices are below
// BLOCK * IPT, so they travel as 32-bit words whatever their output width.
// At the start of each row the CTA prefetches its next row (row + gridDim.x)
// into L2 with one TMA bulk prefetch, so that row's loads do not wait on DRAM.
// kShort: rows shorter than the tile (padded, spread over every warp);
// otherwise every row fills the tile.  The two are separate kernels so that
// each is register-allocated for its own loop.
template <class C, typename V, int IPT, typename VR = V, bool kShort = false>
__global__ void __launch_bounds__(BLOCK, 2) tile_rows_kernel(RowsArgs a) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    constexpr uint32_t TILE = BLOCK * IPT;
    using VS = typename std::conditional<kPairs, VR, uint32_t>::type;
    using VM = typename std::conditional<kPairs, V, uint32_t>::type;
    if (a.skip && *a.skip) return;

    __shared__ TileShared ts;
    __shared__ Cell s_ref;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const Stage<Cell, VS, kPairs, TILE> stage{smem_dyn};
    const uint32_t n = kShort ? a.len : TILE;  // a full-row launch has a.len == TILE
    uint32_t moved = 0;

    for (uint64_t row = blockIdx.x; row < a.rows; row += gridDim.x) {
        const uint64_t next = row + gridDim.x;
        if (threadIdx.x == 0 && next < a.rows) {
            const char* kp = static_cast<const char*>(a.keys_in) + next * n * sizeof(In);
            const uint32_t kb = n * (uint32_t)sizeof(In);
            if ((((uintptr_t)kp | kb) & 15) == 0) bulk_prefetch_l2(kp, kb);
            if (kPairs && !a.iota) {
                const char* vp = static_cast<const char*>(a.vals_in) + next * n * sizeof(VM);
                const uint32_t vb = n * (uint32_t)sizeof(VM);
                if ((((uintptr_t)vp | vb) & 15) == 0) bulk_prefetch_l2(vp, vb);
            }
        }
        if constexpr (kShort)
            moved = sort_row<C, V, IPT, VR, true, false>(a, row * n, n, ts, s_ref, stage);
        else
            moved = sort_row<C, V, IPT, VR, false, false>(a, row * TILE, TILE, ts, s_ref, stage);
    }
    if (a.info && blockIdx.x == 0 && threadIdx.x == 0) {
        a.info->mode = MODE_PASSES;
        a.info->passes_run = moved;
    }
}

}  // namespace rs
