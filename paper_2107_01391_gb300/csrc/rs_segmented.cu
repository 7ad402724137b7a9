// rs_segmented.cu -- rs_sort_segmented: many independent arrays in one launch.
//
// Each segment is an independent sort; in the paper's terms each segment is
// a bucket (§2.2) that is sorted on its own by the hashing and extraction
// cycles.  The batch runs as:
//   1. seg_size_kernel   counts segments per power-of-two size class (a
//                        counting sort of the segments by size, largest first)
//   2. seg_order_kernel  writes the segment ids in that order
//   3. seg_sort_kernel   persistent CTAs take segments from the ordered list:
//        - once the list reaches segments of at most 63 keys (everything
//          after them is as small), a CTA takes eight at a time and each
//          warp sorts one: two keys per lane, each ranked by counting the
//          keys before it in (cell, position) order;
//        - (shapes without step 7) a segment of at most 4096 keys (one
//          tile) is loaded once into registers, spread over every warp, and
//          sorted entirely on chip: one rank-and-scatter through shared
//          memory per 8-bit digit group, then one coalesced write (16 bytes
//          per u32 key+value pair in total);
//        - (shapes without step 7) a longer segment below 2^DEV_MIN_LOG2
//          keys is first read once
//          to count all its digit groups, then sorted by its CTA alone: per
//          non-trivial group a sweep over its tiles in input order with
//          running cell offsets in shared memory (a CTA-sequential
//          extraction cycle, no look-back);
//        - a segment of 2^DEV_MIN_LOG2 keys or more (these come first in the
//          list) is counted the same way (or, when longer than one CTA's
//          share of the batch, tile-parallel by step 5); its groups'
//          raster-order starts and the set of non-trivial groups are left in
//          global memory for the device tier;
//   4. seg_tiles_kernel  (before 3) gives every device-tier segment a
//                        contiguous range of device tiles;
//   5. seg_count_kernel  (before 3) counts every digit group of the device
//                        tier's longest segments, one tile per CTA step
//                        (the others are counted by the CTA that takes them);
//   6. seg_pass_kernel   the device tier, once per digit group: all the
//                        tiles of all device-tier segments in one launch,
//                        each ranked like the device-wide pass and placed
//                        with a decoupled look-back that stops at its
//                        segment's first tile.
//   7. seg_rows_kernel   (4-byte cells with no value, a 4-byte value or an
//                        argsort) the segments of 64 .. 8191 keys, each
//                        sorted whole on chip by one CTA in the row kernel's
//                        8192-key tile; step 3 skips them.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "../../include/rs.h"
#include "rs_sort_impl.cuh"
#include "rs_tile.cuh"

namespace rs {
namespace {

constexpr int SEG_IPT = 16;
constexpr uint32_t SEG_TILE = BLOCK * SEG_IPT;
constexpr int SIZE_CLASSES = 64;
constexpr uint64_t WARP_SEG_MAX = 63;         // segments sorted by one warp
constexpr uint64_t SEG_MAX_LEN = RS_MAX_N;  // look-back words of the device tier hold 30-bit counts
// Segments of at least 2^DEV_MIN_LOG2 keys go to the device tier: exactly the
// size classes 0..DEV_CLASS_MAX (class = leading zeros of the length).
// Shorter ones above one tile are swept by one CTA.  With the device tier's
// L2 prefetch, 2^13 measured best (Run B / Run A, ms: 2^13 5.64 / 115.8,
// 2^14 5.70 / 115.4, 2^15 6.10 / 116.2); without it 2^14 was (2^13 6.27 /
// 133.0, 2^14 6.12 / 132.9).
constexpr uint32_t DEV_MIN_LOG2 = 13;
constexpr uint32_t DEV_CLASS_MAX = 63 - DEV_MIN_LOG2;
static_assert((1u << DEV_MIN_LOG2) > SEG_TILE, "the device tier starts above the on-chip tier");

// Size classes (leading zeros of the 64-bit length) that bound the tiers in
// the ordered list: the row tier holds the classes of 2^ROW_MIN_LOG2 ..
// 2^13-1 keys (ROW_CLASS, the largest, to ROW_LAST_CLASS), and the warp tier
// starts at the class of 32 .. 63 keys.
constexpr uint32_t ROW_MIN_LOG2 = 6;
constexpr uint64_t ROW_MIN = 1ull << ROW_MIN_LOG2;
constexpr uint32_t ROW_CLASS = 63 - 12;
constexpr uint32_t ROW_LAST_CLASS = 63 - ROW_MIN_LOG2;
constexpr uint32_t WARP_CLASS = 63 - 5;
static_assert(ROW_TILE == (1u << 13) && DEV_MIN_LOG2 == 13,
              "the row tier ends where the device tier starts");
static_assert(ROW_MIN > WARP_SEG_MAX && ROW_MIN <= SEG_TILE,
              "the row tier starts above the warp tier and at most one on-chip tile");
static_assert(WARP_SEG_MAX == 63, "the warp tier is the classes of 1 .. 63 keys");

struct SegControl {
    uint32_t class_count[SIZE_CLASSES];
    uint32_t class_cursor[SIZE_CLASSES];
    uint32_t work;
    uint32_t done;
    uint32_t n_large;                  // segments of the device tier (a prefix of the order)
    uint32_t dev_tiles;                // device tiles handed out
    uint32_t dev_counter[MAX_PASSES];  // tile claims of each device-tier pass
    uint32_t long_tiles;               // device tiles of segments counted tile-parallel
};

// One device tile, written when tiles are handed out (seg_tiles_kernel) and
// completed with the segment's moving digit groups when the segment is
// counted (seg_sort_kernel): everything a device-tier pass needs to start
// loading the tile, in one 16-byte read after its claim.
struct TileMeta {
    uint64_t lo;      // first key of the owning segment
    uint32_t len;     // keys in the segment (at most RS_MAX_N)
    uint32_t lt_use;  // bits 0..23: tile index within the segment; 24..31: moving groups
};
static_assert(sizeof(TileMeta) == 16, "one 16-byte load");

struct SegArgs {
    const void* keys_in;
    void* keys_out;
    const void* vals_in;
    void* vals_out;
    void* keys_tmp;
    void* vals_tmp;
    uint64_t n;
    const uint64_t* seg_offsets;  // NULL: equal segments of seg_len keys
    uint64_t seg_len;
    uint64_t num_segs;
    uint32_t iota;                // payload = index of the key within its segment
    const uint32_t* order;
    SegControl* ctl;
    uint32_t passes;
    uint32_t in_is_out;
    CodecParams prm;
    uint32_t* status;
    // device tier
    uint32_t* bins;        // [n_large][passes][RADIX] raster-order starts within the segment
    uint32_t* dev_use;     // [n_large] bit p: digit group p moves data
    uint32_t* tile_start;  // [n_large] first device tile of the segment
    uint32_t* tile_owner;  // [max_tiles] order index of the segment owning a tile
    uint32_t* long_tile;   // [max_tiles] the device tiles of segments of count_par_min keys or more
    TileMeta* tile_meta;   // [max_tiles]
    uint32_t prefetch_ahead;  // device tiles between a tile and the one it prefetches
    uint32_t* lookback[2];
    uint64_t max_tiles;
    uint32_t n_large_max;  // room of bins, dev_use and tile_start
    uint32_t dev_tile;     // keys per device tile
    // device-tier segments of at least this many keys are counted tile by
    // tile by seg_count_kernel; shorter ones by the CTA that takes them
    uint64_t count_par_min;
    // segments of ROW_MIN .. ROW_TILE-1 keys are sorted whole on chip by
    // seg_rows_kernel (4-byte cells with no value, a 4-byte value or an
    // argsort); seg_sort_kernel leaves them out
    uint32_t row_tier;
};

// Size class: 0 holds the largest segments (2^63 and up), 63 the empty ones.
__device__ __forceinline__ uint32_t size_class(uint64_t len) {
    return len ? (uint32_t)__clzll(len) : SIZE_CLASSES - 1;
}

__device__ __forceinline__ bool seg_bounds(const SegArgs& a, uint64_t s, uint64_t& lo,
                                           uint64_t& hi) {
    if (!a.seg_offsets) {
        lo = s * a.seg_len;
        hi = lo + a.seg_len;
        return a.seg_len <= SEG_MAX_LEN;
    }
    lo = a.seg_offsets[s];
    hi = a.seg_offsets[s + 1];
    return lo <= hi && hi <= a.n && hi - lo <= SEG_MAX_LEN;
}

__global__ void __launch_bounds__(BLOCK) seg_size_kernel(SegArgs a) {
    __shared__ uint32_t s_count[SIZE_CLASSES];
    __shared__ uint32_t s_last;
    const uint32_t t = threadIdx.x;
    if (t < SIZE_CLASSES) s_count[t] = 0;
    __syncthreads();
    bool bad = false;
    for (uint64_t s = (uint64_t)blockIdx.x * BLOCK + t; s < a.num_segs;
         s += (uint64_t)gridDim.x * BLOCK) {
        uint64_t lo, hi;
        if (!seg_bounds(a, s, lo, hi)) {
            bad = true;
            continue;
        }
        atomicAdd(&s_count[size_class(hi - lo)], 1u);
    }
    if (bad) atomicOr(a.status, STATUS_RANGE);
    __syncthreads();
    if (t < SIZE_CLASSES && s_count[t]) atomicAdd(&a.ctl->class_count[t], s_count[t]);
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&a.ctl->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (t == 0) {  // exclusive scan of 64 class counts: largest class first
        uint32_t run = 0;
        for (int c = 0; c < SIZE_CLASSES; c++) {
            a.ctl->class_cursor[c] = run;
            run += __ldcg(&a.ctl->class_count[c]);
            // (more large segments than n / 2^DEV_MIN_LOG2 only when
            // segments overlap, which breaks the offsets' contract: it is
            // flagged and the rest are swept by single CTAs)
            if (c == (int)DEV_CLASS_MAX) {
                a.ctl->n_large = min(run, a.n_large_max);
                if (run > a.n_large_max) atomicOr(a.status, STATUS_RANGE);
            }
        }
    }
}

// Device tiles for the large segments (order[0 .. n_large)): each takes a
// contiguous range of ceil(len / dev_tile) tiles from a shared counter, and
// every tile records its owner and description.  Ranges come out in any
// order; within a segment the tiles are in input order.  Each lane claims
// the range of one segment, then the warp writes the entries of its 32
// segments one segment at a time, 32 tiles per step, so that a single long
// segment (an argsort of one array has 2^28 / dev_tile tiles) is not written
// by one thread.
__global__ void __launch_bounds__(BLOCK) seg_tiles_kernel(SegArgs a) {
    const uint32_t n_large = __ldcg(&a.ctl->n_large);
    const uint32_t lane = lane_id();
    for (uint64_t base = (uint64_t)blockIdx.x * BLOCK + (threadIdx.x & ~31u); base < n_large;
         base += (uint64_t)gridDim.x * BLOCK) {
        const uint64_t i = base + lane;
        uint64_t lo = 0, hi = 0;
        uint32_t tiles = 0, start = 0;
        if (i < n_large) {
            seg_bounds(a, a.order[i], lo, hi);  // valid: bad bounds are in the last class
            tiles = (uint32_t)((hi - lo + a.dev_tile - 1) / a.dev_tile);
            start = atomicAdd(&a.ctl->dev_tiles, tiles);
            if ((uint64_t)start + tiles > a.max_tiles) {  // cannot happen: the host's bound
                atomicOr(a.status, STATUS_RANGE);
                a.tile_start[i] = 0xffffffffu;
                tiles = 0;
            } else {
                a.tile_start[i] = start;
            }
        }
        for (int src = 0; src < 32; src++) {
            const uint32_t st = __shfl_sync(0xffffffffu, tiles, src);
            if (st == 0) continue;  // warp-uniform
            const uint32_t s0 = __shfl_sync(0xffffffffu, start, src);
            const uint64_t slo = __shfl_sync(0xffffffffu, lo, src);
            const uint64_t shi = __shfl_sync(0xffffffffu, hi, src);
            const uint32_t owner = (uint32_t)(base + src);
            for (uint32_t j = lane; j < st; j += 32) {
                a.tile_owner[s0 + j] = owner;
                TileMeta m;
                m.lo = slo;
                m.len = (uint32_t)(shi - slo);
                m.lt_use = j;  // the moving groups are added when the segment is counted
                a.tile_meta[s0 + j] = m;
            }
            // a long segment's tiles are listed for seg_count_kernel, which
            // adds their counts into the segment's rows of bins: they start
            // at zero
            if (shi - slo >= a.count_par_min) {
                uint32_t ls = 0;
                if (lane == 0) ls = atomicAdd(&a.ctl->long_tiles, st);  // <= dev_tiles
                ls = __shfl_sync(0xffffffffu, ls, 0);
                for (uint32_t j = lane; j < st; j += 32) a.long_tile[ls + j] = s0 + j;
                for (uint32_t w = lane; w < a.passes * RADIX; w += 32)
                    a.bins[(uint64_t)owner * a.passes * RADIX + w] = 0;
            }
        }
    }
}

// The hashing cycle (§3.1) of the device tier's longest segments (those of
// at least count_par_min keys), one device tile per CTA step (a persistent
// grid): the tile's keys are counted for every digit group in shared memory
// and the non-zero counts are added into the owning segment's rows of bins,
// so such a segment is counted by as many CTAs as it has tiles, not by the
// one CTA of seg_sort_kernel that takes it.  That CTA then turns the counts
// into raster-order starts.
template <class C>
__global__ void __launch_bounds__(BLOCK) seg_count_kernel(SegArgs a) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    constexpr int U = 8;  // loads in flight per thread
    __shared__ uint32_t sh[MAX_PASSES][RADIX];
    __shared__ uint32_t s_slot;
    const uint32_t t = threadIdx.x;
    const uint32_t n_large = __ldcg(&a.ctl->n_large);
    const uint32_t dev_tiles = (uint32_t)min((uint64_t)__ldcg(&a.ctl->dev_tiles), a.max_tiles);
    const uint32_t long_tiles = min(__ldcg(&a.ctl->long_tiles), dev_tiles);
    const uint32_t words = a.passes * RADIX;
    const In* kin = static_cast<const In*>(a.keys_in);
    bool ok = true;
    // The counts of consecutive tiles of one segment (a CTA's tiles k, k+G,
    // ... of the list mostly share their segment) add up in shared memory
    // and reach the segment's rows in global memory once per segment.
    for (uint32_t i = t; i < words; i += BLOCK) (&sh[0][0])[i] = 0;
    if (t == 0) s_slot = 0xffffffffu;
    __syncthreads();
    auto flush = [&]() {
        const uint32_t cur = s_slot;
        if (cur != 0xffffffffu) {
            uint32_t* row = a.bins + (uint64_t)cur * words;
            for (uint32_t i = t; i < words; i += BLOCK) {
                const uint32_t v = (&sh[0][0])[i];
                if (v) atomicAdd(&row[i], v);
                (&sh[0][0])[i] = 0;
            }
        }
    };
    for (uint32_t k = blockIdx.x; k < long_tiles; k += gridDim.x) {
        const uint32_t g = a.long_tile[k];
        if (g >= dev_tiles) continue;  // cannot happen: written by seg_tiles_kernel
        // the tile's description and owner (uniform per CTA)
        const uint4 mw = __ldcg(reinterpret_cast<const uint4*>(&a.tile_meta[g]));
        const uint32_t slot = __ldcg(&a.tile_owner[g]);
        const uint64_t lo = (uint64_t)mw.x | ((uint64_t)mw.y << 32);
        const uint64_t len = mw.z;
        const uint64_t tb = (uint64_t)(mw.w & 0xffffffu) * a.dev_tile;
        if (!(slot < n_large && tb < len && lo + len <= a.n && len >= a.count_par_min)) continue;
        if (slot != s_slot) {  // uniform: every thread read s_slot after the last barrier
            flush();
            __syncthreads();
            if (t == 0) s_slot = slot;
        }
        const uint64_t base = lo + tb;
        const uint64_t end = min(lo + len, base + a.dev_tile);
        for (uint64_t j = base + t; j < end; j += (uint64_t)U * BLOCK) {
            In kv[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint64_t idx = j + (uint64_t)u * BLOCK;
                kv[u] = idx < end ? __ldcs(&kin[idx]) : In(0);
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (j + (uint64_t)u * BLOCK >= end) break;
                const Cell c = C::decode(kv[u], a.prm, ok);
#pragma unroll
                for (uint32_t p = 0; p < sizeof(Cell); p++)
                    if (p < a.passes) atomicAdd(&sh[p][digit_of(c, p * RADIX_BITS)], 1u);
            }
        }
        __syncthreads();  // this tile's counts are in, and s_slot is set
    }
    flush();
    if (!ok) atomicOr(a.status, STATUS_RANGE);
}

__global__ void __launch_bounds__(BLOCK) seg_order_kernel(SegArgs a, uint32_t* order) {
    for (uint64_t s = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; s < a.num_segs;
         s += (uint64_t)gridDim.x * BLOCK) {
        uint64_t lo, hi;
        const uint32_t c = seg_bounds(a, s, lo, hi) ? size_class(hi - lo) : SIZE_CLASSES - 1;
        order[atomicAdd(&a.ctl->class_cursor[c], 1u)] = (uint32_t)s;
    }
}

// Load one tile (positions [base, base+valid) of `src`) warp-striped over
// `rows` item rows per warp (rank_scatter's layout).  With iota_from != ~0
// the values are generated: position - iota_from.
template <class C, typename VS, bool kPairs, bool kDecode>
__device__ __forceinline__ void load_tile(const void* ksrc, const VS* vsrc, uint64_t base,
                                          uint32_t valid, const CodecParams& prm,
                                          uint64_t iota_from, typename C::Cell (&k)[SEG_IPT],
                                          VS (&v)[SEG_IPT], uint32_t* status,
                                          uint32_t rows = SEG_IPT) {
    using Cell = typename C::Cell;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t w0 = warp * 32 * rows + lane;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < SEG_IPT; i++) {
        const uint32_t j = w0 + i * 32;
        if ((uint32_t)i < rows && j < valid) {
            if constexpr (kDecode)
                k[i] = C::decode(static_cast<const typename C::In*>(ksrc)[base + j], prm, ok);
            else
                k[i] = static_cast<const Cell*>(ksrc)[base + j];
            if constexpr (kPairs)
                v[i] = iota_from != ~0ull ? (VS)(base + j - iota_from) : vsrc[base + j];
        }
    }
    if (!ok) atomicOr(status, STATUS_RANGE);
}

// One segment of at most WARP_SEG_MAX keys sorted by one warp: lane l holds
// positions l and l + 32; a key's output position is the number of keys of
// the segment before it in (cell, input position) order, which is its
// stable rank.  Every input is in registers before the first store, so the
// segment may be sorted in place.
template <class C, typename VS, bool kPairs>
__device__ __forceinline__ void warp_sort_segment(const SegArgs& a, uint32_t seg, uint32_t lane) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    using Out = typename C::Out;
    uint64_t lo, hi;
    if (!seg_bounds(a, seg, lo, hi) || hi == lo) return;  // bad bounds were flagged
    const uint32_t len = (uint32_t)(hi - lo);
    Cell c[2];
    VS v[2];
    bool ok = true;
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const uint32_t j = lane + 32 * e;
        c[e] = ~Cell(0);
        v[e] = VS(0);
        if (j < len) {
            c[e] = C::decode(static_cast<const In*>(a.keys_in)[lo + j], a.prm, ok);
            if constexpr (kPairs)
                v[e] = a.iota ? (VS)j : static_cast<const VS*>(a.vals_in)[lo + j];
        }
    }
    if (!ok) atomicOr(a.status, STATUS_RANGE);
    uint32_t r[2] = {0, 0};
#pragma unroll
    for (int e2 = 0; e2 < 2; e2++) {
        for (uint32_t src = 0; src < 32; src++) {
            const Cell o = __shfl_sync(0xffffffffu, c[e2], src);
            const uint32_t po = src + 32 * e2;
            if (po >= len) break;  // uniform across the warp
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const uint32_t pm = lane + 32 * e;
                r[e] += (o < c[e] || (o == c[e] && po < pm)) ? 1u : 0u;
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 2; e++) {
        if (lane + 32 * e < len) {
            static_cast<Out*>(a.keys_out)[lo + r[e]] = C::encode(c[e], a.prm);
            if constexpr (kPairs) static_cast<VS*>(a.vals_out)[lo + r[e]] = v[e];
        }
    }
}

// Resident CTAs per SM: three (80 registers a thread) measured 10% faster
// than two on 2^28 u32 keys + 4-byte values in log-uniform segments; shapes
// with an 8-byte cell or value keep two, since they spill at 80 registers.
template <class C, typename V>
constexpr int seg_ctas_per_sm() {
    return (sizeof(typename C::Cell) == 4 && (!ValTraits<V>::kPairs || sizeof(V) == 4)) ? 3 : 2;
}

template <class C, typename V>
__global__ void __launch_bounds__(BLOCK, seg_ctas_per_sm<C, V>()) seg_sort_kernel(SegArgs a) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    using Out = typename C::Out;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    using VS = typename std::conditional<kPairs, V, uint32_t>::type;

    __shared__ TileShared ts;
    __shared__ uint32_t s_hist[MAX_PASSES][RADIX];  // whole-segment counts (large segments)
    __shared__ uint32_t s_run[RADIX];              // running cell offsets of the sweep
    __shared__ uint32_t s_first, s_take;
    __shared__ uint32_t s_active[MAX_PASSES];
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const Stage<Cell, VS, kPairs, SEG_TILE> stage{smem_dyn};
    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    // The list is ordered by size class, largest first.  One counter step
    // claims one entry before the warp tier, skipping the row tier's (sorted
    // by seg_rows_kernel), or WARPS entries of the warp tier, one per warp.
    const uint64_t warp_from = __ldcg(&a.ctl->class_cursor[WARP_CLASS - 1]);
    const uint64_t row_begin =
        a.row_tier
            ? __ldcg(&a.ctl->class_cursor[ROW_CLASS]) - __ldcg(&a.ctl->class_count[ROW_CLASS])
            : 0;
    const uint64_t row_skip =
        a.row_tier ? __ldcg(&a.ctl->class_cursor[ROW_LAST_CLASS]) - row_begin : 0;

    while (true) {
        if (t == 0) {
            const uint64_t u = atomicAdd(&a.ctl->work, 1u);
            const uint64_t e = u < row_begin ? u : u + row_skip;  // order entry
            const uint64_t first = e < warp_from ? e : warp_from + (e - warp_from) * WARPS;
            s_first = (uint32_t)min(first, (uint64_t)a.num_segs);
            s_take = e < warp_from ? 1u : (uint32_t)WARPS;
        }
        __syncthreads();
        const uint32_t first_w = s_first, take = s_take;
        __syncthreads();
        if (first_w >= a.num_segs) return;
        if (take > 1) {
            if (first_w + warp < a.num_segs)
                warp_sort_segment<C, VS, kPairs>(a, a.order[first_w + warp], lane);
            continue;
        }
        const uint32_t seg = a.order[first_w];
        uint64_t lo, hi;
        if (!seg_bounds(a, seg, lo, hi) || hi == lo) continue;
        const uint64_t len = hi - lo;
        const VS* vin = static_cast<const VS*>(a.vals_in);
        VS* vout = static_cast<VS*>(a.vals_out);

        Cell k[SEG_IPT];
        VS v[SEG_IPT];
        const bool device_tier = first_w < __ldcg(&a.ctl->n_large);
        if (a.row_tier && !device_tier && len >= ROW_MIN && len < ROW_TILE) continue;
        if (!device_tier && len <= SEG_TILE) {
            // ---- one tile: sorted on chip, read once and written once, spread
            // over every warp in ceil(len / BLOCK) item rows ----
            const uint32_t valid = (uint32_t)len;
            const uint32_t rows = (valid + BLOCK - 1) / BLOCK;
            load_tile<C, VS, kPairs, true>(a.keys_in, vin, lo, valid, a.prm,
                                           a.iota ? lo : ~0ull, k, v, a.status, rows);
            const uint32_t w0 = warp * 32 * rows + lane;
            for (uint32_t p = 0; p < a.passes; p++) {
                rank_scatter<Cell, VS, SEG_IPT, kPairs>(k, v, valid, p * RADIX_BITS, ts, stage,
                                                        nullptr, rows);
#pragma unroll
                for (int i = 0; i < SEG_IPT; i++) {
                    const uint32_t j = w0 + i * 32;
                    if ((uint32_t)i < rows && j < valid) stage.get(j, k[i], v[i]);
                }
                __syncthreads();  // the staged tile is rewritten by the next group
            }
#pragma unroll
            for (int i = 0; i < SEG_IPT; i++) {
                const uint32_t j = w0 + i * 32;
                if ((uint32_t)i < rows && j < valid) {
                    static_cast<Out*>(a.keys_out)[lo + j] = C::encode(k[i], a.prm);
                    if constexpr (kPairs) vout[lo + j] = v[i];
                }
            }
            continue;
        }

        // ---- above one tile: count every digit group in one read (the
        // device tier's longest segments were counted tile by tile by
        // seg_count_kernel) ----
        if (device_tier && len >= a.count_par_min) {
            const uint32_t* row = a.bins + (uint64_t)first_w * a.passes * RADIX;
            for (uint32_t i = t; i < a.passes * RADIX; i += BLOCK) (&s_hist[0][0])[i] = row[i];
        } else {
            for (uint32_t i = t; i < MAX_PASSES * RADIX; i += BLOCK) (&s_hist[0][0])[i] = 0;
            __syncthreads();
            bool ok = true;
            const In* kin = static_cast<const In*>(a.keys_in);
            // eight loads in flight per thread, and the segment streaming
            // into L2 ahead of them: one bulk prefetch of the first PF_STEPS
            // loop steps, then each step prefetches the one PF_STEPS on
            constexpr int U = 8;
            constexpr uint64_t STEP = (uint64_t)U * BLOCK;
            constexpr uint64_t PF_STEPS = 8;
            if (t == 0) prefetch_lines_l2(kin + lo, min(len, PF_STEPS * STEP) * sizeof(In));
            for (uint64_t j = lo + t; j < hi; j += STEP) {
                if (t == 0 && j + PF_STEPS * STEP < hi) {  // j is the step's first key
                    const uint64_t pf = j + PF_STEPS * STEP;
                    prefetch_lines_l2(kin + pf, min(hi - pf, STEP) * sizeof(In));
                }
                In kv[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const uint64_t idx = j + (uint64_t)u * BLOCK;
                    kv[u] = idx < hi ? __ldcs(&kin[idx]) : In(0);
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (j + (uint64_t)u * BLOCK >= hi) break;
                    const Cell c = C::decode(kv[u], a.prm, ok);
#pragma unroll
                    for (uint32_t p = 0; p < sizeof(Cell); p++)
                        if (p < a.passes) atomicAdd(&s_hist[p][digit_of(c, p * RADIX_BITS)], 1u);
                }
            }
            if (!ok) atomicOr(a.status, STATUS_RANGE);
        }
        __syncthreads();
        // raster-order starts per group; a group with one occupied cell is an
        // identity permutation and is skipped
        for (uint32_t p = 0; p < a.passes; p++) {
            const uint32_t h = s_hist[p][t];
            uint32_t total;
            const uint32_t e = block_exclusive_scan(h, ts.warp_sum, &total);
            const int occupied = __syncthreads_count(h != 0);
            if (device_tier)
                a.bins[((size_t)first_w * a.passes + p) * RADIX + t] = e;
            else
                s_hist[p][t] = e;
            if (t == 0) s_active[p] = occupied > 1;
        }
        __syncthreads();
        // route as the device-wide sort does: the last moving group writes OUT,
        // earlier ones alternate TMP/OUT, the first reads IN; in place needs an
        // even count of moving groups (a trivial one is switched back on), out
        // of place at least one (two for an in-place argsort, which must write
        // its indices); the pass count is even, so a trivial group is there
        uint32_t use = 0;
        for (uint32_t p = 0; p < a.passes; p++) use |= (s_active[p] ? 1u : 0u) << p;
        {
            const uint32_t act = __popc(use);
            uint32_t need = a.in_is_out ? (act & 1u) : (act == 0);
            if (a.in_is_out && act == 0 && a.iota) need = 2;
            for (uint32_t p = 0; p < a.passes && need; p++)
                if (!(use >> p & 1u)) {
                    use |= 1u << p;
                    need--;
                }
        }
        if (device_tier) {
            // the device tier moves this segment: its starts are stored above
            if (t == 0) a.dev_use[first_w] = use;
            const uint32_t ts0 = a.tile_start[first_w];
            if (ts0 != 0xffffffffu) {
                const uint32_t ntiles = (uint32_t)((len + a.dev_tile - 1) / a.dev_tile);
                for (uint32_t j = t; j < ntiles; j += BLOCK)
                    a.tile_meta[ts0 + j].lt_use = j | (use << 24);
            }
            continue;  // (s_hist is cleared again after the next loop-top barrier)
        }

        // ---- swept by this CTA: per moving group, the segment's tiles in
        // input order with running cell offsets in shared memory ----
        const uint32_t act = __popc(use);
        uint32_t done = 0;
        uint32_t src_buf = BUF_IN;
        for (uint32_t p = 0; p < a.passes; p++) {
            if (!(use >> p & 1u)) continue;
            const uint32_t from_end = act - 1 - done;
            const uint32_t dst_buf = (from_end & 1u) ? BUF_TMP : BUF_OUT;
            const bool first = done == 0, last = from_end == 0;
            // Every buffer is addressed from this segment's own start.  Cells
            // parked in OUT live inside the segment's byte range of OUT, which
            // matters when a cell is narrower than an output key (decimal
            // keys: 32-bit cells in an int64 buffer) -- indexing OUT as a cell
            // array would run into the next segments' bytes.
            auto cell_base = [&](uint32_t b) -> void* {
                if (b == BUF_TMP) return static_cast<Cell*>(a.keys_tmp) + lo;
                return static_cast<unsigned char*>(a.keys_out) + lo * sizeof(Out);
            };
            const void* ksrc = src_buf == BUF_IN
                                   ? static_cast<const void*>(static_cast<const In*>(a.keys_in) + lo)
                                   : cell_base(src_buf);
            const VS* vsrc = static_cast<const VS*>(
                src_buf == BUF_IN ? a.vals_in : (src_buf == BUF_TMP ? a.vals_tmp : a.vals_out));
            if (vsrc) vsrc += lo;
            void* kdst = cell_base(dst_buf);
            VS* vdst = static_cast<VS*>(dst_buf == BUF_TMP ? a.vals_tmp : a.vals_out);
            if (vdst) vdst += lo;
            const uint32_t shift = p * RADIX_BITS;
            s_run[t] = s_hist[p][t];
            ts.count[t] = 0;  // the first tile adds nothing to s_run
            __syncthreads();
            for (uint64_t base = 0; base < len; base += SEG_TILE) {
                const uint32_t valid = (uint32_t)min((uint64_t)SEG_TILE, len - base);
                const uint32_t rows = (valid + BLOCK - 1) / BLOCK;  // the last tile: spread
                if (first)
                    load_tile<C, VS, kPairs, true>(ksrc, vsrc, base, valid, a.prm,
                                                   a.iota ? 0ull : ~0ull, k, v, a.status, rows);
                else
                    load_tile<C, VS, kPairs, false>(ksrc, vsrc, base, valid, a.prm, ~0ull, k, v,
                                                    a.status, rows);
                if (valid == SEG_TILE)  // every tile but a segment's last: no position tests
                    rank_scatter<Cell, VS, SEG_IPT, kPairs, false, true>(k, v, valid, shift, ts,
                                                                         stage, s_run);
                else
                    rank_scatter<Cell, VS, SEG_IPT, kPairs>(k, v, valid, shift, ts, stage, s_run,
                                                            rows);
                for (uint32_t j = t; j < valid; j += BLOCK) {
                    Cell c;
                    VS val;
                    stage.get(j, c, val);
                    const uint32_t d = digit_of(c, shift);
                    const uint64_t g = s_run[d] + (j - ts.excl[d]);  // within the segment
                    if (last)
                        static_cast<Out*>(kdst)[g] = C::encode(c, a.prm);
                    else
                        static_cast<Cell*>(kdst)[g] = c;
                    if constexpr (kPairs) vdst[g] = val;
                }
                // (the next tile's rank_scatter moves s_run on after its
                // first barrier, once every thread is past this write-out)
            }
            // the write-out above reads s_run, the staged tile and ts: done before the
            // next group resets them; also orders this group's global writes
            // before the next group's reads
            __syncthreads();
            src_buf = dst_buf;
            done++;
        }
    }
}

// The row tier: segments of ROW_MIN .. ROW_TILE-1 keys, which are exactly
// the size classes ROW_CLASS .. ROW_LAST_CLASS of the ordered list, each
// sorted whole on chip by one CTA as the row kernel sorts an equal row: one
// read, a rank per non-trivial digit group, one write (16 bytes per key and
// value; the sweep it replaced above 4096 keys moved 4 + 16 per digit
// group).  A row shorter than the tile is padded to a multiple of 4 * BLOCK
// keys and ranked spread over every warp, with no position tests, and the
// table match (the row kernel's 32-key shape has room for its constants).
// One CTA takes every gridDim.x-th entry: the list is ordered by size, so
// each CTA gets the same mix.

template <class C, typename V, typename VR>
__global__ void __launch_bounds__(BLOCK, 2) seg_rows_kernel(SegArgs a) {
    using Cell = typename C::Cell;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    using VS = typename std::conditional<kPairs, VR, uint32_t>::type;
    __shared__ TileShared ts;
    __shared__ Cell s_ref;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const Stage<Cell, VS, kPairs, ROW_TILE> stage{smem_dyn};
    const uint32_t begin =
        __ldcg(&a.ctl->class_cursor[ROW_CLASS]) - __ldcg(&a.ctl->class_count[ROW_CLASS]);
    const uint32_t end = __ldcg(&a.ctl->class_cursor[ROW_LAST_CLASS]);
    RowsArgs ra{};
    ra.keys_in = a.keys_in;
    ra.keys_out = a.keys_out;
    ra.vals_in = a.vals_in;
    ra.vals_out = a.vals_out;
    ra.iota = a.iota;
    ra.passes = a.passes;
    ra.prm = a.prm;
    ra.status = a.status;
    for (uint32_t r = begin + blockIdx.x; r < end; r += gridDim.x) {
        uint64_t lo, hi;
        if (!seg_bounds(a, a.order[r], lo, hi)) continue;  // (uniform per CTA)
        const uint64_t len = hi - lo;
        if (len < ROW_MIN || len >= ROW_TILE) continue;
        sort_row<C, V, ROW_IPT, VR, true, false>(ra, lo, (uint32_t)len, ts, s_ref, stage);
    }
}

// The device tier's count and rank over the first `rows` item rows of a
// warp (all of them with kAll: a full tile, no row test).  rows is a
// multiple of ROWS_Q.
template <bool kAll, int IPT, typename Cell>
__device__ __forceinline__ void count_rows(const Cell (&k)[IPT], uint32_t* wh, uint32_t shift,
                                           uint32_t rows) {
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (!kAll && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;  // block-uniform
        atomicAdd(&wh[digit_of(k[i], shift)], 1u);
    }
}

// Stable rank in (cell, input) order: wh holds the warp's next position of
// each cell; every item is written to its position in `stage`.
template <bool kAll, bool kLut, int IPT, typename Cell, typename VS, bool kPairs, int TILE>
__device__ __forceinline__ void rank_rows(const Cell (&k)[IPT], const VS (&v)[IPT], uint32_t* wh,
                                          uint32_t shift, uint32_t rows, const LaneBits& lbits,
                                          const Stage<Cell, VS, kPairs, TILE>& stage) {
    const uint32_t lt_mask = lanemask_lt(), gt_mask = lanemask_gt();
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if (!kAll && i % ROWS_Q == 0 && (uint32_t)i >= rows) break;  // block-uniform
        const uint32_t dk = digit_of(k[i], shift);
        const uint32_t peers = peer_mask<kLut>(dk, lbits);
        uint32_t* slot_p = &wh[dk];
        const uint32_t pos0 = *slot_p;
        const uint32_t below = __popc(peers & lt_mask);
        __syncwarp();
        if ((peers & gt_mask) == 0) *slot_p = pos0 + below + 1;
        stage.put(pos0 + below, k[i], v[i]);
        __syncwarp();
    }
}

// The device tier: one digit group over every tile of every segment of at
// least SEG_TILE keys.  Persistent CTAs claim device tiles in order from a
// counter, one claim per tile; a tile covers dev_tile consecutive keys of one
// segment.  Like the device-wide pass it counts, publishes its per-cell
// aggregate, ranks in (cell, input) order through shared memory, looks back
// for the counts of the segment's earlier tiles and writes out.  A segment's
// first tile publishes an inclusive prefix, so no look-back walks into
// another segment.  Groups that move no data for a segment (dev_use) are
// skipped, and its buffers alternate over the moving groups only.
// (two CTAs per SM for every shape: the segment bookkeeping of the
// persistent loop does not fit the 80 registers of three)
template <class C, typename V, int IPT>
__global__ void __launch_bounds__(BLOCK, 2) seg_pass_kernel(SegArgs a, uint32_t pass) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    using Out = typename C::Out;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    constexpr uint32_t TILE = BLOCK * IPT;
    using VS = typename std::conditional<kPairs, V, uint32_t>::type;

    __shared__ uint32_t ws[WARPS][RADIX];  // per-warp counts, then next positions
    __shared__ uint32_t s_bin[RADIX];      // segment position of tile-local index 0, per cell
    __shared__ uint32_t s_warp[WARPS];
    __shared__ uint32_t s_tile;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const Stage<Cell, VS, kPairs, TILE> stage{smem_dyn};
    constexpr bool kLut = PassShape<C, V>::kLut && IPT == PassShape<C, V>::kIPT;
    const LaneBits lbits = lane_bits();

    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    const uint32_t n_large = __ldcg(&a.ctl->n_large);
    const uint32_t dev_tiles = (uint32_t)min((uint64_t)__ldcg(&a.ctl->dev_tiles), a.max_tiles);
    uint32_t* const lookback = a.lookback[pass & 1];
    uint32_t* const lookback_next = a.lookback[(pass + 1) & 1];
    const uint32_t shift = pass * RADIX_BITS;

    while (true) {
        if (t == 0) s_tile = atomicAdd(&a.ctl->dev_counter[pass], 1u);
        for (uint32_t d = lane; d < RADIX; d += 32) ws[warp][d] = 0;
        __syncthreads();
        const uint32_t g = s_tile;
        if (g >= dev_tiles) return;
        lookback_next[(uint64_t)g * RADIX + t] = 0;  // the next group's row of this tile
        // the tile's description and owner, one round trip; every thread reads
        // the same words, so the tests are uniform
        const uint4 mw = __ldcg(reinterpret_cast<const uint4*>(&a.tile_meta[g]));
        const uint32_t slot = __ldcg(&a.tile_owner[g]);
        // the tile claimed about half a residency later (tiles are claimed in
        // order): the last thread reads its record in the same round trip and
        // prefetches its keys and values into L2 (a TMA bulk prefetch of the
        // whole 16-byte lines in range), so their loads do not wait on DRAM
        const uint32_t pg = g + a.prefetch_ahead;
        if (a.prefetch_ahead && t == BLOCK - 1 && pg < dev_tiles) {
            const uint4 pm = __ldcg(reinterpret_cast<const uint4*>(&a.tile_meta[pg]));
            const uint64_t plo = (uint64_t)pm.x | ((uint64_t)pm.y << 32);
            const uint64_t plen = pm.z, ptb = (uint64_t)(pm.w & 0xffffffu) * TILE;
            const uint32_t puse = pm.w >> 24;
            if ((puse >> pass & 1u) && ptb < plen && plo + plen <= a.n) {
                const uint64_t pvalid = min((uint64_t)TILE, plen - ptb);
                const uint32_t pf_end = __popc(puse) - 1 - __popc(puse & ((1u << pass) - 1u));
                const bool pfirst = (puse & ((1u << pass) - 1u)) == 0;
                const uint32_t psrc = pfirst ? BUF_IN : (((pf_end + 1) & 1u) ? BUF_TMP : BUF_OUT);
                const char* kp;
                uint64_t kes = sizeof(Cell);
                if (psrc == BUF_IN) {
                    kp = static_cast<const char*>(a.keys_in) + (plo + ptb) * sizeof(In);
                    kes = sizeof(In);
                } else if (psrc == BUF_TMP) {
                    kp = reinterpret_cast<const char*>(static_cast<const Cell*>(a.keys_tmp) + plo + ptb);
                } else {
                    kp = static_cast<const char*>(a.keys_out) + plo * sizeof(Out) + ptb * sizeof(Cell);
                }
                prefetch_lines_l2(kp, pvalid * kes);
                if (kPairs && !(pfirst && a.iota)) {
                    const VS* vb = static_cast<const VS*>(
                        psrc == BUF_IN ? a.vals_in : (psrc == BUF_TMP ? a.vals_tmp : a.vals_out));
                    prefetch_lines_l2(vb + plo + ptb, pvalid * sizeof(VS));
                }
            }
        }
        const uint64_t lo = (uint64_t)mw.x | ((uint64_t)mw.y << 32);
        const uint64_t len = mw.z;
        const uint32_t lt = mw.w & 0xffffffu;  // tile index within the segment
        const uint32_t use = mw.w >> 24;
        const uint64_t tbase = (uint64_t)lt * TILE;
        const bool ok = slot < n_large && tbase < len && lo + len <= a.n;
        if (!ok || !(use >> pass & 1u)) {
            __syncthreads();  // everyone has read s_tile before the next claim
            continue;
        }
        const bool full = tbase + TILE <= len;
        const uint32_t valid = full ? TILE : (uint32_t)(len - tbase);
        // a segment's last tile is spread over every warp in `rows` item rows
        // (a multiple of ROWS_Q), so its count and rank cost what it holds,
        // not a whole tile
        static_assert(IPT % ROWS_Q == 0, "item rows are skipped ROWS_Q at a time");
        const uint32_t rows =
            full ? (uint32_t)IPT
                 : min((uint32_t)IPT, (valid + BLOCK * ROWS_Q - 1) / (BLOCK * ROWS_Q) * ROWS_Q);
        const uint32_t from_end = __popc(use) - 1 - __popc(use & ((1u << pass) - 1u));
        const bool first = (use & ((1u << pass) - 1u)) == 0, last = from_end == 0;
        const uint32_t dstb = (from_end & 1u) ? BUF_TMP : BUF_OUT;
        const uint32_t srcb = first ? BUF_IN : (((from_end + 1) & 1u) ? BUF_TMP : BUF_OUT);
        // Every buffer is addressed from the segment's start.  Cells parked in
        // OUT live inside the segment's byte range of OUT (a cell may be
        // narrower than an output key).
        Cell* const tmp_cells = static_cast<Cell*>(a.keys_tmp) + lo;
        Cell* const out_cells =
            reinterpret_cast<Cell*>(static_cast<unsigned char*>(a.keys_out) + lo * sizeof(Out));

        // ---- load (warp-striped: warp w owns tile items [w*32*rows, (w+1)*32*rows)) ----
        const uint32_t w0 = warp * 32 * rows + lane;
        Cell k[IPT];
        VS v[IPT];
        if (srcb == BUF_IN) {
            const In* in = static_cast<const In*>(a.keys_in) + lo + tbase + w0;
            bool okd = true;  // range errors were recorded when the segment was counted
            if (full) {
#pragma unroll
                for (int i = 0; i < IPT; i++) k[i] = C::decode(__ldcs(&in[i * 32]), a.prm, okd);
            } else {
#pragma unroll
                for (int i = 0; i < IPT; i++)
                    k[i] = (uint32_t)i < rows && w0 + i * 32 < valid
                               ? C::decode(__ldcs(&in[i * 32]), a.prm, okd)
                               : ~Cell(0);
            }
        } else {
            const Cell* in = (srcb == BUF_TMP ? tmp_cells : out_cells) + tbase + w0;
            if (full) {
#pragma unroll
                for (int i = 0; i < IPT; i++) k[i] = __ldcs(&in[i * 32]);
            } else {
#pragma unroll
                for (int i = 0; i < IPT; i++)
                    k[i] = (uint32_t)i < rows && w0 + i * 32 < valid ? __ldcs(&in[i * 32]) : ~Cell(0);
            }
        }
        if constexpr (kPairs) {
            if (first && a.iota) {
#pragma unroll
                for (int i = 0; i < IPT; i++) v[i] = (VS)(tbase + w0 + i * 32);
            } else {
                const VS* vin = static_cast<const VS*>(srcb == BUF_IN ? a.vals_in
                                                       : (srcb == BUF_TMP ? a.vals_tmp : a.vals_out)) +
                                lo + tbase + w0;
                if (full) {
#pragma unroll
                    for (int i = 0; i < IPT; i++) v[i] = __ldcs(&vin[i * 32]);
                } else {
#pragma unroll
                    for (int i = 0; i < IPT; i++)
                        v[i] = (uint32_t)i < rows && w0 + i * 32 < valid ? __ldcs(&vin[i * 32]) : VS(0);
                }
            }
        }

        // ---- counts per (warp, cell), the tile's aggregate, tile-local starts ----
        if (full)
            count_rows<true>(k, ws[warp], shift, rows);
        else
            count_rows<false>(k, ws[warp], shift, rows);
        __syncthreads();
        const uint32_t d = t;  // this thread's cell
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < WARPS; w++) {
            const uint32_t x = ws[w][d];
            ws[w][d] = run;
            run += x;
        }
        // padding items carry cell ~0 (digit 255) and sit after every real item
        const uint32_t count = d == RADIX - 1 ? run - (BLOCK * rows - valid) : run;
        uint32_t* lb = lookback + (uint64_t)g * RADIX;
        st_relaxed(&lb[d], (lt == 0 ? LB_INCLUSIVE : LB_AGGREGATE) | count);
        uint32_t tile_total;
        const uint32_t excl = block_exclusive_scan_n<WARPS>(count, s_warp, &tile_total);
#pragma unroll
        for (int w = 0; w < WARPS; w++) ws[w][d] += excl;
        __syncthreads();

        // ---- stable rank in (cell, input) order, scattered into shared memory ----
        if (full)
            rank_rows<true, kLut>(k, v, ws[warp], shift, rows, lbits, stage);
        else
            rank_rows<false, kLut>(k, v, ws[warp], shift, rows, lbits, stage);

        // ---- look-back over the segment's earlier tiles ----
        uint32_t before = 0;
        if (lt > 0) {
            const uint32_t cell[1] = {d};
            uint32_t bf[1];
            lookback_cells<1>(lookback, g, cell, a.status, bf);
            before = bf[0];
            st_relaxed(&lb[d], LB_INCLUSIVE | ((before + count) & LB_VALUE));
        }
        s_bin[d] = a.bins[((size_t)slot * a.passes + pass) * RADIX + d] + before - excl;
        __syncthreads();

        // ---- coalesced write-out within the segment ----
        // (the clamp only acts after a timed-out wait: output unspecified)
        const uint32_t gmax = (uint32_t)(len - 1);
        if (last) {
            Out* out = static_cast<Out*>(a.keys_out) + lo;
            VS* vout = kPairs ? static_cast<VS*>(a.vals_out) + lo : nullptr;
            for (uint32_t j = t; j < valid; j += BLOCK) {
                Cell c;
                VS val;
                stage.get(j, c, val);
                const uint32_t gp = min(s_bin[digit_of(c, shift)] + j, gmax);
                __stcs(&out[gp], C::encode(c, a.prm));
                if constexpr (kPairs) __stcs(&vout[gp], val);
            }
        } else {
            Cell* out = dstb == BUF_TMP ? tmp_cells : out_cells;
            VS* vout = kPairs ? static_cast<VS*>(dstb == BUF_TMP ? a.vals_tmp : a.vals_out) + lo
                              : nullptr;
            for (uint32_t j = t; j < valid; j += BLOCK) {
                Cell c;
                VS val;
                stage.get(j, c, val);
                const uint32_t gp = min(s_bin[digit_of(c, shift)] + j, gmax);
                out[gp] = c;
                if constexpr (kPairs) vout[gp] = val;
            }
        }
        __syncthreads();  // the staged tile, s_bin and s_tile are reused by the next tile
    }
}

// Workspace of one segmented call.  The device tier needs, per possible
// large segment (at most n / SEG_TILE of them), the group starts and the
// moving-group mask, and per possible device tile (a large segment of len
// keys has ceil(len / dev_tile) <= len / dev_tile + 1 of them) an owner, an
// entry of the list of tiles counted tile-parallel, and two look-back rows.
struct SegLayout {
    size_t ctl, order, keys_tmp, vals_tmp, bins, dev_use, tile_start, tile_owner, long_tile,
        tile_meta, lookback0, lookback1, total;
    size_t n_large_max, max_tiles;
};

inline SegLayout seg_layout(size_t n, size_t num_segs, bool equal_segments, size_t cell_bytes,
                            size_t val_bytes, uint32_t passes, uint32_t dev_tile) {
    SegLayout L{};
    // equal segments: the host knows whether any reaches the device tier
    const bool device_tier = equal_segments
                                 ? num_segs && (n / num_segs) >= ((size_t)1 << DEV_MIN_LOG2)
                                 : true;
    L.n_large_max = device_tier ? std::min<size_t>(num_segs, n >> DEV_MIN_LOG2) : 0;
    L.max_tiles = L.n_large_max ? (n + dev_tile - 1) / dev_tile + L.n_large_max : 0;
    size_t at = 0;
    L.ctl = at;         at += align_up(sizeof(SegControl));
    L.order = at;       at += align_up(sizeof(uint32_t) * std::max<size_t>(num_segs, 1));
    L.keys_tmp = at;    at += align_up(cell_bytes * std::max<size_t>(n, 1));
    L.vals_tmp = at;    at += align_up(val_bytes * std::max<size_t>(n, 1));
    L.bins = at;        at += align_up(sizeof(uint32_t) * L.n_large_max * passes * RADIX);
    L.dev_use = at;     at += align_up(sizeof(uint32_t) * L.n_large_max);
    L.tile_start = at;  at += align_up(sizeof(uint32_t) * L.n_large_max);
    L.tile_owner = at;  at += align_up(sizeof(uint32_t) * L.max_tiles);
    L.long_tile = at;   at += align_up(sizeof(uint32_t) * L.max_tiles);
    L.tile_meta = at;   at += align_up(sizeof(TileMeta) * L.max_tiles);
    L.lookback0 = at;   at += align_up(sizeof(uint32_t) * RADIX * L.max_tiles);
    L.lookback1 = at;   at += align_up(sizeof(uint32_t) * RADIX * L.max_tiles);
    L.total = at;
    return L;
}

template <class C, typename V>
rs_status run_segmented(rs_ctx* ctx, const void* keys_in, void* keys_out, const void* vals_in,
                        void* vals_out, size_t n, const uint64_t* seg_offsets, size_t num_segs,
                        CodecParams prm, uint32_t cell_bits, void* temp, size_t* temp_bytes,
                        cudaStream_t st, bool iota) {
    using Cell = typename C::Cell;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    using VS = typename std::conditional<kPairs, V, uint32_t>::type;
    const size_t vbytes = kPairs ? sizeof(V) : 0;
    constexpr int DIPT = ipt_for<C, V>();
    constexpr uint32_t DTILE = BLOCK * DIPT;
    const uint32_t passes = passes_for(cell_bits);
    const SegLayout L = seg_layout(n, num_segs, seg_offsets == nullptr, sizeof(Cell), vbytes,
                                   passes, DTILE);
    if (!temp) {
        *temp_bytes = L.total;
        return RS_OK;
    }
    if (*temp_bytes < L.total) return RS_ERR_TEMP_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(temp) % 256) return RS_ERR_INVALID;
    if (num_segs == 0 || n == 0) return RS_OK;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;

    // equal rows of 64 .. ROW_TILE keys: one CTA per row sorts it on chip in
    // one read and one write (no size classes, no workspace).  Rows above
    // SMALL_TILE hold 32 keys per thread, which leaves room for 4-byte
    // values only; an argsort's indices travel as 32-bit words.
    const bool narrow_values = !kPairs || sizeof(VS) == 4 || iota;
    if (!seg_offsets && n / num_segs > WARP_SEG_MAX &&
        (n / num_segs <= SMALL_TILE || (n / num_segs <= ROW_TILE && narrow_values))) {
        const uint32_t len = (uint32_t)(n / num_segs);
        RowsArgs ra{};
        ra.keys_in = keys_in;
        ra.keys_out = keys_out;
        ra.vals_in = vals_in;
        ra.vals_out = vals_out;
        ra.rows = num_segs;
        ra.len = len;
        ra.iota = iota;
        ra.passes = passes_for(cell_bits);
        ra.prm = prm;
        ra.status = ctx->d_status;
        const int sms = sm_count(ctx->device);
        auto launch = [&](auto kern, uint32_t tile, size_t val_bytes) -> rs_status {
            const size_t smem = tile * (sizeof(Cell) + val_bytes);
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return RS_ERR_CUDA;
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem) !=
                    cudaSuccess ||
                per_sm < 1)
                per_sm = 1;
            const int grid = (int)std::min<size_t>((size_t)sms * per_sm, num_segs);
            LaunchTimer lt(ctx, KC_SEG, st);
            kern<<<grid, BLOCK, smem, st>>>(ra);
            return RS_OK;
        };
        const size_t vb = kPairs ? sizeof(VS) : 0;
        rs_status rs_;
        if (len == SMALL_TILE) {
            rs_ = launch(tile_rows_kernel<C, V, SMALL_IPT>, SMALL_TILE, vb);
        } else if (len < SMALL_TILE) {
            rs_ = launch(tile_rows_kernel<C, V, SMALL_IPT, V, true>, SMALL_TILE, vb);
        } else {
            if constexpr (!kPairs || sizeof(VS) == 4) {
                if (len == ROW_TILE)
                    rs_ = launch(tile_rows_kernel<C, V, ROW_IPT>, ROW_TILE, vb);
                else
                    rs_ = launch(tile_rows_kernel<C, V, ROW_IPT, V, true>, ROW_TILE, vb);
            } else {  // an argsort with 8-byte indices: carried as 32-bit words
                if (len == ROW_TILE)
                    rs_ = launch(tile_rows_kernel<C, V, ROW_IPT, uint32_t>, ROW_TILE, 4);
                else
                    rs_ = launch(tile_rows_kernel<C, V, ROW_IPT, uint32_t, true>, ROW_TILE, 4);
            }
        }
        if (rs_ != RS_OK) return rs_;
        return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
    }
    unsigned char* T = static_cast<unsigned char*>(temp);
    SegControl* ctl = reinterpret_cast<SegControl*>(T + L.ctl);
    uint32_t* order = reinterpret_cast<uint32_t*>(T + L.order);
    void* keys_tmp = T + L.keys_tmp;
    void* vals_tmp = kPairs ? (void*)(T + L.vals_tmp) : nullptr;

    if (cudaMemsetAsync(ctl, 0, sizeof(SegControl), st) != cudaSuccess) return RS_ERR_CUDA;
    // the device tier's first look-back buffer starts zeroed; each of its
    // passes clears the other buffer's rows for the next one
    if (L.max_tiles &&
        cudaMemsetAsync(T + L.lookback0, 0, sizeof(uint32_t) * RADIX * L.max_tiles, st) != cudaSuccess)
        return RS_ERR_CUDA;
    SegArgs a{};
    a.keys_in = keys_in;
    a.keys_out = keys_out;
    a.vals_in = vals_in;
    a.vals_out = vals_out;
    a.keys_tmp = keys_tmp;
    a.vals_tmp = vals_tmp;
    a.n = n;
    a.seg_offsets = seg_offsets;
    a.seg_len = seg_offsets ? 0 : n / num_segs;
    a.num_segs = num_segs;
    a.iota = iota;
    a.order = order;
    a.ctl = ctl;
    a.passes = passes;
    a.in_is_out = keys_in == keys_out;
    a.prm = prm;
    a.status = ctx->d_status;
    a.bins = reinterpret_cast<uint32_t*>(T + L.bins);
    a.dev_use = reinterpret_cast<uint32_t*>(T + L.dev_use);
    a.tile_start = reinterpret_cast<uint32_t*>(T + L.tile_start);
    a.tile_owner = reinterpret_cast<uint32_t*>(T + L.tile_owner);
    a.long_tile = reinterpret_cast<uint32_t*>(T + L.long_tile);
    a.tile_meta = reinterpret_cast<TileMeta*>(T + L.tile_meta);
    a.lookback[0] = reinterpret_cast<uint32_t*>(T + L.lookback0);
    a.lookback[1] = reinterpret_cast<uint32_t*>(T + L.lookback1);
    a.max_tiles = L.max_tiles;
    a.n_large_max = (uint32_t)L.n_large_max;
    a.dev_tile = DTILE;
    // the row tier holds 32 keys and 32 four-byte values per thread: 4-byte
    // cells with no value, a 4-byte value, or an argsort (indices carried as
    // 32-bit words)
    a.row_tier = sizeof(Cell) == 4 && (!kPairs || sizeof(VS) == 4 || iota);
    const int sms = sm_count(ctx->device);
    const size_t smem = sizeof(Cell) * SEG_TILE + (kPairs ? sizeof(VS) * SEG_TILE : 0);
    auto kern = seg_sort_kernel<C, V>;
    static std::atomic<bool> smem_set[64];  // zero-initialised: false
    if (ctx->device < 64 && !smem_set[ctx->device].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return RS_ERR_CUDA;
        smem_set[ctx->device].store(true, std::memory_order_release);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int grid = (int)std::min<size_t>((size_t)sms * per_sm, num_segs);
    // A segment longer than one CTA's share of the batch would keep its CTA
    // counting after the others are done: such segments (and only those, so
    // that a batch of many long segments still overlaps their counting with
    // the on-chip sorts) are counted tile-parallel.
    a.count_par_min = std::max<uint64_t>(4ull * DTILE, (n + (size_t)grid - 1) / (size_t)grid);
    const int grid_s = (int)std::max<size_t>(1, std::min<size_t>((num_segs + BLOCK - 1) / BLOCK,
                                                                 (size_t)sms * 4));
    {
        LaunchTimer lt(ctx, KC_SEG, st);
        seg_size_kernel<<<grid_s, BLOCK, 0, st>>>(a);
    }
    {
        LaunchTimer lt(ctx, KC_SEG, st);
        seg_order_kernel<<<grid_s, BLOCK, 0, st>>>(a, order);
    }
    if (L.n_large_max) {
        {
            LaunchTimer lt(ctx, KC_SEG, st);
            seg_tiles_kernel<<<grid_s, BLOCK, 0, st>>>(a);
        }
        // the longest segments' counts, tile-parallel (with equal segments
        // the host knows whether there are any)
        if (seg_offsets || n / num_segs >= a.count_par_min) {
            const int grid_c =
                (int)std::max<size_t>(1, std::min<size_t>(L.max_tiles, (size_t)sms * 4));
            LaunchTimer lt(ctx, KC_SEG, st);
            seg_count_kernel<C><<<grid_c, BLOCK, 0, st>>>(a);
        }
    }
    {
        LaunchTimer lt(ctx, KC_SEG, st);
        kern<<<grid, BLOCK, smem, st>>>(a);
    }
    if constexpr (sizeof(Cell) == 4) {
      if (a.row_tier) {
        // (an argsort's indices travel as 32-bit words, as in the row path)
        using VR = typename std::conditional<kPairs && sizeof(VS) == 8, uint32_t, VS>::type;
        auto rkern = seg_rows_kernel<C, V, VR>;
        const size_t rsmem = (size_t)ROW_TILE * (sizeof(Cell) + (kPairs ? sizeof(VR) : 0));
        static std::atomic<bool> rsmem_set[64];  // zero-initialised: false
        if (ctx->device < 64 && !rsmem_set[ctx->device].load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(rkern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)rsmem) != cudaSuccess)
                return RS_ERR_CUDA;
            rsmem_set[ctx->device].store(true, std::memory_order_release);
        }
        LaunchTimer lt(ctx, KC_SEG, st);
        rkern<<<sms * 2, BLOCK, rsmem, st>>>(a);
      }
    }
    if (L.n_large_max) {
        // the device tier: one launch per digit group over all large segments
        using DSmem = PassSmem<Cell, V, DIPT>;
        auto dkern = seg_pass_kernel<C, V, DIPT>;
        static std::atomic<bool> dsmem_set[64];  // zero-initialised: false
        if (ctx->device < 64 && !dsmem_set[ctx->device].load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(dkern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)DSmem::kBytes) != cudaSuccess)
                return RS_ERR_CUDA;
            dsmem_set[ctx->device].store(true, std::memory_order_release);
        }
        static int dper_sm[64] = {};
        int dper_local = 0;
        int& dps = ctx->device < 64 ? dper_sm[ctx->device] : dper_local;
        if (dps <= 0) {
            int occ = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dkern, BLOCK, DSmem::kBytes) !=
                    cudaSuccess ||
                occ < 1)
                occ = 1;
            dps = occ;
        }
        const int dgrid = (int)std::min<size_t>((size_t)sms * dps, L.max_tiles);
        a.prefetch_ahead = prefetch_ahead_for(dgrid);
        for (uint32_t p = 0; p < passes; p++) {
            LaunchTimer lt(ctx, KC_SEG, st);
            dkern<<<dgrid, BLOCK, DSmem::kBytes, st>>>(a, p);
        }
    }
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

// Widen an argsort's 32-bit indices into the caller's 64-bit output: the
// positions inside segments, [offsets[0], offsets[num_segs]) (offsets do not
// decrease), or all n for equal segments; the others stay unwritten.
__global__ void __launch_bounds__(BLOCK) widen_indices_kernel(const uint32_t* in, uint64_t* out,
                                                              const uint64_t* seg_offsets,
                                                              uint64_t num_segs, uint64_t n) {
    uint64_t lo = 0, hi = n;
    if (seg_offsets) {
        lo = seg_offsets[0];
        hi = min(seg_offsets[num_segs], n);
    }
    for (uint64_t j = lo + (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < hi;
         j += (uint64_t)gridDim.x * BLOCK)
        out[j] = in[j];
}

// An argsort with 8-byte indices outside the row path carries the indices as
// 32-bit words (a segment holds fewer than 2^30 keys): every digit pass moves
// 4 fewer bytes in and out per key, and one widening pass writes the 8-byte
// output at the end.  Workspace: the 32-bit sort's, then n 32-bit indices.
template <class C>
rs_status run_segmented_argsort64(rs_ctx* ctx, const void* keys_in, void* keys_out,
                                  void* vals_out, size_t n, const uint64_t* seg_offsets,
                                  size_t num_segs, CodecParams prm, uint32_t cell_bits,
                                  void* temp, size_t* temp_bytes, cudaStream_t st) {
    size_t inner = 0;
    rs_status s = run_segmented<C, uint32_t>(ctx, keys_in, keys_out, nullptr, nullptr, n,
                                             seg_offsets, num_segs, prm, cell_bits, nullptr,
                                             &inner, st, true);
    if (s != RS_OK) return s;
    const size_t idx_off = align_up(inner);
    const size_t total = idx_off + align_up(sizeof(uint32_t) * std::max<size_t>(n, 1));
    if (!temp) {
        *temp_bytes = total;
        return RS_OK;
    }
    if (*temp_bytes < total) return RS_ERR_TEMP_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(temp) % 256) return RS_ERR_INVALID;
    if (num_segs == 0 || n == 0) return RS_OK;
    uint32_t* idx32 = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(temp) + idx_off);
    size_t tb = inner;
    s = run_segmented<C, uint32_t>(ctx, keys_in, keys_out, nullptr, idx32, n, seg_offsets,
                                   num_segs, prm, cell_bits, temp, &tb, st, true);
    if (s != RS_OK) return s;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;
    const int grid = (int)std::max<size_t>(
        1, std::min<size_t>((n + BLOCK - 1) / BLOCK, (size_t)sm_count(ctx->device) * 8));
    LaunchTimer lt(ctx, KC_SEG, st);
    widen_indices_kernel<<<grid, BLOCK, 0, st>>>(idx32, static_cast<uint64_t*>(vals_out),
                                                 seg_offsets, num_segs, n);
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" rs_status rs_sort_segmented(rs_ctx* ctx, rs_key_type kt, const void* keys_in,
                                       void* keys_out, const void* vals_in, void* vals_out,
                                       size_t val_bytes, size_t n, const uint64_t* seg_offsets,
                                       size_t num_segs, const rs_key_params* params, void* temp,
                                       size_t* temp_bytes, rs_stream_t stream) {
    if (!ctx || !temp_bytes) return RS_ERR_INVALID;
    if (n > RS_MAX_SEGMENTED_N || num_segs > 0xfffffffeull) return RS_ERR_INVALID;
    if (kt != RS_KEY_U32 && kt != RS_KEY_U64 && kt != RS_KEY_I64_DEC && kt != RS_KEY_F32 &&
        kt != RS_KEY_F64)
        return RS_ERR_UNSUPPORTED;
    const size_t kbytes = (kt == RS_KEY_U32 || kt == RS_KEY_F32) ? 4 : 8;
    const bool pairs = vals_out != nullptr;
    const bool iota = pairs && vals_in == nullptr;
    if (pairs && val_bytes != 4 && val_bytes != 8) return RS_ERR_INVALID;
    if (!seg_offsets && num_segs > 0 && n % num_segs) return RS_ERR_INVALID;
    if (n > 0) {
        if (!keys_in || !keys_out || (reinterpret_cast<uintptr_t>(keys_in) % kbytes) ||
            (reinterpret_cast<uintptr_t>(keys_out) % kbytes))
            return RS_ERR_INVALID;
        if (pairs && ((reinterpret_cast<uintptr_t>(vals_in) % val_bytes) ||
                      (reinterpret_cast<uintptr_t>(vals_out) % val_bytes)))
            return RS_ERR_INVALID;
        if (pairs && !iota && ((keys_in == keys_out) != (vals_in == vals_out)))
            return RS_ERR_INVALID;
    }
    if (seg_offsets && (reinterpret_cast<uintptr_t>(seg_offsets) % 8)) return RS_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    CodecParams prm{0};
    uint32_t bits = kbytes * 8;
    if (kt == RS_KEY_I64_DEC) {
        if (!params || params->int_digits < 0 || params->frac_digits < 0 ||
            params->int_digits + params->frac_digits < 1 ||
            params->int_digits + params->frac_digits > 18)
            return RS_ERR_INVALID;
        uint64_t p10 = 1;
        for (int i = 0; i < params->int_digits + params->frac_digits; i++) p10 *= 10;
        prm.bias = p10 - 1;
        bits = 1;
        while (bits < 64 && ((2 * prm.bias) >> bits) != 0) bits++;
    }
    rs_status s;
    // an argsort to 8-byte indices that the row path does not take carries
    // 32-bit indices (run_segmented_argsort64); the row path carries them as
    // 32-bit words already
    const bool row_path = !seg_offsets && num_segs > 0 && n / num_segs > WARP_SEG_MAX &&
                          n / num_segs <= ROW_TILE;
    const bool argsort32 = iota && val_bytes == 8 && !row_path;
#define RS_SEG_CALL(CODEC)                                                                      \
    do {                                                                                        \
        if (!pairs)                                                                             \
            s = run_segmented<CODEC, NoVal>(ctx, keys_in, keys_out, nullptr, nullptr, n,        \
                                            seg_offsets, num_segs, prm, bits, temp, temp_bytes, \
                                            st, false);                                         \
        else if (val_bytes == 4)                                                                \
            s = run_segmented<CODEC, uint32_t>(ctx, keys_in, keys_out, vals_in, vals_out, n,    \
                                               seg_offsets, num_segs, prm, bits, temp,          \
                                               temp_bytes, st, iota);                           \
        else if (argsort32)                                                                     \
            s = run_segmented_argsort64<CODEC>(ctx, keys_in, keys_out, vals_out, n, seg_offsets,  \
                                               num_segs, prm, bits, temp, temp_bytes, st);      \
        else                                                                                    \
            s = run_segmented<CODEC, uint64_t>(ctx, keys_in, keys_out, vals_in, vals_out, n,    \
                                               seg_offsets, num_segs, prm, bits, temp,          \
                                               temp_bytes, st, iota);                           \
    } while (0)
    switch (kt) {
    case RS_KEY_U32: RS_SEG_CALL(CodecU32); break;
    case RS_KEY_U64: RS_SEG_CALL(CodecU64); break;
    case RS_KEY_F32: RS_SEG_CALL(CodecF32); break;
    case RS_KEY_F64: RS_SEG_CALL(CodecF64); break;
    default:
        if (2 * prm.bias <= 0xffffffffull)
            RS_SEG_CALL(CodecDec<uint32_t>);
        else
            RS_SEG_CALL(CodecDec<uint64_t>);
    }
#undef RS_SEG_CALL
    if (s != RS_OK && s != RS_ERR_TEMP_TOO_SMALL && s != RS_ERR_INVALID) ctx->host_error = s;
    return s;
}
