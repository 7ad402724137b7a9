// rs_kernels.cuh -- the Recombinant Sort hot path as CUDA kernels (sm_103a).
//
//   count_kernel  the hashing cycle (§3.1, Eq. 1): one read of the keys
//                 counts every key into the 256 cells of each digit group
//                 (and, while every cell index stays below FILL_CELLS, into
//                 one dense count array).  Its last CTA turns the counts into
//                 raster-order cell offsets (the extraction cycle's cursor
//                 overwrite_pos_at, §3.2) and the device-side plan.
//   pass_kernel   one digit group: stable in-tile ranking with warp ballots,
//                 a single-pass decoupled look-back exclusive scan across
//                 tiles in input order, and a scatter staged through shared
//                 memory so global writes coalesce.  Keys and payloads move
//                 together.
//   fill_kernel   keys only, one count array: write every occupied cell's
//                 key, rebuilt from its coordinates (Eq. 16), count times.
#pragma once

#include <type_traits>

#include "rs_device.cuh"

namespace rs {

// predecessor words loaded per look-back round trip: with 10240-pair tiles
// 2 measured best (1.163 ms per pass; 4: 1.168, 8: 1.176)
constexpr int LOOKBACK_WINDOW = 2;

// Tiles are claimed in input order, so while a CTA works on tile t the tiles
// claimed over the next part of a residency period are t + 1 .. t + R (R =
// resident CTAs of the grid).  Each tile starts an L2 prefetch of the keys and
// values of tile t + PassArgs::prefetch_ahead (the host sets it to a fraction
// PREFETCH_FRACTION of R), so that tile's loads find its data in L2 instead
// of waiting on DRAM.  Too far ahead and the lines are evicted before use.
constexpr float PREFETCH_FRACTION = 0.5f;

struct CountArgs {
    const void* keys_in;
    uint64_t n;
    uint32_t passes;        // digit groups of the cell index
    uint32_t fill_allowed;  // keys-only call: the dense count array may be used
    uint32_t in_is_out;     // keys_in == keys_out (an odd pass count is not allowed)
    uint32_t pad_;
    CodecParams prm;
    DevPlan* plan;
    uint32_t* hist;          // [passes][RADIX] counts
    uint32_t* bin_offsets;   // [passes][RADIX] raster-order exclusive offsets
    uint32_t* fill_hist;     // [FILL_CELLS]
    uint32_t* fill_offsets;  // [FILL_CELLS + 1]
    uint32_t* status;
    DevInfo* info;
    const uint32_t* skip;  // nullable: a non-zero word makes the whole sort a no-op
};

// ----------------------------------------------------------------------------
// Hashing cycle: count every key into each digit group's 256 cells.

// Shared-memory counts of 32-bit cells without bank conflicts: each lane owns
// a private copy of every counter, packed as 16-bit halves (cells d and d^1
// share a word), and lane l's copies all sit in bank l.  Word index of
// (group g, cell d, lane l): ((g * RADIX/2 + d/2) * 32 + l); half = d & 1.
// A CTA counts fewer than 32 * 65535 keys per lane copy (n < 2^30 over at
// least min(n / 16384, 8 per SM) CTAs), so the halves cannot overflow.
constexpr uint32_t LANE_HIST_WORDS = 2 * RADIX * 32;  // four groups of a 32-bit cell, two per word

template <class C, bool kFill>
__device__ __forceinline__ void count_one(typename C::In key, const CountArgs& a,
                                          uint32_t (*sh)[RADIX], uint32_t* lh, uint32_t lane,
                                          uint32_t* sfill, bool& ok, bool& big) {
    using Cell = typename C::Cell;
    const Cell cell = C::decode(key, a.prm, ok);
    // every byte of the cell is counted (a group beyond the key's passes is
    // never read by the plan); unrolled, no per-group test
    if constexpr (sizeof(Cell) == 4) {
        // groups 2q and 2q+1 share the word of (pair q, cell, lane): the low
        // half counts group 2q, the high half group 2q+1, so each group's
        // increment is a constant and its word offset is its byte of the
        // cell times 32 (one shift and one mask)
        const uint32_t c = (uint32_t)cell;
        uint32_t* const w = lh + lane;
        atomicAdd(w + ((c << 5) & 0x1FE0u), 1u);
        atomicAdd(w + ((c >> 3) & 0x1FE0u), 0x10000u);
        atomicAdd(w + RADIX * 32 + ((c >> 11) & 0x1FE0u), 1u);
        atomicAdd(w + RADIX * 32 + ((c >> 19) & 0x1FE0u), 0x10000u);
    } else {
#pragma unroll
        for (uint32_t p = 0; p < sizeof(Cell); p++)
            atomicAdd(&sh[p][digit_of(cell, p * RADIX_BITS)], 1u);
    }
    if constexpr (kFill) {
        if (!big) {
            if (cell < (Cell)FILL_CELLS)
                atomicAdd(&sfill[(uint32_t)cell], 1u);
            else
                big = true;
        }
    }
}

// The last CTA of count_kernel: offsets, trivial groups, routing.
static __device__ void make_plan(const CountArgs& a, uint32_t* s_warp) {
    __shared__ uint32_t s_trivial[MAX_PASSES];
    const uint32_t t = threadIdx.x;
    for (uint32_t p = 0; p < a.passes; p++) {
        const uint32_t h = __ldcg(&a.hist[p * RADIX + t]);
        uint32_t total;
        const uint32_t excl = block_exclusive_scan(h, s_warp, &total);
        a.bin_offsets[p * RADIX + t] = excl;
        const int occupied = __syncthreads_count(h != 0);
        if (t == 0) s_trivial[p] = occupied <= 1;  // every key in one cell: identity
    }
    const bool fill = a.fill_allowed && __ldcg(&a.plan->fill_impossible) == 0;
    if (fill) {
        // raster-order offsets of the dense count array: 16 cells per thread
        uint32_t local[FILL_CELLS / BLOCK];
        uint32_t sum = 0;
#pragma unroll
        for (int i = 0; i < (int)(FILL_CELLS / BLOCK); i++) {
            local[i] = __ldcg(&a.fill_hist[t * (FILL_CELLS / BLOCK) + i]);
            sum += local[i];
        }
        uint32_t total;
        uint32_t run = block_exclusive_scan(sum, s_warp, &total);
#pragma unroll
        for (int i = 0; i < (int)(FILL_CELLS / BLOCK); i++) {
            a.fill_offsets[t * (FILL_CELLS / BLOCK) + i] = run;
            run += local[i];
        }
        if (t == BLOCK - 1) a.fill_offsets[FILL_CELLS] = run;
    }
    __syncthreads();
    if (t == 0) {
        DevPlan* P = a.plan;
        uint32_t active[MAX_PASSES];
        uint32_t m = 0;
        for (uint32_t p = 0; p < a.passes; p++) {
            active[p] = fill ? 0u : (s_trivial[p] ? 0u : 1u);
            m += active[p];
        }
        if (!fill) {
            // In place, every pass alternates buffers, so the pass count must
            // be even; out of place, at least one pass must copy.  A trivial
            // group is an identity permutation, so running one costs nothing
            // in correctness.
            const bool need_one_more = a.in_is_out ? (m & 1u) : (m == 0);
            if (need_one_more) {
                for (uint32_t p = 0; p < a.passes; p++)
                    if (!active[p]) {
                        active[p] = 1;
                        m++;
                        break;
                    }
            }
        }
        // Route: the last active pass writes OUT; going backwards the
        // destinations alternate OUT, TMP, OUT, ...; the first reads IN.
        uint32_t k = 0, prev_dst = BUF_IN;
        P->first_active = MAX_PASSES;
        P->last_active = MAX_PASSES;
        for (uint32_t p = 0; p < a.passes; p++) {
            P->active[p] = active[p];
            if (!active[p]) continue;
            const uint32_t from_end = m - 1 - k;
            P->src[p] = prev_dst;
            P->dst[p] = (from_end & 1u) ? BUF_TMP : BUF_OUT;
            prev_dst = P->dst[p];
            if (P->first_active == MAX_PASSES) P->first_active = p;
            P->last_active = p;
            k++;
        }
        P->passes_run = m;
        P->mode = fill ? MODE_FILL : MODE_PASSES;
        a.info->mode = P->mode;
        a.info->passes_run = m;
    }
}

template <class C, bool kFill>
__global__ void __launch_bounds__(BLOCK) count_kernel(CountArgs a) {
    using In = typename C::In;
    if (a.skip && *a.skip) return;  // the plan stays zeroed: every pass inactive
    using Cell = typename C::Cell;
    constexpr bool kLaneHist = sizeof(Cell) == 4;
    __shared__ uint32_t sh[MAX_PASSES][RADIX];
    __shared__ uint32_t sfill[kFill ? FILL_CELLS : 1];
    __shared__ uint32_t s_warp[WARPS];
    __shared__ uint32_t s_last;
    extern __shared__ uint32_t lh[];  // LANE_HIST_WORDS when kLaneHist
    const uint32_t t = threadIdx.x, lane = lane_id();
    for (uint32_t i = t; i < MAX_PASSES * RADIX; i += BLOCK) (&sh[0][0])[i] = 0;
    if constexpr (kLaneHist)
        for (uint32_t i = t; i < LANE_HIST_WORDS; i += BLOCK) lh[i] = 0;
    if constexpr (kFill)
        for (uint32_t i = t; i < FILL_CELLS; i += BLOCK) sfill[i] = 0;
    __syncthreads();

    const In* keys = static_cast<const In*>(a.keys_in);
    bool ok = true;
    bool big = kFill ? (__ldcg(&a.plan->fill_impossible) != 0) : true;
    // 16-byte vector body with a scalar head and tail; n < 2^30, so 32-bit
    // indices suffice
    constexpr uint32_t VEC = 16 / sizeof(In);
    const uint32_t n = (uint32_t)a.n;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    uint32_t head = (uint32_t)(((16 - (addr & 15)) & 15) / sizeof(In));
    if (head > n) head = n;
    const uint32_t nvec = (n - head) / VEC;
    const uint32_t tail0 = head + nvec * VEC;
    const uint32_t gtid = blockIdx.x * BLOCK + t;
    const uint32_t gsize = gridDim.x * BLOCK;
    if (gtid < head) count_one<C, kFill>(keys[gtid], a, sh, lh, lane, sfill, ok, big);
    const uint4* vkeys = reinterpret_cast<const uint4*>(keys + head);
    // four independent 16-byte loads in flight per thread before counting
    uint32_t v = gtid;
    for (; v + 3 * gsize < nvec; v += 4 * gsize) {
        uint4 q[4];
#pragma unroll
        for (int u = 0; u < 4; u++) q[u] = __ldg(&vkeys[v + u * gsize]);
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const In* e = reinterpret_cast<const In*>(&q[u]);
#pragma unroll
            for (uint32_t j = 0; j < VEC; j++) count_one<C, kFill>(e[j], a, sh, lh, lane, sfill, ok, big);
        }
    }
    for (; v < nvec; v += gsize) {
        const uint4 q = __ldg(&vkeys[v]);
        const In* e = reinterpret_cast<const In*>(&q);
#pragma unroll
        for (uint32_t j = 0; j < VEC; j++) count_one<C, kFill>(e[j], a, sh, lh, lane, sfill, ok, big);
    }
    if (tail0 + gtid < n) count_one<C, kFill>(keys[tail0 + gtid], a, sh, lh, lane, sfill, ok, big);
    if (!ok) atomicOr(a.status, STATUS_RANGE);
    if (kFill && big) a.plan->fill_impossible = 1;
    __syncthreads();
    if constexpr (kLaneHist) {
        // fold the 32 lane copies: one row (group pair, cell) per warp step,
        // lane l reads the copy in bank l, a warp sum per 16-bit half
        const uint32_t warp = t >> 5;
        for (uint32_t row = warp; row < 2 * RADIX; row += WARPS) {
            const uint32_t w = lh[(row << 5) + lane];
            uint32_t lo = w & 0xffffu, hi = w >> 16;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo += __shfl_xor_sync(0xffffffffu, lo, o);
                hi += __shfl_xor_sync(0xffffffffu, hi, o);
            }
            if (lane == 0) {
                const uint32_t q = row / RADIX, d = row % RADIX;
                sh[2 * q][d] = lo;
                sh[2 * q + 1][d] = hi;
            }
        }
        __syncthreads();
    }

    for (uint32_t i = t; i < a.passes * RADIX; i += BLOCK) {
        const uint32_t c = (&sh[0][0])[i];
        if (c) atomicAdd(&a.hist[i], c);
    }
    if constexpr (kFill) {
        if (__ldcg(&a.plan->fill_impossible) == 0)
            for (uint32_t i = t; i < FILL_CELLS; i += BLOCK)
                if (sfill[i]) atomicAdd(&a.fill_hist[i], sfill[i]);
    }
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&a.plan->hist_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    make_plan(a, s_warp);
}

// ----------------------------------------------------------------------------
// One digit group: rank, look back, scatter.

struct PassArgs {
    const void* keys_in;
    void* keys_tmp;
    void* keys_out;
    const void* vals_in;
    void* vals_tmp;
    void* vals_out;
    uint64_t n;
    uint32_t pass;
    uint32_t shift;
    CodecParams prm;
    const DevPlan* plan;
    const uint32_t* bin_offsets;  // this group's 256 raster-order offsets
    uint32_t* lookback;           // [tiles][RADIX] for this pass
    uint32_t* lookback_next;      // cleared here for the next pass
    uint32_t* tile_counter;
    uint32_t* status;
    uint32_t prefetch_ahead;  // tiles; 0: no prefetch
};

// The prefetch distance for a grid of `resident` co-resident CTAs.
inline uint32_t prefetch_ahead_for(int resident) {
    return (uint32_t)((float)resident * PREFETCH_FRACTION);
}

struct NoVal {};

template <typename V>
struct ValTraits {
    static constexpr bool kPairs = true;
};
template <>
struct ValTraits<NoVal> {
    static constexpr bool kPairs = false;
};

// Tile shape of the pass kernel per (cell, value) type with 256-thread CTAs:
// keys per thread (kIPT) and the resident CTAs per SM that its register
// budget is compiled for (kCTAs).  Larger tiles amortise the per-tile scans
// and look-back over more keys, so every shape takes the largest tile that
// measured faster on GB300 (2^27-2^28 uniform keys):
//   32-bit cells: keys only 48 (3 CTAs/SM; 64 and 80 at 2 CTAs/SM slower),
//                 4-byte values 40 (2 CTAs/SM; 24 at 3 CTAs/SM, 32, 36, 44,
//                 48 slower), 8-byte values 28;
//   64-bit cells: keys only 40, 4-byte values 28, 8-byte values 24 (two
//                 staging tiles of 96 KB fill the SM's shared memory).
template <class C, typename V>
struct PassShape {
    static constexpr bool kPairs = ValTraits<V>::kPairs;
    static constexpr bool kCell4 = sizeof(typename C::Cell) == 4;
    static constexpr bool kVal8 = kPairs && sizeof(V) == 8;
    static constexpr int kIPT = kCell4 ? (!kPairs ? 48 : (kVal8 ? 28 : 40))
                                       : (!kPairs ? 40 : (kVal8 ? 24 : 28));
    static constexpr int kCTAs = (kCell4 && !kPairs) ? 3 : 2;
    // table match (match_digit_lut) where its five lane constants fit the
    // register budget without spilling; match_digit elsewhere
    static constexpr bool kLut = kCell4 && kPairs && !kVal8;
};

// The narrow tile for small sorts: 16 keys per thread at 3 CTAs per SM, for
// 4-byte cells with no value or a 4-byte value.  A sort of a few hundred
// thousand keys has too few 40-key tiles to occupy 152 SMs; the narrow tile
// gives it 2.5x as many (u32 pairs, whole sort: 2^14 keys 62 -> 50 us, 2^18
// 63 -> 55 us; even at 2^20, 72 vs 75 us; the wide tile from 2^22 on).
template <class C, typename V>
struct NarrowShape {
    static constexpr bool kHas = PassShape<C, V>::kCell4 && !PassShape<C, V>::kVal8;
    static constexpr int kIPT = 16;
    static constexpr int kCTAs = 3;
};

// Resident CTAs per SM a pass-kernel instantiation is compiled for.
template <class C, typename V, int IPT, int PB>
constexpr int pass_ctas() {
    if (PB != 256) return sizeof(typename C::Cell) == 4 ? 6 : 4;
    return IPT == PassShape<C, V>::kIPT ? PassShape<C, V>::kCTAs : NarrowShape<C, V>::kCTAs;
}

template <bool kLut>
__device__ __forceinline__ uint32_t peer_mask(uint32_t d, const LaneBits& L) {
    if constexpr (kLut)
        return match_digit_lut(d, L);
    else
        return match_digit(d);
}

// A ranked tile staged in shared memory.  4-byte cells with 4-byte values
// are kept as one 8-byte item (one shared store per key in the rank, one
// load per item in the write-out); other shapes keep keys and values in two
// arrays.
template <typename Cell, typename VS, bool kPairs, int TILE>
struct Stage {
    static constexpr bool kPacked = kPairs && sizeof(Cell) == 4 && sizeof(VS) == 4;
    unsigned char* base;
    __device__ __forceinline__ void put(uint32_t pos, Cell k, VS v) const {
        if constexpr (kPacked) {
            reinterpret_cast<uint2*>(base)[pos] = make_uint2((uint32_t)k, (uint32_t)v);
        } else {
            reinterpret_cast<Cell*>(base)[pos] = k;
            if constexpr (kPairs) reinterpret_cast<VS*>(base + sizeof(Cell) * TILE)[pos] = v;
        }
    }
    __device__ __forceinline__ Cell key(uint32_t j) const {
        if constexpr (kPacked)
            return (Cell)reinterpret_cast<const uint2*>(base)[j].x;
        else
            return reinterpret_cast<const Cell*>(base)[j];
    }
    __device__ __forceinline__ void get(uint32_t j, Cell& k, VS& v) const {
        if constexpr (kPacked) {
            const uint2 kv = reinterpret_cast<const uint2*>(base)[j];
            k = (Cell)kv.x;
            v = (VS)kv.y;
        } else {
            k = reinterpret_cast<const Cell*>(base)[j];
            if constexpr (kPairs) v = reinterpret_cast<const VS*>(base + sizeof(Cell) * TILE)[j];
        }
    }
};

template <typename Cell, typename V, int IPT, int PB = BLOCK>
struct PassSmem {
    static constexpr int TILE = PB * IPT;
    static constexpr size_t kKeys = sizeof(Cell) * TILE;
    static constexpr size_t kVals = ValTraits<V>::kPairs ? sizeof(V) * TILE : 0;
    static constexpr size_t kBytes = kKeys + kVals;
};

__device__ __forceinline__ const void* pick_src(const PassArgs& a, uint32_t b, bool vals) {
    if (b == BUF_IN) return vals ? a.vals_in : a.keys_in;
    if (b == BUF_TMP) return vals ? a.vals_tmp : a.keys_tmp;
    return vals ? a.vals_out : a.keys_out;
}
__device__ __forceinline__ void* pick_dst(const PassArgs& a, uint32_t b, bool vals) {
    if (b == BUF_TMP) return vals ? a.vals_tmp : a.keys_tmp;
    return vals ? a.vals_out : a.keys_out;
}

// Decoupled look-back for the ND cells a thread owns: for each, the sum of
// its counts over all tiles before `tile`, walking back LOOKBACK_WINDOW
// predecessor words per round trip (the ND walks overlap) until a tile that
// already holds its inclusive prefix.  The wait for an unpublished
// predecessor is bounded by time and by polls; on expiry the status word
// records a timeout and the partial sums are returned so that every tile
// still finishes.
template <int ND>
__device__ __forceinline__ void lookback_cells(const uint32_t* lookback, uint32_t tile,
                                               const uint32_t (&cell)[ND], uint32_t* status,
                                               uint32_t (&before)[ND],
                                               uint64_t timeout_ns = LOOKBACK_TIMEOUT_NS) {
    int64_t j[ND];
    bool done[ND];
#pragma unroll
    for (int e = 0; e < ND; e++) {
        before[e] = 0;
        j[e] = (int64_t)tile - 1;
        done[e] = j[e] < 0;
    }
    const uint64_t t0 = global_ns();
    uint32_t spins = 0;
    while (true) {
        uint32_t sv[ND][LOOKBACK_WINDOW];
#pragma unroll
        for (int e = 0; e < ND; e++)
#pragma unroll
            for (int q = 0; q < LOOKBACK_WINDOW; q++)
                sv[e][q] = (!done[e] && j[e] - q >= 0)
                               ? ld_relaxed(&lookback[(uint64_t)(j[e] - q) * RADIX + cell[e]])
                               : LB_INCLUSIVE;
        bool progress = false, all_done = true;
#pragma unroll
        for (int e = 0; e < ND; e++) {
            if (done[e]) continue;
            int consumed = 0;
            bool blocked = false;
#pragma unroll
            for (int q = 0; q < LOOKBACK_WINDOW; q++) {
                if (done[e] || blocked) continue;
                const uint32_t flag = sv[e][q] & ~LB_VALUE;
                if (flag == 0) {
                    blocked = true;
                    continue;
                }
                before[e] += sv[e][q] & LB_VALUE;
                consumed = q + 1;
                done[e] = flag == LB_INCLUSIVE;
            }
            j[e] -= consumed;
            progress |= consumed > 0;
            all_done &= done[e];
        }
        if (all_done) break;
        if (!progress && (++spins & 15u) == 0 &&
            (global_ns() - t0 > timeout_ns || spins > LOOKBACK_MAX_POLLS)) {
            atomicOr(status, STATUS_TIMEOUT);
            break;  // give up; publish what we have so successors finish
        }
    }
}

// One digit-group pass over one tile of PB * IPT keys; PB threads per CTA,
// each owning ND = 256 / PB consecutive cells in the per-cell phases.
template <class C, typename V, int IPT, int PB>
__global__ void __launch_bounds__(PB, pass_ctas<C, V, IPT, PB>()) pass_kernel(PassArgs a) {
    using Cell = typename C::Cell;
    using In = typename C::In;
    using Out = typename C::Out;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    constexpr int TILE = PB * IPT;
    constexpr int NW = PB / 32;
    constexpr int ND = RADIX / PB;
    static_assert(ND * PB == RADIX, "PB must divide the 256 cells");
    using VS = typename std::conditional<kPairs, V, uint32_t>::type;  // storage type

    // ws[w][d]: first the count of cell d in warp w's slice, then the
    // tile-local position where warp w's next key of cell d goes
    __shared__ uint32_t ws[NW][RADIX];
    __shared__ uint32_t s_bin_global[RADIX];  // global position of tile-local index 0 per cell
    __shared__ uint32_t s_warp[NW];
    __shared__ uint32_t s_tile;
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const Stage<Cell, VS, kPairs, TILE> stage{smem_dyn};

    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;

    // The tile claim goes out first so its round trip overlaps the plan
    // reads and the clearing below.  An inactive pass also claims: its
    // counter is never read.
    uint32_t claimed = 0;
    if (t == 0) claimed = atomicAdd(a.tile_counter, 1u);

    // every plan word this pass reads, loaded together: one round trip that
    // overlaps the tile claim (the plan was written by an earlier launch)
    const DevPlan* P = a.plan;
    const uint32_t p_mode = __ldg(&P->mode), p_active = __ldg(&P->active[a.pass]);
    const uint32_t p_first = __ldg(&P->first_active), p_last = __ldg(&P->last_active);
    const uint32_t src = __ldg(&P->src[a.pass]), dst = __ldg(&P->dst[a.pass]);

    // The next pass's look-back rows are free once this pass started: clear
    // one row per CTA (the grid has one CTA per tile), unless no later pass
    // moves data (the last active pass, the rebuild from cells, or a sort
    // skipped as a whole, whose plan stays zeroed), so that a sort the
    // device skips costs little more than its launches.
    if (p_mode == MODE_PASSES && p_last != MAX_PASSES && p_last > a.pass) {
#pragma unroll
        for (int e = 0; e < ND; e++)
            a.lookback_next[(uint64_t)blockIdx.x * RADIX + e * PB + t] = 0;
    }
    for (uint32_t d = lane; d < RADIX; d += 32) ws[warp][d] = 0;
    if (p_mode != MODE_PASSES || !p_active) return;
    const bool first = p_first == a.pass;
    const bool last = p_last == a.pass;

    if (t == 0) s_tile = claimed;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint64_t tile_base = (uint64_t)tile * TILE;
    const bool full = tile_base + TILE <= a.n;
    const uint32_t valid = full ? TILE : (uint32_t)(a.n - tile_base);

    if (a.prefetch_ahead && t == 0) {
        // whole tiles only, and only where both ranges are 16-byte aligned
        const uint64_t pb = ((uint64_t)tile + a.prefetch_ahead) * TILE;
        if (pb + TILE <= a.n) {
            const size_t kb = first ? sizeof(In) : sizeof(Cell);
            const char* kp = static_cast<const char*>(pick_src(a, src, false)) + pb * kb;
            if (((uintptr_t)kp & 15) == 0) bulk_prefetch_l2(kp, (uint32_t)(TILE * kb));
            if constexpr (kPairs) {
                const char* vp = static_cast<const char*>(pick_src(a, src, true)) + pb * sizeof(VS);
                if (((uintptr_t)vp & 15) == 0) bulk_prefetch_l2(vp, (uint32_t)(TILE * sizeof(VS)));
            }
        }
    }

    // ---- load (warp-striped: warp w owns inputs [w*32*IPT, (w+1)*32*IPT)) ----
    const uint64_t wbase = tile_base + (uint64_t)warp * 32 * IPT + lane;
    Cell k[IPT];
    VS v[IPT];
    if (first) {
        const In* in = static_cast<const In*>(pick_src(a, src, false)) + wbase;
        bool ok = true;
        if (full) {
#pragma unroll
            for (int i = 0; i < IPT; i++) k[i] = C::decode(__ldcs(&in[i * 32]), a.prm, ok);
        } else {
#pragma unroll
            for (int i = 0; i < IPT; i++)
                k[i] = wbase + i * 32 < a.n ? C::decode(__ldcs(&in[i * 32]), a.prm, ok) : ~Cell(0);
        }
    } else {
        const Cell* in = static_cast<const Cell*>(pick_src(a, src, false)) + wbase;
        if (full) {
#pragma unroll
            for (int i = 0; i < IPT; i++) k[i] = __ldcs(&in[i * 32]);
        } else {
#pragma unroll
            for (int i = 0; i < IPT; i++) k[i] = wbase + i * 32 < a.n ? __ldcs(&in[i * 32]) : ~Cell(0);
        }
    }
    if constexpr (kPairs) {
        const VS* vin = static_cast<const VS*>(pick_src(a, src, true)) + wbase;
        if (full) {
#pragma unroll
            for (int i = 0; i < IPT; i++) v[i] = __ldcs(&vin[i * 32]);
        } else {
#pragma unroll
            for (int i = 0; i < IPT; i++) v[i] = wbase + i * 32 < a.n ? __ldcs(&vin[i * 32]) : VS(0);
        }
    }

    // ---- counts per (warp, cell): order does not matter here ----
#pragma unroll
    for (int i = 0; i < IPT; i++) atomicAdd(&ws[warp][digit_of(k[i], a.shift)], 1u);
    __syncthreads();

    // ---- tile count per cell, publish it, then tile-local starts ----
    uint32_t count[ND], excl[ND], cell[ND];
    uint32_t* lb = a.lookback + (uint64_t)tile * RADIX;
    uint32_t mine = 0;
#pragma unroll
    for (int e = 0; e < ND; e++) {
        const uint32_t d = t * ND + e;
        cell[e] = d;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
            const uint32_t x = ws[w][d];
            ws[w][d] = run;
            run += x;
        }
        // padding items carry cell ~0 (digit 255) and sit after every real item
        count[e] = d == RADIX - 1 ? run - (TILE - valid) : run;
        st_relaxed(&lb[d], (tile == 0 ? LB_INCLUSIVE : LB_AGGREGATE) | count[e]);
        mine += count[e];
    }
    uint32_t tile_total;
    uint32_t at = block_exclusive_scan_n<NW>(mine, s_warp, &tile_total);
#pragma unroll
    for (int e = 0; e < ND; e++) {
        excl[e] = at;
        at += count[e];
#pragma unroll
        for (int w = 0; w < NW; w++) ws[w][cell[e]] += excl[e];
    }
    __syncthreads();

    // ---- stable rank in (cell, input) order, scattered into shared memory ----
    const uint32_t lt = lanemask_lt(), gt = lanemask_gt();
    constexpr bool kLut = PB == 256 && PassShape<C, V>::kLut && IPT == PassShape<C, V>::kIPT;
    const LaneBits lb_bits = lane_bits();
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        const uint32_t d = digit_of(k[i], a.shift);
        const uint32_t peers = peer_mask<kLut>(d, lb_bits);
        uint32_t* slot = &ws[warp][d];
        const uint32_t pos0 = *slot;
        const uint32_t below = __popc(peers & lt);
        // every peer has read the slot before the highest one (the last of
        // them in input order) moves it past the group
        __syncwarp();
        if ((peers & gt) == 0) *slot = pos0 + below + 1;
        const uint32_t pos = pos0 + below;
        stage.put(pos, k[i], v[i]);
        __syncwarp();
    }

    // ---- decoupled look-back: these cells' counts in all earlier tiles ----
    // (after the ranking: the predecessors publish while this tile ranks)
    uint32_t before[ND];
    if (tile > 0) {
        lookback_cells<ND>(a.lookback, tile, cell, a.status, before);
#pragma unroll
        for (int e = 0; e < ND; e++)
            st_relaxed(&lb[cell[e]], LB_INCLUSIVE | ((before[e] + count[e]) & LB_VALUE));
    } else {
#pragma unroll
        for (int e = 0; e < ND; e++) before[e] = 0;
    }
#pragma unroll
    for (int e = 0; e < ND; e++)
        s_bin_global[cell[e]] = a.bin_offsets[cell[e]] + before[e] - excl[e];
    __syncthreads();

    // ---- coalesced write-out: consecutive threads, consecutive positions ----
    void* kdst = pick_dst(a, dst, false);
    VS* vdst = kPairs ? static_cast<VS*>(pick_dst(a, dst, true)) : nullptr;
    // (the clamp of g only acts after a timed-out wait: output unspecified)
    const uint32_t gmax = (uint32_t)a.n - 1u;
    if (last) {
        Out* out = static_cast<Out*>(kdst);
        if (full) {
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                const uint32_t j = t + i * PB;
                Cell c;
                VS val;
                stage.get(j, c, val);
                const uint32_t g = min(s_bin_global[digit_of(c, a.shift)] + j, gmax);
                __stcs(&out[g], C::encode(c, a.prm));
                if constexpr (kPairs) __stcs(&vdst[g], val);
            }
        } else {
            for (uint32_t j = t; j < valid; j += PB) {
                Cell c;
                VS val;
                stage.get(j, c, val);
                const uint32_t g = min(s_bin_global[digit_of(c, a.shift)] + j, gmax);
                __stcs(&out[g], C::encode(c, a.prm));
                if constexpr (kPairs) __stcs(&vdst[g], val);
            }
        }
    } else {
        Cell* out = static_cast<Cell*>(kdst);
        if (full) {
#pragma unroll
            for (int i = 0; i < IPT; i++) {
                const uint32_t j = t + i * PB;
                Cell c;
                VS val;
                stage.get(j, c, val);
                const uint32_t g = min(s_bin_global[digit_of(c, a.shift)] + j, gmax);
                out[g] = c;
                if constexpr (kPairs) vdst[g] = val;
            }
        } else {
            for (uint32_t j = t; j < valid; j += PB) {
                Cell c;
                VS val;
                stage.get(j, c, val);
                const uint32_t g = min(s_bin_global[digit_of(c, a.shift)] + j, gmax);
                out[g] = c;
                if constexpr (kPairs) vdst[g] = val;
            }
        }
    }
}

// ----------------------------------------------------------------------------
// Keys only, one count array: the extraction cycle writes each cell's key
// (Eq. 16) once per count.  Warp-strided output positions coalesce.

struct FillArgs {
    void* keys_out;
    uint64_t n;
    CodecParams prm;
    const DevPlan* plan;
    const uint32_t* fill_offsets;  // [FILL_CELLS + 1]
};

constexpr int FILL_IPT = 16;

template <class C>
__global__ void __launch_bounds__(BLOCK) fill_kernel(FillArgs a) {
    using Out = typename C::Out;
    using Cell = typename C::Cell;
    if (a.plan->mode != MODE_FILL) return;
    const uint32_t lane = lane_id();
    const uint64_t warp_g = ((uint64_t)blockIdx.x * BLOCK + threadIdx.x) >> 5;
    const uint64_t base = warp_g * 32 * FILL_IPT;
    if (base >= a.n) return;
    Out* out = static_cast<Out*>(a.keys_out);
    const uint32_t* off = a.fill_offsets;
    // the cell of output position j: the last cell whose offset is <= j
    // (empty cells share their successor's offset and are stepped over)
    uint64_t j = base + lane;
    uint32_t lo = 0, hi = FILL_CELLS;
    if (j < a.n) {
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(&off[mid]) <= j) lo = mid; else hi = mid;
        }
    }
    uint32_t cell = lo;
#pragma unroll 4
    for (int i = 0; i < FILL_IPT; i++, j += 32) {
        if (j >= a.n) break;
        while (cell + 1 < FILL_CELLS && __ldg(&off[cell + 1]) <= j) cell++;
        __stcs(&out[j], C::encode((Cell)cell, a.prm));
    }
}

// Runs the look-back wait of tile 1 against a tile 0 that never publishes
// (a zeroed row): every thread must give up after timeout_ns, record
// STATUS_TIMEOUT and return.  Exercises the bounded wait without a fault.
static __global__ void __launch_bounds__(BLOCK) wait_timeout_kernel(const uint32_t* lookback,
                                                             uint32_t* status,
                                                             uint64_t timeout_ns) {
    const uint32_t cell[1] = {threadIdx.x};
    uint32_t before[1];
    lookback_cells<1>(lookback, 1, cell, status, before, timeout_ns);
}

}  // namespace rs
