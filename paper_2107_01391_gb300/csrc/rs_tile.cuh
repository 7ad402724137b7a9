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

#include "rs_device.cuh"

namespace rs {

struct TileShared {
    uint32_t wh[WARPS][RADIX];  // per-warp counts, then per-warp next positions
    uint32_t count[RADIX];      // keys of each cell in the tile
    uint32_t excl[RADIX];       // tile-local start of each cell
    uint32_t warp_sum[WARPS];
};

// Positions [0, n_valid) of the tile hold keys; the rest are ignored.
// Returns with s_keys/s_vals holding the tile in (cell, input) order and
// ts.count / ts.excl filled.  Every thread of the CTA must call it.
// s_run (optional): running per-cell output offsets of a sweep over several
// tiles; the previous tile's ts.count is added to them once every thread is
// past its write-out (the first barrier below), so the sweep itself needs
// no barrier between tiles.
template <typename Cell, typename VS, int IPT, bool kPairs>
__device__ __forceinline__ void rank_scatter(const Cell (&k)[IPT], const VS (&v)[IPT],
                                             uint32_t n_valid, uint32_t shift, TileShared& ts,
                                             Cell* s_keys, VS* s_vals,
                                             uint32_t* s_run = nullptr) {
    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
    const uint32_t wbase = warp * 32 * IPT;
    for (uint32_t d = lane; d < RADIX; d += 32) ts.wh[warp][d] = 0;
    __syncwarp();
    const uint32_t warp_items = wbase < n_valid ? min(n_valid - wbase, 32u * IPT) : 0u;
#pragma unroll
    for (int i = 0; i < IPT; i++)
        if ((uint32_t)i * 32 + lane < warp_items) atomicAdd(&ts.wh[warp][digit_of(k[i], shift)], 1u);
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
#pragma unroll
    for (int i = 0; i < IPT; i++) {
        if ((uint32_t)i * 32 >= warp_items) break;  // warp-uniform
        const bool valid = (uint32_t)i * 32 + lane < warp_items;
        const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
        const uint32_t d = digit_of(k[i], shift);
        const uint32_t peers = match_digit(d) & vmask;
        uint32_t* slot = &ts.wh[warp][d];
        const uint32_t at = valid ? *slot : 0u;
        const uint32_t below = __popc(peers & lt);
        __syncwarp();
        if (valid) {
            if ((peers & gt) == 0) *slot = at + below + 1;
            const uint32_t pos = at + below;
            s_keys[pos] = k[i];
            if constexpr (kPairs) s_vals[pos] = v[i];
        }
        __syncwarp();
    }
    __syncthreads();
}

}  // namespace rs
