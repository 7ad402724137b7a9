// rs_sort_impl.cuh -- workspace layout and launch sequence of one sort.
//
// Launch sequence (all on the caller's stream, no host synchronisation):
//   1. cudaMemsetAsync: device plan, counters, counts, look-back buffer 0
//   2. count_kernel   hashing cycle + device-side plan (last CTA)
//   3. fill_kernel    keys-only single count array (exits at once otherwise)
//   4. pass_kernel x passes_total, least significant digit group first
//      (each exits at once when the plan marks its group trivial)
#pragma once

#include <algorithm>
#include <atomic>
#include <cstring>

#include "rs_ctx.hpp"
#include "rs_kernels.cuh"
#include "rs_tile.cuh"

#ifndef RS_PASS_BLOCK
#define RS_PASS_BLOCK 256
#endif

namespace rs {

inline size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

// Threads per CTA of the pass kernel.
template <class C, typename V>
constexpr int pass_block() {
    return RS_PASS_BLOCK;
}

// Keys per thread of a pass tile (PassShape).
template <class C, typename V>
constexpr int ipt_for() {
    return PassShape<C, V>::kIPT;
}

struct Layout {
    size_t plan, hist, bin_offsets, fill_hist, fill_offsets, lookback0, lookback1;
    size_t keys_tmp, vals_tmp, total, memset_bytes;
    uint64_t tiles;
};

inline Layout make_layout(size_t n, uint32_t passes, int tile, size_t cell_bytes,
                          size_t val_bytes) {
    Layout L{};
    L.tiles = (n + tile - 1) / tile;
    size_t at = 0;
    L.plan = at;          at += align_up(sizeof(DevPlan));
    L.hist = at;          at += align_up(sizeof(uint32_t) * MAX_PASSES * RADIX);
    L.fill_hist = at;     at += align_up(sizeof(uint32_t) * FILL_CELLS);
    L.lookback0 = at;     at += align_up(sizeof(uint32_t) * RADIX * std::max<uint64_t>(L.tiles, 1));
    L.memset_bytes = at;  // everything above starts at zero
    L.lookback1 = at;     at += align_up(sizeof(uint32_t) * RADIX * std::max<uint64_t>(L.tiles, 1));
    L.bin_offsets = at;   at += align_up(sizeof(uint32_t) * MAX_PASSES * RADIX);
    L.fill_offsets = at;  at += align_up(sizeof(uint32_t) * (FILL_CELLS + 1));
    L.keys_tmp = at;      at += align_up(cell_bytes * std::max<size_t>(n, 1));
    L.vals_tmp = at;      at += align_up(val_bytes * std::max<size_t>(n, 1));
    (void)passes;
    L.total = at;
    return L;
}

// Digit groups of a cell index with cell_bits significant bits, rounded up
// to an even number (never beyond the cell type's width, whose bits are a
// multiple of 16): an in-place sort alternates buffers and so needs an even
// count of data-moving passes, and an extra all-zero group is an identity
// pass the plan can switch on to make the count even.
inline uint32_t passes_for(uint32_t cell_bits) {
    uint32_t p = std::max<uint32_t>(1, (cell_bits + RADIX_BITS - 1) / RADIX_BITS);
    return (p + 1) & ~1u;
}

inline int count_grid(size_t n, int sms, int per_sm = 8) {
    // at least 64 keys per thread, at most per_sm CTAs per SM (8 measured
    // best at 2^28 keys, 3 resident at a time with 64 KB of lane counters),
    // and at most 2^20 keys per CTA: a lane's 16-bit counter collects the
    // keys of its lane in all 8 warps, at most 2^20 / 32 = 32768 of them
    const size_t per_cta = (size_t)BLOCK * 64;
    size_t g = (n + per_cta - 1) / per_cta;
    g = std::min<size_t>(g, (size_t)sms * per_sm);
    g = std::max<size_t>(g, (n + (1u << 20) - 1) >> 20);
    return (int)std::max<size_t>(g, 1);
}

inline int sm_count(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0)
        v = 152;
    return v;
}

// One sort with pass tiles of PB * IPT keys: keys_in (C::In) -> keys_out
// (C::Out), values V (NoVal = keys only).  skip (device pointer, may be
// NULL): when it holds a non-zero word at run time the whole sort is a no-op
// (used by callers that plan on the device).
template <class C, typename V, int IPT>
rs_status run_sort_tile(rs_ctx* ctx, const void* keys_in, void* keys_out, const void* vals_in,
                        void* vals_out, size_t n, CodecParams prm, uint32_t cell_bits,
                        void* temp, size_t* temp_bytes, cudaStream_t stream,
                        const uint32_t* skip) {
    using Cell = typename C::Cell;
    constexpr bool kPairs = ValTraits<V>::kPairs;
    constexpr int PB = pass_block<C, V>();
    constexpr int TILE = PB * IPT;
    const uint32_t passes = passes_for(cell_bits);
    const size_t vbytes = kPairs ? sizeof(V) : 0;
    const Layout L = make_layout(n, passes, TILE, sizeof(Cell), vbytes);

    if (!temp_bytes) return RS_ERR_INVALID;
    if (!temp) {
        *temp_bytes = L.total;
        return RS_OK;
    }
    if (*temp_bytes < L.total) return RS_ERR_TEMP_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(temp) % 256) return RS_ERR_INVALID;
    if (n == 0) return RS_OK;

    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;

    if (n <= SMALL_TILE) {
        // one tile: one CTA sorts it on chip in a single launch (the
        // workspace is not touched)
        // (a full tile and a shorter input are separate kernels)
        const bool full = n == SMALL_TILE;
        auto kern = full ? tile_rows_kernel<C, V, SMALL_IPT>
                         : tile_rows_kernel<C, V, SMALL_IPT, V, true>;
        const size_t smem = SMALL_TILE * (sizeof(Cell) + (kPairs ? sizeof(V) : 0));
        static std::atomic<bool> small_set[2][64];  // zero-initialised: false
        std::atomic<bool>* set = ctx->device < 64 ? &small_set[full][ctx->device] : nullptr;
        if (!set || !set->load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) != cudaSuccess)
                return RS_ERR_CUDA;
            if (set) set->store(true, std::memory_order_release);
        }
        RowsArgs ra{};
        ra.keys_in = keys_in;
        ra.keys_out = keys_out;
        ra.vals_in = vals_in;
        ra.vals_out = vals_out;
        ra.rows = 1;
        ra.len = (uint32_t)n;
        ra.passes = passes;
        ra.prm = prm;
        ra.status = ctx->d_status;
        ra.info = static_cast<DevInfo*>(ctx->d_info);
        ra.skip = skip;
        {
            LaunchTimer lt(ctx, KC_PASS, stream);
            kern<<<1, BLOCK, smem, stream>>>(ra);
        }
        ctx->last_passes_total = passes;
        ctx->last_tiles = 1;
        return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
    }

    unsigned char* T = static_cast<unsigned char*>(temp);
    DevPlan* plan = reinterpret_cast<DevPlan*>(T + L.plan);
    uint32_t* hist = reinterpret_cast<uint32_t*>(T + L.hist);
    uint32_t* bin_offsets = reinterpret_cast<uint32_t*>(T + L.bin_offsets);
    uint32_t* fill_hist = reinterpret_cast<uint32_t*>(T + L.fill_hist);
    uint32_t* fill_offsets = reinterpret_cast<uint32_t*>(T + L.fill_offsets);
    uint32_t* lb[2] = {reinterpret_cast<uint32_t*>(T + L.lookback0),
                       reinterpret_cast<uint32_t*>(T + L.lookback1)};

    if (cudaMemsetAsync(T, 0, L.memset_bytes, stream) != cudaSuccess) return RS_ERR_CUDA;

    const bool fill_allowed = !kPairs;
    {
        CountArgs a{};
        a.keys_in = keys_in;
        a.n = n;
        a.passes = passes;
        a.fill_allowed = fill_allowed;
        a.in_is_out = keys_in == keys_out;
        a.prm = prm;
        a.plan = plan;
        a.hist = hist;
        a.bin_offsets = bin_offsets;
        a.fill_hist = fill_hist;
        a.fill_offsets = fill_offsets;
        a.status = ctx->d_status;
        a.info = static_cast<DevInfo*>(ctx->d_info);
        a.skip = skip;
        LaunchTimer lt(ctx, KC_HIST, stream);
        const size_t lane_hist = sizeof(Cell) == 4 ? LANE_HIST_WORDS * sizeof(uint32_t) : 0;
        const int grid = count_grid(n, sm_count(ctx->device));
        static std::atomic<bool> count_smem_set[64];  // zero-initialised: false
        if (lane_hist && ctx->device < 64 && !count_smem_set[ctx->device].load(std::memory_order_acquire)) {
            if (cudaFuncSetAttribute(count_kernel<C, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)lane_hist) != cudaSuccess ||
                cudaFuncSetAttribute(count_kernel<C, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)lane_hist) != cudaSuccess)
                return RS_ERR_CUDA;
            count_smem_set[ctx->device].store(true, std::memory_order_release);
        }
        if (fill_allowed)
            count_kernel<C, true><<<grid, BLOCK, lane_hist, stream>>>(a);
        else
            count_kernel<C, false><<<grid, BLOCK, lane_hist, stream>>>(a);
    }
    if (fill_allowed) {
        FillArgs f{};
        f.keys_out = keys_out;
        f.n = n;
        f.prm = prm;
        f.plan = plan;
        f.fill_offsets = fill_offsets;
        const size_t per_cta = (size_t)BLOCK * FILL_IPT;
        const unsigned grid = (unsigned)((n + per_cta - 1) / per_cta);
        LaunchTimer lt(ctx, KC_FILL, stream);
        fill_kernel<C><<<grid, BLOCK, 0, stream>>>(f);
    }
    using Smem = PassSmem<Cell, V, IPT, PB>;
    auto kern = pass_kernel<C, V, IPT, PB>;
    // static + dynamic shared memory may exceed the 48 KB default: opt in
    // once per device for this instantiation
    static std::atomic<bool> smem_set[64];  // zero-initialised: false
    if (ctx->device < 64 && !smem_set[ctx->device].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Smem::kBytes) != cudaSuccess)
            return RS_ERR_CUDA;
        smem_set[ctx->device].store(true, std::memory_order_release);
    }
    const uint32_t ahead = prefetch_ahead_for(pass_ctas<C, V, IPT, PB>() * sm_count(ctx->device));
    for (uint32_t p = 0; p < passes; p++) {
        PassArgs a{};
        a.keys_in = keys_in;
        a.keys_tmp = T + L.keys_tmp;
        a.keys_out = keys_out;
        a.vals_in = vals_in;
        a.vals_tmp = kPairs ? (void*)(T + L.vals_tmp) : nullptr;
        a.vals_out = vals_out;
        a.n = n;
        a.pass = p;
        a.shift = p * RADIX_BITS;
        a.prm = prm;
        a.plan = plan;
        a.bin_offsets = bin_offsets + p * RADIX;
        a.lookback = lb[p & 1];
        a.lookback_next = lb[(p + 1) & 1];
        a.tile_counter = &plan->tile_counter[p];
        a.status = ctx->d_status;
        a.prefetch_ahead = ahead;
        LaunchTimer lt(ctx, KC_PASS, stream);
        kern<<<(unsigned)L.tiles, PB, Smem::kBytes, stream>>>(a);
    }
    ctx->last_passes_total = passes;
    ctx->last_tiles = (uint32_t)L.tiles;
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}

// One sort, choosing the pass tile: the narrow one (NarrowShape) for sorts
// of more than one on-chip tile and at most ctx->narrow_max_n keys where the
// shape has one, the wide one (PassShape) otherwise.  A workspace query
// returns room for either, so it needs no context.
template <class C, typename V>
rs_status run_sort(rs_ctx* ctx, const void* keys_in, void* keys_out, const void* vals_in,
                   void* vals_out, size_t n, CodecParams prm, uint32_t cell_bits, void* temp,
                   size_t* temp_bytes, cudaStream_t stream, const uint32_t* skip) {
    constexpr int WIDE = ipt_for<C, V>();
    if constexpr (NarrowShape<C, V>::kHas) {
        constexpr int NARROW = NarrowShape<C, V>::kIPT;
        if (!temp && temp_bytes) {
            size_t wide = 0, narrow = 0;
            rs_status s = run_sort_tile<C, V, WIDE>(ctx, keys_in, keys_out, vals_in, vals_out, n,
                                                    prm, cell_bits, nullptr, &wide, stream, skip);
            if (s != RS_OK) return s;
            s = run_sort_tile<C, V, NARROW>(ctx, keys_in, keys_out, vals_in, vals_out, n, prm,
                                            cell_bits, nullptr, &narrow, stream, skip);
            if (s != RS_OK) return s;
            *temp_bytes = std::max(wide, narrow);
            return RS_OK;
        }
        if (ctx && n > SMALL_TILE && n <= ctx->narrow_max_n)
            return run_sort_tile<C, V, NARROW>(ctx, keys_in, keys_out, vals_in, vals_out, n, prm,
                                               cell_bits, temp, temp_bytes, stream, skip);
    }
    return run_sort_tile<C, V, WIDE>(ctx, keys_in, keys_out, vals_in, vals_out, n, prm,
                                     cell_bits, temp, temp_bytes, stream, skip);
}

#define RS_DECLARE_SORT(C, V)                                                                  \
    template rs_status run_sort<C, V>(rs_ctx*, const void*, void*, const void*, void*, size_t, \
                                      CodecParams, uint32_t, void*, size_t*, cudaStream_t,      \
                                      const uint32_t*);

}  // namespace rs
