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
//        - a segment of at most one tile is loaded once into registers and
//          sorted entirely on chip: one rank-and-scatter through shared
//          memory per 8-bit digit group, then one coalesced write
//          (16 bytes per u32 key+value pair in total);
//        - a larger segment is sorted by its CTA alone: one read to count
//          every digit group, then per non-trivial group a sweep over the
//          segment's tiles in input order with running cell offsets in
//          shared memory (a CTA-sequential extraction cycle, no look-back).

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
constexpr uint64_t SEG_MAX_LEN = 0xffffffffull;  // counts within a segment are 32-bit

struct SegControl {
    uint32_t class_count[SIZE_CLASSES];
    uint32_t class_cursor[SIZE_CLASSES];
    uint32_t work;
    uint32_t done;
};

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
        }
    }
}

__global__ void __launch_bounds__(BLOCK) seg_order_kernel(SegArgs a, uint32_t* order) {
    for (uint64_t s = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; s < a.num_segs;
         s += (uint64_t)gridDim.x * BLOCK) {
        uint64_t lo, hi;
        const uint32_t c = seg_bounds(a, s, lo, hi) ? size_class(hi - lo) : SIZE_CLASSES - 1;
        order[atomicAdd(&a.ctl->class_cursor[c], 1u)] = (uint32_t)s;
    }
}

// Load one tile (positions [base, base+valid) of `src`) warp-striped.  With
// iota_from != ~0 the values are generated: position - iota_from.
template <class C, typename VS, bool kPairs, bool kDecode>
__device__ __forceinline__ void load_tile(const void* ksrc, const VS* vsrc, uint64_t base,
                                          uint32_t valid, const CodecParams& prm,
                                          uint64_t iota_from, typename C::Cell (&k)[SEG_IPT],
                                          VS (&v)[SEG_IPT], uint32_t* status) {
    using Cell = typename C::Cell;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t w0 = warp * 32 * SEG_IPT + lane;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < SEG_IPT; i++) {
        const uint32_t j = w0 + i * 32;
        if (j < valid) {
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
    Cell* s_keys = reinterpret_cast<Cell*>(smem_dyn);
    VS* s_vals = reinterpret_cast<VS*>(smem_dyn + sizeof(Cell) * SEG_TILE);
    const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;

    while (true) {
        if (t == 0) {
            // The list is ordered by size class, largest first: once the next
            // entry is a warp-sized segment every later one is too, so take
            // one per warp.
            uint32_t take = 1;
            const uint32_t peek = ld_relaxed(&a.ctl->work);
            uint64_t plo, phi;
            if (peek < a.num_segs && seg_bounds(a, a.order[peek], plo, phi) &&
                phi - plo <= WARP_SEG_MAX)
                take = WARPS;
            s_first = atomicAdd(&a.ctl->work, take);
            s_take = take;
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
        if (len <= SEG_TILE) {
            // ---- one tile: sorted on chip, read once and written once ----
            const uint32_t valid = (uint32_t)len;
            load_tile<C, VS, kPairs, true>(a.keys_in, vin, lo, valid, a.prm,
                                           a.iota ? lo : ~0ull, k, v, a.status);
            for (uint32_t p = 0; p < a.passes; p++) {
                rank_scatter<Cell, VS, SEG_IPT, kPairs>(k, v, valid, p * RADIX_BITS, ts,
                                                        s_keys, s_vals);
                const uint32_t w0 = warp * 32 * SEG_IPT + lane;
#pragma unroll
                for (int i = 0; i < SEG_IPT; i++) {
                    const uint32_t j = w0 + i * 32;
                    if (j < valid) {
                        k[i] = s_keys[j];
                        if constexpr (kPairs) v[i] = s_vals[j];
                    }
                }
                __syncthreads();  // s_keys is rewritten by the next group
            }
            const uint32_t w0 = warp * 32 * SEG_IPT + lane;
#pragma unroll
            for (int i = 0; i < SEG_IPT; i++) {
                const uint32_t j = w0 + i * 32;
                if (j < valid) {
                    static_cast<Out*>(a.keys_out)[lo + j] = C::encode(k[i], a.prm);
                    if constexpr (kPairs) vout[lo + j] = v[i];
                }
            }
            continue;
        }

        // ---- larger segment: count every digit group in one read ----
        for (uint32_t i = t; i < MAX_PASSES * RADIX; i += BLOCK) (&s_hist[0][0])[i] = 0;
        __syncthreads();
        {
            bool ok = true;
            const In* kin = static_cast<const In*>(a.keys_in);
            for (uint64_t j = lo + t; j < hi; j += BLOCK) {
                const Cell c = C::decode(kin[j], a.prm, ok);
#pragma unroll
                for (uint32_t p = 0; p < sizeof(Cell); p++)
                    if (p < a.passes) atomicAdd(&s_hist[p][digit_of(c, p * RADIX_BITS)], 1u);
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
            s_hist[p][t] = e;
            if (t == 0) s_active[p] = occupied > 1;
        }
        __syncthreads();
        // route as the device-wide sort does: the last active group writes
        // OUT, earlier ones alternate TMP/OUT, the first reads IN; in place
        // needs an even count (one trivial group is re-activated), out of
        // place at least one
        uint32_t act = 0;
        for (uint32_t p = 0; p < a.passes; p++) act += s_active[p];
        bool use[MAX_PASSES];
        for (uint32_t p = 0; p < MAX_PASSES; p++) use[p] = p < a.passes && s_active[p];
        // (the pass count is even, so a trivial group is always there to
        // switch on; an argsort must run at least once to write its indices)
        uint32_t need = a.in_is_out ? (act & 1u) : (act == 0);
        if (a.in_is_out && act == 0 && a.iota) need = 2;
        for (uint32_t p = 0; p < a.passes && need; p++)
            if (!use[p]) {
                use[p] = true;
                act++;
                need--;
            }
        uint32_t done = 0;
        uint32_t src_buf = BUF_IN;
        for (uint32_t p = 0; p < a.passes; p++) {
            if (!use[p]) continue;
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
                if (first)
                    load_tile<C, VS, kPairs, true>(ksrc, vsrc, base, valid, a.prm,
                                                   a.iota ? 0ull : ~0ull, k, v, a.status);
                else
                    load_tile<C, VS, kPairs, false>(ksrc, vsrc, base, valid, a.prm, ~0ull, k, v,
                                                    a.status);
                rank_scatter<Cell, VS, SEG_IPT, kPairs>(k, v, valid, shift, ts, s_keys, s_vals,
                                                        s_run);
                for (uint32_t j = t; j < valid; j += BLOCK) {
                    const Cell c = s_keys[j];
                    const uint32_t d = digit_of(c, shift);
                    const uint64_t g = s_run[d] + (j - ts.excl[d]);  // within the segment
                    if (last)
                        static_cast<Out*>(kdst)[g] = C::encode(c, a.prm);
                    else
                        static_cast<Cell*>(kdst)[g] = c;
                    if constexpr (kPairs) vdst[g] = s_vals[j];
                }
                // (the next tile's rank_scatter moves s_run on after its
                // first barrier, once every thread is past this write-out)
            }
            // the write-out above reads s_run, s_keys and ts: done before the
            // next group resets them; also orders this group's global writes
            // before the next group's reads
            __syncthreads();
            src_buf = dst_buf;
            done++;
        }
        // make this CTA's writes visible before the next segment reuses smem
        __syncthreads();
    }
}

size_t seg_workspace(size_t n, size_t num_segs, size_t cell_bytes, size_t val_bytes) {
    return align_up(sizeof(SegControl)) + align_up(sizeof(uint32_t) * std::max<size_t>(num_segs, 1)) +
           align_up(cell_bytes * std::max<size_t>(n, 1)) + align_up(val_bytes * std::max<size_t>(n, 1));
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
    const size_t total = seg_workspace(n, num_segs, sizeof(Cell), vbytes);
    if (!temp) {
        *temp_bytes = total;
        return RS_OK;
    }
    if (*temp_bytes < total) return RS_ERR_TEMP_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(temp) % 256) return RS_ERR_INVALID;
    if (num_segs == 0 || n == 0) return RS_OK;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;
    unsigned char* T = static_cast<unsigned char*>(temp);
    size_t at = 0;
    SegControl* ctl = reinterpret_cast<SegControl*>(T + at);
    at += align_up(sizeof(SegControl));
    uint32_t* order = reinterpret_cast<uint32_t*>(T + at);
    at += align_up(sizeof(uint32_t) * num_segs);
    void* keys_tmp = T + at;
    at += align_up(sizeof(Cell) * n);
    void* vals_tmp = kPairs ? (void*)(T + at) : nullptr;

    if (cudaMemsetAsync(ctl, 0, sizeof(SegControl), st) != cudaSuccess) return RS_ERR_CUDA;
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
    a.passes = passes_for(cell_bits);
    a.in_is_out = keys_in == keys_out;
    a.prm = prm;
    a.status = ctx->d_status;
    const int sms = sm_count(ctx->device);
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
    {
        LaunchTimer lt(ctx, KC_SEG, st);
        kern<<<grid, BLOCK, smem, st>>>(a);
    }
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
