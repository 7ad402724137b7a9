// rs_device.cuh -- device-side building blocks shared by the sort kernels.
//
// Vocabulary (Kumar et al., "Recombinant Sort", arXiv 2107.01391):
//   key   -> its digit vector (Eq. 1) -> the row-major index of its cell in
//            the count space S (Eq. 2).  For base-10 digits that index is the
//            key itself (scaled by 10^λ for decimals), so a "cell" here is an
//            unsigned integer whose raster order is the key order.
//   digit group -> 8 bits of the cell index: one on-chip dimension group of
//            256 cells.  Groups are counted (hashing cycle, §3.1), prefix-summed
//            in raster order (extraction cycle, §3.2) and scattered stably,
//            least significant group first; the more significant groups act
//            as the paper's buckets (§2.2) for the groups below them.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rs {

constexpr int RADIX_BITS = 8;
constexpr int RADIX = 1 << RADIX_BITS;  // cells per digit group
constexpr int MAX_PASSES = 8;           // 64-bit cells / 8-bit groups
constexpr uint32_t FILL_CELLS = 4096;   // largest count array rebuilt from cells (Eq. 16)
constexpr int BLOCK = 256;              // threads per CTA of every sort kernel
constexpr int WARPS = BLOCK / 32;

// Device status word bits (rs_ctx_status maps them to rs_status codes).
constexpr uint32_t STATUS_RANGE = 1u;
constexpr uint32_t STATUS_TIMEOUT = 2u;

// Look-back words: 2 flag bits over a 30-bit count.
constexpr uint32_t LB_AGGREGATE = 1u << 30;  // this tile's own count only
constexpr uint32_t LB_INCLUSIVE = 2u << 30;  // count of this tile and all before it
constexpr uint32_t LB_VALUE = (1u << 30) - 1u;
// Longest a tile waits for a predecessor before it reports a timeout.
constexpr uint64_t LOOKBACK_TIMEOUT_NS = 2000000000ull;
constexpr uint32_t LOOKBACK_MAX_POLLS = 1u << 24;

// Buffers a pass can read or write.
enum : uint32_t { BUF_IN = 0, BUF_TMP = 1, BUF_OUT = 2 };
enum : uint32_t { MODE_PASSES = 0, MODE_FILL = 1 };

// The plan the device makes for itself from the counts (no host round trip):
// which digit groups need a pass, where each pass reads and writes, and
// whether the whole key space is one count array rebuilt from cells.
struct DevPlan {
    uint32_t mode;
    uint32_t passes_run;
    uint32_t first_active;  // MAX_PASSES if none
    uint32_t last_active;
    uint32_t active[MAX_PASSES];
    uint32_t src[MAX_PASSES];
    uint32_t dst[MAX_PASSES];
    uint32_t hist_done;           // CTAs of the counting kernel that finished
    uint32_t fill_impossible;     // some key's cell is >= FILL_CELLS
    uint32_t tile_counter[MAX_PASSES];
};

// What the last sort decided, kept in the context for diagnostics.
struct DevInfo {
    uint32_t mode;
    uint32_t passes_run;
};

struct CodecParams {
    uint64_t bias;  // fixed-point decimals: 10^D - 1
};

// ------------------------------------------------------------------ codecs
// decode: input key -> cell (sets ok = false for a key outside its space)
// encode: cell -> output key (the key rebuilt from its cell, Eq. 16)

struct CodecU32 {
    using In = uint32_t;
    using Cell = uint32_t;
    using Out = uint32_t;
    __device__ static Cell decode(In k, const CodecParams&, bool&) { return k; }
    __device__ static Out encode(Cell c, const CodecParams&) { return c; }
};

struct CodecU64 {
    using In = uint64_t;
    using Cell = uint64_t;
    using Out = uint64_t;
    __device__ static Cell decode(In k, const CodecParams&, bool&) { return k; }
    __device__ static Out encode(Cell c, const CodecParams&) { return c; }
};

// Fixed-point decimal with D = int_digits + frac_digits digits: the cell of
// v is v + (10^D - 1), a monotone map of [-(10^D-1), 10^D-1] onto
// [0, 2*10^D - 2].  CellT = uint32_t when 2*10^D - 2 < 2^32 (D <= 9).
template <typename CellT>
struct CodecDec {
    using In = int64_t;
    using Cell = CellT;
    using Out = int64_t;
    __device__ static Cell decode(In v, const CodecParams& p, bool& ok) {
        const int64_t b = (int64_t)p.bias;
        if (v < -b || v > b) {
            ok = false;
            v = v < 0 ? -b : b;
        }
        return (Cell)(uint64_t)(v + b);
    }
    __device__ static Out encode(Cell c, const CodecParams& p) {
        return (int64_t)(uint64_t)c - (int64_t)p.bias;
    }
};

// IEEE floats as cells: flipping the sign bit of non-negative values and
// every bit of negative ones makes unsigned order equal numeric order.  Before
// that, -0.0 becomes +0.0 and every NaN the positive quiet NaN, so zeros tie
// and NaNs sort last (the order torch.sort gives); the keys written out are
// those canonical values.
struct CodecF32 {
    using In = uint32_t;  // the float's bits
    using Cell = uint32_t;
    using Out = uint32_t;
    __device__ static Cell decode(In u, const CodecParams&, bool&) {
        if (u == 0x80000000u) u = 0;                                  // -0.0
        if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) u = 0x7fc00000u;  // NaN
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
    __device__ static Out encode(Cell c, const CodecParams&) {
        return (c & 0x80000000u) ? (c & 0x7fffffffu) : ~c;
    }
};

struct CodecF64 {
    using In = uint64_t;  // the double's bits
    using Cell = uint64_t;
    using Out = uint64_t;
    __device__ static Cell decode(In u, const CodecParams&, bool&) {
        constexpr uint64_t SIGN = 0x8000000000000000ull, EXP = 0x7ff0000000000000ull;
        if (u == SIGN) u = 0;
        if ((u & EXP) == EXP && (u & ~(SIGN | EXP))) u = 0x7ff8000000000000ull;
        return (u & SIGN) ? ~u : (u | SIGN);
    }
    __device__ static Out encode(Cell c, const CodecParams&) {
        constexpr uint64_t SIGN = 0x8000000000000000ull;
        return (c & SIGN) ? (c & ~SIGN) : ~c;
    }
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bulk prefetch of [p, p + bytes) into L2 by the copy engine of the SM (TMA),
// with no destination in shared memory.  p and bytes must be multiples of
// 16; the call is a hint and completes asynchronously.
__device__ __forceinline__ void bulk_prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// The whole 16-byte lines inside [p, p + bytes) prefetched into L2 (the
// range's unaligned ends are left out, so nothing outside it is touched).
__device__ __forceinline__ void prefetch_lines_l2(const void* p, uint64_t bytes) {
    const uintptr_t b = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e > b) bulk_prefetch_l2(reinterpret_cast<const void*>(b), (uint32_t)(e - b));
}

// Lanes of the warp holding the same 8-bit digit: one ballot per bit.  Per
// bit b: p = bit set, sx = all ones when set, bal = lanes with the bit set,
// and peers &= ~(bal ^ sx) in one lop3 (truth table 0x90 for a & ~(b ^ c)
// with a = 0xF0, b = 0xCC, c = 0xAA).
template <int B>
__device__ __forceinline__ void match_bit(uint32_t d, uint32_t& m) {
    asm("{\n\t"
        ".reg .pred p;\n\t"
        ".reg .b32 t, sx, bal;\n\t"
        "and.b32 t, %1, %2;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "selp.b32 sx, -1, 0, p;\n\t"
        "vote.sync.ballot.b32 bal, p, 0xffffffff;\n\t"
        "lop3.b32 %0, %0, bal, sx, 0x90;\n\t"
        "}"
        : "+r"(m)
        : "r"(d), "n"(1u << B));
}

__device__ __forceinline__ uint32_t match_digit(uint32_t d) {
    uint32_t m = 0xffffffffu;
    match_bit<0>(d, m);
    match_bit<1>(d, m);
    match_bit<2>(d, m);
    match_bit<3>(d, m);
    match_bit<4>(d, m);
    match_bit<5>(d, m);
    match_bit<6>(d, m);
    match_bit<7>(d, m);
    return m;
}

// The same peer mask from the same eight ballots, with a lookup in place of
// the per-lane selects.  The ballots are warp-uniform, so the peer mask of a
// digit value depends on nothing else: lane l keeps two table entries, T5[l]
// = the lanes whose digit bits 3..7 equal l and T3[l & 7] = the lanes whose
// bits 0..2 equal l & 7, each built against the lane's own index bits (the
// constants sx).  A key's peers are T5[d >> 3] & T3[d & 7], fetched with two
// shuffles (the second within groups of 8 lanes, which all hold T3).  Per key
// row: 8 predicate ops, 8 ballots, 8 table ops, a shift and two shuffles, in
// place of the 8 selects and 8 masks of match_digit.
struct LaneBits {
    uint32_t sx[5];  // all ones where bit b of the lane index is set
};

__device__ __forceinline__ LaneBits lane_bits() {
    LaneBits L;
    const uint32_t lane = lane_id();
#pragma unroll
    for (int b = 0; b < 5; b++) L.sx[b] = 0u - ((lane >> b) & 1u);
    return L;
}

// bal = lanes whose digit has bit B set; m &= ~(bal ^ sx) (lop3 table 0x90)
template <int B>
__device__ __forceinline__ void table_bit(uint32_t d, uint32_t sx, uint32_t& m) {
    asm("{\n\t"
        ".reg .pred p;\n\t"
        ".reg .b32 t, bal;\n\t"
        "and.b32 t, %1, %2;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "vote.sync.ballot.b32 bal, p, 0xffffffff;\n\t"
        "lop3.b32 %0, %0, bal, %3, 0x90;\n\t"
        "}"
        : "+r"(m)
        : "r"(d), "n"(1u << B), "r"(sx));
}

__device__ __forceinline__ uint32_t match_digit_lut(uint32_t d, const LaneBits& L) {
    uint32_t t3 = 0xffffffffu, t5 = 0xffffffffu;
    table_bit<0>(d, L.sx[0], t3);
    table_bit<1>(d, L.sx[1], t3);
    table_bit<2>(d, L.sx[2], t3);
    table_bit<3>(d, L.sx[0], t5);
    table_bit<4>(d, L.sx[1], t5);
    table_bit<5>(d, L.sx[2], t5);
    table_bit<6>(d, L.sx[3], t5);
    table_bit<7>(d, L.sx[4], t5);
    return __shfl_sync(0xffffffffu, t5, d >> 3) & __shfl_sync(0xffffffffu, t3, d, 8);
}

template <typename T>
__device__ __forceinline__ uint32_t digit_of(T cell, uint32_t shift) {
    if constexpr (sizeof(T) == 4) {
        // an 8-bit group is a whole byte: one byte permute extracts it
        return __byte_perm((uint32_t)cell, 0u, 0x4440u | (shift >> 3));
    } else {
        return (uint32_t)(cell >> shift) & (RADIX - 1);
    }
}

__device__ __forceinline__ uint32_t lanemask_gt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_gt;" : "=r"(m));
    return m;
}

// Exclusive scan of one value per thread over a block of NW warps.
// s_warp must hold NW words; *total receives the block sum.
// Contains __syncthreads(); every thread of the block must call it.
template <int NW>
__device__ __forceinline__ uint32_t block_exclusive_scan_n(uint32_t v, uint32_t* s_warp,
                                                           uint32_t* total) {
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t before = 0, sum = 0;
#pragma unroll
    for (int w = 0; w < NW; w++) {
        const uint32_t s = s_warp[w];
        before += (uint32_t)w < warp ? s : 0u;
        sum += s;
    }
    __syncthreads();  // s_warp may be reused by the caller
    *total = sum;
    return before + x - v;
}

// The same over the 256-thread blocks of the other kernels.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp,
                                                         uint32_t* total) {
    return block_exclusive_scan_n<WARPS>(v, s_warp, total);
}

}  // namespace rs
