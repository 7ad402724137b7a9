// rs_strings.cu -- rs_sort_strings: stable sort of byte strings.
//
// The paper claims strings (Table 2, "PS: Yes") without giving an algorithm.
// Reading: one dimension of the count space per character position (Eq. 1,
// Eq. 2), with a padding symbol below every byte for positions past a
// string's end (the §3.1.2 pre-condition of equal digit counts).  The order
// is unsigned-byte lexicographic with a proper prefix first.
//
// GPU form:
//   1. alphabet_kernel: which byte values occur, and the longest string.  The
//      radix of every position is then (distinct bytes + 1): symbol 0 is the
//      pad, byte b maps to 1 + (number of present bytes below b), so symbol
//      order is byte order.  w = bits per symbol (5 for 'a'..'z').
//   2. The positions are grouped into chunks of s = floor(64 / w) symbols,
//      each packed most significant first into a 64-bit cell: a chunk's cell
//      is the row-major index of the chunk's sub-hypercube.
//   3. First attempt, most significant positions first: the first s'
//      symbols (the most that fit 56 bits, so seven digit groups) are packed
//      in input order and sorted as (cell, string index) pairs, out of place.
//   4. tie_kernel: two neighbours of that order with equal cells share their
//      first s' symbols; if either string is longer than s' they may still
//      differ further on.  Only then are the remaining positions needed: the
//      kernel writes the skip words of step 5 (all skipped when no such tie
//      exists, which for random strings longer than s' is the usual case).
//   5. Fallback, the general form: chunks sorted least significant first
//      (the later positions are sorted first, as buckets of the earlier
//      ones, §2.2) as (cell, string index) pairs with the ordinary digit-group
//      passes; every chunk after the first gathers its cells through the
//      permutation so far, and the last (chunk 0) writes perm_out.
// Chunks wholly past the longest string are skipped on the device.

#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/rs.h"
#include "rs_sort_impl.cuh"

namespace rs {


namespace {

constexpr uint32_t kMinSymbolsPerChunk = 7;  // 64 / 9 bits (256 bytes + pad)

// Device-side description of the key space, written by alphabet_plan.
struct StrPlan {
    uint32_t present[RADIX];  // byte value occurs (0/1), then its symbol
    uint32_t longest;         // longest string seen (clamped to max_len)
    uint32_t width;           // bits per symbol
    uint32_t per_chunk;       // symbols per 64-bit cell
    uint32_t chunks;          // chunks that hold any symbol
    uint32_t done;            // CTAs of alphabet_kernel finished
    uint32_t msd_per_chunk;   // symbols of the first attempt's cell (<= 56 bits)
    uint32_t tie;             // the first attempt left a tie that later positions decide
    uint32_t tie_done;        // CTAs of tie_kernel finished
    uint32_t skip[1];         // per-chunk skip flags of the fallback follow (chunks_max entries)
};

// The first attempt packs the most symbols that fit 56 bits: seven 8-bit
// digit groups, one fewer than a full 64-bit cell of s = floor(64 / w).
__host__ __device__ inline uint32_t msd_symbols(uint32_t w) { return 56u / w; }

__global__ void __launch_bounds__(BLOCK) alphabet_kernel(const uint8_t* chars,
                                                         const uint32_t* offsets, uint64_t n,
                                                         uint32_t max_len, uint32_t chunks_max,
                                                         StrPlan* sp, uint32_t* status) {
    __shared__ uint32_t s_present[RADIX];
    __shared__ uint32_t s_longest;
    __shared__ uint32_t s_last;
    const uint32_t t = threadIdx.x;
    s_present[t] = 0;
    if (t == 0) s_longest = 0;
    __syncthreads();
    const uint64_t gtid = (uint64_t)blockIdx.x * BLOCK + t;
    const uint64_t gsize = (uint64_t)gridDim.x * BLOCK;
    bool bad = false;
    uint32_t longest = 0;
    const uint32_t last = n ? offsets[n] : 0;
    for (uint64_t i = gtid; i < n; i += gsize) {
        const uint32_t b = offsets[i], e = offsets[i + 1];
        if (e < b || e > last) {
            bad = true;  // offsets must not decrease nor pass offsets[n]
            continue;
        }
        uint32_t len = e - b;
        if (len > max_len) {
            bad = true;
            len = max_len;
        }
        longest = max(longest, len);
    }
    // bytes that occur: the char buffer between the first and last offset,
    // read 16 bytes at a time, four loads in flight per thread (every writer
    // stores 1: the races are benign)
    const uint32_t c0 = n ? offsets[0] : 0, c1 = last;
    const uint64_t span = c1 > c0 ? c1 - c0 : 0;
    const uint64_t mis = (16 - (reinterpret_cast<uintptr_t>(chars + c0) & 15)) & 15;
    const uint64_t head = mis < span ? mis : span;
    const uint64_t nvec = (span - head) / 16;
    for (uint64_t c = gtid; c < head; c += gsize) s_present[chars[c0 + c]] = 1;
    const uint4* vec = reinterpret_cast<const uint4*>(chars + c0 + head);
    auto mark = [&](const uint4& v) {
        const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int by = 0; by < 4; by++) s_present[(wd[k] >> (8 * by)) & 0xffu] = 1;
    };
    uint64_t q = gtid;
    for (; q + 3 * gsize < nvec; q += 4 * gsize) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++) v[u] = __ldcs(&vec[q + u * gsize]);
#pragma unroll
        for (int u = 0; u < 4; u++) mark(v[u]);
    }
    for (; q < nvec; q += gsize) mark(__ldcs(&vec[q]));
    for (uint64_t c = head + nvec * 16 + gtid; c < span; c += gsize) s_present[chars[c0 + c]] = 1;
    if (bad) atomicOr(status, STATUS_RANGE);
    atomicMax(&s_longest, longest);
    __syncthreads();
    if (s_present[t]) sp->present[t] = 1;
    if (t == 0) atomicMax(&sp->longest, s_longest);
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&sp->done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // last CTA: symbols (exclusive count of present bytes below b, plus one)
    __shared__ uint32_t s_warp[WARPS];
    const uint32_t p = __ldcg(&sp->present[t]);
    uint32_t distinct;
    const uint32_t below = block_exclusive_scan(p, s_warp, &distinct);
    sp->present[t] = p ? below + 1 : 0;
    if (t == 0) {
        uint32_t w = 1;
        while ((1u << w) <= distinct) w++;  // symbols 0..distinct need w bits
        const uint32_t s = 64 / w;
        const uint32_t longest_all = __ldcg(&sp->longest);
        // at least one chunk, so that all-empty input still yields the identity
        const uint32_t chunks = longest_all ? (longest_all + s - 1) / s : 1;
        sp->width = w;
        sp->per_chunk = s;
        sp->chunks = chunks;
        sp->msd_per_chunk = msd_symbols(w);
        // the fallback's chunks stay skipped unless tie_kernel finds a tie
        for (uint32_t c = 0; c < chunks_max; c++) sp->skip[c] = 1;
    }
}

// Length of string i, kept inside chars[0, offsets[n]) and max_len as the
// pack kernel keeps it.
__device__ __forceinline__ uint32_t str_len(const uint32_t* offsets, uint64_t n, uint32_t max_len,
                                            uint32_t i) {
    const uint32_t end = offsets[n];
    const uint32_t b = min(offsets[i], end), e = min(offsets[i + 1], end);
    return e < b ? 0u : min(e - b, max_len);
}

// After the first attempt: neighbours with equal cells agree on their first
// s' symbols, and their input order is final only when neither string is
// longer than s' (then they are equal strings).  Any other tie switches the
// fallback on: its chunks that hold symbols are no longer skipped.
__global__ void __launch_bounds__(BLOCK) tie_kernel(const uint64_t* cells, const uint32_t* perm,
                                                    const uint32_t* offsets, uint64_t n,
                                                    uint32_t max_len, uint32_t chunks_max,
                                                    StrPlan* sp) {
    __shared__ uint32_t s_last;
    const uint32_t t = threadIdx.x;
    const uint32_t s1 = sp->msd_per_chunk;
    bool tie = false;
    for (uint64_t j = 1 + (uint64_t)blockIdx.x * BLOCK + t; j < n;
         j += (uint64_t)gridDim.x * BLOCK) {
        if (cells[j] == cells[j - 1] && (str_len(offsets, n, max_len, perm[j]) > s1 ||
                                         str_len(offsets, n, max_len, perm[j - 1]) > s1))
            tie = true;
    }
    if (__syncthreads_or(tie) && t == 0) atomicOr(&sp->tie, 1u);
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&sp->tie_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const bool fallback = __ldcg(&sp->tie) != 0;
    const uint32_t chunks = sp->chunks;
    for (uint32_t c = t; c < chunks_max; c += BLOCK) sp->skip[c] = !fallback || c >= chunks;
}

// Cells of chunk c: symbols [c*s, (c+1)*s) of each string, packed most
// significant first.  The first chunk processed reads strings in input order;
// later chunks read string perm[j] for output slot j.  msd != 0: the first
// attempt's cell, symbols [0, s') in input order.
// (grid-stride over output slots, so that a skipped chunk costs one short
// launch; the byte -> symbol table is staged in shared memory)
__global__ void __launch_bounds__(BLOCK) pack_kernel(const uint8_t* chars, const uint32_t* offsets,
                                                     uint64_t n, uint32_t max_len, uint32_t c,
                                                     uint32_t msd, const StrPlan* sp,
                                                     uint64_t* cells, uint32_t* idx) {
    if (!msd && sp->skip[c]) return;
    __shared__ uint32_t s_sym[RADIX];
    s_sym[threadIdx.x] = sp->present[threadIdx.x];
    __syncthreads();
    const bool first = msd || c + 1 == sp->chunks;
    // stay inside chars[0, offsets[n]) even for malformed offsets (flagged
    // as RS_ERR_RANGE by alphabet_kernel)
    const uint32_t end = offsets[n];
    const uint32_t w = sp->width, s = msd ? sp->msd_per_chunk : sp->per_chunk;
    const uint32_t p0 = msd ? 0u : c * s;
    for (uint64_t j = (uint64_t)blockIdx.x * BLOCK + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * BLOCK) {
        const uint32_t i = first ? (uint32_t)j : idx[j];
        const uint32_t b = min(offsets[i], end), e = min(offsets[i + 1], end);
        const uint32_t len = e < b ? 0u : min(e - b, max_len);
        const uint8_t* str = chars + b;
        uint64_t cell = 0;
        if (s <= 16) {
            // chunks of at most 16 symbols: independent, unrolled byte loads
            uint32_t byte[16];
#pragma unroll
            for (uint32_t q = 0; q < 16; q++)
                byte[q] = q < s && p0 + q < len ? __ldg(&str[p0 + q]) : 0u;
#pragma unroll
            for (uint32_t q = 0; q < 16; q++)
                if (q < s) cell = (cell << w) | (p0 + q < len ? s_sym[byte[q]] : 0u);
        } else {
            for (uint32_t q = 0; q < s; q++) {
                const uint32_t pos = p0 + q;
                cell = (cell << w) | (pos < len ? s_sym[__ldg(&str[pos])] : 0u);
            }
        }
        cells[j] = cell;
        idx[j] = i;
    }
}

}  // namespace
}  // namespace rs

using namespace rs;

extern "C" rs_status rs_sort_strings(rs_ctx* ctx, const uint8_t* chars, const uint32_t* offsets,
                                     size_t n, uint32_t max_len, uint32_t* perm_out, void* temp,
                                     size_t* temp_bytes, rs_stream_t stream) {
    if (!ctx || !temp_bytes) return RS_ERR_INVALID;
    if (n > RS_MAX_N || max_len == 0 || max_len > RS_MAX_STRING_LEN) return RS_ERR_INVALID;
    if (n > 0 && (!offsets || !perm_out || (reinterpret_cast<uintptr_t>(offsets) % 4) ||
                  (reinterpret_cast<uintptr_t>(perm_out) % 4)))
        return RS_ERR_INVALID;
    const uint32_t chunks_max = (max_len + kMinSymbolsPerChunk - 1) / kMinSymbolsPerChunk;
    cudaStream_t st = (cudaStream_t)stream;

    // workspace: [StrPlan + skip flags][cells u64 n][idx u32 n][sorted cells u64 n]
    //            [pairs-sort workspace]
    size_t sort_bytes = 0;
    rs_status s = run_sort<CodecU64, uint32_t>(ctx, nullptr, nullptr, nullptr, nullptr, n,
                                                    CodecParams{0}, 64, nullptr, &sort_bytes, st,
                                                    nullptr);
    if (s != RS_OK) return s;
    const size_t plan_bytes = align_up(sizeof(StrPlan) + sizeof(uint32_t) * chunks_max);
    const size_t cells_off = plan_bytes;
    const size_t idx_off = cells_off + align_up(sizeof(uint64_t) * std::max<size_t>(n, 1));
    const size_t sorted_off = idx_off + align_up(sizeof(uint32_t) * std::max<size_t>(n, 1));
    const size_t sort_off = sorted_off + align_up(sizeof(uint64_t) * std::max<size_t>(n, 1));
    const size_t total = sort_off + sort_bytes;
    if (!temp) {
        *temp_bytes = total;
        return RS_OK;
    }
    if (*temp_bytes < total) return RS_ERR_TEMP_TOO_SMALL;
    if (reinterpret_cast<uintptr_t>(temp) % 256) return RS_ERR_INVALID;
    if (n == 0) return RS_OK;
    if (!chars) return RS_ERR_INVALID;

    DeviceGuard dg(ctx->device);
    if (!dg.ok) return RS_ERR_CUDA;
    unsigned char* T = static_cast<unsigned char*>(temp);
    StrPlan* sp = reinterpret_cast<StrPlan*>(T);
    uint64_t* cells = reinterpret_cast<uint64_t*>(T + cells_off);
    uint32_t* idx = reinterpret_cast<uint32_t*>(T + idx_off);
    uint64_t* sorted = reinterpret_cast<uint64_t*>(T + sorted_off);
    void* sort_temp = T + sort_off;
    const int sms = sm_count(ctx->device);

    if (cudaMemsetAsync(T, 0, plan_bytes, st) != cudaSuccess) return RS_ERR_CUDA;
    {
        // enough CTAs for the strings and for the bytes (at most n * max_len
        // of them, 16 per load, 8 loads per thread)
        const size_t by_strings = (n + BLOCK * 8 - 1) / (BLOCK * 8);
        const size_t by_bytes = (n * (size_t)max_len + BLOCK * 128 - 1) / (BLOCK * 128);
        const int grid = (int)std::min<size_t>(std::max(by_strings, by_bytes), (size_t)sms * 8);
        LaunchTimer lt(ctx, KC_PACK, st);
        alphabet_kernel<<<std::max(grid, 1), BLOCK, 0, st>>>(chars, offsets, n, max_len,
                                                            chunks_max, sp, ctx->d_status);
    }
    const unsigned grid_n =
        (unsigned)std::min<size_t>((n + BLOCK - 1) / BLOCK, (size_t)sms * 8);
    // first attempt: the leading s' symbols, input order, sorted out of place
    // into (sorted, perm_out)
    {
        LaunchTimer lt(ctx, KC_PACK, st);
        pack_kernel<<<grid_n, BLOCK, 0, st>>>(chars, offsets, n, max_len, 0u, 1u, sp, cells, idx);
    }
    size_t tb = sort_bytes;
    s = run_sort<CodecU64, uint32_t>(ctx, cells, sorted, idx, perm_out, n, CodecParams{0}, 64,
                                     sort_temp, &tb, st, nullptr);
    if (s != RS_OK) return s;
    {
        LaunchTimer lt(ctx, KC_PACK, st);
        tie_kernel<<<grid_n, BLOCK, 0, st>>>(sorted, perm_out, offsets, n, max_len, chunks_max,
                                             sp);
    }
    // fallback (skipped on the device unless a tie needs later positions):
    // chunks least significant first, in place; chunk 0 writes perm_out
    for (int c = (int)chunks_max - 1; c >= 0; c--) {
        {
            LaunchTimer lt(ctx, KC_PACK, st);
            pack_kernel<<<grid_n, BLOCK, 0, st>>>(chars, offsets, n, max_len, (uint32_t)c, 0u, sp,
                                                  cells, idx);
        }
        tb = sort_bytes;
        if (c > 0)
            s = run_sort<CodecU64, uint32_t>(ctx, cells, cells, idx, idx, n, CodecParams{0}, 64,
                                             sort_temp, &tb, st, &sp->skip[c]);
        else
            s = run_sort<CodecU64, uint32_t>(ctx, cells, sorted, idx, perm_out, n,
                                             CodecParams{0}, 64, sort_temp, &tb, st,
                                             &sp->skip[0]);
        if (s != RS_OK) return s;
    }
    return cudaGetLastError() == cudaSuccess ? RS_OK : RS_ERR_CUDA;
}
