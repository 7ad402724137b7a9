/*
 * rs.h -- C ABI of the GB300 Recombinant Sort library (librsort.so).
 *
 * Recombinant Sort (Kumar et al., arXiv 2107.01391) maps each key to the
 * cell of an N-dimensional Cartesian count space whose axes are the key's
 * digits (Eq. 1, Eq. 2), counts the keys per cell (the hashing cycle, §3.1),
 * walks the space in raster order to give each occupied cell its output
 * position (the extraction cycle, §3.2, with the cursor overwrite_pos_at),
 * and writes the keys out in that order, rebuilding keys from cell
 * coordinates where the input is not needed (Eq. 16).  When the space does
 * not fit on chip, the leading dimensions act as buckets (§2.2).
 *
 * Every sort here is STABLE: equal keys (and their payloads) keep their input
 * order.  Order is ascending.
 *
 * Conventions shared by every call:
 *   - All key/value/offset/output pointers are DEVICE pointers owned by the
 *     caller.  The library never allocates per call: each sort takes a
 *     caller-provided device workspace `temp`.  Call once with temp == NULL
 *     to receive the required size in *temp_bytes (nothing is launched), then
 *     again with a buffer of at least that many bytes (256-byte aligned).
 *   - `keys_out` may equal `keys_in` (in-place, as the paper overwrites arr);
 *     any other overlap is undefined.  The same holds for values.
 *   - Work is enqueued asynchronously on `stream` (NULL = the legacy default
 *     stream); the call returns before the sort finishes.
 *   - Host-detectable errors return immediately with nothing launched:
 *     RS_ERR_INVALID (NULL pointer with n > 0, misaligned pointer, n above
 *     RS_MAX_N, bad digit counts), RS_ERR_TEMP_TOO_SMALL, RS_ERR_UNSUPPORTED.
 *     A failed CUDA launch returns RS_ERR_CUDA.
 *   - Device-detected errors (a key outside its declared digit space ->
 *     RS_ERR_RANGE; a look-back wait that exceeded its bound ->
 *     RS_ERR_TIMEOUT) are recorded in the context's status word and
 *     returned by rs_ctx_status().  The output of such a call is unspecified.
 *   - Pointers must be aligned to their element size.
 */
#ifndef RS_H
#define RS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream. */
typedef struct CUstream_st* rs_stream_t;

typedef enum rs_status {
    RS_OK = 0,
    RS_ERR_INVALID = 1,
    RS_ERR_RANGE = 2,
    RS_ERR_TEMP_TOO_SMALL = 3,
    RS_ERR_CUDA = 4,
    RS_ERR_TIMEOUT = 5,
    RS_ERR_UNSUPPORTED = 6
} rs_status;

/* Largest n of one sort (per-tile look-back counts are 30-bit); a segmented
 * batch may hold more (RS_MAX_SEGMENTED_N). */
#define RS_MAX_N ((size_t)((1u << 30) - 1u))

typedef enum rs_key_type {
    RS_KEY_U32 = 0,     /* uint32_t */
    RS_KEY_U64 = 1,     /* uint64_t */
    RS_KEY_I64_DEC = 2, /* int64_t fixed-point decimal, see rs_key_params */
    RS_KEY_F32 = 3,     /* float: -0.0 ties with +0.0 and is written as +0.0;
                           NaNs sort last and are written as the quiet NaN */
    RS_KEY_F64 = 4      /* double, same rules as RS_KEY_F32 */
} rs_key_type;

/* Digit layout of a fixed-point decimal key (RS_KEY_I64_DEC): the value
 * x.y is stored as the integer x.y * 10^frac_digits, and every key must
 * satisfy |key| < 10^(int_digits + frac_digits), 1 <= int_digits +
 * frac_digits <= 18.  frac_digits is the paper's λ, the digit count after the
 * decimal point (§3.1.1, "digit_count_after_decimal"). */
typedef struct rs_key_params {
    int32_t int_digits;
    int32_t frac_digits;
} rs_key_params;

typedef struct rs_ctx rs_ctx;

/* ---------------------------------------------------------------- context */

/* Create a context bound to CUDA device `device`.  Allocates the context's
 * 256-byte device status word once (the only allocation the library makes).
 * RS_ERR_INVALID if ctx is NULL or the device does not exist.  A context
 * keeps host-side counters and timing events: use it from one host thread at
 * a time (one context per thread for concurrent callers).  Calls on
 * different contexts may run from several threads at once, with the one
 * exception of rs_sort_u32_noalloc, whose shared workspace serialises its
 * callers. */
rs_status rs_ctx_create(rs_ctx** ctx, int device);

/* Free the context; waits for nothing (the caller must not destroy a context
 * whose sorts are still running). */
rs_status rs_ctx_destroy(rs_ctx* ctx);

/* Device-detected error of the calls made since the last check, then clear
 * it.  synchronize != 0: wait for the whole device first and read the device
 * status word (RS_OK, RS_ERR_RANGE or RS_ERR_TIMEOUT; a CUDA failure while
 * waiting gives RS_ERR_CUDA).  synchronize == 0: report only errors already
 * known on the host, without touching the device. */
rs_status rs_ctx_status(rs_ctx* ctx, int synchronize);

/* ------------------------------------------------------------------ sorts */

/* Sort n uint32 keys (keys only).  The paper's problem statement (the
 * hashing and extraction cycles, §3.1-§3.2) with λ = 0.  When every key is
 * below RS_FILL_CELLS the whole key space is one count array and the output
 * is rebuilt from the counted cells (Eq. 16) without re-reading the keys;
 * otherwise the key's 8-bit digit groups are the dimensions, sorted as
 * buckets from the least significant group on.  At most 4096 keys are sorted
 * by one CTA in one launch, on chip (every sort call shares this path and
 * leaves the workspace untouched). */
#define RS_FILL_CELLS 4096u
rs_status rs_sort_u32(rs_ctx* ctx, const uint32_t* keys_in, uint32_t* keys_out, size_t n,
                      void* temp, size_t* temp_bytes, rs_stream_t stream);

/* Sort n uint64 keys (keys only).  The hashing and extraction cycles
 * (§3.1-§3.2) with λ = 0 over the 20 base-10 digits of a 64-bit key; the
 * cell index of a key is the key itself, split on the device into eight 8-bit
 * digit groups that act as buckets (§2.2) from the least significant on.
 * Keys below RS_FILL_CELLS are rebuilt from one count array (Eq. 16); at most
 * 4096 keys are sorted by one CTA on chip.  Arguments, workspace, aliasing
 * and errors as for rs_sort_u32. */
rs_status rs_sort_u64(rs_ctx* ctx, const uint64_t* keys_in, uint64_t* keys_out, size_t n,
                      void* temp, size_t* temp_bytes, rs_stream_t stream);

/* Sort n fixed-point decimals (int64 scaled by 10^frac_digits, see
 * rs_key_params): the paper's keys with λ = frac_digits digits after the
 * decimal point, integers and decimals mixed (§3.1.2).  Negative keys sort
 * below positive ones.  A key with |key| >= 10^(int_digits+frac_digits)
 * raises RS_ERR_RANGE (device-detected). */
rs_status rs_sort_fixed_decimal(rs_ctx* ctx, const int64_t* keys_in, int64_t* keys_out,
                                size_t n, int int_digits, int frac_digits, void* temp,
                                size_t* temp_bytes, rs_stream_t stream);

/* Stable key/value sort: the value at input i travels with key i.  This is
 * the counting-sort placement of §2.3 carried through the extraction cycle
 * (§3.2): every key is placed at its cell's running output position in input
 * order, and its payload is placed beside it, so ties keep their input order
 * (Table 2 marks the paper's keys-only extraction unstable; the placement
 * form is stable).  kt selects the key type (params required for RS_KEY_I64_DEC, ignored
 * otherwise); val_bytes is 4 or 8, and vals_in/vals_out are device arrays of
 * n values.  val_bytes == 0 with vals_in == vals_out == NULL sorts the keys
 * alone (the keys-only form for every key type).  Float keys (RS_KEY_F32/F64,
 * not in the paper) are mapped to order-preserving unsigned cells of the
 * same width and written back as rs_key_type describes (-0.0 as +0.0, NaNs
 * last as the quiet NaN). */
rs_status rs_sort_pairs(rs_ctx* ctx, rs_key_type kt, const void* keys_in, void* keys_out,
                        const void* vals_in, void* vals_out, size_t val_bytes, size_t n,
                        const rs_key_params* params, void* temp, size_t* temp_bytes,
                        rs_stream_t stream);

/* Stable sort of n byte strings: string i is chars[offsets[i] ..
 * offsets[i+1]).  The paper's reading for strings (Table 2 claims them, §3
 * gives no algorithm): one dimension of the count space per character
 * position, with a padding symbol below every byte past a string's end, so
 * the order is unsigned-byte lexicographic with a proper prefix first.
 *   chars     device bytes; must cover chars[0 .. offsets[n]);
 *   offsets   device uint32_t[n+1], non-decreasing;
 *   max_len   1..RS_MAX_STRING_LEN, an upper bound on every length;
 *   perm_out  device uint32_t[n]: perm_out[j] = input index of the j-th
 *             smallest string (equal strings keep input order).
 * A string longer than max_len, or offsets that decrease or pass offsets[n],
 * raise RS_ERR_RANGE (device-detected); such strings are cut to fit and the
 * output is unspecified.  Cost: the strings are first sorted by their
 * leading floor(56 / w) symbols (w = bits per symbol of the alphabet present,
 * 5 for 'a'..'z', so 11 symbols in seven digit passes).  Only when two strings
 * agree on those symbols and either is longer does a second, general sort
 * run: positions in chunks of floor(64 / w) symbols, least significant chunk
 * first.  Its launches always run but exit at once on the device when it is
 * not needed (a chunk wholly past the longest string is skipped too), so a
 * max_len close to the longest string is cheapest. */
#define RS_MAX_STRING_LEN 1024u
rs_status rs_sort_strings(rs_ctx* ctx, const uint8_t* chars, const uint32_t* offsets, size_t n,
                          uint32_t max_len, uint32_t* perm_out, void* temp, size_t* temp_bytes,
                          rs_stream_t stream);

/* Segmented sort: num_segs independent stable sorts in one call.  Segment
 * s covers positions [seg_offsets[s], seg_offsets[s+1]) of the arrays; every
 * segment is a bucket of its own (§2.2).  Positions outside every segment
 * are left unwritten.
 *   kt, params  key type as in rs_sort_pairs (RS_KEY_F32/F64 allowed here);
 *   n           length of the key (and value) arrays;
 *   seg_offsets device uint64_t[num_segs+1], non-decreasing, at most n; or
 *               NULL for num_segs equal segments of n / num_segs keys (n
 *               must be a multiple of num_segs);
 *   vals_in/out NULL/NULL: keys only.  vals_in given: values move with
 *               their keys.  vals_in NULL with vals_out given: vals_out
 *               receives, for every output position, the index within its
 *               segment of the key placed there (an argsort), as val_bytes
 *               (4 or 8) unsigned integers.
 * n may exceed RS_MAX_N, up to RS_MAX_SEGMENTED_N; a single segment holds at
 * most RS_MAX_SEGMENT_LEN keys.  Offsets that decrease or pass n, or a longer
 * segment, raise RS_ERR_RANGE (device-detected) and the offending segment is
 * skipped (overlapping segments, from offsets that go back, are flagged too;
 * their output is unspecified).  The segments are sorted largest first by
 * one persistent launch: those of at most 63 keys by one warp each, of at
 * most 4096 keys on chip by one CTA in one read and one write, below 2^13
 * keys by one CTA each (whole on chip in one read and one write for 4-byte
 * keys with no value, a 4-byte value or an argsort; tile by tile for other
 * shapes); longer ones by device-wide passes over all of them
 * at once, one launch per digit group, with a look-back per segment.  A
 * segment longer than one CTA's share of the batch (such as the single
 * segment of an argsort of one array) is counted tile-parallel first, so
 * one long segment costs about what a device-wide sort of it costs.  Equal
 * segments (seg_offsets NULL) of 64..4096 keys, or of up to 8192 keys with
 * no values, 4-byte values or an argsort, take a row path instead: one CTA
 * sorts each whole row on chip in one read and one write. */
#define RS_MAX_SEGMENTED_N (1ull << 40)
#define RS_MAX_SEGMENT_LEN RS_MAX_N
rs_status rs_sort_segmented(rs_ctx* ctx, rs_key_type kt, const void* keys_in, void* keys_out,
                            const void* vals_in, void* vals_out, size_t val_bytes, size_t n,
                            const uint64_t* seg_offsets, size_t num_segs,
                            const rs_key_params* params, void* temp, size_t* temp_bytes,
                            rs_stream_t stream);

/* Backward of a row-wise sort: for every row r < rows and position j < cols,
 * dst[r*cols + perm[r*cols + j]] = src[r*cols + j].  Sorting a row permutes
 * it, so the gradient of the input is the gradient of the sorted output
 * scattered back through the permutation (the paper has no gradient; this is
 * the differentiable form of its output step).
 *   src, dst    device arrays of rows*cols elements of elem_bytes (4 or 8),
 *               not overlapping;
 *   perm        device int64_t[rows*cols], each row a permutation of
 *               0..cols-1 (what rs_sort_segmented's argsort output gives).
 * An index outside [0, cols) raises RS_ERR_RANGE (device-detected) and that
 * element is skipped. */
rs_status rs_scatter_rows(rs_ctx* ctx, const void* src, const int64_t* perm, size_t rows,
                          size_t cols, size_t elem_bytes, void* dst, rs_stream_t stream);

/* The hashing cycle's data structures and the extraction cost, on the
 * device, for fixed-point decimals whose whole digit vector fits one count
 * array: S (one dimension per base-10 digit, Eq. 1 / Eq. 2, preceded by a
 * radix-2 sign dimension when signed_dim != 0), the traverse maps of §3.1.3
 * -- H_Max[row] = largest occupied last-axis coordinate, H_Min[row] =
 * [touched flag, smallest occupied coordinate] -- and the extraction cost k
 * of §5, the cells the extraction cycle visits walking each touched row from
 * H_Min to H_Max.  A row is every coordinate but the last (rows = cells / 10).
 * The sort does not need the maps (they only skip empty cells); this call
 * reports them, e.g. k = 17 for the paper's worked example.
 *   keys        device int64_t[n], |key| < 10^(int_digits+frac_digits);
 *               negative keys need signed_dim (else RS_ERR_RANGE);
 *   S_out       device uint32_t[cells] or NULL; cells = (signed_dim ? 2 : 1)
 *               * 10^(int_digits+frac_digits) <= RS_MAX_MAP_CELLS;
 *   hmax_out    device uint32_t[rows]; hmin_out device uint32_t[2*rows];
 *   k_out       device uint64_t[1];
 *   temp        workspace as for the sorts (4 bytes per row). */
#define RS_MAX_MAP_CELLS ((uint64_t)1 << 28)
rs_status rs_traverse_maps(rs_ctx* ctx, const int64_t* keys, size_t n, int int_digits,
                           int frac_digits, int signed_dim, uint32_t* S_out, uint32_t* hmax_out,
                           uint32_t* hmin_out, uint64_t* k_out, void* temp, size_t* temp_bytes,
                           rs_stream_t stream);

/* ------------------------------------------------------- no allocation */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they sort.  cudaFree waits for the
 * whole device and cudaMalloc can stall, which a latency-bound loop cannot
 * afford, and code that runs inside another framework's memory budget (a
 * plugin or a server that owns every device byte through its own pool) has
 * no allocator it may call and no workspace to pass.
 *
 * rs_sort_u32_noalloc sorts n uint32 keys with the same result as rs_sort_u32
 * and the same counting, rebuild and digit-group kernels, but needs no
 * context and no workspace (unlike rs_sort_u32 it takes that multi-launch
 * path for n <= 4096 too, rather than the single-CTA sort): its
 * workspace is a fixed RS_NOALLOC_SCRATCH_BYTES device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  It allocates nothing.
 *   keys_in, keys_out  device arrays of n keys (keys_out may equal keys_in);
 *   n                  at most RS_NOALLOC_MAX_N, else RS_ERR_TEMP_TOO_SMALL
 *                      and nothing is launched;
 *   status             optional device word (NULL allowed): device-detected
 *                      errors are OR-ed into it (value 2 = a look-back
 *                      wait timed out), so the caller can check it after
 *                      the stream finishes;
 *   stream             the work is enqueued on it; the call does not wait.
 * The call runs on the calling thread's current CUDA device.  Its first call
 * on a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture begins.  All calls on a device
 * share the one array and each clears what must start at zero, so calls whose
 * work overlaps on the GPU (concurrent streams, or host threads without
 * ordering between them) race and must be serialised by the caller. */
#define RS_NOALLOC_MAX_N ((size_t)1 << 20)
#define RS_NOALLOC_SCRATCH_BYTES ((size_t)5 << 20)
rs_status rs_sort_u32_noalloc(const uint32_t* keys_in, uint32_t* keys_out, size_t n,
                              uint32_t* status, rs_stream_t stream);

/* ------------------------------------------------------------ diagnostics */

/* What the device-side plan of the most recent sort on this context chose
 * (synchronises the device).  mode: 0 = digit passes, 1 = one count array
 * rebuilt from cells (Eq. 16).  passes_run: passes that moved data;
 * passes_total: passes the key width allows. */
typedef struct rs_plan_info {
    uint32_t mode;
    uint32_t passes_run;
    uint32_t passes_total;
    uint32_t tiles;
} rs_plan_info;
rs_status rs_ctx_last_plan(rs_ctx* ctx, rs_plan_info* info);

/* Pass-tile selection (not in the paper; the paper sorts on one CPU).  The
 * digit-group passes of rs_sort_u32, rs_sort_fixed_decimal (with at most 9
 * digits) and rs_sort_pairs (4-byte cells with no value or a 4-byte value)
 * come in two tile sizes: a wide tile (40-48 keys per thread, 2-3 CTAs per
 * SM), fastest for large sorts, and a narrow one (16 keys per thread, 3 CTAs
 * per SM) that spreads a sort of a few hundred thousand keys over more SMs.
 * Sorts of more than 4096 keys and at most narrow_max_n keys take the narrow
 * tile.  The default, 2^19, is the crossover measured on GB300;
 * paper_2107_01391_gb300/tune.py measures it on the device at hand.  Both
 * tiles give the same result; a workspace query covers either.
 * RS_ERR_INVALID for a NULL context or output pointer. */
rs_status rs_ctx_set_pass_tile_limit(rs_ctx* ctx, uint64_t narrow_max_n);
rs_status rs_ctx_pass_tile_limit(rs_ctx* ctx, uint64_t* narrow_max_n);

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every launch (off by default).  Kernel classes: "hist" (counting), "pass"
 * (digit-group passes), "fill" (rebuild from cells), "pack" (string alphabet
 * and packing), "seg" (segmented sort).
 * rs_ctx_kernel_time() synchronises, sums the elapsed time of every launch
 * of that class since timing was enabled or last reset, and returns it with
 * the launch count.  At most 65536 launches per class are kept. */
rs_status rs_ctx_set_timing(rs_ctx* ctx, int enable);
rs_status rs_ctx_kernel_time(rs_ctx* ctx, const char* kernel_class, double* total_ms,
                             uint64_t* launches);
rs_status rs_ctx_reset_timing(rs_ctx* ctx);

/* Failure-detection check: runs the sorts' bounded look-back wait against a
 * predecessor tile that never publishes (temp: >= 1024 device bytes, zeroed
 * here), so the wait must give up after timeout_ns (1 ns .. 2 s), record
 * RS_ERR_TIMEOUT in the status word and return; the context stays usable.
 * No GPU fault is involved: the wait is a bounded poll of a word that nothing
 * sets. */
rs_status rs_debug_wait_timeout(rs_ctx* ctx, void* temp, size_t temp_bytes, uint64_t timeout_ns,
                                rs_stream_t stream);

/* Kernels this context launched since creation (all classes). */
uint64_t rs_ctx_launch_count(const rs_ctx* ctx);

/* Library version string. */
const char* rs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RS_H */
