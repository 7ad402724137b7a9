/*
 * rs_oracle.h -- the plain CPU Recombinant Sort used as the parity oracle.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load this code.  It shares
 * nothing with the CUDA path (no headers, no helpers, no tables).
 *
 * Every function follows Kumar et al., "Recombinant Sort" (arXiv 2107.01391):
 *   - key normalisation: the pre-condition of §3.1.2 (pad every key to the
 *     same digit count) and the digit set Λ_Θ of §3.1.1;
 *   - the hashing cycle: Eq. 1 / Eq. 2 and the "Recombinant-hashing"
 *     algorithm of §3.1 (count array S plus traverse maps H_Max, H_Min);
 *   - the extraction cycle: the raster walk of §3.2 and its n-digit form in
 *     the supplementary section, with the output cursor overwrite_pos_at and
 *     the key regeneration of Eq. 16;
 *   - buckets (§2.2) when a key has more dimensions than one count array
 *     holds, and the positional arithmetic of counting sort (§2.3) to place
 *     keys with their payloads.
 *
 * All outputs are caller-allocated.  Return value: 0 on success,
 * ORACLE_ERR_RANGE if a key does not fit the declared digit count,
 * ORACLE_ERR_INVALID for bad arguments, ORACLE_ERR_NOMEM on allocation
 * failure.
 */
#ifndef RS_ORACLE_H
#define RS_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID 1
#define ORACLE_ERR_RANGE 2
#define ORACLE_ERR_NOMEM 3

/* Default upper bound on the cells of one count array S.  1000 = the
 * 10x10x10 space, the largest one the paper tabulates (Table 3). */
#define ORACLE_DEFAULT_CELL_CAP 1000u

typedef struct {
    uint64_t k;          /* extraction cost (§5): cells visited, summed over every extraction cycle */
    uint64_t cycles;     /* hashing+extraction cycles run (one per bucket per level) */
    uint64_t dims;       /* dimensions of the normalised key (digits or character positions) */
    uint64_t top_cells;  /* cells of the first count array S */
    int32_t regenerated; /* 1 if keys_out was written from cell coordinates (Eq. 16) */
    int32_t pad_;
} oracle_stats;

/* Unsigned 32-bit keys.  The digit count D is the number of decimal digits
 * of the largest key (the §3.1.2 pre-condition), at least 1.
 * keys_out (n, nullable) receives the sorted keys; perm_out (n, nullable)
 * receives, for output position j, the input index of the key placed there.
 * cell_cap = 0 selects ORACLE_DEFAULT_CELL_CAP. */
int oracle_sort_u32(const uint32_t* keys, size_t n, uint64_t cell_cap,
                    uint32_t* keys_out, uint64_t* perm_out, oracle_stats* st);

/* Unsigned 64-bit keys, same contract (D up to 20). */
int oracle_sort_u64(const uint64_t* keys, size_t n, uint64_t cell_cap,
                    uint64_t* keys_out, uint64_t* perm_out, oracle_stats* st);

/* Fixed-point decimals stored as int64 scaled by 10^frac_digits (a value
 * x.y with frac_digits = λ is stored as x.y * 10^λ).  Every |key| must be
 * below 10^(int_digits + frac_digits), else ORACLE_ERR_RANGE.  If some key is
 * negative a leading sign dimension of radix 2 is added (negative < positive)
 * and the magnitude digits of a negative key are complemented (9 - digit). */
int oracle_sort_fixed_decimal(const int64_t* keys, size_t n, int int_digits, int frac_digits,
                              uint64_t cell_cap, int64_t* keys_out, uint64_t* perm_out,
                              oracle_stats* st);

/* Byte strings: string i is chars[offsets[i] .. offsets[i+1]).  One dimension
 * per character position, max_len positions (0 = the longest string's
 * length); a string longer than max_len is ORACLE_ERR_RANGE.  Position d of
 * a string holds byte+1, or 0 past its end (the padding symbol ranks below
 * every byte), so the order is unsigned-byte lexicographic with a proper
 * prefix first.  perm_out (n) receives the input index of each output. */
int oracle_sort_strings(const uint8_t* chars, const uint64_t* offsets, size_t n,
                        uint32_t max_len, uint64_t cell_cap, uint64_t* perm_out,
                        oracle_stats* st);

/* IEEE-754 doubles (not in the paper): a class dimension (negative < zero
 * < positive < NaN) then the 19 decimal digits of the magnitude bits,
 * complemented for negatives.  -0.0 ties with +0.0; NaNs tie and sort last.
 * keys_out receives the input keys in sorted order (bits unchanged). */
int oracle_sort_f64(const double* keys, size_t n, uint64_t cell_cap, double* keys_out,
                    uint64_t* perm_out, oracle_stats* st);

/* One hashing cycle over fixed-point decimal keys whose whole digit vector
 * fits a single count array (the worked example's case), exposing the
 * paper's data structures.  radix_out (up to 32 entries) receives the shape
 * of S; *rank_out its number of dimensions.  S_out (cells), hmax_out (rows)
 * and hmin_out (2 * rows, [flag, min] per row) may be NULL to query the
 * shape only; rows = cells / (last radix).  *k_out (nullable) receives the
 * extraction cost of the cycle that follows. */
int oracle_decimal_hashing_cycle(const int64_t* keys, size_t n, int int_digits, int frac_digits,
                                 uint32_t* radix_out, int* rank_out, uint64_t* S_out,
                                 uint32_t* hmax_out, uint32_t* hmin_out, uint64_t* k_out);

#ifdef __cplusplus
}
#endif

#endif /* RS_ORACLE_H */
