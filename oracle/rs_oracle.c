/*
 * rs_oracle.c -- plain, slow, single-threaded CPU Recombinant Sort.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Tests, the smoke check and
 * the benchmark's CPU-baseline leg are the only callers.  Nothing here is
 * shared with the CUDA path, and nothing here is tuned: the code takes the
 * paper's steps in the paper's order so that it can be checked by eye.
 *
 * Source: Kumar, Gangal, Kumari, Tiwari, "Recombinant Sort: N-Dimensional
 * Cartesian Spaced Algorithm ..." (arXiv 2107.01391).
 *
 *   Normalise (§3.1.1, §3.1.2)  every key becomes its digit set Λ_Θ, a vector
 *                               of D digits, most significant first, after
 *                               padding all keys to one digit count.
 *   Hashing cycle (§3.1, Eq. 1) S[digits]++ for each key, while the traverse
 *                               maps H_Max / H_Min keep, per row of S, the
 *                               largest and smallest occupied column.
 *   Extraction cycle (§3.2)     walk S row by row in raster order, each row
 *                               only from H_Min to H_Max, skipping rows whose
 *                               H_Min flag was never set; the running cursor
 *                               overwrite_pos_at gives every occupied cell its
 *                               first output position; stop at `size`.
 *   Output                      keys-only and one count array: write the
 *                               key rebuilt from the cell's coordinates
 *                               S[count] times (Eq. 16).  Otherwise place
 *                               each key (and payload index) at its cell's
 *                               cursor in input order -- the positional
 *                               arithmetic of counting sort (§2.3) -- which
 *                               keeps equal keys in input order.
 *   Buckets (§2.2)              a key with more dimensions than one count
 *                               array holds (cell_cap) is split: the leading
 *                               dimensions form the count array, and each
 *                               occupied cell is a bucket sorted on the
 *                               remaining dimensions by the same two cycles.
 *
 * Readings where the paper is silent or garbled (all output-invariant except
 * where noted):
 *   - The loop "for j = H_Min[i][1] to H_Max[i]+1" is half-open, so a row is
 *     walked from H_Min to H_Max inclusive, and rows whose H_Min flag is 0
 *     are skipped.  With this reading the worked example costs k = 17 (§3.2).
 *   - The n-digit traverse maps are indexed by the prefix of all but the
 *     last dimension of S (rows = cells / last radix); H_Max keeps the
 *     largest last coordinate, H_Min a [flag, smallest] pair.
 *   - Negative decimals: a leading sign dimension of radix 2 (negative
 *     first) is added when some key is negative, and the magnitude digits of
 *     a negative key are complemented (9 - d) so raster order is value order.
 *   - Strings: one dimension per character position, radix 257, symbol 0 =
 *     past the end, byte b -> b + 1.
 *   - Floating-point keys (not in the paper): a leading class dimension of
 *     radix 4 (negative, zero of either sign, positive, NaN), then the 19
 *     base-10 digits of the magnitude's IEEE-754 bit pattern read as an
 *     integer (for finite non-negative doubles that integer grows with the
 *     value), complemented (9 - d) for negative keys.  -0.0 ties with +0.0
 *     and every NaN ties with every other, after all numbers.
 *   - Stability: keys are placed in input order, so equal keys keep their
 *     input order (the paper's keys-only output cannot show the difference).
 */
#include "rs_oracle.h"

#include <stdlib.h>
#include <string.h>

enum { KIND_U32 = 0, KIND_U64 = 1, KIND_DEC = 2, KIND_STR = 3, KIND_F64 = 4 };

#define MAX_DIMS 4096

/* The normalised key space: D dimensions, each with its own radix. */
typedef struct {
    int kind;
    int D;
    uint32_t radix[MAX_DIMS];
    const void* keys;
    const uint8_t* chars;
    const uint64_t* offsets;
    int neg_dim;      /* DEC: 1 if a sign dimension leads the digit vector */
    int mag_digits;   /* DEC: digits of the magnitude (int_digits + frac_digits) */
} keyspace;

static const uint64_t POW10[20] = {
    1ull, 10ull, 100ull, 1000ull, 10000ull, 100000ull, 1000000ull, 10000000ull,
    100000000ull, 1000000000ull, 10000000000ull, 100000000000ull, 1000000000000ull,
    10000000000000ull, 100000000000000ull, 1000000000000000ull, 10000000000000000ull,
    100000000000000000ull, 1000000000000000000ull, 10000000000000000000ull};

/* Number of decimal digits of v (at least 1). */
static int decimal_digits(uint64_t v) {
    int d = 1;
    while (d < 20 && v >= POW10[d]) d++;
    return d;
}

static uint64_t magnitude(int64_t v) {
    return v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
}

/* Digit d (0 = most significant) of item i: one coordinate of the cell
 * S[n1][n2]...[nn] that Eq. 1 increments for the key. */
static uint32_t digit_of(const keyspace* ks, uint64_t i, int d) {
    switch (ks->kind) {
    case KIND_U32: {
        uint64_t v = ((const uint32_t*)ks->keys)[i];
        return (uint32_t)((v / POW10[ks->D - 1 - d]) % 10u);
    }
    case KIND_U64: {
        uint64_t v = ((const uint64_t*)ks->keys)[i];
        return (uint32_t)((v / POW10[ks->D - 1 - d]) % 10u);
    }
    case KIND_DEC: {
        int64_t v = ((const int64_t*)ks->keys)[i];
        if (ks->neg_dim) {
            if (d == 0) return v < 0 ? 0u : 1u;
            d -= 1;
        }
        uint32_t dig = (uint32_t)((magnitude(v) / POW10[ks->mag_digits - 1 - d]) % 10u);
        return v < 0 ? 9u - dig : dig;
    }
    case KIND_F64: {
        double x = ((const double*)ks->keys)[i];
        uint64_t bits;
        memcpy(&bits, &x, sizeof(bits));
        const uint64_t mag = bits & 0x7fffffffffffffffull;
        const int is_nan = (mag >> 52) == 0x7ffull && (mag & 0xfffffffffffffull) != 0;
        const int negative = (bits >> 63) != 0;
        if (d == 0) {
            if (is_nan) return 3u;
            if (mag == 0) return 1u;
            return negative ? 0u : 2u;
        }
        if (is_nan || mag == 0) return 0u;
        uint32_t dig = (uint32_t)((mag / POW10[19 - d]) % 10u);
        return negative ? 9u - dig : dig;
    }
    default: { /* KIND_STR */
        uint64_t beg = ks->offsets[i], len = ks->offsets[i + 1] - beg;
        return (uint64_t)d < len ? (uint32_t)ks->chars[beg + (uint64_t)d] + 1u : 0u;
    }
    }
}

typedef struct {
    uint64_t lo, count;
} bucket;

/* One count array S over dimensions [d0, d0 + g) with its traverse maps.
 * rows = cells / (radix of the last dimension); H_Min holds a [flag, min]
 * pair per row, H_Max the max per row; cursor[] is the extraction output. */
typedef struct {
    int d0, g;
    uint64_t cells, rows, r_last;
    uint64_t* S;
    uint64_t* H_Max;
    uint64_t* H_Min;
    uint64_t* cursor;
} count_array;

/* The count array of the level starting at d0: the next g dimensions whose
 * radix product stays within cell_cap (at least one dimension). */
static int count_array_init(count_array* ca, const keyspace* ks, int d0, uint64_t cell_cap) {
    int g = 1;
    uint64_t cells = ks->radix[d0];
    while (d0 + g < ks->D && cells * ks->radix[d0 + g] <= cell_cap) {
        cells *= ks->radix[d0 + g];
        g++;
    }
    ca->d0 = d0;
    ca->g = g;
    ca->cells = cells;
    ca->r_last = ks->radix[d0 + g - 1];
    ca->rows = cells / ca->r_last;
    ca->S = (uint64_t*)calloc(cells, sizeof(uint64_t));
    ca->cursor = (uint64_t*)calloc(cells, sizeof(uint64_t));
    ca->H_Max = (uint64_t*)calloc(ca->rows, sizeof(uint64_t));
    ca->H_Min = (uint64_t*)calloc(2 * ca->rows, sizeof(uint64_t));
    if (!ca->S || !ca->cursor || !ca->H_Max || !ca->H_Min) return ORACLE_ERR_NOMEM;
    return ORACLE_OK;
}

static void count_array_free(count_array* ca) {
    free(ca->S);
    free(ca->cursor);
    free(ca->H_Max);
    free(ca->H_Min);
    ca->S = ca->cursor = ca->H_Max = ca->H_Min = NULL;
}

/* ---- Hashing cycle (§3.1, Eq. 1): S[n_d0]...[n_d0+g-1]++ per key, in
 * input order, with the traverse-map updates of the hashing algorithm.
 * cell_of[t] receives the cell of items[t]. */
static void hashing_cycle(const keyspace* ks, count_array* ca, const uint64_t* items,
                          uint64_t count, uint64_t* cell_of) {
    for (uint64_t t = 0; t < count; t++) {
        uint64_t c = 0;
        for (int d = ca->d0; d < ca->d0 + ca->g; d++)
            c = c * ks->radix[d] + digit_of(ks, items[t], d);
        cell_of[t] = c;
        ca->S[c] += 1;
        uint64_t row = c / ca->r_last, col = c % ca->r_last;
        if (ca->H_Max[row] < col) ca->H_Max[row] = col;
        if (ca->H_Min[2 * row] == 0) {
            ca->H_Min[2 * row + 1] = col;
            ca->H_Min[2 * row] = 1;
        } else if (ca->H_Min[2 * row + 1] > col) {
            ca->H_Min[2 * row + 1] = col;
        }
    }
}

/* ---- Extraction cycle (§3.2): raster walk of S, each touched row from
 * H_Min to H_Max, with the running cursor overwrite_pos_at; each occupied
 * cell gets its first output position in cursor[].  Stops once all `count`
 * keys are out.  Returns the cells visited (the extraction cost k, §5). */
static uint64_t extraction_cycle(count_array* ca, uint64_t count) {
    uint64_t k = 0, overwrite_pos_at = 0;
    for (uint64_t row = 0; row < ca->rows && overwrite_pos_at < count; row++) {
        if (ca->H_Min[2 * row] == 0) continue; /* row never touched */
        for (uint64_t col = ca->H_Min[2 * row + 1]; col <= ca->H_Max[row]; col++) {
            k++;
            uint64_t c = row * ca->r_last + col;
            if (ca->S[c] != 0) {
                ca->cursor[c] = overwrite_pos_at;
                overwrite_pos_at += ca->S[c];
                if (overwrite_pos_at == count) break; /* every key extracted */
            }
        }
    }
    return k;
}

/*
 * Sort items[lo, lo + count) on dimensions d0.. of the key space: one hashing
 * cycle and one extraction cycle over the count array of the leading
 * dimensions that fit cell_cap, then each occupied cell as a bucket.
 * items[] holds input indices; scratch[] is a same-sized work array.
 */
static int sort_bucket(const keyspace* ks, uint64_t* items, uint64_t* scratch, uint64_t lo,
                       uint64_t count, int d0, uint64_t cell_cap, oracle_stats* st) {
    if (count <= 1 || d0 >= ks->D) return ORACLE_OK; /* one key, or all keys equal */

    count_array ca;
    uint64_t* cell_of = (uint64_t*)malloc(count * sizeof(uint64_t));
    if (count_array_init(&ca, ks, d0, cell_cap) != ORACLE_OK || !cell_of) {
        count_array_free(&ca);
        free(cell_of);
        return ORACLE_ERR_NOMEM;
    }
    st->cycles++;
    hashing_cycle(ks, &ca, items + lo, count, cell_of);
    st->k += extraction_cycle(&ca, count);

    /* ---- Placement in input order (counting sort, §2.3): stable ---- */
    for (uint64_t t = 0; t < count; t++) scratch[lo + ca.cursor[cell_of[t]]++] = items[lo + t];
    memcpy(items + lo, scratch + lo, count * sizeof(uint64_t));
    free(cell_of);

    /* ---- Buckets (§2.2): each occupied cell sorted on the remaining dims ---- */
    int rc = ORACLE_OK;
    const int next = d0 + ca.g;
    if (next < ks->D) {
        uint64_t nb = 0;
        for (uint64_t c = 0; c < ca.cells; c++) nb += ca.S[c] > 1;
        bucket* bk = (bucket*)malloc((nb ? nb : 1) * sizeof(bucket));
        if (!bk) {
            count_array_free(&ca);
            return ORACLE_ERR_NOMEM;
        }
        uint64_t at = lo, b = 0;
        for (uint64_t c = 0; c < ca.cells; c++) {
            if (ca.S[c] > 1) bk[b++] = (bucket){at, ca.S[c]};
            at += ca.S[c];
        }
        count_array_free(&ca);
        for (uint64_t i = 0; i < nb && rc == ORACLE_OK; i++)
            rc = sort_bucket(ks, items, scratch, bk[i].lo, bk[i].count, next, cell_cap, st);
        free(bk);
    } else {
        count_array_free(&ca);
    }
    return rc;
}

/* Run the whole sort: items[] ends as the stable permutation. */
static int run_sort(const keyspace* ks, size_t n, uint64_t cell_cap, uint64_t* items,
                    oracle_stats* st) {
    for (uint64_t i = 0; i < n; i++) items[i] = i;
    uint64_t* scratch = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!scratch) return ORACLE_ERR_NOMEM;
    int rc = sort_bucket(ks, items, scratch, 0, n, 0, cell_cap, st);
    free(scratch);
    return rc;
}

/* Cells of the first count array for a key space under cell_cap. */
static uint64_t top_cells(const keyspace* ks, uint64_t cell_cap, int* g_out) {
    int g = 1;
    uint64_t cells = ks->radix[0];
    while (g < ks->D && cells * ks->radix[g] <= cell_cap) {
        cells *= ks->radix[g];
        g++;
    }
    if (g_out) *g_out = g;
    return cells;
}

static void stats_init(oracle_stats* st, const keyspace* ks, uint64_t cell_cap) {
    memset(st, 0, sizeof(*st));
    st->dims = (uint64_t)ks->D;
    st->top_cells = ks->D > 0 ? top_cells(ks, cell_cap, NULL) : 0;
}

/*
 * Keys-only output when the whole digit vector fits one count array: the
 * extraction cycle writes each occupied cell's key, rebuilt from the cell
 * coordinates (Eq. 16), S[cell] times.  Runs its own hashing and extraction
 * cycle so that the written keys come from cells, not from the input.
 * emit(cell, j) writes output position j.
 */
typedef void (*emit_fn)(const keyspace* ks, uint64_t cell, uint64_t j, void* out);

static int regenerate_keys(const keyspace* ks, size_t n, emit_fn emit, void* out) {
    count_array ca;
    uint64_t* items = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* cell_of = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t cells = 1;
    for (int d = 0; d < ks->D; d++) cells *= ks->radix[d];
    if (count_array_init(&ca, ks, 0, cells) != ORACLE_OK || !items || !cell_of) {
        count_array_free(&ca);
        free(items);
        free(cell_of);
        return ORACLE_ERR_NOMEM;
    }
    for (uint64_t i = 0; i < n; i++) items[i] = i;
    hashing_cycle(ks, &ca, items, n, cell_of);
    extraction_cycle(&ca, n);
    for (uint64_t c = 0; c < ca.cells; c++)
        for (uint64_t z = 0; z < ca.S[c]; z++) emit(ks, c, ca.cursor[c] + z, out);
    free(items);
    free(cell_of);
    count_array_free(&ca);
    return ORACLE_OK;
}

/* Eq. 16 for unsigned integers: the row-major cell index of a base-10
 * hypercube is the number whose digits are the coordinates. */
static void emit_u32(const keyspace* ks, uint64_t cell, uint64_t j, void* out) {
    (void)ks;
    ((uint32_t*)out)[j] = (uint32_t)cell;
}
static void emit_u64(const keyspace* ks, uint64_t cell, uint64_t j, void* out) {
    (void)ks;
    ((uint64_t*)out)[j] = cell;
}
/* Eq. 16 for decimals: coordinates -> sign and magnitude digits. */
static void emit_dec(const keyspace* ks, uint64_t cell, uint64_t j, void* out) {
    uint64_t mag = 0, place = 1;
    int negative = 0;
    for (int d = ks->D - 1; d >= 0; d--) {
        uint32_t coord = (uint32_t)(cell % ks->radix[d]);
        cell /= ks->radix[d];
        if (ks->neg_dim && d == 0) {
            negative = coord == 0;
        } else {
            mag += (uint64_t)coord * place;
            place *= 10u;
        }
    }
    if (negative) {
        /* undo the digit complement: mag holds (10^D - 1) - |v| */
        mag = (POW10[ks->mag_digits] - 1u) - mag;
        ((int64_t*)out)[j] = -(int64_t)mag;
    } else {
        ((int64_t*)out)[j] = (int64_t)mag;
    }
}

static int finish(const keyspace* ks, size_t n, uint64_t cell_cap, void* keys_out,
                  size_t key_bytes, uint64_t* perm_out, oracle_stats* st, emit_fn emit) {
    uint64_t* items = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (!items) return ORACLE_ERR_NOMEM;
    int rc = run_sort(ks, n, cell_cap, items, st);
    if (rc == ORACLE_OK && perm_out) memcpy(perm_out, items, n * sizeof(uint64_t));
    if (rc == ORACLE_OK && keys_out) {
        int g = 0;
        if (n) top_cells(ks, cell_cap, &g);
        if (n && g == ks->D && emit) {
            rc = regenerate_keys(ks, n, emit, keys_out);
            st->regenerated = 1;
        } else {
            const uint8_t* src = (const uint8_t*)ks->keys;
            uint8_t* dst = (uint8_t*)keys_out;
            for (uint64_t j = 0; j < n; j++)
                memcpy(dst + j * key_bytes, src + items[j] * key_bytes, key_bytes);
        }
    }
    free(items);
    return rc;
}

static uint64_t effective_cap(uint64_t cell_cap) {
    return cell_cap ? cell_cap : ORACLE_DEFAULT_CELL_CAP;
}

int oracle_sort_u32(const uint32_t* keys, size_t n, uint64_t cell_cap, uint32_t* keys_out,
                    uint64_t* perm_out, oracle_stats* st_out) {
    if (n && !keys) return ORACLE_ERR_INVALID;
    keyspace ks_storage;
    keyspace* ks = &ks_storage;
    memset(ks, 0, sizeof(*ks));
    ks->kind = KIND_U32;
    ks->keys = keys;
    uint32_t mx = 0;
    for (size_t i = 0; i < n; i++) mx = keys[i] > mx ? keys[i] : mx;
    ks->D = decimal_digits(mx); /* §3.1.2: pad every key to the longest one's digits */
    for (int d = 0; d < ks->D; d++) ks->radix[d] = 10;
    oracle_stats st;
    cell_cap = effective_cap(cell_cap);
    stats_init(&st, ks, cell_cap);
    int rc = finish(ks, n, cell_cap, keys_out, sizeof(uint32_t), perm_out, &st, emit_u32);
    if (st_out) *st_out = st;
    return rc;
}

int oracle_sort_u64(const uint64_t* keys, size_t n, uint64_t cell_cap, uint64_t* keys_out,
                    uint64_t* perm_out, oracle_stats* st_out) {
    if (n && !keys) return ORACLE_ERR_INVALID;
    keyspace ks_storage;
    keyspace* ks = &ks_storage;
    memset(ks, 0, sizeof(*ks));
    ks->kind = KIND_U64;
    ks->keys = keys;
    uint64_t mx = 0;
    for (size_t i = 0; i < n; i++) mx = keys[i] > mx ? keys[i] : mx;
    ks->D = decimal_digits(mx);
    for (int d = 0; d < ks->D; d++) ks->radix[d] = 10;
    oracle_stats st;
    cell_cap = effective_cap(cell_cap);
    stats_init(&st, ks, cell_cap);
    int rc = finish(ks, n, cell_cap, keys_out, sizeof(uint64_t), perm_out, &st, emit_u64);
    if (st_out) *st_out = st;
    return rc;
}

static int decimal_space(keyspace* ks, const int64_t* keys, size_t n, int int_digits,
                         int frac_digits) {
    if (int_digits < 0 || frac_digits < 0 || int_digits + frac_digits < 1 ||
        int_digits + frac_digits > 18)
        return ORACLE_ERR_INVALID;
    if (n && !keys) return ORACLE_ERR_INVALID;
    memset(ks, 0, sizeof(*ks));
    ks->kind = KIND_DEC;
    ks->keys = keys;
    ks->mag_digits = int_digits + frac_digits;
    int any_negative = 0;
    for (size_t i = 0; i < n; i++) {
        if (magnitude(keys[i]) >= POW10[ks->mag_digits]) return ORACLE_ERR_RANGE;
        any_negative |= keys[i] < 0;
    }
    ks->neg_dim = any_negative;
    ks->D = ks->mag_digits + ks->neg_dim;
    for (int d = 0; d < ks->D; d++) ks->radix[d] = 10;
    if (ks->neg_dim) ks->radix[0] = 2;
    return ORACLE_OK;
}

int oracle_sort_fixed_decimal(const int64_t* keys, size_t n, int int_digits, int frac_digits,
                              uint64_t cell_cap, int64_t* keys_out, uint64_t* perm_out,
                              oracle_stats* st_out) {
    keyspace ks_storage;
    keyspace* ks = &ks_storage;
    int rc = decimal_space(ks, keys, n, int_digits, frac_digits);
    if (rc != ORACLE_OK) return rc;
    oracle_stats st;
    cell_cap = effective_cap(cell_cap);
    stats_init(&st, ks, cell_cap);
    rc = finish(ks, n, cell_cap, keys_out, sizeof(int64_t), perm_out, &st, emit_dec);
    if (st_out) *st_out = st;
    return rc;
}

int oracle_sort_strings(const uint8_t* chars, const uint64_t* offsets, size_t n,
                        uint32_t max_len, uint64_t cell_cap, uint64_t* perm_out,
                        oracle_stats* st_out) {
    if (n && (!offsets || (!chars && offsets[n] > offsets[0]))) return ORACLE_ERR_INVALID;
    keyspace ks_storage;
    keyspace* ks = &ks_storage;
    memset(ks, 0, sizeof(*ks));
    ks->kind = KIND_STR;
    ks->chars = chars;
    ks->offsets = offsets;
    uint64_t longest = 0;
    for (size_t i = 0; i < n; i++) {
        if (offsets[i + 1] < offsets[i]) return ORACLE_ERR_INVALID;
        uint64_t len = offsets[i + 1] - offsets[i];
        longest = len > longest ? len : longest;
    }
    if (max_len == 0) max_len = (uint32_t)(longest ? longest : 1);
    if (longest > max_len) return ORACLE_ERR_RANGE;
    if (max_len > MAX_DIMS) return ORACLE_ERR_INVALID;
    ks->D = (int)max_len;
    for (int d = 0; d < ks->D; d++) ks->radix[d] = 257;
    oracle_stats st;
    cell_cap = effective_cap(cell_cap);
    stats_init(&st, ks, cell_cap);
    int rc = finish(ks, n, cell_cap, NULL, 0, perm_out, &st, NULL);
    if (st_out) *st_out = st;
    return rc;
}

int oracle_sort_f64(const double* keys, size_t n, uint64_t cell_cap, double* keys_out,
                    uint64_t* perm_out, oracle_stats* st_out) {
    if (n && !keys) return ORACLE_ERR_INVALID;
    keyspace ks_storage;
    keyspace* ks = &ks_storage;
    memset(ks, 0, sizeof(*ks));
    ks->kind = KIND_F64;
    ks->keys = keys;
    ks->D = 20; /* class + 19 magnitude digits */
    ks->radix[0] = 4;
    for (int d = 1; d < ks->D; d++) ks->radix[d] = 10;
    oracle_stats st;
    cell_cap = effective_cap(cell_cap);
    stats_init(&st, ks, cell_cap);
    int rc = finish(ks, n, cell_cap, keys_out, sizeof(double), perm_out, &st, NULL);
    if (st_out) *st_out = st;
    return rc;
}

int oracle_decimal_hashing_cycle(const int64_t* keys, size_t n, int int_digits, int frac_digits,
                                 uint32_t* radix_out, int* rank_out, uint64_t* S_out,
                                 uint32_t* hmax_out, uint32_t* hmin_out, uint64_t* k_out) {
    keyspace ks_storage;
    keyspace* ks = &ks_storage;
    int rc = decimal_space(ks, keys, n, int_digits, frac_digits);
    if (rc != ORACLE_OK) return rc;
    if (ks->D > 32) return ORACLE_ERR_INVALID;
    uint64_t cells = 1;
    for (int d = 0; d < ks->D; d++) {
        cells *= ks->radix[d];
        if (radix_out) radix_out[d] = ks->radix[d];
    }
    if (rank_out) *rank_out = ks->D;
    if (!S_out && !hmax_out && !hmin_out && !k_out) return ORACLE_OK;
    if (cells > (1ull << 24)) return ORACLE_ERR_INVALID; /* one count array must stay small */

    /* The sort's own hashing and extraction cycles with every dimension in
     * one count array (g = D), over the keys in input order. */
    count_array ca;
    uint64_t* items = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* cell_of = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    if (count_array_init(&ca, ks, 0, cells) != ORACLE_OK || !items || !cell_of) {
        count_array_free(&ca);
        free(items);
        free(cell_of);
        return ORACLE_ERR_NOMEM;
    }
    for (uint64_t i = 0; i < n; i++) items[i] = i;
    hashing_cycle(ks, &ca, items, n, cell_of);
    uint64_t k = extraction_cycle(&ca, n);
    free(items);
    free(cell_of);
    const uint64_t rows = ca.rows;
    uint64_t *S = ca.S, *H_Max = ca.H_Max, *H_Min = ca.H_Min;
    if (S_out) memcpy(S_out, S, cells * sizeof(uint64_t));
    for (uint64_t r = 0; r < rows; r++) {
        if (hmax_out) hmax_out[r] = (uint32_t)H_Max[r];
        if (hmin_out) {
            hmin_out[2 * r] = (uint32_t)H_Min[2 * r];
            hmin_out[2 * r + 1] = (uint32_t)H_Min[2 * r + 1];
        }
    }
    if (k_out) *k_out = k;
    count_array_free(&ca);
    return ORACLE_OK;
}
