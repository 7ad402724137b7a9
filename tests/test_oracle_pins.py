"""Pins for the CPU oracle: checks against what the paper and mathematics fix.

The oracle (``oracle/rs_oracle.c``) is only trusted because these tests tie it
to facts that do not come from the oracle itself:

* the worked example of the paper (golden file ``example1.txt``): sorted
  output, the cells the hashing cycle increments, the row-4 traverse maps, the
  steps that skip map updates, and the extraction cost k = 17;
* Table 3's count-array and traverse-map shapes (``table3_shapes.txt``);
* brute force over every input of a few elements over tiny alphabets,
  against Python's stable ``sorted`` with the input index as tie-breaker;
* numpy's stable argsort and Python's ``bytes`` ordering on random inputs;
* the invariants of §4 (count conservation; sorted, permuted output) and
  stability.
"""
import itertools

import numpy as np
import pytest

from conftest import read_golden

# ------------------------------------------------------------------ example 1


def _example():
    g = read_golden("example1.txt")
    lam = int(g["count_after_decimal"][0])
    scaled = np.array([int(x) for x in g["scaled"]], np.int64)
    return g, lam, scaled


def test_example1_prescaling_matches_input():
    # Steps 1a-10a multiply each element by 10^λ; the golden "scaled" row must
    # be the "input" row under that rule (decimal strings, no float rounding).
    g, lam, scaled = _example()
    for text, s in zip(g["input"], scaled):
        whole, _, frac = text.partition(".")
        frac = (frac + "0" * lam)[:lam]
        assert int(whole + frac) == s


def test_example1_sorted_output(oracle):
    g, lam, scaled = _example()
    out, perm, st = oracle.sort_fixed_decimal(scaled, int_digits=1, frac_digits=lam)
    expected = [int(t.replace(".", "")) for t in g["sorted"]]
    assert out.tolist() == expected
    # keys-only output of a single count array is rebuilt from cells (Eq. 16)
    assert st.regenerated
    assert st.top_cells == 100 and st.dims == 2
    assert st.k == int(g["k"][0]) and st.cycles == 1   # extraction cost of the sort itself
    # equal keys 4.5 (input positions 0 and 6) keep their input order
    assert perm.tolist().index(0) < perm.tolist().index(6)


def test_example1_cells_and_extraction_cost(oracle):
    g, lam, scaled = _example()
    S, hmax, hmin, k = oracle.decimal_hashing_cycle(scaled, 1, lam)
    assert S.shape == (10, 10)
    expected = np.zeros((10, 10), np.int64)
    for cell in g["cells"]:
        r, c = (int(v) for v in cell.split(","))
        expected[r, c] += 1
    assert (S.astype(np.int64) == expected).all()
    assert int(S.sum()) == len(scaled)  # I_Hash at termination (§4.1)
    lo, hi = (int(v) for v in g["row4_hmin_hmax"])
    assert hmin[4].tolist() == [1, lo] and hmax[4] == hi
    assert k == int(g["k"][0])


def test_example1_traverse_map_steps(oracle):
    # Replays the hashing cycle one element at a time: steps the example marks
    # "skipped" leave the map unchanged; the others leave the map at the
    # element's column (H_Max) or at [1, column] (H_Min).
    g, lam, scaled = _example()
    hmax_skip = {int(v) - 1 for v in g["hmax_skipped"]}
    hmin_skip = {int(v) - 1 for v in g["hmin_skipped"]}
    prev_max, prev_min = None, None
    for i in range(len(scaled)):
        _, hmax, hmin, _ = oracle.decimal_hashing_cycle(scaled[: i + 1], 1, lam)
        r, c = divmod(int(scaled[i]), 10)
        if i in hmax_skip:
            assert hmax[r] == prev_max[r]
        else:
            assert hmax[r] == c
        if i in hmin_skip:
            assert hmin[r].tolist() == prev_min[r].tolist()
        else:
            assert hmin[r].tolist() == [1, c]
        prev_max, prev_min = hmax.copy(), hmin.copy()


def test_traverse_maps_definition(oracle):
    # §3.2: each row of H_Min holds the smallest occupied column and a flag,
    # each row of H_Max the largest occupied column.
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1000, 300).astype(np.int64)
    S, hmax, hmin, _ = oracle.decimal_hashing_cycle(keys, 2, 1)
    S2 = S.reshape(-1, S.shape[-1])
    for row in range(S2.shape[0]):
        cols = np.nonzero(S2[row])[0]
        if cols.size == 0:
            assert hmin[row, 0] == 0
        else:
            assert hmin[row].tolist() == [1, cols.min()] and hmax[row] == cols.max()


def test_extraction_cost_by_hand(oracle):
    # k counts the cells walked from H_Min to H_Max of every touched row.
    keys = np.array([5, 95, 91, 99], np.int64)  # rows 0 (col 5) and 9 (cols 1..9)
    _, _, _, k = oracle.decimal_hashing_cycle(keys, 2, 0)
    assert k == 1 + 9
    # the walk stops once every key is out: row 9 ends at its last key
    keys = np.array([90, 91], np.int64)
    assert oracle.decimal_hashing_cycle(keys, 2, 0)[3] == 2


# ------------------------------------------------------------------ table 3


def _table3_rows():
    rows = []
    with open(__import__("os").path.join(__import__("conftest").GOLDEN, "table3_shapes.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rng_part, s, hmin, hmax = (p.strip() for p in line.split("|"))
                lo, hi, cd = (int(v) for v in rng_part.split())
                rows.append((lo, hi, cd, s, hmin, hmax))
    return rows


@pytest.mark.parametrize("row", _table3_rows(), ids=lambda r: f"D({r[0]},{r[1]})cd{r[2]}")
def test_table3_shapes(oracle, row):
    lo, hi, cd, s_printed, hmin_printed, hmax_printed = row
    rng = np.random.default_rng(3)
    # numpy-style half-open range [lo, hi) with cd digits after the point,
    # stored scaled by 10^cd (the §3.1 pre-scaling)
    scaled = rng.integers(lo * 10**cd, hi * 10**cd, 500).astype(np.int64)
    int_digits = len(str(hi - 1))
    shape = oracle.decimal_space_shape(scaled, int_digits, cd)
    assert "x".join(str(d) for d in shape) == s_printed
    S, hmax, hmin, _ = oracle.decimal_hashing_cycle(scaled, int_digits, cd)
    rows = S.size // shape[-1]
    assert hmax.size == rows and hmin.shape == (rows, 2)
    # printed map shapes: a leading "10x" per dimension beyond the first;
    # the trailing factor is 2 for H_Min and 1 for H_Max (the garbled
    # three-dimensional entries "10x22"/"10x11" read as 10x10x2 / 10x10x1)
    def entries(printed, last):
        parts = printed.split("x")
        if len(parts) == 2 and len(parts[1]) == 2 and parts[1] == str(last) * 2:
            return 10 * 10 * last
        return int(np.prod([int(p) for p in parts]))
    assert entries(hmin_printed, 2) == 2 * rows
    assert entries(hmax_printed, 1) == rows


# ------------------------------------------------------------------ brute force


def _stable_reference(keys):
    return [i for _, i in sorted((k, i) for i, k in enumerate(keys))]


@pytest.mark.parametrize("n", range(0, 7))
def test_bruteforce_u32(oracle, n):
    for combo in itertools.product([0, 7, 10], repeat=n):
        keys = np.array(combo, np.uint32)
        out, perm, _ = oracle.sort_u32(keys)
        ref = _stable_reference(combo)
        assert perm.tolist() == ref
        assert out.tolist() == [combo[i] for i in ref]


@pytest.mark.parametrize("n", range(0, 5))
def test_bruteforce_fixed_decimal_signed(oracle, n):
    alphabet = [-11, -10, -1, 0, 1, 10]
    for combo in itertools.product(alphabet, repeat=n):
        keys = np.array(combo, np.int64)
        out, perm, _ = oracle.sort_fixed_decimal(keys, int_digits=1, frac_digits=1)
        ref = _stable_reference(combo)
        assert perm.tolist() == ref
        assert out.tolist() == [combo[i] for i in ref]


@pytest.mark.parametrize("n", range(0, 5))
def test_bruteforce_strings(oracle, n):
    alphabet = [b"", b"a", b"b", b"ab", b"a\x00", b"\xff", b"ba"]
    for combo in itertools.product(alphabet, repeat=n):
        chars = np.frombuffer(b"".join(combo), np.uint8)
        offsets = np.concatenate([[0], np.cumsum([len(s) for s in combo])]).astype(np.uint64)
        perm, _ = oracle.sort_strings(chars, offsets)
        assert perm.tolist() == _stable_reference(combo)


# ------------------------------------------------------------------ library routines


@pytest.mark.parametrize("seed,hi,n", [(1, 2**32, 5000), (2, 1000, 5000), (3, 17, 3000),
                                       (4, 2**32, 1), (5, 10**9, 4000)])
def test_u32_vs_numpy_stable(oracle, seed, hi, n):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, hi, n, dtype=np.uint64).astype(np.uint32)
    out, perm, _ = oracle.sort_u32(keys)
    ref = np.argsort(keys, kind="stable")
    assert (perm.astype(np.int64) == ref).all()
    assert (out == keys[ref]).all()


def test_u32_extremes(oracle):
    keys = np.array([0xFFFFFFFF, 0, 4294967294, 1, 0xFFFFFFFF, 0], np.uint32)
    out, perm, _ = oracle.sort_u32(keys)
    assert out.tolist() == sorted(keys.tolist())
    assert perm.tolist() == [1, 5, 3, 2, 0, 4]


@pytest.mark.parametrize("seed", [1, 2])
def test_u64_vs_numpy_stable(oracle, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2**64 - 1, 4000, dtype=np.uint64, endpoint=True)
    keys[:10] = [0, 2**64 - 1, 2**64 - 1, 10**19, 10**19 - 1, 1, 0, 5, 5, 2**63]
    out, perm, _ = oracle.sort_u64(keys)
    ref = np.argsort(keys, kind="stable")
    assert (perm.astype(np.int64) == ref).all()
    assert (out == keys[ref]).all()


@pytest.mark.parametrize("hi", [1, 10, 1000])
def test_u64_small_keys_regenerated(oracle, hi):
    """u64 keys whose digit vectors fit one count array are rebuilt from their
    cells (Eq. 16) rather than copied: the rebuilt keys must equal numpy's
    stable sort of the input, and the stats must say they were rebuilt."""
    rng = np.random.default_rng(hi)
    keys = rng.integers(0, hi, 3000, dtype=np.uint64)
    keys[:3] = [0, hi - 1, 0]
    out, perm, st = oracle.sort_u64(keys)
    ref = np.argsort(keys, kind="stable")
    assert st.regenerated
    assert out.dtype == np.uint64
    assert (perm.astype(np.int64) == ref).all()
    assert (out == keys[ref]).all()


def test_u32_small_keys_regenerated(oracle):
    """The same for u32 keys of at most three digits (the 10x10x10 space)."""
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1000, 3000, dtype=np.uint64).astype(np.uint32)
    out, perm, st = oracle.sort_u32(keys)
    assert st.regenerated
    assert (out == np.sort(keys, kind="stable")).all()


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fixed_decimal_vs_numpy_stable(oracle, seed):
    rng = np.random.default_rng(seed)
    mag = rng.integers(0, 10**9, 6000)
    sign = np.where(rng.random(6000) < 0.5, -1, 1)
    keys = (sign * mag).astype(np.int64)
    keys[:6] = [0, -999999999, 999999999, -1, 1, 0]
    out, perm, _ = oracle.sort_fixed_decimal(keys, int_digits=6, frac_digits=3)
    ref = np.argsort(keys, kind="stable")
    assert (perm.astype(np.int64) == ref).all()
    assert (out == keys[ref]).all()


def test_fixed_decimal_regenerates_negatives(oracle):
    # sign dimension + 2 digits = 200 cells: one count array, keys rebuilt
    # from the cell coordinates (Eq. 16), negatives included
    rng = np.random.default_rng(9)
    keys = rng.integers(-99, 100, 2000).astype(np.int64)
    out, _, st = oracle.sort_fixed_decimal(keys, int_digits=2, frac_digits=0)
    assert st.regenerated and st.top_cells == 200
    assert (out == np.sort(keys)).all()


def test_fixed_decimal_range_error(oracle):
    with pytest.raises(oracle.OracleError) as e:
        oracle.sort_fixed_decimal(np.array([1, 1000], np.int64), int_digits=2, frac_digits=1)
    assert e.value.code == oracle.ERR_RANGE
    with pytest.raises(oracle.OracleError):
        oracle.sort_fixed_decimal(np.array([-1000], np.int64), int_digits=3, frac_digits=0)


@pytest.mark.parametrize("seed", [1, 2])
def test_strings_vs_python_bytes_order(oracle, seed):
    rng = np.random.default_rng(seed)
    strs = []
    for _ in range(3000):
        ln = int(rng.integers(0, 9))
        alpha = rng.choice([2, 3, 256])
        strs.append(bytes(rng.integers(0, alpha, ln).astype(np.uint8)))
    chars = np.frombuffer(b"".join(strs), np.uint8)
    offsets = np.concatenate([[0], np.cumsum([len(s) for s in strs])]).astype(np.uint64)
    perm, _ = oracle.sort_strings(chars, offsets)
    assert perm.tolist() == _stable_reference(strs)


def test_strings_range_error(oracle):
    chars = np.frombuffer(b"abcdef", np.uint8)
    offsets = np.array([0, 2, 6], np.uint64)
    with pytest.raises(oracle.OracleError) as e:
        oracle.sort_strings(chars, offsets, max_len=3)
    assert e.value.code == oracle.ERR_RANGE


# ------------------------------------------------------------------ invariants


@pytest.mark.parametrize("cap", [10, 100, 1000, 10**6])
def test_output_invariant_under_cell_cap(oracle, cap):
    # The count-array size only decides how many dimensions become buckets;
    # the sorted result never changes (buckets, §2.2).
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 2**32, 3000, dtype=np.uint64).astype(np.uint32)
    keys[::7] = keys[3]
    out, perm, _ = oracle.sort_u32(keys, cell_cap=cap)
    ref = np.argsort(keys, kind="stable")
    assert (perm.astype(np.int64) == ref).all() and (out == keys[ref]).all()


def test_invariants_random(oracle):
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 50, 20000, dtype=np.uint32)
    vals = np.arange(keys.size, dtype=np.uint32)
    out, sorted_vals, _ = oracle.sort_pairs(keys, vals)
    assert (np.diff(out.astype(np.int64)) >= 0).all()                 # non-decreasing
    assert np.array_equal(np.sort(sorted_vals), vals)                  # permutation
    assert (keys[sorted_vals] == out).all()                            # keys follow payloads
    same = out[1:] == out[:-1]
    assert (sorted_vals[1:][same] > sorted_vals[:-1][same]).all()     # stability


def test_single_count_array_cost_bounds(oracle):
    # For one count array, k is at least the number of occupied cells and at
    # most the number of cells (§5).
    rng = np.random.default_rng(8)
    keys = rng.integers(0, 1000, 700).astype(np.uint32)
    _, _, st = oracle.sort_u32(keys)
    assert st.cycles == 1
    assert np.unique(keys).size <= st.k <= 1000


def test_stable_rank_definition(oracle):
    rng = np.random.default_rng(4)
    keys = rng.integers(0, 20, 500, dtype=np.uint32)
    ref = np.argsort(keys, kind="stable")
    pos = np.empty_like(ref)
    pos[ref] = np.arange(ref.size)
    for i in range(0, 500, 37):
        assert oracle.stable_rank(keys, i) == pos[i]


# ------------------------------------------------------------------ floats


def _float_reference(xs):
    # NaN last, -0.0 == +0.0, ties in input order
    return [i for _, _, i in sorted((bool(np.isnan(x)), 0.0 if np.isnan(x) else float(x), i)
                                    for i, x in enumerate(xs))]


@pytest.mark.parametrize("n", range(0, 5))
def test_bruteforce_float(oracle, n):
    alphabet = [-np.inf, -1.5, -0.0, 0.0, 5e-324, 2.0, np.inf, np.nan]
    for combo in itertools.product(alphabet, repeat=n):
        perm = oracle.sort_float(np.array(combo, np.float64))[1]
        assert perm.tolist() == _float_reference(combo)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_float_vs_numpy_stable(oracle, dtype):
    rng = np.random.default_rng(12)
    x = (rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000)).astype(dtype)
    x[::11] = np.round(x[::11])
    x[:8] = [0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 1e-45, -1e-45]
    out, perm, _ = oracle.sort_float(x)
    ref = np.argsort(x, kind="stable")
    assert (perm.astype(np.int64) == ref).all()
    assert np.array_equal(out.view(np.uint8), x[ref].view(np.uint8))
