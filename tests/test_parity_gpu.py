"""Parity of the CUDA path against the CPU oracle, element by element.

Sizes span several tiles (see TILE_KEYS: 256 threads times the keys per
thread of each key/value shape) with ragged tails; every comparison is bit-exact (keys, and payload order for
pairs).  All calls go through the C ABI via the thin binding.
"""
import numpy as np
import pytest
import torch

from gpu_util import from_dev, require_gpu, to_dev
from paper_2107_01391_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# keys per pass tile (256 threads x keys per thread) for each (key, value) shape;
# test_tile_boundaries checks these against the tile count the library reports
TILE_KEYS = {("u32", None): 48 * 256, ("u32", "u32"): 40 * 256, ("u32", "u64"): 28 * 256,
             ("u64", None): 40 * 256, ("u64", "u32"): 28 * 256, ("u64", "u64"): 24 * 256}
_T32 = TILE_KEYS[("u32", None)]
SIZES_U32 = [1, 2, 3, 31, 4095, 4097, _T32 - 1, _T32, _T32 + 1, 3 * _T32 + 17, 100_003]


@pytest.fixture(scope="module")
def rs():
    require_gpu()
    from paper_2107_01391_gb300 import build, binding
    build.build()
    return binding


@pytest.fixture(scope="module")
def ctx(rs):
    c = rs.Context(0)
    yield c
    c.close()


def _sort_u32(rs, ctx, keys, inplace=False):
    d = to_dev(keys)
    out = rs.rs_sort_u32(d, d if inplace else None, ctx=ctx)
    ctx.check()
    return from_dev(out, np.uint32)


# --------------------------------------------------------------- keys only


def test_digits3_fill_path_full_size(rs, ctx, oracle):
    keys = W.digits3(1 << 20)
    ref, _, st = oracle.sort_u32(keys)
    assert st.regenerated  # the oracle also rebuilt keys from cells (Eq. 16)
    got = _sort_u32(rs, ctx, keys)
    assert np.array_equal(got, ref)
    assert ctx.last_plan()["mode"] == "fill"


@pytest.mark.parametrize("n", SIZES_U32)
def test_digits3_small(rs, ctx, oracle, n):
    keys = W.digits3(n, seed_extra=n)
    ref, _, _ = oracle.sort_u32(keys)
    assert np.array_equal(_sort_u32(rs, ctx, keys), ref)


@pytest.mark.parametrize("n", SIZES_U32)
def test_u32_uniform_keys(rs, ctx, oracle, n):
    keys = W.u32_keys(n, "uniform", seed_extra=n)
    ref, _, _ = oracle.sort_u32(keys)
    assert np.array_equal(_sort_u32(rs, ctx, keys), ref)
    assert ctx.last_plan()["mode"] == "passes" or n < 3


@pytest.mark.parametrize("dist", ["zipf", "presorted", "reversed"])
def test_u32_skewed_keys(rs, ctx, oracle, dist):
    if dist == "reversed":  # descending, with runs of ties
        keys = np.sort(W.u32_keys(200_001, "uniform") >> 12)[::-1].copy()
    else:
        keys = W.u32_keys(200_001, dist)
    ref, _, _ = oracle.sort_u32(keys)
    assert np.array_equal(_sort_u32(rs, ctx, keys), ref)


@pytest.mark.parametrize("inplace", [False, True])
@pytest.mark.parametrize("shape", ["one_group", "two_groups", "all_equal", "small_range_big"])
def test_u32_trivial_groups_and_in_place(rs, ctx, oracle, inplace, shape):
    rng = np.random.default_rng(17)
    n = 50_000
    if shape == "one_group":      # only bits 8..15 vary: a single active pass
        keys = (rng.integers(0, 256, n) << 8).astype(np.uint32)
    elif shape == "two_groups":   # bits 0..7 and 24..31 vary
        keys = (rng.integers(0, 256, n) | (rng.integers(0, 256, n) << 24)).astype(np.uint32)
    elif shape == "all_equal":
        keys = np.full(n, 0xDEADBEEF, np.uint32)
    else:                         # every key >= RS_FILL_CELLS but in a narrow range
        keys = rng.integers(5000, 5100, n).astype(np.uint32)
    ref, _, _ = oracle.sort_u32(keys)
    assert np.array_equal(_sort_u32(rs, ctx, keys, inplace=inplace), ref)


def test_u32_extremes(rs, ctx, oracle):
    keys = np.array([0xFFFFFFFF, 0, 1, 0xFFFFFFFE, 0xFFFFFFFF, 0, 0x80000000] * 1000, np.uint32)
    ref, _, _ = oracle.sort_u32(keys)
    assert np.array_equal(_sort_u32(rs, ctx, keys), ref)


def test_empty(rs, ctx):
    d = torch.empty(0, dtype=torch.int32, device="cuda")
    out = rs.rs_sort_u32(d, ctx=ctx)
    ctx.check()
    assert out.numel() == 0


@pytest.mark.parametrize("n", [1, 3071, 3072, 3073, 10_239, 10_241, 70_001])
def test_u64_keys(rs, ctx, oracle, n):
    keys = W.u64_keys(n, seed_extra=n)
    ref, _, _ = oracle.sort_u64(keys)
    d = to_dev(keys)
    out = rs.rs_sort_u64(d, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(out, np.uint64), ref)


@pytest.fixture
def wide_tiles(ctx):
    """Every multi-tile sort on the wide pass tile (no narrow selection)."""
    old = ctx.pass_tile_limit
    ctx.pass_tile_limit = 0
    yield
    ctx.pass_tile_limit = old


@pytest.fixture
def narrow_tiles(ctx):
    """Every multi-tile sort with a 4-byte cell on the narrow pass tile."""
    old = ctx.pass_tile_limit
    ctx.pass_tile_limit = 1 << 62
    yield
    ctx.pass_tile_limit = old


@pytest.mark.parametrize("where", ["minus1", "exact", "plus1", "ragged3"])
@pytest.mark.parametrize("shape", list(TILE_KEYS), ids=lambda s: f"{s[0]}-{s[1]}")
def test_tile_boundaries(rs, ctx, oracle, wide_tiles, shape, where):
    kt, vt = shape
    T = TILE_KEYS[shape]
    n = {"minus1": T - 1, "exact": T, "plus1": T + 1, "ragged3": 3 * T + 17}[where]
    kdt = np.uint32 if kt == "u32" else np.uint64
    keys = (W.u32_keys(n, seed_extra=n) if kt == "u32" else W.u64_keys(n, seed_extra=n))
    keys[1::5] = keys[0::5][: keys[1::5].size]  # ties, so that stability is checked
    if vt is None:
        ref, _, _ = oracle.sort_u32(keys) if kt == "u32" else oracle.sort_u64(keys)
        out = (rs.rs_sort_u32 if kt == "u32" else rs.rs_sort_u64)(to_dev(keys), ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(out, kdt), ref)
    else:
        vdt = np.uint32 if vt == "u32" else np.uint64
        vals = (np.arange(n, dtype=vdt) * vdt(2654435761)) ^ vdt(0x5A5A5A5A)
        ref_k, ref_v, _ = oracle.sort_pairs(keys, vals)
        ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(ko, kdt), ref_k)
        assert np.array_equal(from_dev(vo, vdt), ref_v)
    assert ctx.last_plan()["tiles"] == -(-n // T)


NARROW_TILE = 16 * 256


@pytest.mark.parametrize("n", [4097, 2 * NARROW_TILE - 1, 2 * NARROW_TILE, 2 * NARROW_TILE + 1,
                               5 * NARROW_TILE + 17, 1 << 19, (1 << 19) + 3])
@pytest.mark.parametrize("kind", ["u32_keys", "u32_pairs", "f32_keys", "f32_pairs", "dec_keys",
                                  "dec_pairs"])
def test_narrow_tile_boundaries(rs, ctx, oracle, narrow_tiles, kind, n):
    """The narrow pass tile (16 keys per thread) at its tile boundaries, for
    every shape that has one, against the oracle."""
    rng = np.random.default_rng(n + 7 * len(kind))
    if kind.startswith("u32"):
        keys = W.u32_keys(n, seed_extra=n)
        keys[1::5] = keys[0::5][: keys[1::5].size]  # ties
        ref_k, perm, _ = oracle.sort_u32(keys)
        kdt = np.uint32
    elif kind.startswith("f32"):
        keys = np.round(rng.standard_normal(n) * 100).astype(np.float32)
        _, perm, _ = oracle.sort_float(keys)
        ref_k = keys[perm.astype(np.int64)]
        ref_k[ref_k == 0] = 0.0
        kdt = np.float32
    else:
        keys = W.decimals(n, 6, 3, seed_extra=n)
        ref_k, perm, _ = oracle.sort_fixed_decimal(keys, 6, 3)
        kdt = np.int64
    if kind.endswith("keys"):
        if kind == "u32_keys":
            out = rs.rs_sort_u32(to_dev(keys), ctx=ctx)
        elif kind == "f32_keys":
            out, _ = rs.rs_sort_pairs(to_dev(keys), None, ctx=ctx)
        else:
            out = rs.rs_sort_fixed_decimal(to_dev(keys), 6, 3, ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(out, kdt).view(np.uint8), ref_k.view(np.uint8))
    else:
        vals = np.arange(n, dtype=np.uint32)
        ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals),
                                  decimal=(6, 3) if kind == "dec_pairs" else None, ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(ko, kdt).view(np.uint8), ref_k.view(np.uint8))
        assert np.array_equal(from_dev(vo, np.uint32), perm.astype(np.uint32))
    assert ctx.last_plan()["tiles"] == -(-n // NARROW_TILE)


def test_default_tile_selection(rs, ctx, oracle):
    """With the default limit (2^19) a sort of 2^19 keys takes the narrow tile
    and one of 2^19 + 1 the wide one; both agree with the oracle."""
    assert ctx.pass_tile_limit == 1 << 19
    for n, tile in ((1 << 19, NARROW_TILE), ((1 << 19) + 1, TILE_KEYS[("u32", "u32")])):
        keys, vals = W.u32_pairs(n, "zipf", seed_extra=n)
        ref_k, perm, _ = oracle.sort_u32(keys)
        ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(ko, np.uint32), ref_k)
        assert np.array_equal(from_dev(vo, np.uint32), perm.astype(np.uint32))
        assert ctx.last_plan()["tiles"] == -(-n // tile)


@pytest.mark.parametrize("n", [1, 2, 33, 257, 1000, 1025, 3073, 4095, 4096])
@pytest.mark.parametrize("kind", ["u32_pairs", "u64_pairs", "u32_u64v_in_place", "dec_keys",
                                  "narrow_keys"])
def test_single_tile_sorts(rs, ctx, oracle, kind, n):
    # at most 4096 keys: one CTA sorts the whole input on chip in one launch
    rng = np.random.default_rng(n + len(kind))
    if kind == "u32_pairs":
        keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
        keys[::3] = keys[0]  # ties
        vals = np.arange(n, dtype=np.uint32)
        rk, rv, _ = oracle.sort_pairs(keys, vals)
        ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(ko, np.uint32), rk)
        assert np.array_equal(from_dev(vo, np.uint32), rv)
    elif kind == "u64_pairs":
        keys = W.u64_keys(n, seed_extra=n)
        keys[1::4] = keys[0]
        vals = np.arange(n, dtype=np.uint32) * np.uint32(7)
        rk, rv, _ = oracle.sort_pairs(keys, vals)
        ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(ko, np.uint64), rk)
        assert np.array_equal(from_dev(vo, np.uint32), rv)
    elif kind == "u32_u64v_in_place":
        keys = rng.integers(0, 50, n, dtype=np.uint32)
        vals = np.arange(n, dtype=np.uint64) << np.uint64(33)
        rk, rv, _ = oracle.sort_pairs(keys, vals)
        dk, dv = to_dev(keys), to_dev(vals)
        rs.rs_sort_pairs(dk, dv, dk, dv, ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(dk, np.uint32), rk)
        assert np.array_equal(from_dev(dv, np.uint64), rv)
    elif kind == "dec_keys":
        keys = W.decimals(n, 9, 9, seed_extra=n)  # 64-bit cells, 8 digit groups
        ref, _, _ = oracle.sort_fixed_decimal(keys, 9, 9)
        out = rs.rs_sort_fixed_decimal(to_dev(keys), 9, 9, ctx=ctx)
        ctx.check()
        assert np.array_equal(from_dev(out, np.int64), ref)
    else:  # keys in [0, 1000): the upper digit groups are skipped
        keys = W.digits3(n, seed_extra=n)
        ref, _, _ = oracle.sort_u32(keys)
        assert np.array_equal(_sort_u32(rs, ctx, keys), ref)
        assert ctx.last_plan()["passes_run"] <= 2
    assert ctx.last_plan()["tiles"] == 1


def test_single_tile_boundary(rs, ctx, oracle):
    # 4096 keys take the single-CTA path (one launch), 4097 the device-wide
    # one (count, fill, four digit-group passes)
    for n, launches in ((4096, 1), (4097, 6)):
        keys = W.u32_keys(n, seed_extra=77)
        ref, _, _ = oracle.sort_u32(keys)
        before = ctx.launch_count()
        assert np.array_equal(_sort_u32(rs, ctx, keys), ref)
        assert ctx.launch_count() - before == launches
        assert ctx.last_plan()["mode"] == "passes"


# --------------------------------------------------------------- decimals


@pytest.mark.parametrize("n", [1, 4097, 150_001])
def test_fixed_decimal_6_3(rs, ctx, oracle, n):
    keys = W.decimals(n, 6, 3, seed_extra=n)
    ref, _, _ = oracle.sort_fixed_decimal(keys, 6, 3)
    out = rs.rs_sort_fixed_decimal(to_dev(keys), 6, 3, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(out, np.int64), ref)


@pytest.mark.parametrize("lo,hi,cd", [(1, 10, 0), (1, 10, 1), (1, 10, 2), (1, 100, 0), (1, 100, 1)])
def test_fixed_decimal_table1_cases(rs, ctx, oracle, lo, hi, cd):
    # the paper's five data cases (Table 1) at GPU scale: one count array,
    # output rebuilt from cells
    rng = np.random.default_rng(cd + hi)
    keys = rng.integers(lo * 10**cd, hi * 10**cd, 1 << 18).astype(np.int64)
    int_digits = len(str(hi - 1))
    ref, _, st = oracle.sort_fixed_decimal(keys, int_digits, cd)
    out = rs.rs_sort_fixed_decimal(to_dev(keys), int_digits, cd, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(out, np.int64), ref)
    assert ctx.last_plan()["mode"] == "fill"


def test_fixed_decimal_example1(rs, ctx, oracle):
    keys = np.array([45, 3, 23, 88, 70, 92, 45, 43, 80, 32], np.int64)
    out = rs.rs_sort_fixed_decimal(to_dev(keys), 1, 1, ctx=ctx)
    ctx.check()
    assert from_dev(out, np.int64).tolist() == [3, 23, 32, 43, 45, 45, 70, 80, 88, 92]


def test_fixed_decimal_signed_mixed_and_in_place(rs, ctx, oracle):
    rng = np.random.default_rng(5)
    keys = rng.integers(-(10**12) + 1, 10**12, 60_000).astype(np.int64)
    keys[:4] = [-(10**12) + 1, 10**12 - 1, 0, -1]
    ref, _, _ = oracle.sort_fixed_decimal(keys, 10, 2)
    d = to_dev(keys)
    rs.rs_sort_fixed_decimal(d, 10, 2, out=d, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(d, np.int64), ref)


def test_fixed_decimal_range_error(rs, ctx):
    keys = np.array([1, 2, 10**9, 3] * 100, np.int64)  # 10^9 needs 10 digits
    rs.rs_sort_fixed_decimal(to_dev(keys), 6, 3, ctx=ctx)
    assert ctx.status(True) == rs.RS_ERR_RANGE
    assert ctx.status(True) == rs.RS_OK  # the status word was cleared


# --------------------------------------------------------------- pairs


@pytest.mark.parametrize("dist", ["uniform", "zipf", "presorted"])
@pytest.mark.parametrize("n", [4097, 1_000_003])
def test_u32_pairs(rs, ctx, oracle, dist, n):
    keys, vals = W.u32_pairs(n, dist, seed_extra=n)
    ref_k, ref_perm, _ = oracle.sort_u32(keys)
    ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    assert np.array_equal(from_dev(vo, np.uint32), ref_perm.astype(np.uint32))


@pytest.mark.parametrize("inplace", [False, True])
def test_u32_pairs_u64_values(rs, ctx, oracle, inplace):
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 1000, 77_777).astype(np.uint32)  # many ties; pairs never fill
    vals = rng.integers(0, 2**63, keys.size).astype(np.int64)
    ref_k, perm, _ = oracle.sort_u32(keys)
    dk, dv = to_dev(keys), to_dev(vals)
    if inplace:
        rs.rs_sort_pairs(dk, dv, dk, dv, ctx=ctx)
        ko, vo = dk, dv
    else:
        ko, vo = rs.rs_sort_pairs(dk, dv, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    assert np.array_equal(from_dev(vo, np.int64), vals[perm.astype(np.int64)])


def test_u64_pairs(rs, ctx, oracle):
    keys = W.u64_keys(40_000)
    keys[::3] = keys[5]
    vals = np.arange(keys.size, dtype=np.uint32)
    ref_k, perm, _ = oracle.sort_u64(keys)
    ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint64), ref_k)
    assert np.array_equal(from_dev(vo, np.uint32), perm.astype(np.uint32))


@pytest.mark.parametrize("int_digits,frac_digits", [(4, 2), (1, 0), (9, 9)])
def test_decimal_pairs_in_place(rs, ctx, oracle, int_digits, frac_digits):
    # cells of 21, 5 and 61 bits: odd and even numbers of digit groups
    rng = np.random.default_rng(int_digits)
    lim = 10 ** (int_digits + frac_digits)
    keys = rng.integers(-lim + 1, lim, 50_001).astype(np.int64)
    vals = np.arange(keys.size, dtype=np.uint32)
    ref_k, perm, _ = oracle.sort_fixed_decimal(keys, int_digits, frac_digits)
    dk, dv = to_dev(keys), to_dev(vals)
    rs.rs_sort_pairs(dk, dv, dk, dv, decimal=(int_digits, frac_digits), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(dk, np.int64), ref_k)
    assert np.array_equal(from_dev(dv, np.uint32), perm.astype(np.uint32))


def test_decimal_pairs(rs, ctx, oracle):
    keys = W.decimals(123_457, 6, 3)
    vals = np.arange(keys.size, dtype=np.uint32)
    ref_k, perm, _ = oracle.sort_fixed_decimal(keys, 6, 3)
    ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), decimal=(6, 3), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.int64), ref_k)
    assert np.array_equal(from_dev(vo, np.uint32), perm.astype(np.uint32))


# --------------------------------------------------------------- full size


def _check_stable_sort_properties(keys_in, keys_out, vals_out):
    """On the device: output non-decreasing, payload a permutation, keys follow
    their payloads, equal keys keep input order.  Together these determine
    the stable sort uniquely."""
    n = keys_in.numel()
    ki = keys_in.to(torch.int64) & 0xFFFFFFFF
    ko = keys_out.to(torch.int64) & 0xFFFFFFFF
    v = vals_out.to(torch.int64) & 0xFFFFFFFF
    assert bool((ko[1:] >= ko[:-1]).all())
    seen = torch.zeros(n, dtype=torch.int32, device=keys_in.device)
    seen.index_fill_(0, v, 1)
    assert int(seen.sum()) == n
    assert bool((ki[v] == ko).all())
    same = ko[1:] == ko[:-1]
    assert bool((v[1:][same] > v[:-1][same]).all())


@pytest.mark.parametrize("dist", ["uniform", "zipf", "presorted"])
def test_u32_pairs_full_size(rs, ctx, oracle, dist):
    n = 1 << 28
    keys, vals = W.u32_pairs(n, dist)
    dk, dv = to_dev(keys), to_dev(vals)
    ko, vo = rs.rs_sort_pairs(dk, dv, ctx=ctx)
    ctx.check()
    _check_stable_sort_properties(dk, ko, vo)
    # sampled outputs against the plain definition of the stable rank
    rng = np.random.default_rng(99)
    ko_h, vo_h = from_dev(ko, np.uint32), from_dev(vo, np.uint32)
    for i in rng.integers(0, n, 6):
        r = oracle.stable_rank(keys, int(i))
        assert ko_h[r] == keys[i] and vo_h[r] == i
    del dk, dv, ko, vo
    torch.cuda.empty_cache()


def test_u32_pairs_maximum_size(rs, ctx, oracle):
    # n = RS_MAX_N: per-cell counts reach the 30-bit limit of the look-back words
    n = rs.RS_MAX_N
    keys, vals = W.u32_pairs(n, "uniform", seed_extra=7)
    dk, dv = to_dev(keys), to_dev(vals)
    ko, vo = rs.rs_sort_pairs(dk, dv, ctx=ctx)
    ctx.check()
    assert ctx.last_plan()["tiles"] == -(-n // TILE_KEYS[("u32", "u32")])
    _check_stable_sort_properties(dk, ko, vo)
    rng = np.random.default_rng(98)
    for i in list(rng.integers(0, n, 2)) + [n - 1]:
        r = oracle.stable_rank(keys, int(i))
        assert int(ko[r].item()) & 0xFFFFFFFF == keys[i] and int(vo[r].item()) == i
    del dk, dv, ko, vo
    torch.cuda.empty_cache()


def test_fixed_decimal_6_3_full_size(rs, ctx, oracle):
    """2^26 signed decimals with 6 integer and 3 fraction digits (the
    decimal workload at its full size), keys and the stable permutation,
    element by element against the oracle."""
    n = 1 << 26
    keys = W.decimals(n, 6, 3)
    ref_k, perm, _ = oracle.sort_fixed_decimal(keys, 6, 3)
    dk = to_dev(keys)
    out = rs.rs_sort_fixed_decimal(dk, 6, 3, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(out, np.int64), ref_k)
    del out
    vals = np.arange(n, dtype=np.uint32)
    ko, vo = rs.rs_sort_pairs(dk, to_dev(vals), decimal=(6, 3), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.int64), ref_k)
    assert np.array_equal(from_dev(vo, np.uint32), perm.astype(np.uint32))
    del dk, ko, vo
    torch.cuda.empty_cache()


def test_timing_and_launch_count(rs, ctx):
    keys = to_dev(W.u32_keys(1 << 20))
    ctx.set_timing(True)
    ctx.reset_timing()
    before = ctx.launch_count()
    rs.rs_sort_u32(keys, ctx=ctx)
    ctx.check()
    ms, launches = ctx.kernel_time("pass")
    assert launches == 4 and ms > 0
    assert ctx.launch_count() - before == 6  # count + fill + 4 passes
    ctx.set_timing(False)


# --------------------------------------------------------------- float keys


def _canonical(keys):
    """What the library writes for float keys: -0.0 as +0.0, every NaN as the
    quiet NaN of its width (the order is decided before, by the oracle)."""
    out = keys.copy()
    out[out == 0] = 0.0
    out[np.isnan(out)] = np.nan
    return out


@pytest.mark.parametrize("fdt", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 7, 7168 + 3, 3 * 10240 + 17, 100_003])
def test_float_pairs(rs, ctx, oracle, fdt, n):
    rng = np.random.default_rng(n + (0 if fdt == np.float32 else 1))
    keys = rng.standard_normal(n).astype(fdt)
    keys[::5] = np.round(keys[::5])  # ties, including +0.0 and -0.0
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 1e-45, -1e-45], fdt)
    # NaNs that carry a payload, a sign or the signalling bit pattern
    ub = np.uint32 if fdt == np.float32 else np.uint64
    nan_bits = ([0x7FC00001, 0xFFC00123, 0x7F800001, 0xFFFFFFFF] if fdt == np.float32 else
                [0x7FF8000000000001, 0xFFF8000000000123, 0x7FF0000000000001,
                 0xFFFFFFFFFFFFFFFF])
    special = np.concatenate([special, np.array(nan_bits, ub).view(fdt)])
    m = min(n, special.size)
    keys[rng.permutation(n)[:m]] = special[:m]
    vals = np.arange(n, dtype=np.uint32)
    _, perm, _ = oracle.sort_float(keys)
    perm = perm.astype(np.int64)
    ko, vo = rs.rs_sort_pairs(to_dev(keys), to_dev(vals), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(vo, np.uint32).astype(np.int64), perm)
    want = _canonical(keys[perm])
    got = from_dev(ko, fdt)
    assert np.array_equal(got.view(np.uint32 if fdt == np.float32 else np.uint64),
                          want.view(np.uint32 if fdt == np.float32 else np.uint64))
