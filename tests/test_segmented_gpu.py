"""Parity of rs_sort_segmented against the CPU oracle, segment by segment."""
import numpy as np
import pytest
import torch

from gpu_util import from_dev, require_gpu, to_dev
from paper_2107_01391_gb300 import workloads as W

pytestmark = pytest.mark.gpu


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


# around the tier boundaries: 63 (warp), 4096 (on chip), 8192 (device tier)
SIZES = [0, 1, 2, 17, 31, 32, 33, 255, 256, 257, 1000, 4095, 4096, 4097, 5000, 8191, 8192, 8193,
         12_289, 70_000, 3, 0]


def _offsets(sizes):
    off = np.zeros(len(sizes) + 1, np.uint64)
    np.cumsum(np.asarray(sizes, np.uint64), out=off[1:])
    return off


def _oracle_segments(oracle, keys, off, sort_fn):
    out = np.empty_like(keys)
    perm = np.empty(keys.size, np.int64)
    for s in range(off.size - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        k, p, _ = sort_fn(keys[lo:hi])
        out[lo:hi] = k
        perm[lo:hi] = p.astype(np.int64)
    return out, perm


@pytest.mark.parametrize("inplace", [False, True])
def test_u32_pairs_mixed_sizes(rs, ctx, oracle, inplace):
    rng = np.random.default_rng(1)
    off = _offsets(SIZES)
    n = int(off[-1])
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
    keys[5000:9000] = keys[5000]  # a long run of ties
    vals = np.arange(n, dtype=np.uint32)
    ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
    dk, dv, doff = to_dev(keys), to_dev(vals), to_dev(off)
    if inplace:
        rs.rs_sort_segmented(dk, doff, dv, dk, dv, ctx=ctx)
        ko, vo = dk, dv
    else:
        ko, vo = rs.rs_sort_segmented(dk, doff, dv, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    base = np.repeat(off[:-1].astype(np.int64), np.diff(off).astype(np.int64))
    assert np.array_equal(from_dev(vo, np.uint32).astype(np.int64), base + perm)


@pytest.mark.parametrize("index_dtype", [torch.int64, torch.int32])
def test_argsort_mode(rs, ctx, oracle, index_dtype):
    rng = np.random.default_rng(2)
    off = _offsets(SIZES)
    n = int(off[-1])
    keys = rng.integers(0, 300, n, dtype=np.uint32)  # many ties
    ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
    ko, idx = rs.rs_sort_segmented(to_dev(keys), to_dev(off), argsort=True,
                                   index_dtype=index_dtype, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), perm)


def test_long_segments_many_device_tiles(rs, ctx, oracle):
    # segments of hundreds of device tiles: each is counted by many CTAs
    off = _offsets([3, (1 << 22) + 123, 70_000, (1 << 21) + 5, 1])
    n = int(off[-1])
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
    keys[100_000:300_000] = keys[100_000]  # a long run of ties inside the long segment
    ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
    ko, idx = rs.rs_sort_segmented(to_dev(keys), to_dev(off), argsort=True, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    assert np.array_equal(idx.cpu().numpy(), perm)


def test_one_segment_argsort(rs, ctx, oracle):
    # the whole array one segment: the argsort form of a single sort
    n = (1 << 23) + 77
    keys = W.u32_keys(n)
    ref_k, perm, _ = oracle.sort_u32(keys)
    ko, idx = rs.rs_sort_segmented(to_dev(keys), None, num_segs=1, argsort=True, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    assert np.array_equal(idx.cpu().numpy(), perm.astype(np.int64))


def test_device_tier_range_error_flagged(rs, ctx):
    # a decimal key beyond its declared digits inside a device-tier segment
    off = _offsets([10, 40_000, 5])
    dec = W.decimals(int(off[-1]), 6, 3)
    dec[20_000] = 10 ** 9  # needs ten digits
    rs.rs_sort_segmented(to_dev(dec), to_dev(off), decimal=(6, 3), ctx=ctx)
    assert ctx.status(True) == rs.RS_ERR_RANGE


def test_argsort_in_place_all_equal(rs, ctx):
    keys = np.full(3 * 9000, 7, np.uint32)
    dk = to_dev(keys)
    ko, idx = rs.rs_sort_segmented(dk, None, keys_out=dk, num_segs=3, argsort=True, ctx=ctx)
    ctx.check()
    assert np.array_equal(idx.cpu().numpy(), np.tile(np.arange(9000), 3))


def test_u64_and_decimal_keys(rs, ctx, oracle):
    off = _offsets([5, 4096, 6000, 1, 33_333])
    n = int(off[-1])
    k64 = W.u64_keys(n)
    ref, _ = _oracle_segments(oracle, k64, off, oracle.sort_u64)
    out = rs.rs_sort_segmented(to_dev(k64), to_dev(off), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(out, np.uint64), ref)
    dec = W.decimals(n, 6, 3)
    ref, perm = _oracle_segments(oracle, dec, off,
                                 lambda k: oracle.sort_fixed_decimal(k, 6, 3))
    ko, idx = rs.rs_sort_segmented(to_dev(dec), to_dev(off), argsort=True, decimal=(6, 3), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.int64), ref)
    assert np.array_equal(idx.cpu().numpy(), perm)


def _oracle_float_rows(oracle, x):
    """Per-row stable order from the oracle's float path, and the keys the
    library writes for it (-0.0 as +0.0, every NaN as the quiet NaN)."""
    ref = np.stack([oracle.sort_float(r)[1].astype(np.int64) for r in x])
    want = np.take_along_axis(x, ref, axis=1)
    want[want == 0] = 0.0
    want[np.isnan(want)] = np.nan
    return ref, want


def test_f32_rows_against_oracle(rs, ctx, oracle):
    rng = np.random.default_rng(3)
    rows, length = 64, 5000
    x = rng.standard_normal((rows, length)).astype(np.float32)
    x[:, ::7] = np.round(x[:, ::7])  # ties
    x[0, :4] = [0.0, -0.0, np.inf, -np.inf]
    x[1, :3] = np.array([0x7FC00001, 0xFFC00000, 0x7F800001], np.uint32).view(np.float32)
    ko, idx = rs.rs_sort_segmented(torch.from_numpy(x).cuda().reshape(-1), None,
                                   num_segs=rows, argsort=True, ctx=ctx)
    ctx.check()
    ref, want = _oracle_float_rows(oracle, x)
    assert np.array_equal(idx.cpu().numpy().reshape(rows, length), ref)
    assert np.array_equal(ko.cpu().numpy().reshape(rows, length).view(np.uint32),
                          want.view(np.uint32))


# ---- warp tier: segments of at most 63 keys are sorted by one warp each ----


@pytest.mark.parametrize("inplace", [False, True])
def test_warp_tier_tiny_segments_pairs(rs, ctx, oracle, inplace):
    rng = np.random.default_rng(11)
    sizes = rng.integers(0, 64, 5000)
    sizes[:8] = [63, 62, 33, 32, 31, 1, 0, 2]
    off = _offsets(sizes)
    n = int(off[-1])
    keys = rng.integers(0, 40, n, dtype=np.uint32)  # many ties inside each segment
    vals = rng.integers(0, 1 << 32, n, dtype=np.uint32)
    ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
    dk, dv, doff = to_dev(keys), to_dev(vals), to_dev(off)
    if inplace:
        rs.rs_sort_segmented(dk, doff, dv, dk, dv, ctx=ctx)
        ko, vo = dk, dv
    else:
        ko, vo = rs.rs_sort_segmented(dk, doff, dv, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    base = np.repeat(off[:-1].astype(np.int64), np.diff(off).astype(np.int64))
    assert np.array_equal(from_dev(vo, np.uint32), vals[base + perm])


def test_warp_tier_u64_decimal_and_argsort(rs, ctx, oracle):
    rng = np.random.default_rng(12)
    sizes = rng.integers(1, 64, 3000)
    off = _offsets(sizes)
    n = int(off[-1])
    k64 = W.u64_keys(n, seed_extra=5)
    k64[1::3] = k64[0::3][: k64[1::3].size]  # ties
    ref, perm = _oracle_segments(oracle, k64, off, oracle.sort_u64)
    ko, idx = rs.rs_sort_segmented(to_dev(k64), to_dev(off), argsort=True, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint64), ref)
    assert np.array_equal(idx.cpu().numpy(), perm)
    dec = W.decimals(n, 3, 2, seed_extra=6)
    ref, perm = _oracle_segments(oracle, dec, off,
                                 lambda k: oracle.sort_fixed_decimal(k, 3, 2))
    ko, idx = rs.rs_sort_segmented(to_dev(dec), to_dev(off), argsort=True, decimal=(3, 2),
                                   index_dtype=torch.int32, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.int64), ref)
    assert np.array_equal(idx.cpu().numpy().astype(np.int64), perm)


def test_warp_tier_uniform_rows(rs, ctx, oracle):
    # equal segments of 50 keys (no offsets array): every row goes to the warp tier
    rng = np.random.default_rng(13)
    rows, length = 4000, 50
    x = rng.standard_normal((rows, length)).astype(np.float32)
    x[:, ::3] = np.round(x[:, ::3])  # ties, including -0.0 and +0.0
    x[7, :2] = np.array([0xFFC00123, 0x7FC00000], np.uint32).view(np.float32)
    ko, idx = rs.rs_sort_segmented(torch.from_numpy(x).cuda().reshape(-1), None,
                                   num_segs=rows, argsort=True, ctx=ctx)
    ctx.check()
    ref, want = _oracle_float_rows(oracle, x)
    assert np.array_equal(idx.cpu().numpy().reshape(rows, length), ref)
    assert np.array_equal(ko.cpu().numpy().reshape(rows, length).view(np.uint32),
                          want.view(np.uint32))


# ---- equal rows of 64 .. 8192 keys: one CTA sorts a row on chip ----


@pytest.mark.parametrize("rows,length", [(100, 64), (37, 4096), (9, 4097), (5, 8192)])
@pytest.mark.parametrize("kind", ["u32_pairs", "u64_u64v", "f32_argsort64", "dec_in_place"])
def test_equal_rows(rs, ctx, oracle, rows, length, kind):
    rng = np.random.default_rng(rows * length + len(kind))
    n = rows * length
    off = np.arange(0, n + 1, length, dtype=np.uint64)
    if kind == "u32_pairs":
        keys = rng.integers(0, 1000, n, dtype=np.uint32)  # ties; upper groups trivial
        vals = rng.integers(0, 1 << 32, n, dtype=np.uint32)
        ko, vo = rs.rs_sort_segmented(to_dev(keys), None, to_dev(vals), num_segs=rows, ctx=ctx)
        ctx.check()
        ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
        base = np.repeat(off[:-1].astype(np.int64), length)
        assert np.array_equal(from_dev(ko, np.uint32), ref_k)
        assert np.array_equal(from_dev(vo, np.uint32), vals[base + perm])
    elif kind == "u64_u64v":  # 8-byte values above 4096 keys take the general path
        keys = W.u64_keys(n, seed_extra=rows)
        keys[::5] = keys[0]
        vals = rng.integers(0, 1 << 63, n, dtype=np.uint64)
        ko, vo = rs.rs_sort_segmented(to_dev(keys), None, to_dev(vals), num_segs=rows, ctx=ctx)
        ctx.check()
        ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u64)
        base = np.repeat(off[:-1].astype(np.int64), length)
        assert np.array_equal(from_dev(ko, np.uint64), ref_k)
        assert np.array_equal(from_dev(vo, np.uint64), vals[base + perm])
    elif kind == "f32_argsort64":
        x = rng.standard_normal(n).astype(np.float32)
        x[::7] = np.round(x[::7])
        ko, idx = rs.rs_sort_segmented(to_dev(x), None, num_segs=rows, argsort=True, ctx=ctx)
        ctx.check()
        ref = np.argsort(x.reshape(rows, length), axis=1, kind="stable")
        assert np.array_equal(idx.cpu().numpy().reshape(rows, length), ref)
    else:
        keys = W.decimals(n, 4, 2, seed_extra=rows)
        dk = to_dev(keys)
        rs.rs_sort_segmented(dk, None, keys_out=dk, num_segs=rows, decimal=(4, 2), ctx=ctx)
        ctx.check()
        ref, _ = _oracle_segments(oracle, keys, off, lambda k: oracle.sort_fixed_decimal(k, 4, 2))
        assert np.array_equal(from_dev(dk, np.int64), ref)


def test_bad_offsets_flagged(rs, ctx):
    keys = to_dev(np.arange(100, dtype=np.uint32)[::-1].copy())
    off = to_dev(np.array([0, 50, 40, 100], np.uint64))
    rs.rs_sort_segmented(keys, off, ctx=ctx)
    assert ctx.status(True) == rs.RS_ERR_RANGE


def test_overlapping_offsets_flagged(rs, ctx):
    # offsets that go back make segments overlap (outside the contract): more
    # large segments than the workspace was sized for; the extra one is
    # flagged and skipped, nothing is accessed out of bounds
    n = 8192
    keys = to_dev(np.arange(n, dtype=np.uint32)[::-1].copy())
    off = to_dev(np.array([0, n, 0, n, 0, n], np.uint64))
    rs.rs_sort_segmented(keys, off, ctx=ctx)
    assert ctx.status(True) == rs.RS_ERR_RANGE


def test_run_b_full_size(rs, ctx):
    # 65536 segments, log-uniform sizes scaled to a total of 2^28 keys
    sizes = W.segment_sizes(65536, total=1 << 28)
    keys, vals, off = W.segments(sizes)
    dk, doff = to_dev(keys), to_dev(off)
    dv = to_dev(np.arange(keys.size, dtype=np.uint32))
    ko, vo = rs.rs_sort_segmented(dk, doff, dv, ctx=ctx)
    ctx.check()
    n = keys.size
    seg_id = torch.repeat_interleave(torch.arange(sizes.size, device="cuda"),
                                     torch.from_numpy(sizes).cuda())
    ki = dk.to(torch.int64) & 0xFFFFFFFF
    kk = ko.to(torch.int64) & 0xFFFFFFFF
    v = vo.to(torch.int64) & 0xFFFFFFFF
    same_seg = seg_id[1:] == seg_id[:-1]
    assert bool((kk[1:] >= kk[:-1])[same_seg].all())            # sorted within segments
    assert bool((seg_id[v] == seg_id).all())                     # payload stays in its segment
    seen = torch.zeros(n, dtype=torch.int32, device="cuda")
    seen.index_fill_(0, v, 1)
    assert int(seen.sum()) == n                                  # a permutation
    assert bool((ki[v] == kk).all())                             # keys follow payloads
    tie = same_seg & (kk[1:] == kk[:-1])
    assert bool((v[1:][tie] > v[:-1][tie]).all())                # stable
    # three segments (smallest, one tile, largest) against the oracle
    from oracle import oracle as O
    ko_h, vo_h = from_dev(ko, np.uint32), from_dev(vo, np.uint32)
    for s in [int(np.argmin(sizes)), int(np.argmin(np.abs(sizes - 4096))), int(np.argmax(sizes))]:
        lo, hi = int(off[s]), int(off[s + 1])
        rk, rp, _ = O.sort_u32(keys[lo:hi])
        assert np.array_equal(ko_h[lo:hi], rk)
        assert np.array_equal(vo_h[lo:hi].astype(np.int64), lo + rp.astype(np.int64))


@pytest.mark.parametrize("index_dtype", [torch.int64, torch.int32])
@pytest.mark.parametrize("sizes", [[5, 9000, 300], [20_000], [100, 5000, 70_000, 0, 17]])
def test_argsort_leaves_positions_outside_segments(rs, ctx, oracle, index_dtype, sizes):
    """Segments that start after position 0 and end before n: the keys and
    indices at positions outside every segment keep what the caller put
    there, and each segment's indices (8-byte ones carried as 32-bit words
    and widened at the end) are the oracle's."""
    rng = np.random.default_rng(len(sizes) + sum(sizes))
    head, tail = 37, 53
    off = _offsets(sizes) + np.uint64(head)
    n = int(off[-1]) + tail
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
    keys[head: head + 40] = keys[head]  # ties
    dk, doff = to_dev(keys), to_dev(off)
    ko = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    io = torch.full((n,), -9, dtype=index_dtype, device="cuda")
    rs.rs_sort_segmented(dk, doff, None, ko, io, argsort=True, index_dtype=index_dtype, ctx=ctx)
    ctx.check()
    got_k, got_i = from_dev(ko, np.uint32), io.cpu().numpy().astype(np.int64)
    for s in range(len(sizes)):
        lo, hi = int(off[s]), int(off[s + 1])
        ref_k, perm, _ = oracle.sort_u32(keys[lo:hi])
        assert np.array_equal(got_k[lo:hi], ref_k)
        assert np.array_equal(got_i[lo:hi], perm.astype(np.int64))
    assert (got_i[:head] == -9).all() and (got_i[n - tail:] == -9).all()
    assert (got_k[:head] == np.uint32(0xFFFFFFF9)).all()
    assert (got_k[n - tail:] == np.uint32(0xFFFFFFF9)).all()


# ---- partial tiles spread over every warp: lengths around multiples of the
# block (256 keys) and of 4 item rows (1024 keys), in every tier, with keys
# equal to the largest cell, which the padding of a short tile shares ----

SPREAD_SIZES = [64, 65, 255, 257, 511, 767, 768, 769, 1023, 1025, 2049, 3071, 4095,  # on chip
                4097, 4353, 5119, 5120, 5121, 6143, 7169, 8191,                       # row tier
                8192, 9000, 10_239, 10_241, 10_240 + 255, 10_240 + 257, 10_240 + 1025,
                2 * 10_240 + 3072, 2 * 10_240 + 3073, 3 * 10_240 - 1]                # device tier


@pytest.mark.parametrize("spread", ["random", "ties_top"])
def test_spread_partial_tiles(rs, ctx, oracle, spread):
    rng = np.random.default_rng(11 if spread == "random" else 12)
    off = _offsets(SPREAD_SIZES)
    n = int(off[-1])
    if spread == "random":
        keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
        keys[::97] = 0xFFFFFFFF
    else:  # few values, the largest among them: trivial and moving groups mixed
        keys = rng.choice(np.array([0, 1, 0xFFFFFF00, 0xFFFFFFFF], np.uint32), n)
    vals = np.arange(n, dtype=np.uint32)
    ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
    ko, vo = rs.rs_sort_segmented(to_dev(keys), to_dev(off), to_dev(vals), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    base = np.repeat(off[:-1].astype(np.int64), np.diff(off).astype(np.int64))
    assert np.array_equal(from_dev(vo, np.uint32).astype(np.int64), base + perm)
    ko, idx = rs.rs_sort_segmented(to_dev(keys), to_dev(off), argsort=True, ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(ko, np.uint32), ref_k)
    assert np.array_equal(idx.cpu().numpy(), perm)


@pytest.mark.parametrize("length", [100, 300, 1025, 4000, 4097, 5000, 8000])
@pytest.mark.parametrize("kind", ["u32_pairs", "f32_argsort64", "u64_u64v"])
def test_equal_short_rows_spread(rs, ctx, oracle, length, kind):
    """Equal rows shorter than their tile: each row is ranked padded, spread
    over every warp."""
    rows = 7
    rng = np.random.default_rng(length + len(kind))
    n = rows * length
    off = np.arange(0, n + 1, length, dtype=np.uint64)
    base = np.repeat(off[:-1].astype(np.int64), length)
    if kind == "u32_pairs":
        keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
        keys[::13] = 0xFFFFFFFF
        vals = rng.integers(0, 1 << 32, n, dtype=np.uint32)
        ko, vo = rs.rs_sort_segmented(to_dev(keys), None, to_dev(vals), num_segs=rows, ctx=ctx)
        ctx.check()
        ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u32)
        assert np.array_equal(from_dev(ko, np.uint32), ref_k)
        assert np.array_equal(from_dev(vo, np.uint32), vals[base + perm])
    elif kind == "u64_u64v":
        keys = W.u64_keys(n, seed_extra=length)
        keys[::11] = np.uint64(0xFFFFFFFFFFFFFFFF)
        vals = rng.integers(0, 1 << 63, n, dtype=np.uint64)
        ko, vo = rs.rs_sort_segmented(to_dev(keys), None, to_dev(vals), num_segs=rows, ctx=ctx)
        ctx.check()
        ref_k, perm = _oracle_segments(oracle, keys, off, oracle.sort_u64)
        assert np.array_equal(from_dev(ko, np.uint64), ref_k)
        assert np.array_equal(from_dev(vo, np.uint64), vals[base + perm])
    else:
        x = rng.standard_normal(n).astype(np.float32)
        x[::9] = np.float32(np.nan)  # NaN: the largest cell
        ko, idx = rs.rs_sort_segmented(to_dev(x), None, num_segs=rows, argsort=True, ctx=ctx)
        ctx.check()
        ref, want = _oracle_float_rows(oracle, x.reshape(rows, length))
        assert np.array_equal(idx.cpu().numpy().reshape(rows, length), ref)
        assert np.array_equal(ko.cpu().numpy().reshape(rows, length).view(np.uint32),
                              want.view(np.uint32))
