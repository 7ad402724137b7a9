"""Parity of rs_sort_strings against the CPU oracle (radix-257 character
dimensions), permutations compared element by element."""
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


def _pack(strs):
    chars = np.frombuffer(b"".join(strs), np.uint8) if strs else np.zeros(0, np.uint8)
    offsets = np.zeros(len(strs) + 1, np.uint32)
    np.cumsum([len(x) for x in strs], out=offsets[1:]) if strs else None
    return chars, offsets


def _gpu_perm(rs, ctx, chars, offsets, max_len):
    dc = torch.from_numpy(chars.copy()).cuda() if chars.size else torch.zeros(0, dtype=torch.uint8, device="cuda")
    perm = rs.rs_sort_strings(dc, to_dev(offsets), max_len, ctx=ctx)
    ctx.check()
    return from_dev(perm, np.uint32)


@pytest.mark.parametrize("n", [1, 2, 4095, 4097, 100_003])
def test_lowercase_strings(rs, ctx, oracle, n):
    chars, offsets = W.strings(n, seed_extra=n)
    ref, _ = oracle.sort_strings(chars, offsets.astype(np.uint64))
    got = _gpu_perm(rs, ctx, chars, offsets, 16)
    assert np.array_equal(got, ref.astype(np.uint32))


def test_strings_full_size(rs, ctx, oracle):
    """The 2^24-string workload at its full size: the whole permutation
    against the oracle, element by element."""
    n = 1 << 24
    chars, offsets = W.strings(n)
    ref, _ = oracle.sort_strings(chars, offsets.astype(np.uint64))
    got = _gpu_perm(rs, ctx, chars, offsets, 16)
    assert np.array_equal(got, ref.astype(np.uint32))


def test_strings_full_size_sampled(rs, ctx, oracle):
    n = 1 << 24
    chars, offsets = W.strings(n)
    got = _gpu_perm(rs, ctx, chars, offsets, 16)
    # property check on every output: consecutive strings ordered as Python bytes,
    # equal neighbours in input order; the permutation is a bijection
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32))
    off = offsets.astype(np.int64)
    rng = np.random.default_rng(1)
    for j in rng.integers(0, n - 1, 20000):
        a, b = int(got[j]), int(got[j + 1])
        sa = chars[off[a]:off[a + 1]].tobytes()
        sb = chars[off[b]:off[b + 1]].tobytes()
        assert sa < sb or (sa == sb and a < b)
    # a 2^20 prefix of the same workload against the oracle, element by element
    m = 1 << 20
    ref, _ = oracle.sort_strings(chars[: off[m]], offsets[: m + 1].astype(np.uint64))
    got_m = _gpu_perm(rs, ctx, chars[: off[m]], offsets[: m + 1], 16)
    assert np.array_equal(got_m, ref.astype(np.uint32))


@pytest.mark.parametrize("case", ["binary", "prefixes", "empty_mix", "all_equal", "long",
                                  "maximum_length"])
def test_edge_strings(rs, ctx, oracle, case):
    rng = np.random.default_rng(7)
    if case == "binary":      # every byte value, including 0x00 and 0xff: 9-bit symbols
        strs = [bytes(rng.integers(0, 256, int(rng.integers(0, 20))).astype(np.uint8))
                for _ in range(30_000)]
        strs.append(bytes(range(256))[:20])
    elif case == "prefixes":  # proper prefixes sort first; "a\\0" after "a"
        base = [b"", b"a", b"a\x00", b"a\x00\x00", b"ab", b"abc", b"b", b"\x00", b"\xff"]
        strs = [base[i] for i in rng.integers(0, len(base), 20_000)]
    elif case == "empty_mix":
        strs = [b"" if rng.random() < 0.5 else b"x" * int(rng.integers(1, 4)) for _ in range(9000)]
    elif case == "all_equal":
        strs = [b"same-string"] * 12_345
    elif case == "long":      # long strings spanning several 64-bit cells
        strs = [bytes(rng.integers(97, 100, int(rng.integers(30, 200))).astype(np.uint8))
                for _ in range(5000)]
    else:                     # up to RS_MAX_STRING_LEN bytes, equal for the first 1000
        prefix = bytes(rng.integers(97, 99, 1000).astype(np.uint8))
        strs = [prefix + bytes(rng.integers(97, 99, int(rng.integers(0, 25))).astype(np.uint8))
                for _ in range(3000)]
        strs.append(prefix + b"b" * (rs.RS_MAX_STRING_LEN - 1000))
    max_len = (rs.RS_MAX_STRING_LEN if case == "maximum_length"
               else max(1, max(len(x) for x in strs)))
    chars, offsets = _pack(strs)
    ref, _ = oracle.sort_strings(chars, offsets.astype(np.uint64))
    got = _gpu_perm(rs, ctx, chars, offsets, max_len)
    assert np.array_equal(got, ref.astype(np.uint32))


@pytest.mark.parametrize("case", ["differ_after_11", "equal_11", "mixed_lengths"])
def test_first_attempt_boundary(rs, ctx, oracle, case):
    """The first attempt sorts by the leading 11 symbols of a 'a'..'z'
    alphabet (56 bits of 5-bit symbols).  Strings that agree there and are
    longer must go through the general sort; strings of at most 11 symbols
    that agree there are equal and keep their input order."""
    rng = np.random.default_rng(len(case))
    head = [bytes(rng.integers(97, 123, 11).astype(np.uint8)) for _ in range(50)]
    strs = []
    for _ in range(20_000):
        h = head[int(rng.integers(0, len(head)))]
        if case == "differ_after_11":
            strs.append(h + bytes(rng.integers(97, 123, int(rng.integers(1, 6))).astype(np.uint8)))
        elif case == "equal_11":
            strs.append(h)
        else:
            tail = int(rng.integers(0, 3))
            strs.append(h[: int(rng.integers(9, 12))] if tail == 0 else
                        h + bytes(rng.integers(97, 123, tail).astype(np.uint8)))
    chars, offsets = _pack(strs)
    ref, _ = oracle.sort_strings(chars, offsets.astype(np.uint64))
    got = _gpu_perm(rs, ctx, chars, offsets, 16)
    assert np.array_equal(got, ref.astype(np.uint32))


def test_all_empty_strings(rs, ctx):
    n = 777
    chars = np.zeros(0, np.uint8)
    offsets = np.zeros(n + 1, np.uint32)
    got = _gpu_perm(rs, ctx, chars, offsets, 4)
    assert np.array_equal(got, np.arange(n, dtype=np.uint32))


def test_string_longer_than_max_len(rs, ctx):
    chars, offsets = _pack([b"abc", b"toolongstring", b"x"])
    dc = torch.from_numpy(chars.copy()).cuda()
    rs.rs_sort_strings(dc, to_dev(offsets), 5, ctx=ctx)
    assert ctx.status(True) == rs.RS_ERR_RANGE
