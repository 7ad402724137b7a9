"""The torch-level entry point ``sort`` routes every argument shape to the
right C-ABI call; each route is checked against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import from_dev, require_gpu, to_dev
from paper_2107_01391_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 3 * 10240 + 17  # several pass tiles of every shape, ragged


@pytest.fixture(scope="module")
def rs():
    require_gpu()
    from paper_2107_01391_gb300 import build
    build.build()
    import paper_2107_01391_gb300 as pkg
    return pkg


def test_integer_keys(rs, oracle):
    k32 = W.u32_keys(N, seed_extra=41)
    want, _, _ = oracle.sort_u32(k32)
    assert np.array_equal(from_dev(rs.sort(to_dev(k32)), np.uint32), want)
    k64 = W.u64_keys(N, seed_extra=42)
    want, _, _ = oracle.sort_u64(k64)
    assert np.array_equal(from_dev(rs.sort(to_dev(k64)), np.uint64), want)


def test_decimal_keys_and_pairs(rs, oracle):
    dec = W.decimals(N, 4, 2, seed_extra=43)
    want, perm, _ = oracle.sort_fixed_decimal(dec, 4, 2)
    assert np.array_equal(from_dev(rs.sort(to_dev(dec), decimal=(4, 2)), np.int64), want)
    vals = np.arange(N, dtype=np.uint32)
    ko, vo = rs.sort(to_dev(dec), to_dev(vals), decimal=(4, 2))
    assert np.array_equal(from_dev(ko, np.int64), want)
    assert np.array_equal(from_dev(vo, np.uint32).astype(np.int64), perm.astype(np.int64))


@pytest.mark.parametrize("fdt", [np.float32, np.float64])
def test_float_keys_only(rs, oracle, fdt):
    rng = np.random.default_rng(44)
    keys = rng.standard_normal(N).astype(fdt)
    keys[::9] = -0.0
    keys[5::97] = np.nan
    _, perm, _ = oracle.sort_float(keys)
    want = keys[perm.astype(np.int64)]
    want[want == 0] = 0.0
    got = from_dev(rs.sort(to_dev(keys)), fdt)
    ut = np.uint32 if fdt == np.float32 else np.uint64
    want[np.isnan(want)] = np.nan
    assert np.array_equal(got.view(ut), want.view(ut))


def test_pairs_segments_and_argsort(rs, oracle):
    keys = W.u32_keys(N, seed_extra=45)
    vals = np.arange(N, dtype=np.uint32) * np.uint32(3)
    want_k, want_v, _ = oracle.sort_pairs(keys, vals)
    ko, vo = rs.sort(to_dev(keys), to_dev(vals))
    assert np.array_equal(from_dev(ko, np.uint32), want_k)
    assert np.array_equal(from_dev(vo, np.uint32), want_v)

    # equal segments given as a count, argsort within each
    segs = 17
    n = (N // segs) * segs
    k = keys[:n]
    ko, idx = rs.sort(to_dev(k), segments=segs, argsort=True)
    L = n // segs
    for s in (0, segs // 2, segs - 1):
        ref_k, ref_p, _ = oracle.sort_u32(k[s * L:(s + 1) * L])
        assert np.array_equal(from_dev(ko, np.uint32)[s * L:(s + 1) * L], ref_k)
        assert np.array_equal(idx.cpu().numpy()[s * L:(s + 1) * L], ref_p.astype(np.int64))

    # uneven segments given as offsets, with values
    off = np.array([0, 5, 5, 4000, 4063, N], np.int64)
    ko, vo = rs.sort(to_dev(keys), to_dev(vals), segments=torch.from_numpy(off).cuda())
    for s in range(off.size - 1):
        lo, hi = int(off[s]), int(off[s + 1])
        ref_k, ref_v, _ = oracle.sort_pairs(keys[lo:hi], vals[lo:hi])
        assert np.array_equal(from_dev(ko, np.uint32)[lo:hi], ref_k)
        assert np.array_equal(from_dev(vo, np.uint32)[lo:hi], ref_v)


def test_strings_and_sortfn(rs, oracle):
    chars, offs = W.strings(5000, seed_extra=46)
    perm = rs.sort_strings(to_dev(chars), to_dev(offs), 16)
    ref, _ = oracle.sort_strings(chars, offs.astype(np.uint64), 16)
    assert np.array_equal(perm.cpu().numpy().view(np.uint32).astype(np.int64),
                          ref.astype(np.int64))
    x = torch.randn(8, 300, device="cuda", dtype=torch.float64, requires_grad=True)
    values, idx = rs.SortFn.apply(x)
    ref_v, ref_i = torch.sort(x.detach(), stable=True)
    assert torch.equal(values.detach(), ref_v) and torch.equal(idx, ref_i)
