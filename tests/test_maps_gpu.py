"""The traverse maps and extraction cost on the device against the oracle's
hashing cycle and the paper's worked example (k = 17)."""
import numpy as np
import pytest

from conftest import read_golden
from gpu_util import require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    require_gpu()
    from paper_2107_01391_gb300 import build, binding
    build.build()
    return binding


def test_worked_example(rs):
    g = read_golden("example1.txt")
    keys = np.array([int(x) for x in g["scaled"]], np.int64)
    S, hmax, hmin, k = rs.rs_traverse_maps(to_dev(keys), 1, 1)
    assert int(k.item()) == int(g["k"][0])
    lo, hi = (int(v) for v in g["row4_hmin_hmax"])
    assert hmin[4].tolist() == [1, lo] and int(hmax[4]) == hi
    expected = np.zeros((10, 10), np.int64)
    for cell in g["cells"]:
        r, c = (int(v) for v in cell.split(","))
        expected[r, c] += 1
    assert np.array_equal(S.cpu().numpy(), expected)


@pytest.mark.parametrize("int_digits,frac_digits,n", [(1, 2, 500), (2, 1, 30_000), (3, 3, 200_000),
                                                      (4, 2, 3_000_000)])
def test_maps_vs_oracle(rs, oracle, int_digits, frac_digits, n):
    rng = np.random.default_rng(n)
    hi = 10 ** (int_digits + frac_digits)
    keys = rng.integers(0, hi // 3, n).astype(np.int64) * 3  # leaves empty cells and rows
    S_ref, hmax_ref, hmin_ref, k_ref = oracle.decimal_hashing_cycle(keys, int_digits, frac_digits)
    S, hmax, hmin, k = rs.rs_traverse_maps(to_dev(keys), int_digits, frac_digits)
    assert np.array_equal(S.cpu().numpy(), S_ref.astype(np.int64))
    assert np.array_equal(hmax.cpu().numpy(), hmax_ref.astype(np.int64))
    assert np.array_equal(hmin.cpu().numpy(), hmin_ref.astype(np.int64))
    assert int(k.item()) == k_ref


def test_maps_signed(rs, oracle):
    rng = np.random.default_rng(9)
    keys = rng.integers(-999, 1000, 50_000).astype(np.int64)
    S_ref, hmax_ref, hmin_ref, k_ref = oracle.decimal_hashing_cycle(keys, 2, 1)
    S, hmax, hmin, k = rs.rs_traverse_maps(to_dev(keys), 2, 1, signed_dim=True)
    assert S_ref.shape == (2, 10, 10, 10)
    assert np.array_equal(S.cpu().numpy(), S_ref.astype(np.int64))
    assert np.array_equal(hmax.cpu().numpy(), hmax_ref.astype(np.int64))
    assert np.array_equal(hmin.cpu().numpy(), hmin_ref.astype(np.int64))
    assert int(k.item()) == k_ref


def test_maps_range_error(rs):
    ctx = rs.Context(0)
    rs.rs_traverse_maps(to_dev(np.array([5, -3], np.int64)), 1, 0, ctx=ctx)
    assert ctx.status(True) == rs.RS_ERR_RANGE
    ctx.close()
