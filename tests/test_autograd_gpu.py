"""The differentiable sort: forward parity with the oracle and torch.sort,
backward equal to the reference scatter bit for bit, and FP64 finite
differences (the Jacobian of a sort of distinct keys is a 0/1 permutation)."""
import numpy as np
import pytest
import torch

from gpu_util import require_gpu
from paper_2107_01391_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    require_gpu()
    from paper_2107_01391_gb300 import build
    build.build()
    from paper_2107_01391_gb300 import autograd
    return autograd


def test_forward_matches_oracle_rows(ag, oracle):
    x = W.distinct_rows(16, 5000)
    x[3, :10] = x[3, 10:20]  # ties inside one row
    vals, perm = ag.sort(torch.from_numpy(x).cuda())
    vals, perm = vals.cpu().numpy(), perm.cpu().numpy()
    for r in range(x.shape[0]):
        ref_k, ref_p, _ = oracle.sort_float(x[r])
        assert np.array_equal(perm[r], ref_p.astype(np.int64))
        assert np.array_equal(vals[r], ref_k)


def test_forward_matches_torch_sort(ag):
    x = torch.from_numpy(W.distinct_rows(64, 8192)).cuda()
    vals, perm = ag.sort(x)
    ref = torch.sort(x, dim=-1, stable=True)
    assert torch.equal(vals, ref.values) and torch.equal(perm, ref.indices)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("cols", [1000, 8192, 20_000])
def test_forward_signed_zeros_and_nans(ag, oracle, dtype, cols):
    """Rows holding -0.0, +0.0 and NaNs with payloads and either sign.  The
    permutation is the oracle's: -0.0 ties with +0.0 (input order kept) and
    every NaN sorts last, in input order (torch.sort's order for zeros and
    quiet NaNs).  The values are x gathered through that permutation, except
    that the library writes every zero as +0.0 and every NaN as the quiet NaN
    (its cells have the key's own width, so tied keys cannot keep distinct
    bits)."""
    rng = np.random.default_rng(cols)
    x = np.round(rng.standard_normal((6, cols)) * 3).astype(np.float64)
    x[:, ::7] = -0.0
    x[:, 3::11] = 0.0
    bits = np.array([0x7FF8000000000001, 0xFFF8000000000123, 0x7FF0000000000001,
                     0xFFFFFFFFFFFFFFFF], np.uint64)
    if dtype == torch.float32:
        x = x.astype(np.float32)
        bits = np.array([0x7FC00001, 0xFFC00123, 0x7F800001, 0xFFFFFFFF], np.uint32)
    nan = bits.view(x.dtype)
    for r in range(x.shape[0]):
        x[r, rng.permutation(cols)[:9]] = nan[rng.integers(0, nan.size, 9)]
    vals, perm = ag.sort(torch.from_numpy(x).cuda())
    vals, perm = vals.cpu().numpy(), perm.cpu().numpy()
    ub = np.uint32 if dtype == torch.float32 else np.uint64
    for r in range(x.shape[0]):
        _, ref_p, _ = oracle.sort_float(x[r])
        ref_p = ref_p.astype(np.int64)
        assert np.array_equal(perm[r], ref_p)
        want = x[r][ref_p].copy()
        want[want == 0] = 0.0          # -0.0 written as +0.0
        want[np.isnan(want)] = np.nan  # every NaN as the quiet NaN
        assert np.array_equal(vals[r].view(ub), want.view(ub))
        assert np.isnan(vals[r][-9:]).all()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_backward_is_the_reference_scatter(ag, dtype):
    x = torch.from_numpy(W.distinct_rows(32, 3000)).to(dtype).cuda().requires_grad_(True)
    g = torch.randn(32, 3000, dtype=dtype, device="cuda")
    vals, perm = ag.sort(x)
    (gx,) = torch.autograd.grad(vals, x, g)
    ref = torch.zeros_like(x).scatter_(1, perm, g)
    assert torch.equal(gx, ref)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_long_rows_forward_and_backward(ag, dtype):
    # rows longer than the backward's shared-memory row (96 KB), and long
    # enough for the segmented sort's device tier in the forward
    x = torch.from_numpy(W.distinct_rows(3, 40_000)).to(dtype).cuda().requires_grad_(True)
    vals, perm = ag.sort(x)
    ref = torch.sort(x.detach(), dim=-1, stable=True)
    assert torch.equal(vals, ref.values) and torch.equal(perm, ref.indices)
    g = torch.randn_like(vals)
    (gx,) = torch.autograd.grad(vals, x, g)
    assert torch.equal(gx, torch.zeros_like(g).scatter_(1, perm, g))


def test_fp64_finite_differences(ag):
    x = torch.from_numpy(W.distinct_rows(4, 64).astype(np.float64)).cuda().requires_grad_(True)
    # keys differ by at least 1, so a 1e-6 step never reorders a row
    assert torch.autograd.gradcheck(lambda t: ag.sort(t)[0], (x,), eps=1e-6, atol=1e-6)
    # the numerical Jacobian itself is a permutation matrix per row
    jac = torch.autograd.functional.jacobian(lambda t: ag.sort(t)[0], x.detach())
    j = jac.reshape(x.numel(), x.numel()).cpu()
    assert torch.all((j - j.round()).abs() < 1e-6)
    assert torch.all(j.sum(0) == 1) and torch.all(j.sum(1) == 1)


def test_full_shape_4096x8192(ag):
    x = torch.from_numpy(W.distinct_rows(4096, 8192)).cuda().requires_grad_(True)
    vals, perm = ag.sort(x)
    ref = torch.sort(x.detach(), dim=-1, stable=True)
    assert torch.equal(vals, ref.values) and torch.equal(perm, ref.indices)
    g = torch.randn_like(vals)
    (gx,) = torch.autograd.grad(vals, x, g)
    assert torch.equal(gx, torch.zeros_like(g).scatter_(1, perm, g))
