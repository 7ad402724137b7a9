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
