"""The allocation-free sort entry point (rs_sort_u32_noalloc).

It exists for callers that cannot allocate device memory while they sort
(cudaFree waits for the whole device; a plugin inside another framework's
memory pool has no allocator to call).  Its workspace is a fixed array built
into the library and shared by every call, so these tests check, through the
C ABI, that two calls in a row each give exactly what rs_sort_u32 gives: the
second call must not see anything the first one left behind.

The file is named to be collected last; it passes alone in a fresh process
and after the other tests.
"""
import ctypes

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


def _call_noalloc(rs, keys_dev, out_dev, status_dev):
    fn = rs.lib().rs_sort_u32_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return fn(ctypes.c_void_p(keys_dev.data_ptr()), ctypes.c_void_p(out_dev.data_ptr()),
              keys_dev.numel(), ctypes.c_void_p(status_dev.data_ptr()), stream)


def test_noalloc_matches_rs_sort_u32_twice_in_a_row(rs, oracle):
    ctx = rs.Context(0)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cases = [
        W.u32_keys(rs.RS_NOALLOC_MAX_N, "uniform", seed_extra=1),  # the largest size, 4 passes
        W.digits3(300_001, seed_extra=2),                          # small keys: rebuilt from cells
        W.u32_keys(777_777, "presorted", seed_extra=4),            # back to the pass path
    ]
    for keys in cases:
        d = to_dev(keys)
        want = rs.rs_sort_u32(d, ctx=ctx)
        ctx.check()
        ref, _, _ = oracle.sort_u32(keys)
        assert np.array_equal(from_dev(want, np.uint32), ref)
        got = torch.empty_like(d)
        assert _call_noalloc(rs, d, got, status) == rs.RS_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(from_dev(got, np.uint32), ref)
    ctx.close()


# Small inputs: unlike rs_sort_u32, which sorts at most 4096 keys in one
# single-CTA launch, the allocation-free call always runs the counting,
# rebuild and digit-group launches, here over one partial tile (a tile is
# 48 x 256 = 12288 keys) or just past one.
@pytest.mark.parametrize("n", [1, 2, 31, 4096, 4097, 12288, 12289])
@pytest.mark.parametrize("kind", ["uniform", "digits3"])
def test_noalloc_small_inputs_against_oracle(rs, oracle, n, kind):
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    keys = (W.u32_keys(n, "uniform", seed_extra=n) if kind == "uniform"
            else W.digits3(n, seed_extra=n))
    ref, _, _ = oracle.sort_u32(keys)
    d = to_dev(keys)
    for _ in range(2):  # a second call must not see what the first left behind
        got = torch.empty_like(d)
        assert _call_noalloc(rs, d, got, status) == rs.RS_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(from_dev(got, np.uint32), ref)


def test_noalloc_in_place_and_binding(rs):
    keys = W.u32_keys(123_457, "zipf", seed_extra=3)
    d = to_dev(keys)
    want = from_dev(rs.rs_sort_u32(d, ctx=rs.default_context(0)), np.uint32)
    rs.rs_sort_u32_noalloc(d, out=d)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(d, np.uint32), want)


def test_noalloc_binding_checks_buffers(rs):
    d = to_dev(W.u32_keys(1000, "uniform", seed_extra=9))
    with pytest.raises(ValueError):
        rs.rs_sort_u32_noalloc(d, out=torch.empty(999, dtype=torch.int32, device="cuda"))
    with pytest.raises(TypeError):
        rs.rs_sort_u32_noalloc(d, status=torch.zeros(1, dtype=torch.int32))  # host memory
    with pytest.raises(TypeError):
        rs.rs_sort_u32_noalloc(d, status=torch.zeros(1, dtype=torch.int64, device="cuda"))


def test_noalloc_rejects_more_than_its_workspace(rs):
    big = torch.empty(rs.RS_NOALLOC_MAX_N + 1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call_noalloc(rs, big, big, status) == rs.RS_ERR_TEMP_TOO_SMALL
