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


def test_noalloc_matches_rs_sort_u32_twice_in_a_row(rs):
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
        got = torch.empty_like(d)
        assert _call_noalloc(rs, d, got, status) == rs.RS_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert np.array_equal(from_dev(got, np.uint32), from_dev(want, np.uint32))
    ctx.close()


def test_noalloc_in_place_and_binding(rs):
    keys = W.u32_keys(123_457, "zipf", seed_extra=3)
    d = to_dev(keys)
    want = from_dev(rs.rs_sort_u32(d, ctx=rs.default_context(0)), np.uint32)
    rs.rs_sort_u32_noalloc(d, out=d)
    torch.cuda.synchronize()
    assert np.array_equal(from_dev(d, np.uint32), want)


def test_noalloc_rejects_more_than_its_workspace(rs):
    big = torch.empty(rs.RS_NOALLOC_MAX_N + 1, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call_noalloc(rs, big, big, status) == rs.RS_ERR_TEMP_TOO_SMALL
