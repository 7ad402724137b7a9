"""Failure detection without a GPU fault: the look-back wait gives up.

The decoupled look-back is the only wait in the sort kernels.  Here it polls
a predecessor that never publishes (a zeroed word nothing sets); it must stop
after its bound, report RS_ERR_TIMEOUT through the status word, and leave
the context able to sort correctly afterwards."""
import ctypes
import time

import numpy as np
import pytest
import torch

from gpu_util import from_dev, require_gpu, to_dev
from paper_2107_01391_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives(oracle):
    require_gpu()
    from paper_2107_01391_gb300 import build, binding
    build.build()
    ctx = binding.Context(0)
    L = binding.lib()
    fn = L.rs_debug_wait_timeout
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64,
                   ctypes.c_void_p]
    fn.restype = ctypes.c_int
    temp = torch.empty(4096, dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    t0 = time.perf_counter()
    assert fn(ctx.handle, ctypes.c_void_p(temp.data_ptr()), temp.numel(), 50_000_000, stream) == 0
    assert ctx.status(True) == binding.RS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    assert ctx.status(True) == binding.RS_OK  # cleared
    keys = W.u32_keys(100_000, "uniform", seed_extra=5)
    out = binding.rs_sort_u32(to_dev(keys), ctx=ctx)
    ctx.check()
    assert np.array_equal(from_dev(out, np.uint32), oracle.sort_u32(keys)[0])
    ctx.close()
