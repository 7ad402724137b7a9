"""Sorts captured in a CUDA graph and replayed on new inputs.

The library plans on the device and never synchronises with the host, so a
whole sort (memset, count, plan, passes) can be captured once and replayed
with new keys written into the captured input buffers.  Every replay must
match the oracle bit for bit, including when the new keys choose a different
plan (the fill path, a different set of trivial digit groups) than the keys
seen at capture time.
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


@pytest.fixture(scope="module")
def ctx(rs):
    c = rs.Context(0)
    yield c
    c.close()


def _capture(fn):
    """Capture fn() on a side stream into a CUDA graph (after one eager run)."""
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g


def test_graph_replay_pairs(rs, ctx, oracle):
    n = 3 * 6144 + 17
    inputs = [W.u32_keys(n, "uniform", seed_extra=31),
              W.u32_keys(n, "zipf", seed_extra=32),
              (W.u32_keys(n, "uniform", seed_extra=33) & np.uint32(0x00FF00FF)),  # 2 active groups
              np.full(n, 7, np.uint32)]                                      # every group trivial
    vals = np.arange(n, dtype=np.uint32)
    dk, dv = to_dev(inputs[0]), to_dev(vals)
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    temp = torch.empty(rs.workspace_bytes("rs_sort_pairs_u32", n), dtype=torch.uint8,
                       device="cuda")
    g = _capture(lambda: rs.rs_sort_pairs(dk, dv, ko, vo, ctx=ctx, temp=temp))
    for keys in inputs:
        dk.copy_(to_dev(keys))
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        want_k, want_v, _ = oracle.sort_pairs(keys, vals)
        np.testing.assert_array_equal(from_dev(ko, np.uint32), want_k)
        np.testing.assert_array_equal(from_dev(vo, np.uint32), want_v)


def test_graph_replay_keys_switches_plan(rs, ctx, oracle):
    # captured on keys that need the digit passes, replayed on keys whose
    # whole space fits one count array (the fill path), and back
    n = 100_003
    wide = W.u32_keys(n, "uniform", seed_extra=34)
    narrow = W.digits3(n, seed_extra=35)
    dk = to_dev(wide)
    out = torch.empty_like(dk)
    temp = torch.empty(rs.workspace_bytes("rs_sort_u32", n), dtype=torch.uint8, device="cuda")
    g = _capture(lambda: rs.rs_sort_u32(dk, out, ctx=ctx, temp=temp))
    for keys in (narrow, wide, narrow):
        dk.copy_(to_dev(keys))
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        want, _, _ = oracle.sort_u32(keys)
        np.testing.assert_array_equal(from_dev(out, np.uint32), want)


def test_graph_replay_segmented_mixed_tiers(rs, ctx, oracle):
    """One rs_sort_segmented call (size ordering, the persistent warp, on-chip
    and CTA tiers, the device tier's passes) captured once with an offsets
    tensor, then replayed on new keys and values: every segment must match
    the oracle each time."""
    sizes = [0, 5, 63, 64, 700, 4096, 4097, 9000, 20_000, 50_000, 1, 31]
    off = np.zeros(len(sizes) + 1, np.uint64)
    np.cumsum(np.asarray(sizes, np.uint64), out=off[1:])
    n = int(off[-1])
    rng = np.random.default_rng(41)
    inputs = [rng.integers(0, 1 << 32, n, dtype=np.uint32),
              rng.integers(0, 50, n, dtype=np.uint32),            # many ties
              (rng.integers(0, 1 << 32, n, dtype=np.uint32) & np.uint32(0xFF0000FF))]
    dk = to_dev(inputs[0])
    dv = torch.empty(n, dtype=torch.float32, device="cuda")
    doff = to_dev(off)
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    need = ctypes.c_size_t(0)
    L = rs.lib()
    prm = rs.KeyParams(0, 0)
    z = ctypes.c_void_p(256)
    assert L.rs_sort_segmented(ctx.handle, rs.RS_KEY_U32, z, z, z, z, 4, n, z, len(sizes),
                               ctypes.byref(prm), None, ctypes.byref(need), None) == rs.RS_OK
    temp = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    g = _capture(lambda: rs.rs_sort_segmented(dk, doff, dv, ko, vo, ctx=ctx, temp=temp))
    for t, keys in enumerate(inputs):
        vals = rng.standard_normal(n).astype(np.float32)
        dk.copy_(to_dev(keys))
        dv.copy_(torch.from_numpy(vals).cuda())
        g.replay()
        torch.cuda.synchronize()
        ctx.check()
        got_k, got_v = from_dev(ko, np.uint32), vo.cpu().numpy()
        for s_ in range(len(sizes)):
            lo, hi = int(off[s_]), int(off[s_ + 1])
            want_k, perm, _ = oracle.sort_u32(keys[lo:hi])
            np.testing.assert_array_equal(got_k[lo:hi], want_k)
            np.testing.assert_array_equal(got_v[lo:hi].view(np.uint32),
                                          vals[lo:hi][perm.astype(np.int64)].view(np.uint32))
