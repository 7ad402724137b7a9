"""CPU checks of the C ABI: the library loads, exports every declared entry
point, and its host-side logic (argument checks, workspace sizing) behaves as
``include/rs.h`` documents.  Nothing here launches GPU work."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rs.h")


@pytest.fixture(scope="module")
def rs():
    from paper_2107_01391_gb300 import build, binding
    build.build()
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rs_sort_u32", "rs_sort_u64", "rs_sort_fixed_decimal", "rs_sort_pairs",
                     "rs_ctx_create", "rs_ctx_destroy", "rs_ctx_status"):
        assert required in names


def test_library_exports_every_declared_symbol(rs):
    out = subprocess.run(["nm", "-D", "--defined-only", rs.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (rs_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert set(rs.EXPORTS) <= exported
    lib = rs.lib()
    for f in declared_functions():
        assert getattr(lib, f) is not None


def test_version(rs):
    assert "sm_103a" in rs.version()


def test_workspace_query_grows_with_n(rs):
    sizes = [rs.workspace_bytes("rs_sort_u32", n) for n in (0, 1, 4096, 1 << 20, 1 << 28)]
    assert all(s > 0 and s % 256 == 0 for s in sizes)
    assert sizes == sorted(sizes)
    # keys-only u32 at 2^28: one ping-pong key buffer (1 GiB) plus look-back rows
    assert (1 << 30) <= sizes[-1] <= (1 << 30) + (256 << 20)
    pairs = rs.workspace_bytes("rs_sort_pairs_u32", 1 << 28)
    assert pairs >= sizes[-1] + (1 << 30)


def _call_u32(rs, ctx, src, dst, n, temp, tb):
    need = ctypes.c_size_t(tb)
    return rs.lib().rs_sort_u32(ctx, ctypes.c_void_p(src), ctypes.c_void_p(dst), n,
                                ctypes.c_void_p(temp) if temp else None, ctypes.byref(need), None)


def test_argument_checks(rs):
    L = rs.lib()
    fake = ctypes.c_void_p(1)
    assert L.rs_sort_u32(None, None, None, 0, None, None, None) == rs.RS_ERR_INVALID
    # NULL keys with n > 0
    assert _call_u32(rs, fake, 0, 0, 10, 0, 0) == rs.RS_ERR_INVALID
    # misaligned key pointer
    assert _call_u32(rs, fake, 258, 512, 10, 0, 0) == rs.RS_ERR_INVALID
    # n above the documented maximum
    assert _call_u32(rs, fake, 256, 512, rs.RS_MAX_N + 1, 0, 0) == rs.RS_ERR_INVALID
    # workspace too small (nothing launched: the check comes first)
    assert _call_u32(rs, fake, 256, 512, 1000, 4096, 16) == rs.RS_ERR_TEMP_TOO_SMALL
    # fixed-point digit counts out of range
    need = ctypes.c_size_t(0)
    z = ctypes.c_void_p(256)
    assert L.rs_sort_fixed_decimal(fake, z, z, 10, 10, 9, None, ctypes.byref(need),
                                   None) == rs.RS_ERR_INVALID
    assert L.rs_sort_fixed_decimal(fake, z, z, 10, 0, 0, None, ctypes.byref(need),
                                   None) == rs.RS_ERR_INVALID
    assert L.rs_sort_fixed_decimal(fake, z, z, 10, 6, 3, None, ctypes.byref(need),
                                   None) == rs.RS_OK
    # payload width other than 4 or 8
    assert L.rs_sort_pairs(fake, rs.RS_KEY_U32, z, z, z, z, 3, 10, None, None,
                           ctypes.byref(need), None) == rs.RS_ERR_INVALID
    # unknown key type
    assert L.rs_sort_pairs(fake, 9, z, z, z, z, 4, 10, None, None, ctypes.byref(need),
                           None) == rs.RS_ERR_UNSUPPORTED
    # float keys: a size query succeeds for both widths and payload sizes
    for kt in (rs.RS_KEY_F32, rs.RS_KEY_F64):
        for vb in (4, 8):
            assert L.rs_sort_pairs(fake, kt, z, z, z, z, vb, 10, None, None,
                                   ctypes.byref(need), None) == rs.RS_OK
    # decimal pairs need their digit counts
    assert L.rs_sort_pairs(fake, rs.RS_KEY_I64_DEC, z, z, z, z, 4, 10, None, None,
                           ctypes.byref(need), None) == rs.RS_ERR_INVALID


def test_segmented_size_limits(rs):
    L = rs.lib()
    fn = L.rs_sort_segmented
    fake, z = ctypes.c_void_p(1), ctypes.c_void_p(256)
    need = ctypes.c_size_t(0)
    # a batch may hold more keys than one sort (segments are sorted apart)
    n = rs.RS_MAX_N + 1
    assert fn(fake, rs.RS_KEY_U32, z, z, None, z, 4, n, z, 1000, None, None,
              ctypes.byref(need), None) == rs.RS_OK
    assert need.value >= 8 * n  # cell and value ping-pong buffers
    assert fn(fake, rs.RS_KEY_U32, z, z, None, z, 4, rs.RS_MAX_SEGMENTED_N + 1, z, 1000, None,
              None, ctypes.byref(need), None) == rs.RS_ERR_INVALID


def test_context_needs_a_device(rs):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert rs.lib().rs_ctx_create(ctypes.byref(h), 0) == rs.RS_ERR_INVALID
    assert rs.lib().rs_ctx_status(None, 0) == rs.RS_ERR_INVALID
    with pytest.raises(RuntimeError):
        rs.Context(0)


def test_segmented_workspace_layout(rs):
    """Host-side sizing of a segmented call: equal segments below the device
    tier (2^13 keys) reserve no device-tier room, offsets always do; an
    argsort to 8-byte indices carries 32-bit indices, so it needs the 4-byte
    argsort's workspace plus n 32-bit words."""
    fn = rs.lib().rs_sort_segmented
    fake, z = ctypes.c_void_p(1), ctypes.c_void_p(256)

    def ws(n, segs, offsets, vals_in, vb):
        need = ctypes.c_size_t(0)
        assert fn(fake, rs.RS_KEY_U32, z, z, z if vals_in else None, z, vb, n,
                  z if offsets else None, segs, None, None, ctypes.byref(need), None) == rs.RS_OK
        assert need.value % 256 == 0
        return need.value

    n = 1 << 24
    short_equal = ws(n, n >> 12, False, True, 4)   # rows of 4096 keys
    long_equal = ws(n, n >> 14, False, True, 4)    # rows of 16384 keys: device tier
    with_offsets = ws(n, n >> 12, True, True, 4)
    assert short_equal < with_offsets
    assert long_equal == ws(n, n >> 14, True, True, 4)
    assert short_equal >= 8 * n                     # cell and value ping-pong buffers
    arg32 = ws(n, n >> 12, True, False, 4)
    arg64 = ws(n, n >> 12, True, False, 8)
    assert arg64 >= arg32 + 4 * n
