"""Thin Python binding of the C ABI in ``include/rs.h`` (``librsort.so``).

Argument marshalling only: torch supplies device memory (outputs and the
workspace) and the current CUDA stream; every step of the sort runs in the
library's CUDA kernels.  There is no CPU fallback: without the built library
or a CUDA device every call raises.

The function names mirror the C entry points (``rs_sort_u32`` ...).  Each
takes CUDA tensors, allocates the outputs and the workspace unless given,
enqueues the sort on the current stream and returns without waiting.
Device-side errors surface through ``Context.status(synchronize=True)``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librsort.so")

RS_OK, RS_ERR_INVALID, RS_ERR_RANGE, RS_ERR_TEMP_TOO_SMALL = 0, 1, 2, 3
RS_ERR_CUDA, RS_ERR_TIMEOUT, RS_ERR_UNSUPPORTED = 4, 5, 6
STATUS_NAMES = {0: "RS_OK", 1: "RS_ERR_INVALID", 2: "RS_ERR_RANGE", 3: "RS_ERR_TEMP_TOO_SMALL",
                4: "RS_ERR_CUDA", 5: "RS_ERR_TIMEOUT", 6: "RS_ERR_UNSUPPORTED"}
RS_KEY_U32, RS_KEY_U64, RS_KEY_I64_DEC, RS_KEY_F32, RS_KEY_F64 = 0, 1, 2, 3, 4
RS_MAX_N = (1 << 30) - 1
RS_MAX_SEGMENTED_N = 1 << 40
RS_MAX_SEGMENT_LEN = RS_MAX_N
RS_FILL_CELLS = 4096

# Every function the header declares (the CPU test checks the export table).
EXPORTS = ("rs_ctx_create", "rs_ctx_destroy", "rs_ctx_status", "rs_sort_u32", "rs_sort_u64",
           "rs_sort_fixed_decimal", "rs_sort_pairs", "rs_ctx_last_plan", "rs_ctx_set_timing",
           "rs_ctx_kernel_time", "rs_ctx_reset_timing", "rs_ctx_launch_count", "rs_version",
           "rs_sort_strings", "rs_sort_segmented", "rs_scatter_rows", "rs_traverse_maps",
           "rs_sort_u32_noalloc", "rs_debug_wait_timeout", "rs_ctx_set_pass_tile_limit",
           "rs_ctx_pass_tile_limit")


class RsError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what} failed: {STATUS_NAMES.get(code, code)}")
        self.code = code


class KeyParams(ctypes.Structure):
    _fields_ = [("int_digits", ctypes.c_int32), ("frac_digits", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("passes_run", ctypes.c_uint32),
                ("passes_total", ctypes.c_uint32), ("tiles", ctypes.c_uint32)]


_lib = None
_lib_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load librsort.so (built by ``paper_2107_01391_gb300.build``); raise if absent."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2107_01391_gb300/build.py "
                               "(nvcc, sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        p, sz, st = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        psz = ctypes.POINTER(ctypes.c_size_t)
        L.rs_ctx_create.argtypes = [ctypes.POINTER(p), ctypes.c_int]
        L.rs_ctx_destroy.argtypes = [p]
        L.rs_ctx_status.argtypes = [p, ctypes.c_int]
        L.rs_ctx_last_plan.argtypes = [p, ctypes.POINTER(PlanInfo)]
        L.rs_ctx_set_timing.argtypes = [p, ctypes.c_int]
        L.rs_ctx_reset_timing.argtypes = [p]
        L.rs_ctx_kernel_time.argtypes = [p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_uint64)]
        L.rs_ctx_launch_count.argtypes = [p]
        L.rs_ctx_launch_count.restype = ctypes.c_uint64
        L.rs_version.restype = ctypes.c_char_p
        L.rs_sort_u32.argtypes = [p, p, p, sz, p, psz, p]
        L.rs_sort_u64.argtypes = [p, p, p, sz, p, psz, p]
        L.rs_sort_fixed_decimal.argtypes = [p, p, p, sz, ctypes.c_int, ctypes.c_int, p, psz, p]
        L.rs_sort_pairs.argtypes = [p, ctypes.c_int, p, p, p, p, sz, sz,
                                    ctypes.POINTER(KeyParams), p, psz, p]
        L.rs_sort_strings.argtypes = [p, p, p, sz, ctypes.c_uint32, p, p, psz, p]
        L.rs_sort_segmented.argtypes = [p, ctypes.c_int, p, p, p, p, sz, sz, p, sz,
                                        ctypes.POINTER(KeyParams), p, psz, p]
        L.rs_scatter_rows.argtypes = [p, p, p, sz, sz, sz, p, p]
        L.rs_traverse_maps.argtypes = [p, p, sz, ctypes.c_int, ctypes.c_int, ctypes.c_int, p, p,
                                       p, p, p, psz, p]
        L.rs_sort_u32_noalloc.argtypes = [p, p, sz, p, p]
        L.rs_ctx_set_pass_tile_limit.argtypes = [p, ctypes.c_uint64]
        L.rs_ctx_pass_tile_limit.argtypes = [p, ctypes.POINTER(ctypes.c_uint64)]
        for name in ("rs_sort_strings", "rs_sort_segmented", "rs_scatter_rows",
                     "rs_traverse_maps", "rs_sort_u32_noalloc", "rs_ctx_set_pass_tile_limit",
                     "rs_ctx_pass_tile_limit"):
            getattr(L, name).restype = st
        for name in ("rs_ctx_create", "rs_ctx_destroy", "rs_ctx_status", "rs_ctx_last_plan",
                     "rs_ctx_set_timing", "rs_ctx_reset_timing", "rs_ctx_kernel_time",
                     "rs_sort_u32", "rs_sort_u64", "rs_sort_fixed_decimal", "rs_sort_pairs"):
            getattr(L, name).restype = st
        _lib = L
        return L


def _check(code: int, what: str):
    if code != RS_OK:
        raise RsError(code, what)


class Context:
    """Owns an ``rs_ctx`` (the device status word and the timing state)."""

    def __init__(self, device: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("rsort needs a CUDA device; there is no CPU fallback")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._h = ctypes.c_void_p()
        _check(lib().rs_ctx_create(ctypes.byref(self._h), self.device), "rs_ctx_create")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().rs_ctx_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, synchronize: bool = True) -> int:
        return lib().rs_ctx_status(self._h, int(synchronize))

    def check(self):
        """Wait for the device and raise on a device-detected error."""
        _check(self.status(True), "device-side sort")

    def last_plan(self) -> dict:
        info = PlanInfo()
        _check(lib().rs_ctx_last_plan(self._h, ctypes.byref(info)), "rs_ctx_last_plan")
        return {"mode": "fill" if info.mode == 1 else "passes", "passes_run": info.passes_run,
                "passes_total": info.passes_total, "tiles": info.tiles}

    def set_timing(self, enable: bool):
        _check(lib().rs_ctx_set_timing(self._h, int(enable)), "rs_ctx_set_timing")

    def reset_timing(self):
        _check(lib().rs_ctx_reset_timing(self._h), "rs_ctx_reset_timing")

    def kernel_time(self, kernel_class: str):
        """(total milliseconds, launches) of one kernel class: hist, pass or fill."""
        ms, n = ctypes.c_double(), ctypes.c_uint64()
        _check(lib().rs_ctx_kernel_time(self._h, kernel_class.encode(), ctypes.byref(ms),
                                        ctypes.byref(n)), "rs_ctx_kernel_time")
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(lib().rs_ctx_launch_count(self._h))

    @property
    def pass_tile_limit(self) -> int:
        """Sorts of more than 4096 and at most this many keys take the narrow
        pass tile (rs_ctx_set_pass_tile_limit)."""
        v = ctypes.c_uint64()
        _check(lib().rs_ctx_pass_tile_limit(self._h, ctypes.byref(v)), "rs_ctx_pass_tile_limit")
        return int(v.value)

    @pass_tile_limit.setter
    def pass_tile_limit(self, narrow_max_n: int):
        _check(lib().rs_ctx_set_pass_tile_limit(self._h, int(narrow_max_n)),
               "rs_ctx_set_pass_tile_limit")

    def apply_tuning(self, path: str | None = None) -> bool:
        """Apply a tuning table written by ``paper_2107_01391_gb300.tune`` (the
        file at ``path``, else $RS_TUNE_FILE) if it was measured on this
        device's model; returns whether it was applied."""
        import json
        path = path or os.environ.get("RS_TUNE_FILE")
        if not path or not os.path.exists(path):
            return False
        with open(path) as f:
            table = json.load(f)
        if table.get("device_name") != torch.cuda.get_device_name(self.device):
            return False
        self.pass_tile_limit = int(table["narrow_max_n"])
        return True


_default_ctx: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    """The per-device context the wrappers use when given none; a tuning table
    named by $RS_TUNE_FILE is applied to it when created."""
    dev = torch.cuda.current_device() if device is None else int(device)
    if dev not in _default_ctx:
        c = Context(dev)
        c.apply_tuning()
        _default_ctx[dev] = c
    return _default_ctx[dev]


def _cuda(t: torch.Tensor, name: str, nbytes: int, dtypes) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name}: dtype {t.dtype} not in {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _out(t: torch.Tensor, like: torch.Tensor, name: str, dtypes=None,
         numel: int | None = None) -> torch.Tensor:
    """Check a caller-given output buffer.

    The C ABI takes bare device pointers and cannot see a buffer's length or
    device, so an output that is too short or on another GPU would turn into
    out-of-bounds device writes.  It must be a contiguous CUDA tensor on the
    input's device with exactly ``numel`` elements (default: as many as
    ``like``) of an allowed dtype (default: ``like``'s element size).
    """
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtypes is not None and t.dtype not in dtypes:
        raise TypeError(f"{name}: dtype {t.dtype} not in {dtypes}")
    if dtypes is None and t.element_size() != like.element_size():
        raise TypeError(f"{name}: {t.element_size()}-byte elements, "
                        f"{like.element_size()} expected")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    want = like.numel() if numel is None else numel
    if t.numel() != want:
        raise ValueError(f"{name} has {t.numel()} elements, {want} expected")
    if t.device != like.device:
        raise ValueError(f"{name} is on {t.device}, the input on {like.device}")
    return t


def _context(ctx: "Context | None", t: torch.Tensor) -> "Context":
    """The given context (which must belong to t's device) or t's default one."""
    if ctx is None:
        return default_context(t.device.index)
    if ctx.device != t.device.index:
        raise ValueError(f"context of cuda:{ctx.device} used with a tensor on {t.device}")
    return ctx


def _stream(t: torch.Tensor, stream):
    s = torch.cuda.current_stream(t.device) if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


def _workspace(query, device, temp):
    need = ctypes.c_size_t(0)
    _check(query(None, ctypes.byref(need)), "workspace query")
    if temp is not None:
        _cuda(temp, "temp", 1, (torch.uint8,))
        if temp.device != torch.device(device):
            raise ValueError(f"temp is on {temp.device}, the input on {device}")
    if temp is None or temp.numel() < need.value:
        temp = torch.empty(max(need.value, 1), dtype=torch.uint8, device=device)
    return temp, ctypes.c_size_t(temp.numel())


U32_DTYPES = (torch.uint32, torch.int32)
U64_DTYPES = (torch.uint64, torch.int64)


def rs_sort_u32(keys: torch.Tensor, out: torch.Tensor | None = None, *, ctx: Context | None = None,
                stream=None, temp: torch.Tensor | None = None) -> torch.Tensor:
    """Stable ascending sort of uint32 keys (int32 tensors are read as their uint32 bits)."""
    _cuda(keys, "keys", 4, U32_DTYPES)
    out = torch.empty_like(keys) if out is None else _out(out, keys, "out", U32_DTYPES)
    ctx = _context(ctx, keys)
    n, s, L = keys.numel(), _stream(keys, stream), lib()
    temp, tb = _workspace(lambda t, b: L.rs_sort_u32(ctx.handle, _ptr(keys), _ptr(out), n, t, b, s),
                          keys.device, temp)
    _check(L.rs_sort_u32(ctx.handle, _ptr(keys), _ptr(out), n, _ptr(temp), ctypes.byref(tb), s),
           "rs_sort_u32")
    return out


def rs_sort_u64(keys: torch.Tensor, out: torch.Tensor | None = None, *, ctx: Context | None = None,
                stream=None, temp: torch.Tensor | None = None) -> torch.Tensor:
    """Stable ascending sort of uint64 keys (int64 tensors are read as their uint64 bits)."""
    _cuda(keys, "keys", 8, U64_DTYPES)
    out = torch.empty_like(keys) if out is None else _out(out, keys, "out", U64_DTYPES)
    ctx = _context(ctx, keys)
    n, s, L = keys.numel(), _stream(keys, stream), lib()
    temp, tb = _workspace(lambda t, b: L.rs_sort_u64(ctx.handle, _ptr(keys), _ptr(out), n, t, b, s),
                          keys.device, temp)
    _check(L.rs_sort_u64(ctx.handle, _ptr(keys), _ptr(out), n, _ptr(temp), ctypes.byref(tb), s),
           "rs_sort_u64")
    return out


def rs_sort_fixed_decimal(keys: torch.Tensor, int_digits: int, frac_digits: int,
                          out: torch.Tensor | None = None, *, ctx: Context | None = None,
                          stream=None, temp: torch.Tensor | None = None) -> torch.Tensor:
    """Stable ascending sort of int64 fixed-point decimals scaled by 10^frac_digits."""
    _cuda(keys, "keys", 8, (torch.int64,))
    out = torch.empty_like(keys) if out is None else _out(out, keys, "out", (torch.int64,))
    ctx = _context(ctx, keys)
    n, s, L = keys.numel(), _stream(keys, stream), lib()
    temp, tb = _workspace(
        lambda t, b: L.rs_sort_fixed_decimal(ctx.handle, _ptr(keys), _ptr(out), n, int_digits,
                                             frac_digits, t, b, s), keys.device, temp)
    _check(L.rs_sort_fixed_decimal(ctx.handle, _ptr(keys), _ptr(out), n, int_digits, frac_digits,
                                   _ptr(temp), ctypes.byref(tb), s), "rs_sort_fixed_decimal")
    return out


def _key_type(keys: torch.Tensor, decimal: tuple[int, int] | None) -> int:
    if decimal is not None:
        _cuda(keys, "keys", 8, (torch.int64,))
        return RS_KEY_I64_DEC
    if keys.dtype in U32_DTYPES:
        return RS_KEY_U32
    if keys.dtype in U64_DTYPES:
        return RS_KEY_U64
    if keys.dtype == torch.float32:
        return RS_KEY_F32
    if keys.dtype == torch.float64:
        return RS_KEY_F64
    raise TypeError(f"unsupported key dtype {keys.dtype}")


def rs_sort_pairs(keys: torch.Tensor, values: torch.Tensor | None,
                  keys_out: torch.Tensor | None = None,
                  values_out: torch.Tensor | None = None, *, decimal: tuple[int, int] | None = None,
                  ctx: Context | None = None, stream=None, temp: torch.Tensor | None = None):
    """Stable key/value sort; returns (sorted keys, values in the same order).

    ``decimal=(int_digits, frac_digits)`` sorts int64 keys as fixed-point
    decimals; float32/float64 keys sort as numbers (-0.0 ties +0.0 and is
    written as +0.0, NaNs last); other 4-byte keys are uint32 and 8-byte keys
    uint64.  Values may be any 4- or 8-byte dtype (moved as raw bits);
    ``values=None`` sorts the keys alone and returns (sorted keys, None).
    """
    kt = _key_type(keys, decimal)
    _cuda(keys, "keys", keys.element_size(), (keys.dtype,))
    if values is None:
        vb = 0
        values_out = None
    else:
        if values.numel() != keys.numel():
            raise ValueError("keys and values must have the same length")
        vb = values.element_size()
        if vb not in (4, 8):
            raise TypeError("values must be 4 or 8 bytes per element")
        _cuda(values, "values", vb, (values.dtype,))
        if values.device != keys.device:
            raise ValueError("keys and values must be on the same device")
        values_out = (torch.empty_like(values) if values_out is None
                      else _out(values_out, values, "values_out"))
    keys_out = torch.empty_like(keys) if keys_out is None else _out(keys_out, keys, "keys_out")
    ctx = _context(ctx, keys)
    prm = KeyParams(*(decimal or (0, 0)))
    pp = ctypes.byref(prm)
    n, s, L = keys.numel(), _stream(keys, stream), lib()

    def call(t, b):
        return L.rs_sort_pairs(ctx.handle, kt, _ptr(keys), _ptr(keys_out), _ptr(values),
                               _ptr(values_out), vb, n, pp, t, b, s)

    temp, tb = _workspace(call, keys.device, temp)
    _check(call(_ptr(temp), ctypes.byref(tb)), "rs_sort_pairs")
    return keys_out, values_out


def workspace_bytes(fn_name: str, n: int, **kw) -> int:
    """Workspace size a call of ``fn_name`` needs for n keys (no launch)."""
    L = lib()
    need = ctypes.c_size_t(0)
    # A size query launches nothing and never dereferences the context or the
    # key pointers; placeholders only have to pass the argument checks.
    h = ctypes.c_void_p(1)
    z = ctypes.c_void_p(256)
    if fn_name == "rs_sort_u32":
        code = L.rs_sort_u32(h, z, z, n, None, ctypes.byref(need), None)
    elif fn_name == "rs_sort_u64":
        code = L.rs_sort_u64(h, z, z, n, None, ctypes.byref(need), None)
    elif fn_name == "rs_sort_fixed_decimal":
        code = L.rs_sort_fixed_decimal(h, z, z, n, kw["int_digits"], kw["frac_digits"], None,
                                       ctypes.byref(need), None)
    elif fn_name == "rs_sort_strings":
        code = L.rs_sort_strings(h, z, z, n, kw.get("max_len", RS_MAX_STRING_LEN), z, None,
                                 ctypes.byref(need), None)
    elif fn_name == "rs_sort_pairs_u32":
        code = L.rs_sort_pairs(h, RS_KEY_U32, z, z, z, z, kw.get("val_bytes", 4), n, None, None,
                               ctypes.byref(need), None)
    else:
        raise ValueError(fn_name)
    _check(code, f"{fn_name} workspace query")
    return need.value


RS_MAX_STRING_LEN = 1024


def rs_sort_strings(chars: torch.Tensor, offsets: torch.Tensor, max_len: int,
                    perm_out: torch.Tensor | None = None, *, ctx: Context | None = None,
                    stream=None, temp: torch.Tensor | None = None) -> torch.Tensor:
    """Stable sort of byte strings; returns perm (int32 tensor holding uint32
    indices): perm[j] is the input index of the j-th smallest string.

    String i is ``chars[offsets[i]:offsets[i+1]]``; ``offsets`` has n+1
    entries (int32/uint32 bits), ``chars`` is uint8.
    """
    _cuda(chars, "chars", 1, (torch.uint8,))
    _cuda(offsets, "offsets", 4, U32_DTYPES)
    n = offsets.numel() - 1
    if n < 0:
        raise ValueError("offsets needs n+1 entries")
    if chars.device != offsets.device:
        raise ValueError("chars and offsets must be on the same device")
    perm_out = (torch.empty(n, dtype=torch.int32, device=offsets.device) if perm_out is None
                else _out(perm_out, offsets, "perm_out", U32_DTYPES, numel=n))
    ctx = _context(ctx, offsets)
    L = lib()
    fn = L.rs_sort_strings
    s = _stream(offsets, stream)
    cptr = ctypes.c_void_p(chars.data_ptr()) if chars.numel() else ctypes.c_void_p(
        offsets.data_ptr())  # any valid device address; no byte is read when empty

    def call(t, b):
        return fn(ctx.handle, cptr, _ptr(offsets), n, max_len, _ptr(perm_out), t, b, s)

    temp, tb = _workspace(call, offsets.device, temp)
    _check(call(_ptr(temp), ctypes.byref(tb)), "rs_sort_strings")
    return perm_out


def _seg_key_type(keys: torch.Tensor, decimal):
    if decimal is not None:
        return RS_KEY_I64_DEC
    return {torch.uint32: RS_KEY_U32, torch.int32: RS_KEY_U32, torch.uint64: RS_KEY_U64,
            torch.int64: RS_KEY_U64, torch.float32: RS_KEY_F32,
            torch.float64: RS_KEY_F64}[keys.dtype]


def rs_sort_segmented(keys: torch.Tensor, seg_offsets: torch.Tensor | None,
                      values: torch.Tensor | None = None, keys_out: torch.Tensor | None = None,
                      values_out: torch.Tensor | None = None, *, num_segs: int | None = None,
                      argsort: bool = False, index_dtype=torch.int64,
                      decimal: tuple[int, int] | None = None, ctx: Context | None = None,
                      stream=None, temp: torch.Tensor | None = None):
    """Sort every segment of ``keys`` independently and stably.

    ``seg_offsets`` (int64 CUDA tensor, num_segs+1 entries) delimits the
    segments; ``None`` with ``num_segs`` means equal segments.  Returns
    (sorted keys, sorted values) when ``values`` is given, (sorted keys,
    indices within each segment) when ``argsort``, else the sorted keys.
    Float keys: -0.0 ties with +0.0 and comes out as +0.0; NaNs sort last.
    """
    kt = _seg_key_type(keys, decimal)
    _cuda(keys, "keys", keys.element_size(), (keys.dtype,))
    n = keys.numel()
    if seg_offsets is not None:
        _cuda(seg_offsets, "seg_offsets", 8, (torch.int64, torch.uint64))
        if seg_offsets.device != keys.device:
            raise ValueError("seg_offsets must be on the keys' device")
        num_segs = seg_offsets.numel() - 1
    elif num_segs is None:
        raise ValueError("give seg_offsets or num_segs")
    keys_out = torch.empty_like(keys) if keys_out is None else _out(keys_out, keys, "keys_out")
    if values is not None:
        vb = values.element_size()
        _cuda(values, "values", vb, (values.dtype,))
        if values.numel() != n or values.device != keys.device:
            raise ValueError("values must match the keys' length and device")
        values_out = (torch.empty_like(values) if values_out is None
                      else _out(values_out, values, "values_out"))
    elif argsort:
        values_out = (torch.empty(keys.shape, dtype=index_dtype, device=keys.device)
                      if values_out is None
                      else _out(values_out, keys, "values_out",
                                (torch.int32, torch.uint32, torch.int64, torch.uint64)))
        vb = values_out.element_size()
    else:
        vb = 0
    ctx = _context(ctx, keys)
    L = lib()
    fn = L.rs_sort_segmented
    prm = KeyParams(*(decimal or (0, 0)))
    s = _stream(keys, stream)
    vin = _ptr(values) if values is not None else ctypes.c_void_p(0)
    vout = _ptr(values_out) if values_out is not None else ctypes.c_void_p(0)
    offs = _ptr(seg_offsets) if seg_offsets is not None else ctypes.c_void_p(0)

    def call(t, b):
        return fn(ctx.handle, kt, _ptr(keys), _ptr(keys_out), vin, vout, vb, n, offs, num_segs,
                  ctypes.byref(prm), t, b, s)

    temp, tb = _workspace(call, keys.device, temp)
    _check(call(_ptr(temp), ctypes.byref(tb)), "rs_sort_segmented")
    if values_out is not None:
        return keys_out, values_out
    return keys_out


def rs_scatter_rows(src: torch.Tensor, perm: torch.Tensor, out: torch.Tensor | None = None, *,
                    ctx: Context | None = None, stream=None) -> torch.Tensor:
    """out[r, perm[r, j]] = src[r, j] for 2-D src/perm (the backward of a row sort)."""
    if src.dim() != 2 or perm.shape != src.shape:
        raise ValueError("src and perm must be 2-D and of the same shape")
    _cuda(src, "src", src.element_size(), (src.dtype,))
    _cuda(perm, "perm", 8, (torch.int64,))
    if perm.device != src.device:
        raise ValueError("src and perm must be on the same device")
    out = torch.empty_like(src) if out is None else _out(out, src, "out")
    ctx = _context(ctx, src)
    L = lib()
    fn = L.rs_scatter_rows
    _check(fn(ctx.handle, _ptr(src), _ptr(perm), src.shape[0], src.shape[1],
              src.element_size(), _ptr(out), _stream(src, stream)), "rs_scatter_rows")
    return out


def rs_traverse_maps(keys: torch.Tensor, int_digits: int, frac_digits: int,
                     signed_dim: bool = False, with_counts: bool = True, *,
                     ctx: Context | None = None, stream=None):
    """Count array S, traverse maps H_Max / H_Min and extraction cost k of the
    paper's hashing and extraction cycles, computed on the device.

    Returns (S or None, hmax [rows], hmin [rows, 2], k) as CUDA tensors (S
    shaped like the hypercube); k is a one-element int64 tensor.
    """
    _cuda(keys, "keys", 8, (torch.int64,))
    D = int_digits + frac_digits
    cells = (2 if signed_dim else 1) * 10 ** D
    rows = cells // 10
    dev = keys.device
    S = torch.empty(cells, dtype=torch.int32, device=dev) if with_counts else None
    hmax = torch.empty(rows, dtype=torch.int32, device=dev)
    hmin = torch.empty(rows, 2, dtype=torch.int32, device=dev)
    k = torch.empty(1, dtype=torch.int64, device=dev)
    ctx = _context(ctx, keys)
    L = lib()
    fn = L.rs_traverse_maps
    s = _stream(keys, stream)
    sp = _ptr(S) if S is not None else ctypes.c_void_p(0)

    def call(t, b):
        return fn(ctx.handle, _ptr(keys), keys.numel(), int_digits, frac_digits, int(signed_dim),
                  sp, _ptr(hmax), _ptr(hmin), _ptr(k), t, b, s)

    temp, tb = _workspace(call, dev, temp=None)
    _check(call(_ptr(temp), ctypes.byref(tb)), "rs_traverse_maps")
    shape = ((2,) if signed_dim else ()) + (10,) * D
    return (S.view(shape) if S is not None else None), hmax, hmin, k


def rs_sort_u32_noalloc(keys: torch.Tensor, out: torch.Tensor | None = None,
                        status: torch.Tensor | None = None, *, stream=None) -> torch.Tensor:
    """The uint32 keys-only sort whose workspace is built into the library.

    For callers that cannot allocate device memory while sorting: the C call
    allocates nothing (this wrapper only allocates ``out`` when it is not
    given).  At most ``RS_NOALLOC_MAX_N`` keys.  ``status`` is an optional
    one-element int32 CUDA tensor that collects device-side error bits.
    Calls whose work overlaps on the GPU share one built-in workspace and race.
    """
    L = lib()
    fn = L.rs_sort_u32_noalloc
    _cuda(keys, "keys", 4, U32_DTYPES)
    out = torch.empty_like(keys) if out is None else _out(out, keys, "out", U32_DTYPES)
    if status is not None:
        # the kernels OR error bits into this word: it must be a device int32
        # on the keys' GPU
        _cuda(status, "status", 4, (torch.int32, torch.uint32))
        if status.numel() < 1 or status.device != keys.device:
            raise ValueError("status must be a one-element int32 tensor on the keys' device")
    st = _ptr(status) if status is not None else ctypes.c_void_p(0)
    # the C call runs on the current device: make it the keys' device, whose
    # stream is passed
    with torch.cuda.device(keys.device):
        _check(fn(_ptr(keys), _ptr(out), keys.numel(), st, _stream(keys, stream)),
               "rs_sort_u32_noalloc")
    return out


RS_NOALLOC_MAX_N = 1 << 20


def version() -> str:
    return lib().rs_version().decode()
