"""Python face of the plain CPU Recombinant Sort oracle (``rs_oracle.c``).

TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only ``tests/``, the smoke
check and the benchmark's CPU-baseline leg may import this module.  It shares
no code with the CUDA path: it compiles and loads its own C file with gcc.

Every call returns numpy arrays.  The algorithm is the paper's (Kumar et al.,
arXiv 2107.01391): hashing cycle (§3.1, Eq. 1), extraction cycle (§3.2,
Eq. 16), buckets (§2.2); see the header comment of ``rs_oracle.c``.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rs_oracle.c")
_HDR = os.path.join(_HERE, "rs_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_RANGE, ERR_NOMEM = 0, 1, 2, 3
DEFAULT_CELL_CAP = 1000


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


class _Stats(ctypes.Structure):
    _fields_ = [
        ("k", ctypes.c_uint64),
        ("cycles", ctypes.c_uint64),
        ("dims", ctypes.c_uint64),
        ("top_cells", ctypes.c_uint64),
        ("regenerated", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
    ]


@dataclass
class Stats:
    k: int            # extraction cost (§5), summed over all extraction cycles
    cycles: int       # hashing+extraction cycles run
    dims: int         # dimensions of the normalised key
    top_cells: int    # cells of the first count array
    regenerated: bool  # keys_out rebuilt from cell coordinates (Eq. 16)


def build(force: bool = False) -> str:
    """Compile ``rs_oracle.c`` into ``liboracle.so`` beside it (gcc, -O2)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or any(
            os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-shared",
                                   "-fPIC", _SRC, "-o", tmp])
            os.replace(tmp, _LIB)
    return _LIB


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    p = ctypes.c_void_p
    sz = ctypes.c_size_t
    u64 = ctypes.c_uint64
    st = ctypes.POINTER(_Stats)
    lib.oracle_sort_u32.argtypes = [p, sz, u64, p, p, st]
    lib.oracle_sort_u64.argtypes = [p, sz, u64, p, p, st]
    lib.oracle_sort_fixed_decimal.argtypes = [p, sz, ctypes.c_int, ctypes.c_int, u64, p, p, st]
    lib.oracle_sort_strings.argtypes = [p, p, sz, ctypes.c_uint32, u64, p, st]
    lib.oracle_sort_f64.argtypes = [p, sz, u64, p, p, st]
    lib.oracle_sort_f64.restype = ctypes.c_int
    lib.oracle_decimal_hashing_cycle.argtypes = [p, sz, ctypes.c_int, ctypes.c_int, p,
                                                 ctypes.POINTER(ctypes.c_int), p, p, p,
                                                 ctypes.POINTER(ctypes.c_uint64)]
    for f in (lib.oracle_sort_u32, lib.oracle_sort_u64, lib.oracle_sort_fixed_decimal,
              lib.oracle_sort_strings, lib.oracle_decimal_hashing_cycle):
        f.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Run the wrappers against another build of the oracle (mutation tests)."""
    global _lib
    saved = _lib
    _lib = _configure(ctypes.CDLL(path))
    try:
        yield
    finally:
        _lib = saved


def _ptr(a: np.ndarray | None):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _stats(s: _Stats) -> Stats:
    return Stats(int(s.k), int(s.cycles), int(s.dims), int(s.top_cells), bool(s.regenerated))


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(rc, what)


def sort_u32(keys, cell_cap: int = 0, want_keys: bool = True):
    """Stable Recombinant Sort of uint32 keys -> (sorted_keys, perm, Stats)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    n = keys.size
    out = np.empty(n, np.uint32) if want_keys else None
    perm = np.empty(n, np.uint64)
    s = _Stats()
    _check(_load().oracle_sort_u32(_ptr(keys), n, cell_cap, _ptr(out), _ptr(perm), ctypes.byref(s)),
           "oracle_sort_u32")
    return out, perm, _stats(s)


def sort_u64(keys, cell_cap: int = 0, want_keys: bool = True):
    """Stable Recombinant Sort of uint64 keys -> (sorted_keys, perm, Stats)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    n = keys.size
    out = np.empty(n, np.uint64) if want_keys else None
    perm = np.empty(n, np.uint64)
    s = _Stats()
    _check(_load().oracle_sort_u64(_ptr(keys), n, cell_cap, _ptr(out), _ptr(perm), ctypes.byref(s)),
           "oracle_sort_u64")
    return out, perm, _stats(s)


def sort_fixed_decimal(keys, int_digits: int, frac_digits: int, cell_cap: int = 0,
                       want_keys: bool = True):
    """Stable Recombinant Sort of int64 fixed-point decimals (scaled by 10^frac_digits)."""
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    n = keys.size
    out = np.empty(n, np.int64) if want_keys else None
    perm = np.empty(n, np.uint64)
    s = _Stats()
    _check(_load().oracle_sort_fixed_decimal(_ptr(keys), n, int_digits, frac_digits, cell_cap,
                                             _ptr(out), _ptr(perm), ctypes.byref(s)),
           "oracle_sort_fixed_decimal")
    return out, perm, _stats(s)


def sort_float(keys, cell_cap: int = 0, want_keys: bool = True):
    """Stable sort of float32/float64 keys (-0.0 ties +0.0, NaN last).

    float32 keys are widened to float64 first (exact and order-preserving;
    a signalling NaN widens to a quiet NaN, still a NaN).
    Returns (sorted keys in the input dtype, perm, Stats).
    """
    keys = np.asarray(keys)
    with np.errstate(invalid="ignore"):
        kd = np.ascontiguousarray(keys, dtype=np.float64)
    n = kd.size
    out = np.empty(n, np.float64) if want_keys else None
    perm = np.empty(n, np.uint64)
    s = _Stats()
    _check(_load().oracle_sort_f64(_ptr(kd), n, cell_cap, _ptr(out), _ptr(perm), ctypes.byref(s)),
           "oracle_sort_f64")
    if want_keys and keys.dtype == np.float32:
        out = keys[perm.astype(np.int64)]
    return out, perm, _stats(s)


def sort_strings(chars, offsets, max_len: int = 0, cell_cap: int = 0):
    """Stable Recombinant Sort of byte strings -> (perm, Stats).

    String i is ``chars[offsets[i]:offsets[i+1]]``.
    """
    chars = np.ascontiguousarray(chars, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = offsets.size - 1
    if n < 0:
        raise ValueError("offsets needs n+1 entries")
    perm = np.empty(n, np.uint64)
    s = _Stats()
    _check(_load().oracle_sort_strings(_ptr(chars if chars.size else np.zeros(1, np.uint8)),
                                       _ptr(offsets), n, max_len, cell_cap, _ptr(perm),
                                       ctypes.byref(s)),
           "oracle_sort_strings")
    return perm, _stats(s)


def sort_pairs(keys, values, **kw):
    """Stable key/value sort: the payload follows its key's permutation."""
    keys = np.asarray(keys)
    if keys.dtype == np.uint32:
        k, perm, st = sort_u32(keys, **kw)
    elif keys.dtype == np.uint64:
        k, perm, st = sort_u64(keys, **kw)
    else:
        raise TypeError(f"unsupported key dtype {keys.dtype}")
    return k, np.asarray(values)[perm.astype(np.int64)], st


def decimal_hashing_cycle(keys, int_digits: int, frac_digits: int):
    """One hashing cycle over fixed-point decimals whose digits fit one count array.

    Returns (S with the paper's shape, H_Max (rows,), H_Min (rows, 2), k).
    """
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    radix = np.zeros(32, np.uint32)
    rank = ctypes.c_int(0)
    _check(lib.oracle_decimal_hashing_cycle(_ptr(keys), keys.size, int_digits, frac_digits,
                                            _ptr(radix), ctypes.byref(rank), None, None, None,
                                            None), "oracle_decimal_hashing_cycle(shape)")
    shape = tuple(int(r) for r in radix[: rank.value])
    cells = int(np.prod(shape))
    rows = cells // shape[-1]
    S = np.zeros(cells, np.uint64)
    hmax = np.zeros(rows, np.uint32)
    hmin = np.zeros(2 * rows, np.uint32)
    k = ctypes.c_uint64(0)
    _check(lib.oracle_decimal_hashing_cycle(_ptr(keys), keys.size, int_digits, frac_digits, None,
                                            None, _ptr(S), _ptr(hmax), _ptr(hmin),
                                            ctypes.byref(k)), "oracle_decimal_hashing_cycle")
    return S.reshape(shape), hmax, hmin.reshape(rows, 2), int(k.value)


def decimal_space_shape(keys, int_digits: int, frac_digits: int):
    """Shape of the count array S for these decimals (one dimension per digit)."""
    lib = _load()
    keys = np.ascontiguousarray(keys, dtype=np.int64)
    radix = np.zeros(32, np.uint32)
    rank = ctypes.c_int(0)
    _check(lib.oracle_decimal_hashing_cycle(_ptr(keys), keys.size, int_digits, frac_digits,
                                            _ptr(radix), ctypes.byref(rank), None, None, None,
                                            None), "oracle_decimal_hashing_cycle(shape)")
    return tuple(int(r) for r in radix[: rank.value])


def stable_rank(keys: np.ndarray, i: int) -> int:
    """Output position of input element i under a stable ascending sort.

    The plain definition: the number of keys smaller than keys[i], plus the
    number of keys equal to it that come earlier in the input.  O(n) per call;
    used to check sampled outputs of very large sorts one by one.
    """
    k = keys[i]
    return int(np.count_nonzero(keys < k) + np.count_nonzero(keys[:i] == k))
