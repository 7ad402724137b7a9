"""One entry point for the library's sorts: ``sort(keys, values=None, segments=None)``.

It picks the C-ABI call from its arguments and marshals the tensors; every
step of the sort runs in the library's CUDA kernels.  There is no CPU path:
keys that are not on a CUDA device raise.

* one array, keys only: ``rs_sort_u32`` (4-byte integer keys),
  ``rs_sort_u64`` (8-byte integer keys), ``rs_sort_fixed_decimal``
  (``decimal=(int_digits, frac_digits)``), or the keys-only form of
  ``rs_sort_pairs`` (float32/float64 keys);
* one array with values: ``rs_sort_pairs``;
* ``segments`` (an int for that many equal segments, or an int64 CUDA tensor
  of num_segs+1 offsets), or ``argsort=True``: ``rs_sort_segmented``, every
  segment a bucket of its own (§2.2).

Integer keys compare as unsigned numbers of their width (int32 -1 sorts last);
float keys compare as numbers, -0.0 ties with +0.0 and is written as +0.0,
NaNs sort last.  Every sort is stable.

``SortFn.apply(x)`` is the differentiable row sort of ``autograd``.
"""
from __future__ import annotations

import torch

from . import autograd, binding

SortFn = autograd.RSSortFunction

_INT4 = (torch.int32, torch.uint32)
_INT8 = (torch.int64, torch.uint64)
_FLOAT = (torch.float32, torch.float64)


def sort(keys: torch.Tensor, values: torch.Tensor | None = None, segments=None, *,
         decimal: tuple[int, int] | None = None, argsort: bool = False,
         index_dtype=torch.int64, ctx: binding.Context | None = None, stream=None):
    """Stable ascending sort of a contiguous 1-D CUDA tensor.

    Returns the sorted keys, or (sorted keys, values in the same order) when
    ``values`` is given, or (sorted keys, index of each key within its
    segment) when ``argsort`` is set.
    """
    if not isinstance(keys, torch.Tensor) or not keys.is_cuda:
        raise TypeError("keys must be a CUDA tensor: the library has no CPU path")
    if keys.dim() != 1:
        raise ValueError("keys must be 1-D (reshape rows into segments instead)")
    if values is not None and argsort:
        raise ValueError("give values or argsort, not both")
    if decimal is not None and keys.dtype != torch.int64:
        raise TypeError("decimal keys are int64 values scaled by 10^frac_digits")
    if keys.dtype not in _INT4 + _INT8 + _FLOAT:
        raise TypeError(f"unsupported key dtype {keys.dtype}")

    if segments is not None or argsort:
        if segments is None:
            segments = 1
        if isinstance(segments, int):
            if segments < 1 or keys.numel() % segments:
                raise ValueError("equal segments must divide the key count")
            return binding.rs_sort_segmented(keys, None, values, num_segs=segments,
                                             argsort=argsort, index_dtype=index_dtype,
                                             decimal=decimal, ctx=ctx, stream=stream)
        return binding.rs_sort_segmented(keys, segments, values, argsort=argsort,
                                         index_dtype=index_dtype, decimal=decimal, ctx=ctx,
                                         stream=stream)

    if values is not None:
        return binding.rs_sort_pairs(keys, values, decimal=decimal, ctx=ctx, stream=stream)
    if decimal is not None:
        return binding.rs_sort_fixed_decimal(keys, decimal[0], decimal[1], ctx=ctx, stream=stream)
    if keys.dtype in _INT4:
        return binding.rs_sort_u32(keys, ctx=ctx, stream=stream)
    if keys.dtype in _INT8:
        return binding.rs_sort_u64(keys, ctx=ctx, stream=stream)
    return binding.rs_sort_pairs(keys, None, ctx=ctx, stream=stream)[0]


def sort_strings(chars: torch.Tensor, offsets: torch.Tensor, max_len: int, *,
                 ctx: binding.Context | None = None, stream=None) -> torch.Tensor:
    """Stable permutation of byte strings (``rs_sort_strings``): string i is
    ``chars[offsets[i]:offsets[i+1]]``; returns perm (int32 holding uint32
    indices), perm[j] = input index of the j-th smallest string."""
    return binding.rs_sort_strings(chars, offsets, max_len, ctx=ctx, stream=stream)
