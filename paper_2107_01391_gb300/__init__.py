"""GB300-native Recombinant Sort (Kumar et al., arXiv 2107.01391).

The sorting path is a C-ABI CUDA library (``include/rs.h``); ``binding``
marshals torch tensors into its calls.  Nothing here computes on the CPU.

``sort(keys, values=None, segments=None)``, ``sort_strings`` and ``SortFn``
(the differentiable row sort) are the torch-level entry points (``api``).
"""

_API = ("sort", "sort_strings", "SortFn")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
