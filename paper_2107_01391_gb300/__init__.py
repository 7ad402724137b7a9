"""GB300-native Recombinant Sort (Kumar et al., arXiv 2107.01391).

The sorting path is a C-ABI CUDA library (``include/rs.h``); ``binding``
marshals torch tensors into its calls.  Nothing here computes on the CPU.
"""
