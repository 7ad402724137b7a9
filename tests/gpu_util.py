"""Helpers for the GPU tests: move numpy arrays to CUDA tensors and back
bit-for-bit (unsigned keys travel as signed torch tensors of the same width)."""
import numpy as np
import torch

_TO_TORCH = {np.dtype(np.uint32): np.int32, np.dtype(np.int32): np.int32,
             np.dtype(np.uint64): np.int64, np.dtype(np.int64): np.int64,
             np.dtype(np.float32): np.float32, np.dtype(np.float64): np.float64,
             np.dtype(np.uint8): np.uint8}


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(_TO_TORCH[a.dtype])).cuda()


def from_dev(t: torch.Tensor, dtype) -> np.ndarray:
    return t.cpu().numpy().view(dtype)


def require_gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
