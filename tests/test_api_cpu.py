"""The torch-level entry point refuses what it cannot run on the GPU: there is
no CPU path, so CPU tensors and malformed arguments raise before any call."""
import pytest
import torch

import paper_2107_01391_gb300 as rs


def test_cpu_tensors_raise():
    with pytest.raises(TypeError, match="CUDA"):
        rs.sort(torch.arange(10, dtype=torch.int32))
    with pytest.raises(TypeError, match="CUDA"):
        rs.sort(torch.randn(10), torch.arange(10))


def test_api_names():
    assert callable(rs.sort) and callable(rs.sort_strings)
    assert issubclass(rs.SortFn, torch.autograd.Function)
    with pytest.raises(AttributeError):
        rs.no_such_name  # noqa: B018
