"""Host-side argument checks of the Python binding that run before any launch (CPU)."""
import pytest
import torch

from paper_2604_05065_gb300 import aplicur as api


def _check(A, x, y=None):
    api._check_noalloc_args(torch, A, x, y)


def test_noalloc_rejects_half_precision_matrices():
    for dt in (torch.float16, torch.bfloat16, torch.int32):
        with pytest.raises(TypeError):
            _check(torch.zeros(4, 3, dtype=dt), torch.zeros(4, dtype=torch.float64))


def test_noalloc_rejects_wrong_vector_sizes():
    A = torch.zeros(5, 3, dtype=torch.float32)
    with pytest.raises(ValueError, match="x must"):
        _check(A, torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="y must"):
        _check(A, torch.zeros(5, dtype=torch.float64), torch.zeros(2, dtype=torch.float64))
    with pytest.raises(TypeError, match="y must be float64"):
        _check(A, torch.zeros(5, dtype=torch.float64), torch.zeros(3, dtype=torch.float32))


def test_noalloc_rejects_non_row_major_and_host_matrices():
    A = torch.zeros(3, 5, dtype=torch.float64).t()
    with pytest.raises(ValueError, match="row-major"):
        _check(A, torch.zeros(5, dtype=torch.float64))
    with pytest.raises(ValueError, match="CUDA"):
        _check(torch.zeros(5, 3, dtype=torch.float64), torch.zeros(5, dtype=torch.float64))
