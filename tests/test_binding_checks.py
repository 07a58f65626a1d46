"""Argument checks of the Python binding that run before any call into the
C ABI (CPU only): a tensor of the wrong dtype, layout, device or length
would make the library's kernels read or write out of bounds, so the
binding refuses it first."""
import pytest
import torch

from paper_2112_03851_gb300._lib import check_local_vector


def test_accepts_a_matching_vector():
    check_local_vector(torch.zeros(10, dtype=torch.float64), 10, torch.device("cpu"), "x")


@pytest.mark.parametrize("bad, why", [
    (torch.zeros(10, dtype=torch.float32), "float64"),
    (torch.zeros(9, dtype=torch.float64), "10 values"),
    (torch.zeros(20, dtype=torch.float64)[::2], "contiguous"),
    (torch.zeros((2, 5), dtype=torch.float64).t(), "contiguous"),
    ([0.0] * 10, "torch tensor"),
])
def test_refuses_wrong_vectors(bad, why):
    with pytest.raises((ValueError, TypeError), match=why):
        check_local_vector(bad, 10, torch.device("cpu"), "x")


def test_refuses_a_vector_on_another_device():
    with pytest.raises(ValueError, match="must be on"):
        check_local_vector(torch.zeros(10, dtype=torch.float64), 10, torch.device("cuda", 0), "y")
