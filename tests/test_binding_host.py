"""Argument checks of the Python binding that run before any library call:
device arguments of smc_forward / smc_gradient must be contiguous float64
CUDA tensors of sufficient size, host buffers of smc_move_host contiguous
float64 host arrays (numpy or CPU tensors).  On CPU, with stand-in tensors for
the CUDA cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2503_16028_gb300 import smcgm  # noqa: E402


class _FakeCuda:
    """Quacks like a CUDA tensor for the checks (no device needed)."""

    def __init__(self, n, dtype=torch.float64, contiguous=True):
        self.is_cuda, self.dtype, self._n, self._c = True, dtype, n, contiguous

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n


def test_device_arguments():
    assert smcgm._device_f64(_FakeCuda(12), 12, "X") is not None
    with pytest.raises(ValueError, match="CUDA tensor"):
        smcgm._device_f64(torch.zeros(12, dtype=torch.float64), 12, "X")
    with pytest.raises(ValueError, match="CUDA tensor"):
        smcgm._device_f64(np.zeros(12), 12, "X")
    with pytest.raises(ValueError, match="float64"):
        smcgm._device_f64(_FakeCuda(12, dtype=torch.float32), 12, "X")
    with pytest.raises(ValueError, match="contiguous"):
        smcgm._device_f64(_FakeCuda(12, contiguous=False), 12, "X")
    with pytest.raises(ValueError, match="13 needed"):
        smcgm._device_f64(_FakeCuda(12), 13, "X")


def test_host_arguments():
    a = np.zeros((3, 4))
    assert smcgm._host_f64(a, 12, "X") is a
    t = torch.zeros((3, 4), dtype=torch.float64)
    assert smcgm._host_f64(t, 12, "X") is t
    with pytest.raises(ValueError, match="host memory"):
        smcgm._host_f64(_FakeCuda(12), 12, "X")
    with pytest.raises(ValueError, match="float64"):
        smcgm._host_f64(np.zeros(12, dtype=np.float32), 12, "X")
    with pytest.raises(ValueError, match="contiguous"):
        smcgm._host_f64(np.zeros((3, 8))[:, ::2], 12, "X")
    with pytest.raises(ValueError, match="contiguous"):
        smcgm._host_f64(torch.zeros((3, 8), dtype=torch.float64)[:, ::2], 12, "X")
    with pytest.raises(ValueError, match="13 needed"):
        smcgm._host_f64(a, 13, "X")
