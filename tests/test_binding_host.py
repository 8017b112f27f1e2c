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


def test_concurrent_builds_use_private_objects(tmp_path, monkeypatch):
    """Two builds at once (threads standing in for processes): no object file is written by
    both, the library ends up in place, and the private directories are removed."""
    import concurrent.futures as cf
    import os
    import subprocess
    import threading
    import time
    from paper_2503_16028_gb300 import build
    monkeypatch.setattr(build, "BUILD", str(tmp_path / "_build"))
    monkeypatch.setattr(build, "LIB", str(tmp_path / "libsmcgm.so"))
    monkeypatch.setattr(build, "nvcc", lambda: "nvcc")
    written, lock = [], threading.Lock()

    def fake_run(cmd, capture_output=True, text=True):
        out = cmd[cmd.index("-o") + 1]
        with lock:
            written.append(out)
        time.sleep(0.005)
        with open(out, "w") as fh:
            fh.write("x")
        return subprocess.CompletedProcess(cmd, 0, "", "")

    monkeypatch.setattr(build.subprocess, "run", fake_run)
    with cf.ThreadPoolExecutor(2) as ex:
        libs = list(ex.map(lambda _: build.build(force=True), range(2)))
    objs = [o for o in written if o.endswith(".o")]
    assert len(objs) == 2 * len(build.sources()) and len(set(objs)) == len(objs)
    assert libs == [build.LIB, build.LIB] and os.path.exists(build.LIB)
    assert os.listdir(build.BUILD) == []


def test_choose_solve_batch():
    """The largest batch whose workspace fits the budget: a workspace of base + B * per bytes."""
    base, per, N = 1000, 37, 4096
    size = lambda b: base + b * per
    assert smcgm.choose_solve_batch(size, N, size(N)) == N
    assert smcgm.choose_solve_batch(size, N, 10 ** 12) == N
    for budget in (size(1), size(2) - 1, size(777), size(777) + per - 1, size(N) - 1):
        b = smcgm.choose_solve_batch(size, N, budget)
        assert size(b) <= budget and (b == N or size(b + 1) > budget), (budget, b)
    with pytest.raises(MemoryError):
        smcgm.choose_solve_batch(size, N, size(1) - 1)
