"""The warp-tile kernels' index arithmetic and launch resources, checked on the
CPU: tests/kernel_geometry.cu includes the kernels' headers, is compiled with
nvcc as an ordinary host program and run (it makes no CUDA call).  It checks
that every quad of a smoothing region is owned exactly once, that the TMA boxes
start on 16-byte boundaries, cover the region and sit 128-byte aligned, and
that the shared memory of the resident blocks each launch asks for fits an SM."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_kernel_geometry(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "kernel_geometry")
    build = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-o", exe, os.path.join(HERE, "kernel_geometry.cu")], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and "kernel geometry ok" in run.stdout, run.stdout + run.stderr
