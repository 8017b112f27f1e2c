"""The C ABI library builds, loads and exports every entry point that
include/smcgm.h declares; host-only calls (no GPU work) behave as documented."""
import ctypes
import os
import re
import shutil

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc unavailable")
    from paper_2503_16028_gb300 import build, smcgm
    build.build()
    return smcgm.load_library()


def _declared():
    src = open(os.path.join(ROOT, "include", "smcgm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(smc_[a-z_0-9]+|gm_fit)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2503_16028_gb300 import smcgm
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in smcgm.EXPORTS, "binding lacks " + n


def test_config_layout_and_defaults(lib):
    from paper_2503_16028_gb300 import smcgm
    assert lib.smc_config_size() == ctypes.sizeof(smcgm.smc_config)
    cfg = smcgm.smc_config()
    assert lib.smc_config_init(ctypes.byref(cfg)) == 0
    assert cfg.dim == 2 and cfg.smooth_sweeps == 2 and cfg.coarse_scale == 2.0


def test_workspace_size_and_validation(lib):
    from paper_2503_16028_gb300 import inputs, smcgm
    wl = inputs.load_workload("darcy256_precision")
    cfg = smcgm.make_config(wl)
    size = ctypes.c_size_t()
    assert lib.smc_workspace_size(ctypes.byref(cfg), ctypes.byref(size)) == 0
    n, N = 256, 4096
    # at least: particles (3 N d FP64) + FP64 coefficients/solution + FP32 CG vectors
    assert size.value > 3 * N * 128 * 128 * 8 + 4 * N * n * n * 8 + 7 * N * n * n * 4
    assert size.value < 64 << 30
    bad = smcgm.make_config(wl, n=200)
    assert lib.smc_workspace_size(ctypes.byref(bad), ctypes.byref(size)) == smcgm.SMC_EINVAL
    # the largest 2D grid is 512^2 (the cosine-transform block's shared memory)
    ok = smcgm.make_config(wl, n=512)
    assert lib.smc_workspace_size(ctypes.byref(ok), ctypes.byref(size)) == 0
    bad = smcgm.make_config(wl, n=1024)
    assert lib.smc_workspace_size(ctypes.byref(bad), ctypes.byref(size)) == smcgm.SMC_EINVAL
    assert b"512" in lib.smc_last_error(None)
    bad = smcgm.make_config(wl, n_particles=40000)
    assert lib.smc_workspace_size(ctypes.byref(bad), ctypes.byref(size)) == smcgm.SMC_EINVAL
    bad = smcgm.make_config(wl, n_particles=1)           # a single particle's weights carry no information
    assert lib.smc_workspace_size(ctypes.byref(bad), ctypes.byref(size)) == smcgm.SMC_EINVAL
    assert b"n_particles" in lib.smc_last_error(None)
    obs = np.array([[0.5, 1.5]])
    bad = smcgm.make_config(dict(wl, obs=obs, data=np.zeros(1)))
    assert lib.smc_workspace_size(ctypes.byref(bad), ctypes.byref(size)) == smcgm.SMC_EINVAL


def test_init_rejects_small_workspace_without_touching_the_gpu(lib):
    from paper_2503_16028_gb300 import inputs, smcgm
    wl = inputs.load_workload("darcy64_bimodal")
    cfg = smcgm.make_config(wl)
    ctx = ctypes.c_void_p()
    assert lib.smc_init(ctypes.byref(cfg), ctypes.c_void_p(256), 1024, None, ctypes.byref(ctx)) == smcgm.SMC_ENOMEM
    assert b"workspace" in lib.smc_last_error(None)
    assert lib.smc_temper_step(None, None, None, None, None) == smcgm.SMC_EINVAL


def test_batch_calls_reject_null_arguments_without_touching_the_gpu(lib):
    from paper_2503_16028_gb300 import smcgm
    out = ctypes.c_void_p()
    assert lib.smc_batch_create(None, 1, 1, ctypes.byref(out)) == smcgm.SMC_EINVAL
    assert lib.smc_batch_move(None, None) == smcgm.SMC_EINVAL
    assert lib.smc_batch_move_host(None, None, None, None, None, None) == smcgm.SMC_EINVAL
    lib.smc_batch_destroy(None)                     # a no-op


def test_default_solve_batch_is_capped_at_2_28_cells(lib):
    """solve_batch = 0 leaves the batch to the library: all particles, up to 2^28 grid cells per
    batch (4096 particles at 256^2, 1024 at 512^2); the workspace shows which batch was planned."""
    from paper_2503_16028_gb300 import inputs, smcgm
    wl = inputs.load_workload("darcy256_precision")
    size = ctypes.c_size_t()

    def ws(**over):
        cfg = smcgm.make_config(wl, **over)
        assert lib.smc_workspace_size(ctypes.byref(cfg), ctypes.byref(size)) == 0
        return size.value
    assert ws(n_particles=16384, solve_batch=0) == ws(n_particles=16384, solve_batch=4096)
    assert ws(n_particles=16384, solve_batch=0) < ws(n_particles=16384, solve_batch=8192)
    assert ws(n_particles=2048, solve_batch=0) == ws(n_particles=2048, solve_batch=2048)
    assert ws(n=512, n_particles=4096, solve_batch=0) == ws(n=512, n_particles=4096, solve_batch=1024)
