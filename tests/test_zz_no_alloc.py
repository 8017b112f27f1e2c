"""The allocation-free resampling entry point (smc_resample_indices_static) gives
the same indices as the context-based smc_resample(), and the oracle's systematic
indices at the metric workload's 4096 particles and at its cap of 32768.

Callers that cannot give the library device memory -- an application whose own
pool owns all device memory, or a loop that must not risk cudaMalloc's implicit
synchronisation -- use the static variant, whose scratch is a fixed device array
inside the library.  This file sorts last so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build, smcgm
    build.build()
    return smcgm.load_library()


def test_static_resampling_matches_context_resampling_twice(lib):
    from paper_2503_16028_gb300 import inputs, smcgm
    wl = inputs.load_workload("darcy64_bimodal")
    N = 300
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N))
    s.smc_temper_step()
    s.smc_resample()
    _, _, _, logw_ptr, idx_ptr = s.diagnostics_pointers()
    ref = s.to_host(idx_ptr, N, np.int32)
    assert ref.min() >= 0 and ref.max() < N and np.all(np.diff(ref) >= 0)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # two calls in a row share the static scratch
        out.fill_(-1)
        st = lib.smc_resample_indices_static(ctypes.c_void_p(logw_ptr), N, wl["seed"], 0,
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == smcgm.SMC_OK, lib.smc_last_error(None)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
    s.close()


def test_static_resampling_rejects_oversize(lib):
    from paper_2503_16028_gb300 import smcgm
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    st = lib.smc_resample_indices_static(ctypes.c_void_p(out.data_ptr()), smcgm.SMC_STATIC_RESAMPLE_MAX + 1, 1, 0,
                                         ctypes.c_void_p(out.data_ptr()), None)
    assert st == smcgm.SMC_EINVAL
    assert b"SMC_STATIC_RESAMPLE_MAX" in lib.smc_last_error(None)


@pytest.mark.parametrize("N", [4096, 32768])
def test_static_resampling_matches_oracle_at_scale(lib, N):
    """Seeded log weights with a tie for the largest weight, a run of equal weights and one
    dominant weight, at layer 7, twice in a row: the indices equal the oracle's systematic
    indices (after checking that no systematic point is a near-tie)."""
    from paper_2503_16028_gb300 import inputs, smcgm
    from oracle import smc as osmc
    assert N <= smcgm.SMC_STATIC_RESAMPLE_MAX == 32768
    seed, layer = 2503016028, 7
    logw = inputs.structured_log_weights(N + 3, N)
    u48 = osmc.resample_u48(seed, layer)
    assert osmc.resampling_near_ties(logw, u48) == []
    ref = osmc.systematic_indices(logw, u48)
    d_logw = torch.tensor(logw, dtype=torch.float64, device="cuda")
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out.fill_(-1)
        st = lib.smc_resample_indices_static(ctypes.c_void_p(d_logw.data_ptr()), N, seed, layer,
                                             ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert st == smcgm.SMC_OK, lib.smc_last_error(None)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref)
