"""Independent problems run concurrently (one context, stream and host thread
each) give exactly the results they give run one by one; the autotuner
returns one of its candidates."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import batch, inputs, smcgm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()


def _configs():
    wl = inputs.load_workload("darcy64_bimodal")
    specs = [dict(n_particles=64, sigma=0.005, seed=11), dict(n_particles=128, sigma=0.01, seed=12),
             dict(n_particles=96, sigma=0.02, seed=13, n=128, kl_modes=32), dict(n_particles=64, sigma=0.008, seed=14)]
    return [smcgm.make_config(wl, n_components=2, em_iters=10, **sp) for sp in specs]


def test_concurrent_batch_equals_sequential():
    res_c, _ = batch.run_batch(batch.make_samplers(_configs()), mcmc_steps=3, max_layers=4, concurrent=True)
    torch.cuda.synchronize()
    res_s, _ = batch.run_batch(batch.make_samplers(_configs()), mcmc_steps=3, max_layers=4, concurrent=False)
    for a, b in zip(res_c, res_s):
        assert len(a["layers"]) == len(b["layers"])
        for la, lb in zip(a["layers"], b["layers"]):
            assert la == lb
        assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["Phi"], b["Phi"])


def test_autotune_returns_a_candidate():
    wl = inputs.load_workload("darcy64_bimodal")
    cands = (dict(), dict(smooth_sweeps=1))
    best, timings = batch.autotune(wl, candidates=cands, n_particles=64, steps=1, reps=1, n_components=2, em_iters=5)
    assert best in cands
    assert len(timings) == 2 and all(t > 0 for _, t in timings)


def test_mesh_independence_of_the_tempering_schedule():
    """Sec. 3.2 (mesh independence): the same prior, data and random streams on
    64^2 and 128^2 grids give the same number of layers and nearly the same
    temperatures (they differ only through the discretisation of Phi)."""
    wl = inputs.load_workload("darcy256_precision")
    temps, _ = batch.mesh_sweep(wl, [64, 128], n_particles=1024, kl_modes=32, mcmc_steps=10, max_layers=60,
                                n_components=8, em_iters=30)
    a, b = temps[64], temps[128]
    assert a[-1] == 1.0 and b[-1] == 1.0
    assert abs(len(a) - len(b)) <= 2, (len(a), len(b))
    for ta, tb in zip(a[:-3], b[:-3]):
        assert abs(ta - tb) <= 0.25 * max(ta, tb) + 1e-3, (a, b)
