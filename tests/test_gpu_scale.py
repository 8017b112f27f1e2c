"""Parity at the sizes the product runs, through the C ABI, against the FP64 oracle.

The single-block kernels of the layer step (tempering, resampling, the EM fit) give
each of their 1024 threads a contiguous chunk of ceil(N / 1024) particles.  At the
metric workload's N = 4096 a chunk holds 4 particles, at the library's cap of 32768
it holds 32: the per-chunk sums, the per-chunk argmax with its cross-chunk tie rule,
the remainder fix-up and the chunk scan all run there and are compared here.

* Tempering and resampling at N = 4096 and 32768 on seeded potentials with ties for
  the largest weight, a run of equal weights and one dominant weight, at a nonzero
  layer (the resampling uniform depends on it).
* The metric workload's own first layer (256^2, N = 4096, K = 8, r = 64, 50 EM
  iterations): temperature, indices, gathered particles and the fitted mixture.
* A 512^2 grid (the largest the library accepts: the cosine-transform block at its
  shared-memory limit, one more multigrid level): initial potentials and one pCN-GM
  move of 2 particles, in every precision of the solver (FP64, FP32 + refinement, and
  FP32 + refinement with the BF16 smoother).

Resampling indices must be identical.  Weights come from floating-point exponentials,
so each test first asks the oracle for the systematic points within 64 CDF units of a
CDF boundary (near-ties, where two correct implementations may differ) and requires
there to be none, as the accept tests require no accept near-ties.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402
from oracle import problem as oproblem, smc as osmc, gm as ogm, pcngm as opcngm  # noqa: E402

NEAR_TIE = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("N", [4096, 32768])
def test_temper_and_resample_at_scale(N):
    wl = inputs.load_workload("darcy64_bimodal")
    cfg = smcgm.make_config(wl, n_particles=N, n_components=2, solve_batch=4096)
    s = smcgm.Sampler(cfg)
    X, _ = s.particles()
    Phi = inputs.structured_potentials(17 + N, N)
    s.smc_set_particles(X, Phi)
    layer, t = 5, 0.3
    s.smc_set_schedule(t, 0.2, layer, 0)
    h, ess, lz, done = s.smc_temper_step()
    ref_h = osmc.bisect_h(Phi, t, cfg.ess_frac * N)
    assert abs(h - ref_h) <= 1e-9 * ref_h
    assert abs(ess - osmc.ess_of_h(Phi, h)) <= 1e-9 * ess
    assert ess >= cfg.ess_frac * N
    assert abs(lz - osmc.log_z_increment(Phi, h)) <= 1e-9 * max(1.0, abs(lz))
    logw = s.diagnostics()["logw"]
    ref_logw = -h * Phi - opcngm.logsumexp(-h * Phi)
    assert np.max(np.abs(logw - ref_logw)) <= 1e-12 * max(1.0, np.max(np.abs(ref_logw)))
    s.smc_resample()
    u48 = osmc.resample_u48(wl["seed"], layer)
    assert osmc.resampling_near_ties(-h * Phi, u48) == []
    idx = s.diagnostics()["indices"]
    ref_idx = osmc.systematic_indices(-h * Phi, u48)
    assert np.array_equal(idx, ref_idx)
    X2, Phi2 = s.particles()
    assert np.array_equal(X2, X[ref_idx]) and np.array_equal(Phi2, Phi[ref_idx])
    s.close()


def test_metric_workload_first_layer_matches_oracle():
    """256^2, N = 4096, K = 8, r = 64, 50 EM iterations (the bench's configuration)."""
    wl = inputs.load_workload("darcy256_precision")
    cfg = smcgm.make_config(wl)
    assert (cfg.n_particles, cfg.n_components, cfg.gm_rank, cfg.em_iters) == (4096, 8, 64, 50)
    s = smcgm.Sampler(cfg)
    N = cfg.n_particles
    X, Phi = s.particles()
    h, ess, lz, done = s.smc_temper_step()
    ref_h = osmc.bisect_h(Phi, 0.0, cfg.ess_frac * N)
    assert abs(h - ref_h) <= 1e-9 * ref_h
    assert abs(lz - osmc.log_z_increment(Phi, h)) <= 1e-9 * max(1.0, abs(lz))
    s.smc_resample()
    u48 = osmc.resample_u48(wl["seed"], 0)
    assert osmc.resampling_near_ties(-h * Phi, u48) == []
    ref_idx = osmc.systematic_indices(-h * Phi, u48)
    assert np.array_equal(s.diagnostics()["indices"], ref_idx)
    X2, Phi2 = s.particles()
    assert np.array_equal(Phi2, Phi[ref_idx])
    ll = s.gm_fit()
    prob = oproblem.from_workload(wl)
    S = prob.gm_modes(cfg.gm_rank)
    mix, hist = ogm.fit(X2[:, S], np.arange(len(S)), prob.lam[S], 8, 50, wl["seed"], 0, var_floor=cfg.var_floor)
    w, m, lam, modes = s.smc_get_mixture()
    assert np.array_equal(modes, S)
    assert np.allclose(w, mix.w, rtol=1e-7, atol=1e-12)
    assert np.allclose(m, mix.m, rtol=1e-7, atol=1e-9 * np.sqrt(np.max(prob.lam)))
    assert np.allclose(lam, mix.lam, rtol=1e-7, atol=1e-14)
    assert abs(ll - hist[-1]) <= 1e-8 * abs(hist[-1])
    s.close()


@pytest.mark.parametrize("precision", [smcgm.SMC_P_FP64, smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE])
def test_grid_512_init_and_move(precision):
    wl = dict(inputs.load_workload("darcy256_precision"))
    wl["n"] = 512
    N = 2
    cfg = smcgm.make_config(wl, n_particles=N, n_components=2, precision=precision)
    s = smcgm.Sampler(cfg)
    prob = oproblem.from_workload(wl)
    X, Phi = s.particles()
    for n in range(N):
        assert _rel(X[n], osmc.prior_draw(wl["seed"], prob.lam, n)) < 1e-14
        ref = prob.potential(X[n])
        assert abs(Phi[n] - ref) <= 1e-10 * abs(ref), (n, Phi[n], ref)
    w, m, lam, modes = s.smc_get_mixture()
    rng = np.random.default_rng(512)
    w = np.array([0.4, 0.6])
    m = rng.standard_normal(m.shape) * np.sqrt(lam) * 0.5
    s.smc_set_mixture(w, m, lam)
    mix = opcngm.Mixture(modes, w, m, lam, prob.lam)
    t, beta, step = 0.05, 0.2, 3
    s.smc_set_schedule(t, beta, 0, step)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    for n in range(N):
        x, ph, acc, la, pv = osmc.move_particle(X[n], Phi[n], mix, beta, t, wl["seed"], n, step, prob.potential)
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv), (n, dg["phi_proposed"][n], pv)
        U = float(osmc.philox.uniforms(wl["seed"], 0, n, step, osmc.philox.ACCEPT))
        assert abs(np.log(U) - la) >= NEAR_TIE
        assert bool(dg["accepted"][n]) == bool(acc)
        assert _rel(X2[n], x) < 1e-13
        assert abs(Phi2[n] - ph) <= 1e-10 * abs(ph)
    s.close()
