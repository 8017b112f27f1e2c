"""Full-covariance mixtures (cfg.full_cov) against the oracle (oracle/gm.py
fit_full, oracle/pcngm.py with Mixture.cov, pinned by direct densities):
the EM fit on resampled particles, a pCN-GM move and an independence move
with a given full-covariance mixture, and the checkpoint round trip."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402
from oracle import gm as ogm, pcngm as opcngm, problem as oproblem, smc as osmc  # noqa: E402

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


def test_full_covariance_em_matches_oracle():
    wl = inputs.load_workload("darcy64_bimodal")
    N, K, r, iters = 300, 3, 16, 15
    cfg = smcgm.make_config(wl, n_particles=N, n_components=K, gm_rank=r, em_iters=iters, full_cov=1)
    s = smcgm.Sampler(cfg)
    s.smc_temper_step()
    s.smc_resample()
    X2, _ = s.particles()
    ll = s.gm_fit()
    prob = oproblem.from_workload(wl)
    mix, hist = ogm.fit_full(X2, prob.gm_modes(r), prob.lam, K, iters, wl["seed"], 0, var_floor=cfg.var_floor)
    w, m, lam, modes = s.smc_get_mixture()
    cov = s.smc_get_mixture_cov()
    assert np.array_equal(modes, mix.S)
    assert np.allclose(w, mix.w, rtol=1e-7, atol=1e-12)
    assert _rel(m, mix.m) < 1e-7
    assert _rel(cov, mix.cov) < 1e-7
    assert np.allclose(lam, np.stack([np.diag(c) for c in cov]), rtol=0, atol=0)
    assert abs(ll - hist[-1]) <= 1e-8 * abs(hist[-1])
    s.close()


def _random_full_mixture(s, prob, K, rng):
    w, m, lam, modes = s.smc_get_mixture()
    r = len(modes)
    w = rng.dirichlet(np.ones(K) * 3)
    m = rng.standard_normal((K, r)) * np.sqrt(prob.lam[modes]) * 0.8
    cov = []
    for _ in range(K):
        A = rng.standard_normal((r, r)) * 0.3
        sd = np.sqrt(prob.lam[modes])
        cov.append(np.outer(sd, sd) * (A @ A.T / r + np.eye(r)) * rng.uniform(0.4, 1.2))
    cov = np.stack(cov)
    s.smc_set_mixture_cov(w, m, cov)
    return opcngm.Mixture(modes, w, m, np.stack([np.diag(c) for c in cov]), prob.lam, cov=cov)


@pytest.mark.parametrize("kernel", [smcgm.SMC_K_PCN_GM, smcgm.SMC_K_GM_INDEP])
def test_full_covariance_move_matches_oracle(kernel):
    wl = inputs.load_workload("darcy64_bimodal")
    N, K, r = 8, 3, 16
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=N, n_components=K, gm_rank=r, full_cov=1, kernel=kernel))
    prob = oproblem.from_workload(wl)
    mix = _random_full_mixture(s, prob, K, np.random.default_rng(17))
    X, Phi = s.particles()
    indep = kernel == smcgm.SMC_K_GM_INDEP
    t, beta, step = 0.05, (1.0 if indep else 0.3), 4
    s.smc_set_schedule(t, beta, 0, step)
    s.smc_move(1)
    X2, Phi2 = s.particles()
    dg = s.diagnostics()
    for n in range(N):
        x, ph, acc, la, pv = osmc.move_particle(X[n], Phi[n], mix, beta, t, wl["seed"], n, step, prob.potential,
                                                always_accept=indep)
        assert abs(dg["phi_proposed"][n] - pv) <= 1e-10 * abs(pv), n
        if not indep:
            assert abs(dg["log_alpha"][n] - la) <= 1e-8 * max(1.0, abs(la)), (n, dg["log_alpha"][n], la)
            U = float(osmc.philox.uniforms(wl["seed"], 0, n, step, osmc.philox.ACCEPT))
            if abs(np.log(U) - la) < NEAR_TIE:
                continue
        assert bool(dg["accepted"][n]) == bool(acc), n
        assert _rel(X2[n], x) < 1e-12, n
    s.close()


def test_full_covariance_checkpoint_roundtrip():
    wl = inputs.load_workload("darcy64_bimodal")
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=8, n_components=2, gm_rank=8, full_cov=1))
    prob = oproblem.from_workload(wl)
    _random_full_mixture(s, prob, 2, np.random.default_rng(3))
    cov = s.smc_get_mixture_cov()
    buf = s.smc_save()
    _random_full_mixture(s, prob, 2, np.random.default_rng(4))
    s.smc_load(buf)
    assert np.array_equal(s.smc_get_mixture_cov(), cov)
    s.close()


@pytest.mark.parametrize("N,K,r,iters", [(4096, 8, 64, 20), (1000, 3, 40, 10)])
def test_full_covariance_em_at_scale(N, K, r, iters):
    """The EM fit with full covariances at the metric workload's sizes (N = 4096, K = 8,
    r = 64: whole 32 x 32 tiles of the blocked covariance contraction, particle chunks of
    512) and at a ragged mode count (r = 40: a partial tile), against the oracle."""
    wl = inputs.load_workload("darcy64_bimodal")
    cfg = smcgm.make_config(wl, n_particles=N, n_components=K, gm_rank=r, em_iters=iters, full_cov=1, solve_batch=1024)
    s = smcgm.Sampler(cfg)
    s.smc_temper_step()
    s.smc_resample()
    X2, _ = s.particles()
    ll = s.gm_fit()
    prob = oproblem.from_workload(wl)
    mix, hist = ogm.fit_full(X2, prob.gm_modes(r), prob.lam, K, iters, wl["seed"], 0, var_floor=cfg.var_floor)
    w, m, lam, modes = s.smc_get_mixture()
    cov = s.smc_get_mixture_cov()
    assert np.allclose(w, mix.w, rtol=1e-7, atol=1e-12)
    assert _rel(m, mix.m) < 1e-7
    assert _rel(cov, mix.cov) < 1e-7
    assert np.array_equal(cov, np.swapaxes(cov, 1, 2))
    assert abs(ll - hist[-1]) <= 1e-8 * abs(hist[-1])
    s.close()


def test_covariance_that_is_not_positive_definite_is_rejected():
    """smc_set_mixture_cov with a C_j that is not positive definite: the device factorisation
    finds a pivot <= 0, the call returns SMC_EINVAL and the context holds no usable mixture
    (smc_move returns SMC_ESTATE) until a valid one is set."""
    wl = inputs.load_workload("darcy64_bimodal")
    s = smcgm.Sampler(smcgm.make_config(wl, n_particles=8, n_components=2, gm_rank=8, full_cov=1))
    prob = oproblem.from_workload(wl)
    mix = _random_full_mixture(s, prob, 2, np.random.default_rng(5))
    bad = mix.cov.copy()
    bad[1, 3, 3] = -1.0
    with pytest.raises(smcgm.SMCError) as ei:
        s.smc_set_mixture_cov(mix.w, mix.m, bad)
    assert ei.value.status == smcgm.SMC_EINVAL and "positive definite" in str(ei.value)
    s.smc_set_schedule(0.1, 0.2, 0, 0)
    with pytest.raises(smcgm.SMCError) as ei:
        s.smc_move(1)
    assert ei.value.status == smcgm.SMC_ESTATE
    _random_full_mixture(s, prob, 2, np.random.default_rng(6))
    s.smc_move(1)
    s.close()
