"""Whole SMC-pCN-GM runs on the 2D Darcy workload (64^2, mirror-pair data) on the GPU.

* Parity: the run of Alg. 1 with Alg. 2 as mutation, from the prior to t = 1, in FP64
  and in both mixed-precision modes (FP32 + refinement, with FP32 or BF16 smoother
  faces), against the oracle's own run (96 particles, K = 4, L = 10, 50 EM
  iterations): every layer's temperature increment and acceptance rate, the log
  evidence, and the final particles and potentials.  The oracle's run is computed once
  for all precisions.
* The mirror invariant of this workload: the observation points come in pairs
  (x, y) / (1 - x, y) with pair-averaged data, and the prior, the source and the grid
  are symmetric under x -> 1 - x, so Phi(Ru) = Phi(u) for the reflection R, which flips
  the sign of every KL coefficient with odd k (cos(k pi (1 - x)) = (-1)^k cos(k pi x)).
  The posterior is R-invariant and its mean vanishes on odd-k coefficients.  The SMC
  estimate of that mean is checked to be zero within 4 Monte Carlo standard errors,
  the standard errors taken from the spread of independent runs (different seeds) of
  the full workload (1024 particles).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2503_16028_gb300 import inputs, smcgm  # noqa: E402
from oracle import problem as oproblem, smc as osmc  # noqa: E402

N_PARITY = 96


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_16028_gb300 import build
    build.build()
    smcgm.load_library()


@pytest.fixture(scope="module")
def oracle_run():
    wl = inputs.load_workload("darcy64_bimodal")
    prob = oproblem.from_workload(wl)
    return osmc.run(prob, N=N_PARITY, K=wl["n_components"], r=wl["gm_rank"], L=wl["mcmc_steps"], beta0=wl["beta0"],
                    ess_frac=wl["ess_frac"], seed=wl["seed"], em_iters=50, max_layers=100)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.mark.parametrize("precision", [smcgm.SMC_P_FP64, smcgm.SMC_P_FP32_REFINE, smcgm.SMC_P_BF16SMOOTH_REFINE])
def test_darcy64_full_run_matches_oracle(oracle_run, precision):
    wl = inputs.load_workload("darcy64_bimodal")
    cfg = smcgm.make_config(wl, n_particles=N_PARITY, em_iters=50, precision=precision)
    s = smcgm.Sampler(cfg)
    ref = oracle_run
    assert ref["t"] == 1.0
    logz = 0.0
    for k, lay in enumerate(ref["layers"]):
        h, ess, lz, done = s.smc_temper_step()
        logz += lz
        assert abs(h - lay["h"]) <= 1e-9 * lay["h"], (k, h, lay["h"])
        assert done == (k == len(ref["layers"]) - 1)
        s.smc_resample()
        s.gm_fit()
        acc, _ = s.smc_move(wl["mcmc_steps"])
        assert abs(acc - lay["acc"]) < 1e-12, (k, acc, lay["acc"])
    assert abs(logz - ref["logZ"]) <= 1e-9 * abs(ref["logZ"])
    X, Phi = s.particles()
    assert _rel(X, ref["X"]) < 1e-10
    assert _rel(Phi, ref["Phi"]) < 1e-10
    s.close()


def _posterior_mean(seed):
    wl = inputs.load_workload("darcy64_bimodal")
    cfg = smcgm.make_config(wl, seed=seed)
    assert (cfg.n_particles, cfg.n_components) == (1024, 4)
    s = smcgm.Sampler(cfg)
    done = False
    layers = 0
    while not done:
        _, _, _, done = s.smc_temper_step()
        s.smc_resample()
        s.gm_fit()
        s.smc_move(wl["mcmc_steps"])
        layers += 1
        assert layers < 200
    mean, _ = s.smc_posterior_moments()
    s.close()
    return mean


def test_mirror_invariant_posterior_mean_of_odd_modes():
    wl = inputs.load_workload("darcy64_bimodal")
    Km = wl["kl_modes"]
    prob = oproblem.from_workload(wl)
    # the three odd-k coefficients of largest prior variance: (k, l) = (1, 0), (1, 1), (1, 2)
    odd = [1 * Km + 0, 1 * Km + 1, 1 * Km + 2]
    even = [0, 1, 2 * Km]            # (0, 0), (0, 1), (2, 0): left free
    assert all(prob.lam[i] > 0.01 for i in odd)
    means = np.array([_posterior_mean(wl["seed"] + 1000 * s) for s in range(8)])
    M = means.mean(axis=0)
    se = means.std(axis=0, ddof=1) / np.sqrt(means.shape[0])
    assert np.all(se[odd] > 0)
    z = M[odd] / se[odd]
    assert np.all(np.abs(z) < 4.0), (M[odd], se[odd], z)
    # the statistic is not vacuous: the data move the even-k means away from the prior's 0
    assert np.max(np.abs(M[even]) / se[even]) > 4.0
