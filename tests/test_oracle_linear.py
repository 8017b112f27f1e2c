"""Whole-method pins for the oracle's SMC driver (Alg. 1 + Alg. 2): a linear
forward map has a closed-form Gaussian posterior (Sec. 2.1 with linear F),
and Phi = 0 leaves the prior invariant with a_pCN = 1 (eq. a in pCN)."""
import numpy as np

from oracle import prior, smc


class LinearProblem:
    def __init__(self, d, G, data, sigma, alpha=0.01):
        self.lam = prior.eigenvalues_1d(d, alpha)
        self.G = G
        self.data = data
        self.sigma = sigma

    def gm_modes(self, r):
        return np.arange(min(r, self.lam.shape[0]))

    def potential(self, v):
        r = self.G @ v - self.data
        return float(r @ r / (2 * self.sigma ** 2))


def test_linear_forward_map_matches_gaussian_posterior():
    rng = np.random.default_rng(0)
    d = 6
    lam = prior.eigenvalues_1d(d, 0.01)
    G = rng.standard_normal((3, d))
    sigma = 0.4
    truth = np.sqrt(lam) * rng.standard_normal(d)
    data = G @ truth + sigma * rng.standard_normal(3)
    prob = LinearProblem(d, G, data, sigma)
    P = np.diag(1 / lam) + G.T @ G / sigma ** 2
    cov = np.linalg.inv(P)
    mean = cov @ G.T @ data / sigma ** 2
    N = 2000
    out = smc.run(prob, N=N, K=2, r=d, L=8, beta0=0.5, ess_frac=0.5, seed=42, em_iters=20)
    assert out["t"] == 1.0
    m, v = smc.posterior_moments(out["X"])
    se = np.sqrt(np.diag(cov) / (N / 4))
    assert np.all(np.abs(m - mean) < 5 * se), (m, mean, se)
    assert np.all(np.abs(v / np.diag(cov) - 1) < 0.25), (v, np.diag(cov))


def test_zero_potential_pcn_accepts_everything_and_keeps_prior():
    class Zero(LinearProblem):
        def potential(self, v):
            return 0.0
    d = 4
    prob = Zero(d, np.zeros((1, d)), np.zeros(1), 1.0)
    out = smc.run(prob, N=3000, K=1, r=d, L=5, beta0=0.5, ess_frac=0.5, seed=3, kernel="pcn")
    assert len(out["layers"]) == 1 and out["layers"][0]["acc"] == 1.0
    m, v = smc.posterior_moments(out["X"])
    lam = prob.lam
    assert np.all(np.abs(m) < 5 * np.sqrt(lam / 3000))
    assert np.all(np.abs(v / lam - 1) < 0.1)
