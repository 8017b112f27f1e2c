"""Pins of the oracle's full-covariance mixtures (pcngm with Mixture.cov,
gm.fit_full): the diagonal special case, detailed balance against the
mixture proposal densities written out, the single-component closed form of
EM, and recovery of a correlated two-component mixture."""
import numpy as np
import pytest

from oracle import gm, pcngm


def _spd(r, rng, scale):
    A = rng.standard_normal((r, r)) * 0.4
    return scale * (A @ A.T + np.eye(r))


def _mix(d, r, K, seed, full=True):
    rng = np.random.default_rng(seed)
    lam0 = (1.0 + 0.3 * np.arange(d)) ** -2.0
    S = np.arange(r)
    w = rng.dirichlet(np.ones(K) * 2)
    m = rng.standard_normal((K, r)) * np.sqrt(lam0[S]) * 0.6
    cov = np.stack([_spd(r, rng, 0.3 * lam0[0]) for _ in range(K)])
    lam = np.stack([np.diag(c) for c in cov])
    return pcngm.Mixture(S, w, m, lam, lam0, cov=cov if full else None)


def _log_gauss_full(x, mean, C):
    dev = x - mean
    _, logdet = np.linalg.slogdet(2 * np.pi * C)
    return float(-0.5 * logdet - 0.5 * dev @ np.linalg.solve(C, dev))


def test_diagonal_covariance_is_the_diagonal_kernel():
    mix = _mix(7, 4, 3, 1)
    diag = pcngm.Mixture(mix.S, mix.w, mix.m, mix.lam, mix.lam0)
    full = pcngm.Mixture(mix.S, mix.w, mix.m, mix.lam, mix.lam0, cov=np.stack([np.diag(l) for l in mix.lam]))
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal(7), rng.standard_normal(7)
    assert np.allclose(pcngm.log_r(b, a, full, 0.4), pcngm.log_r(b, a, diag, 0.4), rtol=1e-12, atol=1e-12)
    z = rng.standard_normal(7)
    assert np.allclose(pcngm.propose(a, 1, z, full, 0.4), pcngm.propose(a, 1, z, diag, 0.4), rtol=0, atol=1e-14)


@pytest.mark.parametrize("beta", [0.3, 0.8, 1.0])
def test_ratio_equals_direct_mixture_densities(beta):
    d, r, K = 7, 4, 3
    mix = _mix(d, r, K, 5)
    g = pcngm.gamma_of(beta)
    S, off = mix.S, np.arange(r, d)

    def log_q(a, b):              # log sum_j w_j N(b; gamma a + (1-gamma) m_j, beta^2 (C_j + diag lambda off S))
        terms = []
        for j in range(K):
            mean = g * a.copy()
            mean[S] += (1 - g) * mix.m[j]
            C = np.zeros((d, d))
            C[np.ix_(S, S)] = beta ** 2 * mix.cov[j]
            C[off, off] = beta ** 2 * mix.lam0[off]
            terms.append(np.log(mix.w[j]) + _log_gauss_full(b, mean, C))
        return pcngm.logsumexp(np.array(terms))

    log_pi0 = lambda x: _log_gauss_full(x, np.zeros(d), np.diag(mix.lam0))
    rng = np.random.default_rng(6)
    for _ in range(4):
        u = np.sqrt(mix.lam0) * rng.standard_normal(d)
        v = np.sqrt(mix.lam0) * rng.standard_normal(d)
        direct = (log_pi0(v) + log_q(v, u)) - (log_pi0(u) + log_q(u, v))
        assert pcngm.log_mixture_ratio(u, v, mix, beta) == pytest.approx(direct, rel=1e-10, abs=1e-10)


def test_single_component_is_sample_mean_and_covariance():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((500, 6)) @ np.diag([1.0, 0.5, 0.3, 0.2, 0.1, 0.05])
    X[:, 1] += 0.4 * X[:, 0]
    S = np.arange(4)
    lam0 = np.linspace(1.0, 0.2, 6)
    mix, _ = gm.fit_full(X, S, lam0, 1, 3, seed=1, layer=0, var_floor=1e-3)
    xs = X[:, S]
    mean = xs.mean(axis=0)
    cov = (xs - mean).T @ (xs - mean) / xs.shape[0] + np.diag(1e-3 * lam0[S])
    assert np.allclose(mix.m[0], mean, atol=1e-14)
    assert np.allclose(mix.cov[0], cov, atol=1e-14)
    assert mix.w[0] == 1.0


def test_recovers_correlated_mixture_and_loglik_monotone():
    rng = np.random.default_rng(4)
    N = 20000
    C1 = np.array([[0.04, 0.03], [0.03, 0.05]])
    C2 = np.array([[0.03, -0.02], [-0.02, 0.04]])
    lab = rng.random(N) < 0.35
    X = np.where(lab[:, None], rng.multivariate_normal([1.0, 0.0], C1, N), rng.multivariate_normal([-1.0, 0.5], C2, N))
    mix, hist = gm.fit_full(X, np.arange(2), np.array([1.0, 1.0]), 2, 40, seed=2, layer=0, var_floor=1e-6)
    assert np.all(np.diff(hist) > -1e-8 * np.abs(hist[1:]))
    j1 = int(np.argmin(np.abs(mix.m[:, 0] - 1.0)))
    j2 = 1 - j1
    assert mix.w[j1] == pytest.approx(0.35, abs=0.01)
    assert np.allclose(mix.m[j1], [1.0, 0.0], atol=0.01) and np.allclose(mix.m[j2], [-1.0, 0.5], atol=0.01)
    assert np.allclose(mix.cov[j1], C1, atol=0.004) and np.allclose(mix.cov[j2], C2, atol=0.004)


def test_full_e_step_against_scipy_densities():
    """Responsibilities g_nj = w_j N(x_n; m_j, C_j) / sum_k w_k N(x_n; m_k, C_k) and the
    log-likelihood sum_n log sum_j w_j N(x_n; m_j, C_j), with the densities from scipy."""
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(8)
    N, r, K = 40, 5, 3
    xs = rng.standard_normal((N, r))
    w = rng.dirichlet(np.ones(K))
    m = 0.5 * rng.standard_normal((K, r))
    cov = np.stack([_spd(r, rng, 0.8) for _ in range(K)])
    g, ll = gm.e_step_full(xs, w, m, cov)
    dens = np.stack([w[j] * stats.multivariate_normal(m[j], cov[j]).pdf(xs) for j in range(K)], axis=1)
    assert np.allclose(g, dens / dens.sum(axis=1, keepdims=True), rtol=1e-12, atol=1e-15)
    assert ll == pytest.approx(float(np.sum(np.log(dens.sum(axis=1)))), rel=1e-12)
