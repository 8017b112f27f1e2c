"""Pins of the oracle's pCN-Langevin kernel (oracle/langevin.py).

* Detailed balance written out with full Gaussian densities: for a quadratic
  potential with a closed-form gradient, log alpha(u, v) must equal
  [log pi_t(v) + log q(v, u)] - [log pi_t(u) + log q(u, v)] with
  pi_t = exp(-t Phi) N(0, C) and q(u, .) = N(gamma u - (1-gamma) t C DPhi(u),
  beta^2 C) evaluated directly (not through the prior-relative form).
* No drift (t = 0, or a zero gradient): the pCN proposal and acceptance.
* The Crank-Nicolson step: beta = sqrt(8 delta)/(2 + delta) gives
  gamma = (2 - delta)/(2 + delta) and a drift factor 2 delta/(2 + delta).
* The samplers against the densities: both proposals are affine in z, with
  the mean and the per-coordinate scale of the Gaussians the detailed-balance
  tests write out.
* The move's wiring: t = 0 accepts the Philox-driven proposal, a potential of
  +inf at the proposal rejects it and keeps the particle.
"""
import numpy as np
import pytest

from oracle import langevin, pcngm


def _quadratic(d, seed):
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((d + 2, d))
    y = rng.standard_normal(d + 2)
    phi = lambda x: 0.5 * float(np.sum((H @ x - y) ** 2))
    grad = lambda x: H.T @ (H @ x - y)
    return phi, grad


def _log_gauss(x, m, var):
    return float(-0.5 * np.sum((x - m) ** 2 / var) - 0.5 * np.sum(np.log(2 * np.pi * var)))


@pytest.mark.parametrize("t,beta", [(0.3, 0.2), (1.0, 0.5), (0.05, 0.9)])
def test_detailed_balance_direct_densities(t, beta):
    d = 6
    lam = (1.0 + 0.3 * np.arange(d)) ** -2.0
    phi, grad = _quadratic(d, 3)
    rng = np.random.default_rng(5)
    gm = np.sqrt(1 - beta ** 2)
    for _ in range(5):
        u = np.sqrt(lam) * rng.standard_normal(d)
        v = np.sqrt(lam) * rng.standard_normal(d)
        la = langevin.log_alpha(u, v, phi(u), phi(v), grad(u), grad(v), lam, beta, t)

        def log_pi(x):
            return -t * phi(x) + _log_gauss(x, 0.0, lam)

        def log_q(a, b):
            return _log_gauss(b, gm * a - (1 - gm) * t * lam * grad(a), beta ** 2 * lam)

        direct = (log_pi(v) + log_q(v, u)) - (log_pi(u) + log_q(u, v))
        assert abs(la - direct) <= 1e-10 * max(1.0, abs(direct)), (la, direct)


def test_no_drift_is_pcn():
    d = 5
    lam = np.linspace(1.0, 0.1, d)
    rng = np.random.default_rng(8)
    u, z = rng.standard_normal(d), rng.standard_normal(d)
    g = rng.standard_normal(d)
    beta = 0.3
    v0 = langevin.propose(u, g, lam, beta, 0.0, z)
    assert np.allclose(v0, np.sqrt(1 - beta ** 2) * u + beta * np.sqrt(lam) * z, rtol=0, atol=1e-15)
    v = langevin.propose(u, np.zeros(d), lam, beta, 0.7, z)
    assert np.array_equal(v, v0)
    la = langevin.log_alpha(u, v, 2.0, 1.5, np.zeros(d), np.zeros(d), lam, beta, 0.7)
    assert la == pytest.approx(0.7 * 0.5, abs=1e-15)


def test_crank_nicolson_step():
    for delta in (0.01, 0.2, 1.0, 1.9):          # delta <= 2: beta <= 1 and gamma >= 0
        beta = np.sqrt(8 * delta) / (2 + delta)
        gm = langevin.gamma_of(beta)
        assert gm == pytest.approx((2 - delta) / (2 + delta), rel=1e-13)
        assert 1 - gm == pytest.approx(2 * delta / (2 + delta), rel=1e-12)


def _mixture(d, r, K, seed):
    rng = np.random.default_rng(seed)
    lam0 = (1.0 + 0.3 * np.arange(d)) ** -2.0
    S = np.arange(r)
    w = rng.dirichlet(np.ones(K) * 2)
    m = rng.standard_normal((K, r)) * np.sqrt(lam0[S]) * 0.7
    lam = lam0[S] * rng.uniform(0.3, 1.5, size=(K, r))
    return pcngm.Mixture(S, w, m, lam, lam0)


@pytest.mark.parametrize("t,beta", [(0.3, 0.2), (1.0, 0.6)])
def test_gm_detailed_balance_direct_densities(t, beta):
    """GMpCN-Langevin: log alpha against the mixture proposal densities and the
    tempered posterior written out in full."""
    d, r, K = 7, 4, 3
    mix = _mixture(d, r, K, 9)
    lam = mix.lam0
    phi, grad = _quadratic(d, 4)
    gm = np.sqrt(1 - beta ** 2)
    rng = np.random.default_rng(12)

    def log_q(a, b):
        terms = []
        for j in range(K):
            lamj = lam.copy(); lamj[mix.S] = mix.lam[j]
            mj = np.zeros(d); mj[mix.S] = mix.m[j]
            mean = gm * a + (1 - gm) * mj - (1 - gm) * t * lamj * grad(a)
            terms.append(np.log(mix.w[j]) + _log_gauss(b, mean, beta ** 2 * lamj))
        return pcngm.logsumexp(np.array(terms))

    for _ in range(5):
        u = np.sqrt(lam) * rng.standard_normal(d)
        v = np.sqrt(lam) * rng.standard_normal(d)
        la = langevin.gm_log_alpha(u, v, phi(u), phi(v), grad(u), grad(v), mix, beta, t)
        direct = (-t * phi(v) + _log_gauss(v, 0.0, lam) + log_q(v, u)) - (-t * phi(u) + _log_gauss(u, 0.0, lam) + log_q(u, v))
        assert abs(la - direct) <= 1e-10 * max(1.0, abs(direct)), (la, direct)


def test_gm_special_cases():
    d, r = 6, 3
    lam0 = (1.0 + 0.3 * np.arange(d)) ** -2.0
    rng = np.random.default_rng(2)
    u, v, g_u, g_v = (rng.standard_normal(d) for _ in range(4))
    # one prior component: the pCN-Langevin kernel
    prior_mix = pcngm.Mixture.prior(lam0, np.arange(r), K=1)
    a = langevin.gm_log_alpha(u, v, 1.0, 0.5, g_u, g_v, prior_mix, 0.3, 0.4)
    b = langevin.log_alpha(u, v, 1.0, 0.5, g_u, g_v, lam0, 0.3, 0.4)
    assert a == pytest.approx(b, rel=1e-12, abs=1e-12)
    # zero drift: the pCN-GM kernel
    mix = _mixture(d, r, 2, 5)
    a = langevin.gm_log_alpha(u, v, 1.0, 0.5, g_u, g_v, mix, 0.3, 0.0)
    b = pcngm.log_alpha(0.0, 1.0, 0.5, pcngm.log_mixture_ratio(u, v, mix, 0.3))
    assert a == pytest.approx(b, rel=1e-12, abs=1e-12)


def test_propose_is_mean_plus_scaled_noise():
    """v is affine in z: z = 0 gives the drifted mean gamma u - (1 - gamma) t C g that the
    detailed-balance test writes into q(u, .), and z = e_i adds beta sqrt(lambda_i) e_i."""
    d = 6
    lam = (1.0 + 0.3 * np.arange(d)) ** -2.0
    rng = np.random.default_rng(21)
    u, g = rng.standard_normal(d), rng.standard_normal(d)
    beta, t = 0.4, 0.6
    gm = np.sqrt(1 - beta ** 2)
    mean = langevin.propose(u, g, lam, beta, t, np.zeros(d))
    assert np.allclose(mean, gm * u - (1 - gm) * t * lam * g, rtol=0, atol=1e-15)
    for i in range(d):
        e = np.zeros(d); e[i] = 1.0
        step = langevin.propose(u, g, lam, beta, t, e) - mean
        expect = np.zeros(d); expect[i] = beta * np.sqrt(lam[i])
        assert np.allclose(step, expect, rtol=0, atol=1e-15)


def test_gm_propose_is_component_mean_plus_scaled_noise():
    """The GMpCN-Langevin proposal from component j: z = 0 gives gamma u + (1 - gamma) m_j -
    (1 - gamma) t C_j g (m_j and C_j = diag(lambda_j) on S, 0 and the prior off S), and z = e_i
    adds beta sqrt(C_j,ii) e_i."""
    d, r, K = 7, 4, 3
    mix = _mixture(d, r, K, 13)
    rng = np.random.default_rng(22)
    u, g = rng.standard_normal(d), rng.standard_normal(d)
    beta, t = 0.5, 0.3
    gm = np.sqrt(1 - beta ** 2)
    for j in range(K):
        lamj = mix.lam0.copy(); lamj[:r] = mix.lam[j]
        mj = np.zeros(d); mj[:r] = mix.m[j]
        mean = langevin.gm_propose(u, g, j, np.zeros(d), mix, beta, t)
        assert np.allclose(mean, gm * u + (1 - gm) * mj - (1 - gm) * t * lamj * g, rtol=0, atol=1e-15)
        for i in range(d):
            e = np.zeros(d); e[i] = 1.0
            step = langevin.gm_propose(u, g, j, e, mix, beta, t) - mean
            assert step[i] == pytest.approx(beta * np.sqrt(lamj[i]), rel=1e-14)
            assert np.count_nonzero(np.abs(step) > 1e-15) == 1


def test_move_particle_accepts_and_rejects():
    """At t = 0 every proposal is accepted (log alpha = 0) and the new state is the proposal
    from the Philox normals; with a potential of +inf at the proposal (t > 0) it is rejected
    and the particle, its potential and gradient stay."""
    from oracle import philox
    d = 5
    lam = np.linspace(1.0, 0.2, d)
    x = np.linspace(-0.3, 0.4, d)
    g = np.ones(d)
    seed, n, step, beta = 7, 3, 2, 0.3
    z = philox.normals(seed, d, n, step, philox.NORMAL)
    v = langevin.propose(x, g, lam, beta, 0.0, z)
    x2, phi2, g2, acc, la, pv = langevin.move_particle(x, 1.0, g, lam, beta, 0.0, seed, n, step,
                                                       lambda y: (2.0, -y))
    assert acc and la == 0.0 and pv == 2.0 and phi2 == 2.0
    assert np.array_equal(x2, v) and np.array_equal(g2, -v)
    x3, phi3, g3, acc3, la3, _ = langevin.move_particle(x, 1.0, g, lam, beta, 0.5, seed, n, step,
                                                        lambda y: (np.inf, np.zeros(d)))
    assert not acc3 and la3 == -np.inf
    assert np.array_equal(x3, x) and phi3 == 1.0 and np.array_equal(g3, g)
