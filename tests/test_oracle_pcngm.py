"""Pins for the pCN-GM kernel (Sec. 2.3, Thm 2, eqs. auv of pCN-GMM..GMM4, App. B)."""
import numpy as np
from scipy import stats

from oracle import pcngm, philox


def _random_mixture(rng, lam0, S, K):
    r = len(S)
    w = rng.dirichlet(np.ones(K))
    m = rng.standard_normal((K, r)) * np.sqrt(lam0[S])
    lam = lam0[S] * rng.uniform(0.2, 2.0, size=(K, r))
    return pcngm.Mixture(S, w, m, lam, lam0)


def _joint_blocks(mix, beta, j):
    """Thm 2 (a): component j of mu_0(du)Q(u,dv) and of mu_0(dv)Q(v,du) on H x H."""
    g = pcngm.gamma_of(beta)
    d = mix.lam0.shape[0]
    C = np.diag(mix.lam0)
    lj = mix.lam0.copy()
    lj[mix.S] = mix.lam[j]
    mj = np.zeros(d)
    mj[mix.S] = mix.m[j]
    Cj = np.diag(lj)
    V = np.block([[C, g * C], [g * C, beta ** 2 * Cj + g ** 2 * C]])
    Vp = np.block([[beta ** 2 * Cj + g ** 2 * C, g * C], [g * C, C]])
    mean = np.concatenate([np.zeros(d), (1 - g) * mj])
    meanp = np.concatenate([(1 - g) * mj, np.zeros(d)])
    return mean, V, meanp, Vp


def test_prior_mixture_gives_pcn():
    """M = 1, m = 0, C_1 = C: the ratio is 1 and a = a_pCN (eq. a in pCN)."""
    rng = np.random.default_rng(0)
    lam0 = rng.uniform(0.1, 1.0, 6)
    mix = pcngm.Mixture.prior(lam0, np.array([0, 2, 3]))
    for beta in (0.1, 0.5, 1.0):
        u, v = rng.standard_normal(6), rng.standard_normal(6)
        assert abs(pcngm.log_mixture_ratio(u, v, mix, beta)) < 1e-14


def test_ratio_equals_theorem2_block_gaussian_densities():
    """Brute force in H x H: log sum_j w_j rho'_j(u, v) - log sum_j w_j rho_j(u, v)."""
    rng = np.random.default_rng(1)
    for (d, S, K, beta) in [(3, [0, 1, 2], 3, 0.4), (4, [1, 3], 2, 0.7), (2, [0, 1], 4, 0.15), (3, [2], 2, 0.95)]:
        lam0 = rng.uniform(0.2, 1.5, d)
        mix = _random_mixture(rng, lam0, np.array(S), K)
        for _ in range(5):
            u, v = rng.standard_normal(d), rng.standard_normal(d)
            uv = np.concatenate([u, v])
            num, den = [], []
            for j in range(K):
                mean, V, meanp, Vp = _joint_blocks(mix, beta, j)
                num.append(np.log(mix.w[j]) + stats.multivariate_normal(meanp, Vp).logpdf(uv))
                den.append(np.log(mix.w[j]) + stats.multivariate_normal(mean, V).logpdf(uv))
            ref = pcngm.logsumexp(np.array(num)) - pcngm.logsumexp(np.array(den))
            got = pcngm.log_mixture_ratio(u, v, mix, beta)
            assert abs(got - ref) < 1e-11 * max(1.0, abs(ref)), (got, ref)


def test_block_covariance_eigenvalues_and_trace():
    """Per mode, V_j has eigenvalues (1 + gamma t^+-) lambda_i with t^+- from the proof of Thm 2;
    the trace of V_j is (1 + gamma^2) tr C + beta^2 tr C_j."""
    rng = np.random.default_rng(2)
    lam0 = rng.uniform(0.2, 1.5, 3)
    mix = _random_mixture(rng, lam0, np.array([0, 1, 2]), 2)
    beta = 0.6
    g = pcngm.gamma_of(beta)
    for j in range(2):
        _, V, _, _ = _joint_blocks(mix, beta, j)
        ev = np.sort(np.linalg.eigvalsh(V))
        mine = []
        for i in range(3):
            li, lji = lam0[i], mix.lam[j][i]
            a = beta ** 2 / (2 * g * li) * (lji - li)
            tp = a + np.sqrt(a * a + 1)
            tm = a - np.sqrt(a * a + 1)
            mine += [(1 + g * tp) * li, (1 + g * tm) * li]
        assert np.allclose(ev, np.sort(mine), rtol=1e-12)
        assert np.isclose(np.trace(V), (1 + g * g) * lam0.sum() + beta ** 2 * mix.lam[j].sum(), rtol=1e-13)


def test_beta_one_is_independence_sampler_ratio():
    """beta = 1: the ratio is [Q(u)/mu_0(u)] / [Q(v)/mu_0(v)] with Q = sum_j w_j N(m_j, C_j)."""
    rng = np.random.default_rng(3)
    lam0 = rng.uniform(0.2, 1.5, 4)
    S = np.array([0, 1, 2, 3])
    mix = _random_mixture(rng, lam0, S, 3)
    for _ in range(5):
        u, v = rng.standard_normal(4), rng.standard_normal(4)

        def logq_over_prior(x):
            q = [np.log(mix.w[j]) + stats.multivariate_normal(mix.m[j], np.diag(mix.lam[j])).logpdf(x) for j in range(3)]
            return pcngm.logsumexp(np.array(q)) - stats.multivariate_normal(np.zeros(4), np.diag(lam0)).logpdf(x)
        ref = logq_over_prior(u) - logq_over_prior(v)
        assert abs(pcngm.log_mixture_ratio(u, v, mix, 1.0) - ref) < 1e-11
        assert abs(pcngm.log_density_kl(u, mix) - logq_over_prior(u)) < 1e-11


def test_proposal_mean_and_components():
    rng = np.random.default_rng(4)
    lam0 = rng.uniform(0.2, 1.5, 5)
    mix = _random_mixture(rng, lam0, np.array([1, 4]), 2)
    u = rng.standard_normal(5)
    beta = 0.3
    g = pcngm.gamma_of(beta)
    v = pcngm.propose(u, 1, np.zeros(5), mix, beta)
    assert np.allclose(v[[0, 2, 3]], g * u[[0, 2, 3]])
    assert np.allclose(v[[1, 4]], g * u[[1, 4]] + (1 - g) * mix.m[1])
    U = philox.uniforms(8, np.arange(40000), 0, 0, philox.COMP)
    picks = np.array([pcngm.choose_component(mix.w, x) for x in U])
    assert abs(np.mean(picks == 0) - mix.w[0]) < 0.01


def test_beta_from_crank_nicolson_step():
    """App. B: beta = sqrt(8 delta)/(2 + delta) and gamma = (2 - delta)/(2 + delta) satisfy beta^2 + gamma^2 = 1."""
    for delta in (0.01, 0.3, 1.0, 2.0, 5.0):
        b = pcngm.beta_from_delta(delta)
        assert abs(b * b + ((2 - delta) / (2 + delta)) ** 2 - 1) < 1e-15


def test_kernel_leaves_prior_invariant_when_potential_is_zero():
    """Phi = 0: the pCN-GM chain started at mu_0 stays at mu_0 for any mixture (Sec. 2.3)."""
    rng = np.random.default_rng(5)
    lam0 = np.array([1.0, 0.4])
    S = np.array([0, 1])
    mix = pcngm.Mixture(S, np.array([0.5, 0.5]), np.array([[1.6, 0.0], [-1.6, 0.5]]),
                        np.array([[0.3, 0.2], [0.5, 0.1]]), lam0)
    M, steps, beta = 3000, 15, 0.8
    X = np.sqrt(lam0) * rng.standard_normal((M, 2))
    acc = 0
    for s in range(steps):
        for n in range(M):
            j = pcngm.choose_component(mix.w, rng.uniform())
            v = pcngm.propose(X[n], j, rng.standard_normal(2), mix, beta)
            la = pcngm.log_mixture_ratio(X[n], v, mix, beta)
            if pcngm.accept(la, rng.uniform()):
                X[n] = v
                acc += 1
    assert 0.05 < acc / (M * steps) < 0.95
    for i in range(2):
        assert stats.kstest(X[:, i] / np.sqrt(lam0[i]), "norm").pvalue > 1e-3


def test_accept_with_probability_min_one_alpha():
    """The Metropolis-Hastings rule: a move with ratio alpha is taken with probability
    min(1, alpha).  Over 40000 uniforms the accepted fraction matches it to 4 binomial
    standard deviations; concrete cases on either side of alpha = 0.3; alpha >= 1 always."""
    rng = np.random.default_rng(17)
    U = rng.random(40000)
    for alpha in (0.02, 0.3, 0.75, 1.0, 3.0):
        frac = np.mean([pcngm.accept(np.log(alpha), u) for u in U])
        p = min(1.0, alpha)
        assert abs(frac - p) <= 4 * np.sqrt(max(p * (1 - p), 1e-12) / U.size) + 1e-12, (alpha, frac)
    assert pcngm.accept(np.log(0.3), 0.2) and not pcngm.accept(np.log(0.3), 0.4)
    assert pcngm.accept(0.0, 0.999999) and pcngm.accept(2.0, 0.5)
    assert not pcngm.accept(-np.inf, 1e-300)


def test_component_draw_at_the_cumulative_boundaries():
    """j = min{j : U < w_1 + ... + w_j}: the intervals [c_{j-1}, c_j) are closed on the left,
    so a uniform exactly on a boundary (binary fractions make the sums exact) belongs to the
    next component; the last component takes the rest."""
    w = np.array([0.25, 0.25, 0.5])
    assert [pcngm.choose_component(w, u) for u in (0.0, 0.2499, 0.25, 0.4999, 0.5, 0.75, 0.9999)] == [0, 0, 1, 1, 2, 2, 2]
    assert pcngm.choose_component(np.array([0.5, 0.5]), 0.5) == 1


def test_log_alpha_is_detailed_balance_for_the_tempered_target():
    """log alpha(u, v) = [log pi_t(v) + log Q(v, u)] - [log pi_t(u) + log Q(u, v)] for the
    tempered target pi_t(x) ~ exp(-t Phi(x)) N(x; 0, C) and the mixture proposal
    Q(u, .) = sum_j w_j N(gamma u + (1 - gamma) m_j, beta^2 C_j), all densities written out
    (a quadratic Phi, so that Phi(u) and Phi(v) differ)."""
    rng = np.random.default_rng(23)
    d = 5
    lam0 = rng.uniform(0.2, 1.5, d)
    S = np.array([0, 1, 2])
    mix = _random_mixture(rng, lam0, S, 3)
    H = rng.standard_normal((4, d))
    phi = lambda x: 0.5 * float(np.sum((H @ x - 0.3) ** 2))
    for t, beta in ((0.2, 0.3), (0.9, 0.7)):
        g = pcngm.gamma_of(beta)

        def log_q(a, b):
            terms = []
            for j in range(3):
                lj = lam0.copy(); lj[S] = mix.lam[j]
                mean = g * a.copy(); mean[S] += (1 - g) * mix.m[j]
                terms.append(np.log(mix.w[j]) + stats.multivariate_normal(mean, beta ** 2 * np.diag(lj)).logpdf(b))
            return pcngm.logsumexp(np.array(terms))

        def log_pi(x):
            return -t * phi(x) + stats.multivariate_normal(np.zeros(d), np.diag(lam0)).logpdf(x)

        for _ in range(4):
            u, v = np.sqrt(lam0) * rng.standard_normal(d), np.sqrt(lam0) * rng.standard_normal(d)
            direct = (log_pi(v) + log_q(v, u)) - (log_pi(u) + log_q(u, v))
            la = pcngm.log_alpha(t, phi(u), phi(v), pcngm.log_mixture_ratio(u, v, mix, beta))
            assert abs(la - direct) <= 1e-10 * max(1.0, abs(direct)), (la, direct)
