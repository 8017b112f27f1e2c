"""pCN-GM transition kernel of Sec. 2.3 (Alg. 2) in truncated KL coordinates.

Proposal (eq. pCN-GM proposal, component-wise reading):
  Q(u, .) = sum_j w_j N(gamma u + (1 - gamma) m_j, beta^2 C_j),  gamma = sqrt(1 - beta^2).
The printed proposal places the mixture weights on the shift sum_j w_j m_j;
the characteristic function in the proof of Thm 2 and the block means
[0, (1 - gamma) m_j] of Thm 2 (a) fix the per-component shift (1 - gamma) m_j,
which is the reading used here.  C_j shares the prior eigenfunctions
(eq. C_j phi_i = lambda_ji phi_i), so it is diagonal in KL coordinates.  The
mixture lives on a set S of r leading modes; outside S, m_j = 0 and
lambda_j = lambda (prior), so those coordinates follow the plain pCN move.

Acceptance (eqs. auv of pCN-GMM / -GMM2): with rho = exp(-t Phi) mu_0,
  a(u, v) = min{1, exp(t (Phi(u) - Phi(v))) * [mu_0(dv) Q(v, du)] / [mu_0(du) Q(u, dv)]}.
The mixture Radon-Nikodym factor (eqs. auv of pCN-GMM3/4, Thm 2) is computed
in the prior-relative form: the base pCN kernel q0(b|a) = N(gamma a, beta^2 C)
is mu_0-reversible, so
  mu_0(dv)Q(v,du) / mu_0(du)Q(u,dv) = sum_j w_j r_j(u|v) / sum_j w_j r_j(v|u),
  r_j(b|a) = N(e; (1-gamma) m_j, beta^2 C_j) / N(e; 0, beta^2 C),  e = b - gamma a,
  log r_j(b|a) = sum_{i in S} [ 1/2 log(lambda_i / lambda_ji)
                               - (e_i - (1-gamma) m_ji)^2 / (2 beta^2 lambda_ji)
                               + e_i^2 / (2 beta^2 lambda_i) ].
In finite dimension this equals the ratio of the two Gaussian-mixture densities
on H x H of Thm 2 (the tests check that by brute force).  M = 1, m = 0,
lambda_1 = lambda gives log-ratio 0 and a_pCN (eq. a in pCN).
"""
import numpy as np


def gamma_of(beta):
    return np.sqrt(1.0 - beta * beta)


def beta_from_delta(delta):
    """App. B: the Crank-Nicolson step delta maps to beta = sqrt(8 delta) / (2 + delta)."""
    return np.sqrt(8.0 * delta) / (2.0 + delta)


def logsumexp(a, axis=-1):
    a = np.asarray(a, dtype=np.float64)
    m = np.max(a, axis=axis, keepdims=True)
    return np.squeeze(m, axis=axis) + np.log(np.sum(np.exp(a - m), axis=axis))


class Mixture:
    """Gaussian mixture sum_j w_j N(m_j, C_j) in KL coordinates.

    S      : (r,) mode indices carrying the mixture
    w      : (K,) weights, sum 1
    m      : (K, r) means on S
    lam    : (K, r) eigenvalues lambda_ji of C_j on S
    lam0   : (d,) prior eigenvalues lambda_i
    """

    def __init__(self, S, w, m, lam, lam0, cov=None):
        self.S = np.asarray(S, dtype=np.int64)
        self.w = np.asarray(w, dtype=np.float64)
        self.m = np.asarray(m, dtype=np.float64)
        self.lam = np.asarray(lam, dtype=np.float64)
        self.lam0 = np.asarray(lam0, dtype=np.float64)
        # full covariances (K, r, r) on S, or None for the diagonal lambda_j of Sec. 2.3
        self.cov = None if cov is None else np.asarray(cov, dtype=np.float64)

    @property
    def K(self):
        return self.w.shape[0]

    @staticmethod
    def prior(lam0, S, K=1):
        """M components equal to the prior: the pCN special case."""
        r = len(S)
        return Mixture(S, np.full(K, 1.0 / K), np.zeros((K, r)),
                       np.tile(np.asarray(lam0)[S], (K, 1)), lam0)

    def copy(self):
        return Mixture(self.S.copy(), self.w.copy(), self.m.copy(), self.lam.copy(), self.lam0.copy(),
                       None if self.cov is None else self.cov.copy())


def choose_component(w, U):
    """j = min{j : U < w_1 + ... + w_j} (cumulative sum in index order); K-1 if none."""
    c = 0.0
    for j, wj in enumerate(w):
        c += wj
        if U < c:
            return j
    return len(w) - 1


def propose(u, j, z, mix, beta):
    """v = gamma u + (1 - gamma) m_j + beta sqrt(lambda_j) z  (eq. pCN-GM proposal);
    with full covariances, beta L_j z_S on S, C_j = L_j L_j^T (Cholesky)."""
    g = gamma_of(beta)
    v = g * u + beta * np.sqrt(mix.lam0) * z
    S = mix.S
    if mix.cov is not None:
        L = np.linalg.cholesky(mix.cov[j])
        v[S] = g * u[S] + (1.0 - g) * mix.m[j] + beta * (L @ z[S])
        return v
    v[S] = g * u[S] + (1.0 - g) * mix.m[j] + beta * np.sqrt(mix.lam[j]) * z[S]
    return v


def log_r(b, a, mix, beta):
    """(K,) array of log r_j(b|a) over the mixture modes S (module docstring)."""
    g = gamma_of(beta)
    S = mix.S
    e = b[S] - g * a[S]
    l0 = mix.lam0[S]
    out = np.empty(mix.K)
    if mix.cov is not None:
        # log N(e; (1-gamma) m_j, beta^2 C_j) - log N(e; 0, beta^2 diag(lambda_S)), written out
        for j in range(mix.K):
            C = beta * beta * mix.cov[j]
            dev = e - (1.0 - g) * mix.m[j]
            _, logdet = np.linalg.slogdet(C)
            out[j] = (-0.5 * logdet - 0.5 * dev @ np.linalg.solve(C, dev)
                      + 0.5 * np.sum(np.log(beta * beta * l0)) + np.sum(e * e / (2.0 * beta * beta * l0)))
        return out
    for j in range(mix.K):
        lj = mix.lam[j]
        out[j] = np.sum(0.5 * np.log(l0 / lj)
                        - (e - (1.0 - g) * mix.m[j]) ** 2 / (2.0 * beta * beta * lj)
                        + e * e / (2.0 * beta * beta * l0))
    return out


def log_mixture_ratio(u, v, mix, beta):
    """log [mu_0(dv) Q(v,du) / mu_0(du) Q(u,dv)]."""
    lw = np.log(mix.w)
    return logsumexp(lw + log_r(u, v, mix, beta)) - logsumexp(lw + log_r(v, u, mix, beta))


def log_alpha(t, phi_u, phi_v, log_ratio):
    """log of the MH ratio for rho = exp(-t Phi) mu_0 (eqs. auv of pCN-GMM / -GMM2)."""
    return t * (phi_u - phi_v) + log_ratio


def accept(log_a, U):
    """Accept iff U < min(1, alpha), tested as log U < log alpha."""
    return bool(log_a >= 0.0 or np.log(U) < log_a)


def log_density_kl(x, mix):
    """log of the mixture density relative to the prior on the modes S,
    log [sum_j w_j N(x_S; m_j, C_j) / N(x_S; 0, C)] (used by the beta = 1 check)."""
    S = mix.S
    xs = x[S]
    l0 = mix.lam0[S]
    terms = np.empty(mix.K)
    for j in range(mix.K):
        lj = mix.lam[j]
        terms[j] = np.log(mix.w[j]) + np.sum(0.5 * np.log(l0 / lj) - (xs - mix.m[j]) ** 2 / (2 * lj) + xs ** 2 / (2 * l0))
    return logsumexp(terms)
