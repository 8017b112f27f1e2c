"""pCN-Langevin mutation: the Langevin equation of App. B with its drift kept.

App. B starts from du/ds = -K (L u + gamma D Phi(u)) + sqrt(2K) db/ds with
L = C^{-1}, K = C and drops the drift (gamma = 0) to reach the pCN(-GM)
proposal; Sec. 1 and Sec. 2.4 cite the pCN Langevin kernel without giving it.
Keeping the drift for the tempered target pi_t(du) ~ exp(-t Phi(u)) mu0(du)
(so gamma = t), and discretising the linear part by Crank-Nicolson and the
drift explicitly, as App. B does for the rest:

  (1 + delta/2) v = (1 - delta/2) u - delta t C DPhi(u) + sqrt(2 delta) C^{1/2} z,

and with beta = sqrt(8 delta)/(2 + delta) (App. B's step), gamma_b =
sqrt(1 - beta^2) = (2 - delta)/(2 + delta), 2 delta/(2 + delta) = 1 - gamma_b:

  v = gamma_b u - (1 - gamma_b) t C DPhi(u) + beta C^{1/2} z,   z ~ N(0, I).

Metropolis-Hastings against pi_t.  The drift-free kernel q0(u, .) =
N(gamma_b u, beta^2 C) is mu0-reversible, so the ratio reduces to
Cameron-Martin terms that stay finite in infinite dimensions:

  log alpha = t (Phi(u) - Phi(v)) + rho(v, u) - rho(u, v),
  rho(a, b) = log q(a, b) - log q0(a, b)
            = -(1 - gamma_b) t <g_a, b - gamma_b a> / beta^2
              - (1 - gamma_b)^2 t^2 <g_a, C g_a> / (2 beta^2),

with g_a = DPhi(a) in KL coordinates, C = diag(lambda).  With g = 0 (or
t = 0) this is the pCN kernel and its acceptance t (Phi(u) - Phi(v)).
Random numbers: the normals and the accept uniform of the pCN-GM move
(Philox purposes NORMAL and ACCEPT with the same counters).

GMpCN-Langevin (a definition: the paper gives neither Langevin kernel).  The
pCN-GM proposal of Sec. 2.3 with the same drift, preconditioned by the
drawn component's covariance:

  v = gamma u + (1 - gamma) m_j - (1 - gamma) t C_j DPhi(u) + beta C_j^{1/2} z,

C_j = diag(lambda_j) on the mixture modes S and C elsewhere.  Against the
mu0-reversible pCN kernel the acceptance is

  log alpha = t (Phi(u) - Phi(v)) + log sum_j w_j R_j(v, u) - log sum_j w_j R_j(u, v),
  R_j(a, b) = N(b; gamma a + (1-gamma) m_j - (1-gamma) t C_j DPhi(a), beta^2 C_j)
              / N(b; gamma a, beta^2 C)      (over all d modes).

With DPhi = 0 it is the pCN-GM kernel; with one prior component, pCN-Langevin.
"""
import numpy as np

from . import pcngm, philox


def gamma_of(beta):
    return np.sqrt(1.0 - beta * beta)


def propose(x, g, lam, beta, t, z):
    """v = gamma u - (1 - gamma) t C g + beta C^{1/2} z."""
    gm = gamma_of(beta)
    return gm * x - (1.0 - gm) * t * lam * g + beta * np.sqrt(lam) * z


def rho(a, b, g_a, lam, beta, t):
    """log q(a, b) - log q0(a, b) for the drift shift -(1 - gamma) t C g_a."""
    gm = gamma_of(beta)
    k = (1.0 - gm) * t
    return -k * float(g_a @ (b - gm * a)) / beta ** 2 - k * k * float(g_a @ (lam * g_a)) / (2.0 * beta ** 2)


def log_alpha(x, v, phi_x, phi_v, g_x, g_v, lam, beta, t):
    return t * (phi_x - phi_v) + rho(v, x, g_v, lam, beta, t) - rho(x, v, g_x, lam, beta, t)


def move_particle(x, phi_x, g_x, lam, beta, t, seed, n, step, potential_and_gradient):
    """One pCN-Langevin step for particle n; returns (x', phi', g', accepted, log_alpha, phi_v).

    potential_and_gradient(v) -> (Phi(v), DPhi(v))."""
    z = philox.normals(seed, x.shape[0], n, step, philox.NORMAL)
    v = propose(x, g_x, lam, beta, t, z)
    phi_v, g_v = potential_and_gradient(v)
    la = log_alpha(x, v, phi_x, phi_v, g_x, g_v, lam, beta, t)
    Ua = float(philox.uniforms(seed, 0, n, step, philox.ACCEPT))
    if pcngm.accept(la, Ua):
        return v, phi_v, g_v, True, la, phi_v
    return x, phi_x, g_x, False, la, phi_v


def _component_lams(mix, j):
    """(mean shift (1-gamma) m_j and variance factors lambda_j) as full d-vectors."""
    lamj = mix.lam0.copy()
    lamj[mix.S] = mix.lam[j]
    mj = np.zeros_like(mix.lam0)
    mj[mix.S] = mix.m[j]
    return mj, lamj


def gm_propose(x, g, j, z, mix, beta, t):
    """v = gamma u + (1 - gamma) m_j - (1 - gamma) t C_j g + beta C_j^{1/2} z."""
    gm = gamma_of(beta)
    mj, lamj = _component_lams(mix, j)
    return gm * x + (1.0 - gm) * mj - (1.0 - gm) * t * lamj * g + beta * np.sqrt(lamj) * z


def gm_log_R(b, a, g_a, mix, beta, t):
    """(K,) log R_j(a, b), every mode written out."""
    gm = gamma_of(beta)
    out = np.empty(mix.K)
    base = gm * a
    q0 = -0.5 * np.sum((b - base) ** 2 / (beta ** 2 * mix.lam0) + np.log(beta ** 2 * mix.lam0))
    for j in range(mix.K):
        mj, lamj = _component_lams(mix, j)
        mean = base + (1.0 - gm) * mj - (1.0 - gm) * t * lamj * g_a
        out[j] = -0.5 * np.sum((b - mean) ** 2 / (beta ** 2 * lamj) + np.log(beta ** 2 * lamj)) - q0
    return out


def gm_log_alpha(x, v, phi_x, phi_v, g_x, g_v, mix, beta, t):
    lw = np.log(mix.w)
    return (t * (phi_x - phi_v) + pcngm.logsumexp(lw + gm_log_R(x, v, g_v, mix, beta, t))
            - pcngm.logsumexp(lw + gm_log_R(v, x, g_x, mix, beta, t)))


def gm_move_particle(x, phi_x, g_x, mix, beta, t, seed, n, step, potential_and_gradient):
    """One GMpCN-Langevin step (component draw, normals and accept uniform as in the pCN-GM move)."""
    Uc = float(philox.uniforms(seed, 0, n, step, philox.COMP))
    j = pcngm.choose_component(mix.w, Uc)
    z = philox.normals(seed, x.shape[0], n, step, philox.NORMAL)
    v = gm_propose(x, g_x, j, z, mix, beta, t)
    phi_v, g_v = potential_and_gradient(v)
    la = gm_log_alpha(x, v, phi_x, phi_v, g_x, g_v, mix, beta, t)
    Ua = float(philox.uniforms(seed, 0, n, step, philox.ACCEPT))
    if pcngm.accept(la, Ua):
        return v, phi_v, g_v, True, la, phi_v
    return x, phi_x, g_x, False, la, phi_v
