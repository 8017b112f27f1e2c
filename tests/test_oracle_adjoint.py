"""Pins of the oracle's adjoint gradient (oracle/adjoint.py) against what the
mathematics fixes: the observation matrix reproduces the observation
operator, the analysis is the exact transpose of the synthesis, and the
gradient matches central finite differences of the oracle's own potential,
both on the grid (per cell, walls and corners included) and in KL
coordinates (random directions)."""
import numpy as np
import pytest

from oracle import adjoint, darcy, observe, prior, problem
import scipy.sparse.linalg as spla


def _problem(n=16, Km=8, nobs=12, seed=7):
    rng = np.random.default_rng(seed)
    obs = rng.uniform(0.03, 0.97, size=(nobs, 2))
    obs[0] = (0.01, 0.5)          # near the west wall: ghost cells in the interpolation
    obs[1] = (0.99, 0.995)        # near the north-east corner
    data = rng.normal(0.0, 0.05, nobs)
    return problem.Problem(dim=2, n=n, kl_modes=Km, alpha=0.02, sigma=0.02, source_kind=1, src_amp=10.0,
                           src_width=50.0, obs=obs, data=data)


def _phi_of_u(prob, u):
    n = prob.n
    w = darcy.solve_2d(u, prob.f)
    y = observe.observe_2d(w, prob.obs)
    return float(observe.potential(y, prob.data, prob.sigma))


def test_observation_matrix_matches_operator():
    prob = _problem()
    rng = np.random.default_rng(1)
    O = adjoint.observation_matrix_2d(prob.n, prob.obs)
    for _ in range(3):
        w = rng.standard_normal((prob.n, prob.n))
        assert np.allclose(O @ w.ravel(), observe.observe_2d(w, prob.obs), rtol=0, atol=1e-14)


def test_analysis_is_transpose_of_synthesis():
    rng = np.random.default_rng(2)
    n, Km = 16, 8
    x = rng.standard_normal(Km * Km)
    g = rng.standard_normal((n, n))
    lhs = float(np.sum(prior.synthesize_2d(x, n, Km) * g))
    rhs = float(x @ adjoint.analysis_2d(g, Km))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def test_grid_gradient_matches_finite_differences_per_cell():
    prob = _problem()
    n = prob.n
    x = np.sqrt(prob.lam) * np.random.default_rng(3).standard_normal(prob.d)
    u = prob.field(x)
    kc = np.exp(u)
    A = darcy.assemble_2d(kc)
    lu = spla.splu(A)
    w = lu.solve((prob.f / (n * n)).ravel())
    O = adjoint.observation_matrix_2d(n, prob.obs)
    lam = lu.solve(O.T @ (O @ w - prob.data) / prob.sigma ** 2)
    g = adjoint.grad_u_from_adjoint(kc, w.reshape(n, n), lam.reshape(n, n))
    eps = 1e-6
    cells = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (0, 5), (7, 0), (n - 1, 9), (4, n - 1), (6, 9), (11, 3)]
    for (j, i) in cells:
        up, um = u.copy(), u.copy()
        up[j, i] += eps
        um[j, i] -= eps
        fd = (_phi_of_u(prob, up) - _phi_of_u(prob, um)) / (2 * eps)
        assert abs(fd - g[j, i]) <= 1e-6 * np.abs(g).max(), (j, i, fd, g[j, i])


@pytest.mark.parametrize("seed", [4, 5])
def test_kl_gradient_matches_finite_differences(seed):
    prob = _problem(seed=seed)
    rng = np.random.default_rng(seed)
    x = np.sqrt(prob.lam) * rng.standard_normal(prob.d)
    phi, grad, _, _ = adjoint.potential_and_gradient_2d(prob, x)
    assert abs(phi - prob.potential(x)) <= 1e-12 * phi
    eps = 1e-6
    for _ in range(6):
        e = rng.standard_normal(prob.d)
        e /= np.linalg.norm(e)
        fd = (prob.potential(x + eps * e) - prob.potential(x - eps * e)) / (2 * eps)
        assert abs(fd - grad @ e) <= 1e-6 * np.linalg.norm(grad), (fd, grad @ e)
