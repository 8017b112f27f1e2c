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


def test_face_derivatives_against_central_differences():
    """The face coefficients are the harmonic means 2 k_a k_b / (k_a + k_b) (walls: 2 k_c), and
    each derivative with respect to u = log k is the central difference of those faces: a
    cell's own west/south face, its east/north neighbour's west/south face (as that face's
    neighbour), and the east/north wall faces of the last column/row; no other face moves."""
    rng = np.random.default_rng(31)
    n, eps = 6, 1e-6
    u = 0.7 * rng.standard_normal((n, n))
    k = np.exp(u)
    Kw, Ks, dWo, dWn, dSo, dSn, Ke, Kn = adjoint.face_derivatives(k)
    assert np.allclose(Kw[:, 1:], 2 * k[:, 1:] * k[:, :-1] / (k[:, 1:] + k[:, :-1]), rtol=1e-14, atol=0)
    assert np.allclose(Ks[1:, :], 2 * k[1:, :] * k[:-1, :] / (k[1:, :] + k[:-1, :]), rtol=1e-14, atol=0)
    assert np.array_equal(Kw[:, 0], 2 * k[:, 0]) and np.array_equal(Ks[0, :], 2 * k[0, :])
    assert np.array_equal(Ke, 2 * k[:, -1]) and np.array_equal(Kn, 2 * k[-1, :])
    for j, i in [(2, 3), (0, 0), (5, 5), (0, 4), (3, 0), (5, 1)]:
        up, um = u.copy(), u.copy()
        up[j, i] += eps
        um[j, i] -= eps
        P = adjoint.face_derivatives(np.exp(up))
        M = adjoint.face_derivatives(np.exp(um))
        dKw, dKs = (P[0] - M[0]) / (2 * eps), (P[1] - M[1]) / (2 * eps)
        dKe, dKn = (P[6] - M[6]) / (2 * eps), (P[7] - M[7]) / (2 * eps)
        ew, es = np.zeros((n, n)), np.zeros((n, n))
        ew[j, i] = dWo[j, i]
        es[j, i] = dSo[j, i]
        if i + 1 < n:
            ew[j, i + 1] = dWn[j, i + 1]
        if j + 1 < n:
            es[j + 1, i] = dSn[j + 1, i]
        assert np.allclose(dKw, ew, rtol=1e-8, atol=1e-9), (j, i)
        assert np.allclose(dKs, es, rtol=1e-8, atol=1e-9), (j, i)
        ee, en = np.zeros(n), np.zeros(n)
        if i == n - 1:
            ee[j] = Ke[j]
        if j == n - 1:
            en[i] = Kn[i]
        assert np.allclose(dKe, ee, rtol=1e-8, atol=1e-9) and np.allclose(dKn, en, rtol=1e-8, atol=1e-9), (j, i)
