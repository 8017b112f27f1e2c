"""Pins for the oracle's prior: KL eigenpairs, synthesis, draws (Sec. 2.1, Sec. 3)."""
import math

import numpy as np
import sympy as sp

from oracle import prior


def test_cosine_modes_are_neumann_laplacian_eigenfunctions():
    """-Lap phi_kl = pi^2 (k^2 + l^2) phi_kl with zero normal derivative, by symbolic
    differentiation; hence (I - alpha Lap)^-2 has eigenvalue (1 + alpha mu)^-2."""
    x, y = sp.symbols("x y")
    for (k, l) in [(0, 0), (1, 0), (0, 3), (2, 5), (7, 4)]:
        ck = 1 if k == 0 else sp.sqrt(2)
        cl = 1 if l == 0 else sp.sqrt(2)
        phi = ck * cl * sp.cos(k * sp.pi * x) * sp.cos(l * sp.pi * y)
        lap = sp.diff(phi, x, 2) + sp.diff(phi, y, 2)
        mu = sp.simplify(-lap / phi) if phi != 0 else None
        assert sp.simplify(mu - sp.pi ** 2 * (k ** 2 + l ** 2)) == 0
        for xb in (0, 1):
            assert sp.simplify(sp.diff(phi, x).subs(x, xb)) == 0
        lam = prior.eigenvalues_2d(8, 0.02).reshape(8, 8)[k, l]
        assert abs(lam - float((1 + 0.02 * mu) ** -2)) < 1e-15


def test_sine_modes_are_dirichlet_eigenfunctions():
    x = sp.symbols("x")
    for k in (1, 2, 9):
        phi = sp.sqrt(2) * sp.sin(k * sp.pi * x)
        mu = sp.simplify(-sp.diff(phi, x, 2) / phi)
        assert sp.simplify(mu - (k * sp.pi) ** 2) == 0
        assert phi.subs(x, 0) == 0 and sp.simplify(phi.subs(x, 1)) == 0
        assert abs(prior.eigenvalues_1d(10, 0.01)[k - 1] - float((1 + 0.01 * mu) ** -2)) < 1e-15


def test_basis_orthonormal_on_cell_centres():
    """The midpoint rule is exact for these trigonometric products (discrete cosine orthogonality)."""
    n, Km = 64, 32
    B = prior.cosine_basis_1d(n, Km)
    assert np.allclose(B.T @ B / n, np.eye(Km), atol=1e-13)
    # and against the continuous inner product by adaptive quadrature for two modes
    from scipy.integrate import quad
    f = lambda t: 2 * math.cos(3 * math.pi * t) * math.cos(3 * math.pi * t)
    assert abs(quad(f, 0, 1)[0] - 1.0) < 1e-12


def test_synthesis_against_pointwise_sum():
    n, Km = 6, 4
    rng = np.random.default_rng(1)
    v = rng.standard_normal(Km * Km)
    U = prior.synthesize_2d(v, n, Km)
    for j in range(n):
        for i in range(n):
            xi, yj = (i + 0.5) / n, (j + 0.5) / n
            s = 0.0
            for k in range(Km):
                for l in range(Km):
                    ck = 1.0 if k == 0 else math.sqrt(2.0)
                    cl = 1.0 if l == 0 else math.sqrt(2.0)
                    s += v[k * Km + l] * ck * math.cos(k * math.pi * xi) * cl * math.cos(l * math.pi * yj)
            assert abs(U[j, i] - s) < 1e-13


def test_synthesis_1d_against_pointwise_sum():
    n, Km = 8, 5
    v = np.random.default_rng(2).standard_normal(Km)
    u = prior.synthesize_1d(v, n, Km)
    for i in range(n):
        x = (i + 0.5) / n
        s = sum(v[k - 1] * math.sqrt(2) * math.sin(k * math.pi * x) for k in range(1, Km + 1))
        assert abs(u[i] - s) < 1e-13


def test_gm_modes_are_the_largest_eigenvalues():
    lam = prior.eigenvalues_2d(16, 0.02)
    S = prior.gm_modes(2, 16, 20)
    rest = np.setdiff1d(np.arange(lam.size), S)
    assert len(S) == 20 and lam[S].min() >= lam[rest].max()
