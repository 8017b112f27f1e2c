"""Pins for the oracle's Darcy solver (Sec. 3.2, eq. example2:PDE)."""
import numpy as np
import pytest
import sympy as sp

from oracle import darcy


def _manufactured_2d():
    x, y = sp.symbols("x y")
    u = sp.Rational(1, 2) * sp.cos(sp.pi * x) * sp.cos(sp.pi * y)
    w = sp.sin(sp.pi * x) * sp.sin(sp.pi * y)
    k = sp.exp(u)
    f = -(sp.diff(k * sp.diff(w, x), x) + sp.diff(k * sp.diff(w, y), y))
    return (sp.lambdify((x, y), u, "numpy"), sp.lambdify((x, y), w, "numpy"), sp.lambdify((x, y), f, "numpy"))


def test_manufactured_solution_second_order():
    """Error of the cell-centred scheme on a manufactured solution falls ~4x per halving of h."""
    uf, wf, ff = _manufactured_2d()
    errs = []
    for n in (16, 32, 64, 128):
        c = (np.arange(n) + 0.5) / n
        X, Y = np.meshgrid(c, c, indexing="xy")
        w = darcy.solve_2d(uf(X, Y), ff(X, Y))
        errs.append(np.max(np.abs(w - wf(X, Y))))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios), (errs, ratios)


def test_assembled_operator_matches_flux_definition():
    """Dense matrix from a loop over cells and their four faces equals the assembled one."""
    n = 5
    rng = np.random.default_rng(3)
    kc = np.exp(rng.standard_normal((n, n)))
    A = darcy.assemble_2d(kc).toarray()
    B = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            c = j * n + i
            for (di, dj) in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < n and 0 <= jj < n:
                    kf = 2 * kc[j, i] * kc[jj, ii] / (kc[j, i] + kc[jj, ii])
                    B[c, c] += kf
                    B[c, jj * n + ii] -= kf
                else:
                    B[c, c] += 2 * kc[j, i]
    assert np.array_equal(A, A.T)
    assert np.allclose(A, B, rtol=1e-15, atol=1e-15)
    # and the solve equals a dense solve
    f = rng.standard_normal((n, n))
    w = darcy.solve_2d(np.log(kc), f)
    assert np.allclose(w.ravel(), np.linalg.solve(B, f.ravel() / n ** 2), rtol=1e-13, atol=1e-15)


def test_apply_operator_equals_matrix_product():
    n = 7
    rng = np.random.default_rng(4)
    kc = np.exp(rng.standard_normal((n, n)))
    w = rng.standard_normal((n, n))
    Kw, Ks, D = darcy.face_coefficients(kc)
    assert np.allclose(darcy.apply_operator(Kw, Ks, D, w).ravel(), darcy.assemble_2d(kc) @ w.ravel(), rtol=1e-14, atol=1e-14)


def test_constant_coefficient_symmetries_and_positivity():
    n = 16
    w = darcy.solve_2d(np.zeros((n, n)), np.ones((n, n)))
    assert np.all(w > 0)
    assert np.allclose(w, w[::-1, :], atol=1e-15) and np.allclose(w, w[:, ::-1], atol=1e-15)
    assert np.allclose(w, w.T, atol=1e-15)


def test_manufactured_solution_1d_second_order():
    x = sp.symbols("x")
    u = sp.Rational(3, 10) * sp.cos(2 * sp.pi * x)
    w = sp.sin(sp.pi * x)
    f = -sp.diff(sp.exp(u) * sp.diff(w, x), x)
    uf, wf, ff = (sp.lambdify(x, e, "numpy") for e in (u, w, f))
    errs = []
    for n in (32, 64, 128, 256):
        xm = (np.arange(n) + 0.5) / n
        xn = np.arange(1, n) / n
        errs.append(np.max(np.abs(darcy.solve_1d(uf(xm), ff(xn)) - wf(xn))))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.5 < r < 4.5 for r in ratios), (errs, ratios)


def test_sources_at_cell_centres_and_nodes():
    """The Gaussian source of the 2D workloads: symmetric under x -> 1 - x and y -> 1 - y, the
    value at a cell centre from the formula, and a midpoint sum equal to the integral of the
    Gaussian over the plane, amp pi / width (the mass outside the unit square is below 1e-5 of
    it at width 50); the 1D source at the interior nodes i/n; the constant kind."""
    n, amp, width = 256, 10.0, 50.0
    f = darcy.source_2d(n, 1, amp, width)
    assert f.shape == (n, n)
    assert np.array_equal(f, f[:, ::-1]) and np.array_equal(f, f[::-1, :]) and np.array_equal(f, f.T)
    i, j = 37, 201
    assert f[j, i] == pytest.approx(amp * np.exp(-width * (((i + 0.5) / n - 0.5) ** 2 + ((j + 0.5) / n - 0.5) ** 2)), rel=1e-15)
    assert f.sum() / n ** 2 == pytest.approx(amp * np.pi / width, rel=1e-5)
    assert np.array_equal(darcy.source_2d(8, 0, 3.0, 0.0), np.full((8, 8), 3.0))
    g = darcy.source_1d(16, 1, amp, width)
    assert g.shape == (15,) and g[7] == amp                        # node 8/16 = 1/2
    assert g[2] == pytest.approx(amp * np.exp(-width * (3 / 16 - 0.5) ** 2), rel=1e-15)
    assert np.array_equal(darcy.source_1d(16, 0, 1.0, 0.0), np.ones(15))
