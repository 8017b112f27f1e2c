"""Pins for the observation operator and the potential (Sec. 2.1 eq. Phi, Sec. 3.2)."""
import numpy as np

from oracle import observe


def test_cell_centre_points_select_exactly():
    n = 8
    w = np.random.default_rng(0).standard_normal((n, n))
    pts = np.array([[(i + 0.5) / n, (j + 0.5) / n] for (i, j) in [(0, 0), (3, 5), (7, 7), (2, 6)]])
    y = observe.observe_2d(w, pts)
    assert np.array_equal(y, np.array([w[0, 0], w[5, 3], w[7, 7], w[6, 2]]))


def test_bilinear_reproduces_affine_fields_inside():
    n = 10
    c = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(c, c, indexing="xy")
    w = 0.3 + 1.7 * X - 2.2 * Y + 0.4 * X * Y
    pts = np.random.default_rng(1).uniform(0.06, 0.94, size=(50, 2))
    y = observe.observe_2d(w, pts)
    ref = 0.3 + 1.7 * pts[:, 0] - 2.2 * pts[:, 1] + 0.4 * pts[:, 0] * pts[:, 1]
    assert np.allclose(y, ref, atol=1e-13)


def test_interpolant_vanishes_on_walls():
    n = 6
    w = np.random.default_rng(2).standard_normal((n, n))
    pts = np.array([[0.0, 0.37], [1.0, 0.61], [0.25, 0.0], [0.8, 1.0]])
    assert np.allclose(observe.observe_2d(w, pts), 0.0, atol=1e-15)


def test_linear_1d():
    n = 8
    xn = np.arange(1, n) / n
    w = 2.0 * xn + 0.5
    pts = np.array([0.13, 0.5, 0.77])
    assert np.allclose(observe.observe_1d(w, np.array([0.5])), [1.5])
    full = np.concatenate([[0.0], w, [0.0]])
    assert np.allclose(observe.observe_1d(w, pts), np.interp(pts, np.arange(n + 1) / n, full))


def test_potential():
    y = np.array([1.0, 2.0, 3.0])
    assert observe.potential(y, y, 0.1) == 0.0
    assert np.isclose(observe.potential(y, y + 0.2, 0.1), 3 * 0.04 / 0.02)
    assert observe.potential(np.random.default_rng(3).standard_normal((5, 3)), y, 0.5).min() >= 0.0
