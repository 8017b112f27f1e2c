"""Pins for the Gaussian-mixture fit (Sec. 2.4 / Alg. 3 mutation; EM reading)."""
import numpy as np

from oracle import gm


def test_single_component_is_sample_moments():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((500, 6)) * np.array([1, 2, 0.5, 1, 1, 3]) + 1.0
    S = np.array([0, 2, 5])
    lam0 = np.ones(6)
    mix, _ = gm.fit(X, S, lam0, 1, 3, seed=1, layer=0)
    assert np.allclose(mix.m[0], X[:, S].mean(0), rtol=1e-13)
    assert np.allclose(mix.lam[0], X[:, S].var(0), rtol=1e-12)
    assert mix.w[0] == 1.0


def test_recovers_separated_mixture_and_loglik_monotone():
    rng = np.random.default_rng(1)
    N = 20000
    z = rng.uniform(size=N) < 0.3
    X = np.where(z[:, None], rng.normal([4.0, -3.0], [0.5, 0.8], (N, 2)), rng.normal([-2.0, 2.0], [1.0, 0.3], (N, 2)))
    mix, hist = gm.fit(X, np.array([0, 1]), np.array([10.0, 10.0]), 2, 40, seed=3, layer=1)
    a = int(np.argmax(mix.m[:, 0]))
    b = 1 - a
    assert abs(mix.w[a] - 0.3) < 0.015
    assert np.allclose(mix.m[a], [4.0, -3.0], atol=0.03) and np.allclose(mix.m[b], [-2.0, 2.0], atol=0.03)
    assert np.allclose(np.sqrt(mix.lam[a]), [0.5, 0.8], rtol=0.05) and np.allclose(np.sqrt(mix.lam[b]), [1.0, 0.3], rtol=0.05)
    assert all(hist[i + 1] >= hist[i] - 1e-9 * abs(hist[i]) for i in range(len(hist) - 1))


def test_collapse_reseeds_and_keeps_weights_normalised():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((40, 3))
    X[0] += 50.0
    mix, _ = gm.fit(X, np.array([0, 1, 2]), np.ones(3), 4, 10, seed=5, layer=0)
    assert np.isclose(mix.w.sum(), 1.0, rtol=1e-15)
    assert np.all(np.isfinite(mix.m)) and np.all(mix.lam > 0)


def test_init_indices_distinct():
    for N, K in [(4, 4), (10, 8), (1000, 8)]:
        idx = gm.init_indices(11, 2, N, K)
        assert len(set(idx)) == K and all(0 <= i < N for i in idx)
