"""Pins for the Gaussian-mixture fit (Sec. 2.4 / Alg. 3 mutation; EM reading)."""
import numpy as np

from oracle import gm, philox


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


def _init_picks(seed, layer, N, K):
    """The initial particles by the stated rule, from the (separately pinned) Philox words:
    floor(word * N / 2^32), a repeat moves to the next index mod N."""
    out = []
    for k in range(K):
        c = (int(philox.word32(seed, k, 0, layer, philox.EMINIT)) * N) >> 32
        while c in out:
            c = (c + 1) % N
        out.append(c)
    return out


def test_collapse_reseeds_at_lowest_max_responsibility():
    """Two components initialised at 0 and 100 on 1000 points: 998 at 0, one at 100 and one at
    50.  With the pooled variance (12.4775) the points at 0 and 100 belong to their own
    component with responsibility 1 to double precision (the other is e^-400), and the point
    at 50 is split 1/2 : 1/2.  So N_0 = 998.5 and N_1 = 1.5 < 2: component 1 collapses and is
    re-seeded at the point with the lowest max-responsibility, the one at 50, with the pooled
    variance and weight 1/N before the weights are renormalised; component 0 gets weight
    N_0/N and mean 25/998.5 (one M-step)."""
    N, seed, layer = 1000, 21, 4
    a, b = _init_picks(seed, layer, N, 2)
    assert gm.init_indices(seed, layer, N, 2) == [a, b]
    c = next(i for i in range(N) if i not in (a, b))
    x = np.zeros((N, 1))
    x[b, 0] = 100.0
    x[c, 0] = 50.0
    mean = 150.0 / N
    pooled = ((N - 2) * mean ** 2 + (50.0 - mean) ** 2 + (100.0 - mean) ** 2) / N
    assert abs(pooled - 12.4775) < 1e-12
    mix, _ = gm.fit(x, np.array([0]), np.array([1.0]), 2, 1, seed, layer)
    assert mix.m[1, 0] == 50.0
    assert abs(mix.lam[1, 0] - pooled) <= 1e-14 * pooled
    assert abs(mix.w[1] / mix.w[0] - (1.0 / N) / (998.5 / N)) < 1e-12
    assert abs(mix.w.sum() - 1.0) < 1e-15
    assert abs(mix.m[0, 0] - 25.0 / 998.5) < 1e-14
    m0 = 25.0 / 998.5
    assert abs(mix.lam[0, 0] - ((N - 2) * m0 ** 2 + 0.5 * (50.0 - m0) ** 2) / 998.5) < 1e-12


def test_variance_floor_binds_on_a_constant_coordinate():
    """A coordinate on which every particle is 3.0 has zero spread: its pooled variance and
    every component's variance are the floor 1e-3 * lambda_i exactly (here 1e-3 * 2.0); the
    other coordinate keeps its fitted variance above its floor."""
    rng = np.random.default_rng(7)
    X = np.stack([rng.standard_normal(200) * 1.5, np.full(200, 3.0)], axis=1)
    lam0 = np.array([1.0, 2.0])
    mix, _ = gm.fit(X, np.array([0, 1]), lam0, 2, 3, seed=2, layer=1, var_floor=1e-3)
    assert np.all(mix.lam[:, 1] == 1e-3 * 2.0)
    assert np.all(mix.lam[:, 0] > 1e-3 * 1.0)
    assert np.all(np.abs(mix.m[:, 1] - 3.0) < 1e-14)
