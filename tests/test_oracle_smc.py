"""Pins for tempering, reweighting, resampling and the beta rule (Alg. 1, App. C)."""
import math
from fractions import Fraction
from itertools import product

import numpy as np

from oracle import smc


def test_ess_limits_and_monotonicity():
    rng = np.random.default_rng(0)
    phi = rng.uniform(0, 50, 300)
    assert smc.ess_of_h(phi, 0.0) == 300.0
    hs = np.linspace(0, 1, 200)
    e = [smc.ess_of_h(phi, h) for h in hs]
    assert all(e[i + 1] <= e[i] * (1 + 1e-14) for i in range(len(e) - 1))
    assert abs(smc.ess_of_h(np.full(50, 3.7), 0.9) - 50.0) < 1e-12
    # ESS equals (sum w^2)^-1 for the normalised weights (App. C)
    w = np.exp(-0.3 * phi)
    w /= w.sum()
    assert abs(smc.ess_of_h(phi, 0.3) - 1.0 / np.sum(w * w)) < 1e-9


def test_bisection_brackets_target():
    rng = np.random.default_rng(1)
    phi = rng.exponential(40.0, 500)
    target = 250.0
    h = smc.bisect_h(phi, 0.0, target)
    assert 0 < h < 1
    assert smc.ess_of_h(phi, h) >= target
    assert smc.ess_of_h(phi, h * (1 + 1e-9) + 1e-15) < target
    assert smc.bisect_h(np.full(10, 2.0), 0.25, 5.0) == 0.75


def test_log_z_increment_direct_sum():
    phi = np.random.default_rng(2).uniform(0, 30, 64)
    h = 0.137
    ref = math.log(math.fsum(math.exp(-h * p) for p in phi) / 64)
    assert abs(smc.log_z_increment(phi, h) - ref) < 1e-12


def _exact_indices(logw, u48):
    w = smc.normalised_weights(np.asarray(logw))
    cdf = smc.fixed_point_cdf(w)
    N = len(w)
    T = smc.RESAMPLE_T
    U = Fraction(2 * u48 + 1, 2 * T)
    out = []
    for k in range(N):
        p = (k + U) / N
        out.append(min(i for i in range(N) if Fraction(cdf[i], T) > p))
    return out, cdf


def test_systematic_resampling_brute_force():
    rng = np.random.default_rng(3)
    for N in range(1, 7):
        for _ in range(30):
            logw = rng.normal(0, 2, N)
            u48 = int(rng.integers(0, smc.RESAMPLE_T))
            got = smc.systematic_indices(logw, u48)
            ref, cdf = _exact_indices(logw, u48)
            assert list(got) == ref
            q = np.diff([0] + cdf)
            assert sum(q) == smc.RESAMPLE_T
            counts = np.bincount(got, minlength=N)
            for i in range(N):
                assert math.floor(N * q[i] / smc.RESAMPLE_T) <= counts[i] <= math.ceil(N * q[i] / smc.RESAMPLE_T)


def test_equal_weights_identity_and_extremes():
    for N in (1, 5, 64):
        assert list(smc.systematic_indices(np.zeros(N), 12345)) == list(range(N))
        assert list(smc.systematic_indices(np.zeros(N), smc.RESAMPLE_T - 1)) == list(range(N))
    # N a power of two: the fixed-point CDF is exact, so with the smallest uniform every
    # systematic point (k + 2^-49)/N lies just above a CDF boundary and must still map to k
    for N in (2, 8, 64):
        assert list(smc.systematic_indices(np.zeros(N), 0)) == list(range(N))
    logw = np.array([0.0, -800.0, -800.0])
    assert list(smc.systematic_indices(logw, 7)) == [0, 0, 0]


def test_beta_rule_table():
    for (acc, out) in [(0.31, 0.4), (0.3, 0.2), (0.2, 0.2), (0.15, 0.2), (0.149, 0.1), (0.0, 0.1)]:
        assert smc.beta_rule(0.2, acc) == out
    assert smc.beta_rule(0.8, 0.9) == 1.0


def test_posterior_moments_closed_form():
    """Mean and population variance (divisor N) of the particles: two particles per
    coordinate pair give mean (a + b)/2 and variance ((a - b)/2)^2; an affine map of the
    particles maps the moments as c mean + s and c^2 var."""
    X = np.array([[1.0, 2.0, -5.0], [3.0, 6.0, -5.0]])
    m, v = smc.posterior_moments(X)
    assert np.array_equal(m, [2.0, 4.0, -5.0]) and np.array_equal(v, [1.0, 4.0, 0.0])
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((50, 4))
    m1, v1 = smc.posterior_moments(Y)
    m2, v2 = smc.posterior_moments(-3.0 * Y + 0.5)
    assert np.allclose(m2, -3.0 * m1 + 0.5, rtol=1e-13) and np.allclose(v2, 9.0 * v1, rtol=1e-13)


def test_prior_draws_have_the_prior_moments():
    """x_n = sqrt(lambda) z_n: over 20000 particles the coordinates have mean 0 and variance
    lambda (4 standard errors), and draws of different particles are uncorrelated."""
    lam = np.array([1.0, 0.25, 0.04, 1e-4])
    N = 20000
    X = np.stack([smc.prior_draw(7, lam, n) for n in range(N)])
    assert np.all(np.abs(X.mean(axis=0)) < 4 * np.sqrt(lam / N))
    assert np.all(np.abs(X.var(axis=0) / lam - 1.0) < 4 * np.sqrt(2.0 / N))
    assert abs(np.corrcoef(X[:-1, 0], X[1:, 0])[0, 1]) < 4 / np.sqrt(N)


# Fixed-point CDFs written out by hand (Alg. 1 resampling; the reading: T = 2^48, floor, the
# remainder to the largest weight, lowest index among equal largest weights).  Each weight's
# binary expansion is stated so that the floors can be checked without running anything.
T48 = 1 << 48
HAND_CDFS = [
    # 1/8, 3/8, 1/2 are exact: q = 2^45, 3 * 2^45, 2^47 and nothing is left over
    ([0.125, 0.375, 0.5], [35184372088832, 140737488355328, 281474976710656]),
    # the double nearest 1/3 is 6004799503160661 * 2^-54, so w T = 93824992236885.328125;
    # three floors leave 1, which goes to index 0 (a three-way tie for the largest weight)
    ([1 / 3, 1 / 3, 1 / 3], [93824992236886, 187649984473771, 281474976710656]),
    # 0.2 = 3602879701896397 * 2^-54 -> 56294995342131.203125, 0.4 -> 112589990684262.40625;
    # the floors leave 1, which goes to index 1 (tie between 1 and 2: lowest index)
    ([0.2, 0.4, 0.4], [56294995342131, 168884986026394, 281474976710656]),
    # 0.1 -> 28147497671065.6015625, 0.3 -> 84442493013196.796875; the floors leave 2,
    # which go to the largest weight 0.4 (index 3)
    ([0.1, 0.2, 0.3, 0.4], [28147497671065, 84442493013196, 168884986026392, 281474976710656]),
    # five weights: the floors leave 3, which go to index 0 (0.3 twice: lowest index)
    ([0.3, 0.3, 0.2, 0.1, 0.1], [84442493013199, 168884986026395, 225179981368526, 253327479039591,
                                 281474976710656]),
]


def test_fixed_point_cdf_hand_computed():
    assert smc.RESAMPLE_T == T48
    for w, cdf in HAND_CDFS:
        assert list(smc.fixed_point_cdf(np.array(w))) == cdf, w


def test_systematic_indices_hand_computed():
    """logw = (log 2, 0, 0) normalises to exactly (1/2, 1/4, 1/4): CDF/T = (1/2, 3/4, 1), and
    the points (k + U)/3 with U = (u48 + 1/2)/2^48 fall, by hand:
      u48 = 0:           ~0, ~1/3, ~2/3          -> 0, 0, 1
      u48 = 2^47 - 1:    U = 1/2 - 2^-49: 1/6, 1/2 - 2^-49/3, 5/6 - ...  -> 0, 0, 2
      u48 = 2^47:        U = 1/2 + 2^-49: 1/6, 1/2 + 2^-49/3, 5/6 + ...  -> 0, 1, 2
      u48 = 2^48 - 1:    ~1/3, ~2/3, ~1 (below)  -> 0, 1, 2
    The second and third straddle the CDF boundary 1/2: index i is taken only when the
    point lies strictly below CDF_i."""
    logw = np.array([np.log(2.0), 0.0, 0.0])
    assert list(smc.normalised_weights(logw)) == [0.5, 0.25, 0.25]
    for u48, ref in [(0, [0, 0, 1]), ((1 << 47) - 1, [0, 0, 2]), (1 << 47, [0, 1, 2]), (T48 - 1, [0, 1, 2])]:
        assert list(smc.systematic_indices(logw, u48)) == ref, u48


def test_resampling_near_ties_hand_computed():
    """Weights (1/2, 1/4, 1/4), N = 3: with u48 = 2^47 - 1 the second point is
    (3/2 - 2^-49)/3 = 1/2 - 2^-49/3, i.e. half a CDF unit below the boundary 1/2 on the
    scale N * CDF (2 * 3 * 2^47 - (2 (2^48 + 2^47 - 1) + 1) = 1): a near-tie for any margin.
    With u48 = 2^46 (U just above 1/4) the third point is (2 + 1/4)/3 = 3/4 plus a
    fraction of a unit, on the boundary 3/4; with u48 = 2^45 (U ~ 1/8) the points 1/24,
    3/8, 17/24 stay at least T/24 from the boundaries 1/2 and 3/4: none."""
    logw = np.array([np.log(2.0), 0.0, 0.0])
    assert smc.resampling_near_ties(logw, (1 << 47) - 1, units=1) == [1]
    assert smc.resampling_near_ties(logw, 1 << 46, units=1) == [2]
    assert smc.resampling_near_ties(logw, 1 << 45, units=1 << 40) == []
    assert smc.resampling_near_ties(logw, 1 << 47, units=1) == [1]
    # equal weights with N a power of two: CDF_i = (i + 1) T / N exactly, the points sit
    # u48 + 1/2 units above k T, i.e. u48 + 1/2 above the boundary below them
    assert smc.resampling_near_ties(np.zeros(4), 10, units=11) == [1, 2, 3]
    assert smc.resampling_near_ties(np.zeros(4), 10, units=10) == [1, 2, 3]
    assert smc.resampling_near_ties(np.zeros(4), 10, units=2) == []
