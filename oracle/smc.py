"""SMC driver of Alg. 1 (reweight, resample, mutate) with the pCN-GM mutation
of Alg. 2, the tempering rule and the beta rule of App. C, and the posterior
moments reported in Sec. 3.2.

Tempering (App. C, "Determine the temperatures"): weights are uniform before
reweighting (Alg. 1, "Set w_j = 1/N"), so the reweighted weights of step h are
proportional to exp(-h Phi_n) and
  ESS(h) = (sum_n exp(-h Phi_n))^2 / sum_n exp(-2 h Phi_n),
which is the paper's (sum w_i^2)^-1 for normalised w.  If ESS(1 - t) >= target
the last step h = 1 - t is taken; otherwise exactly 64 bisection steps on
[0, 1 - t] keep the lower bracket, so ESS(h) >= target.  The paper's target is
0.6 N; the workloads here use ess_frac (0.5 by default).
log Z increment: log((1/N) sum_n exp(-h Phi_n)).

Resampling (Alg. 1, "resampling from sum_n w_n delta_{v_n}"; the scheme is not
stated): systematic resampling on an integer CDF so that any summation order
gives the same indices.  Normalised weights are scaled to T = 2^48 and
floored; the remainder goes to the largest weight (lowest index on ties);
CDF_i = q_0 + ... + q_i.  One Philox draw gives u48 in [0, 2^48); particle k
(k = 0..N-1) takes index min{i : N * CDF_i > k T + u48 + 1/2}, i.e. the point
(k + U)/N with U = (u48 + 1/2)/2^48.  Requires N <= 2^15.

Beta rule (App. C, "Settings of pCN transition kernel"): beta doubles when
the layer's mean acceptance rate exceeds 0.3, halves below 0.15; it is
capped at 1 (the paper is silent on the cap).

Accept test (Alg. 2): U < min(1, alpha) with U = (u53 + 1/2) 2^-53.
"""
import bisect

import numpy as np
from . import philox, pcngm, gm

RESAMPLE_T = 1 << 48


def ess_of_h(phi, h):
    a = -h * (phi - np.min(phi))
    e = np.exp(a)
    return np.sum(e) ** 2 / np.sum(e * e)


def bisect_h(phi, t, target, iters=64):
    rest = 1.0 - t
    if ess_of_h(phi, rest) >= target:
        return rest
    lo, hi = 0.0, rest
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if ess_of_h(phi, mid) >= target:
            lo = mid
        else:
            hi = mid
    return lo


def log_z_increment(phi, h):
    return pcngm.logsumexp(-h * phi) - np.log(phi.shape[0])


def normalised_weights(logw):
    return np.exp(logw - pcngm.logsumexp(logw))


def fixed_point_cdf(w):
    q = [int(np.floor(wi * RESAMPLE_T)) for wi in w]
    rem = RESAMPLE_T - sum(q)
    q[int(np.argmax(w))] += rem
    cdf = []
    acc = 0
    for qi in q:
        acc += qi
        cdf.append(acc)
    return cdf


def resample_u48(seed, layer):
    w = philox.philox4x32_10(0, 0, layer, philox.RESAMPLE, *philox.key_of(seed))
    return (int(w[0]) << 16) | (int(w[1]) >> 16)


def systematic_indices(logw, u48):
    N = len(logw)
    assert N <= (1 << 15)
    cdf = fixed_point_cdf(normalised_weights(np.asarray(logw, dtype=np.float64)))
    out = np.empty(N, dtype=np.int64)
    i = 0
    for k in range(N):
        target = k * RESAMPLE_T + u48          # need N * CDF_i > target + 1/2
        while N * cdf[i] <= target:
            i += 1
        out[k] = i
    return out


def resampling_near_ties(logw, u48, units=64):
    """Systematic points that lie within `units` CDF units (of 2^48) of a CDF boundary.

    Particle k's point sits at k T + u48 + 1/2 on the scale of N * CDF, and the index
    changes where it crosses N * CDF_i.  The weights come from floating-point exponentials
    and a log-sum-exp, whose last bits depend on the summation order and the exp routine, so
    two correct implementations may floor a w_i T differently by one unit and shift later
    CDF entries by a few units.  A point farther than `units` from every boundary gets the
    same index under any such difference; the points returned here are the near-ties."""
    N = len(logw)
    cdf = fixed_point_cdf(normalised_weights(np.asarray(logw, dtype=np.float64)))
    bounds = [2 * N * c for c in cdf[:-1]]      # twice the scaled boundaries: integers
    ties = []
    for k in range(N):
        p2 = 2 * (k * RESAMPLE_T + u48) + 1     # twice the point
        i = bisect.bisect_left(bounds, p2)      # bounds[i - 1] < p2 <= bounds[i]
        gaps = [abs(bounds[j] - p2) for j in (i - 1, i) if 0 <= j < len(bounds)]
        if gaps and min(gaps) < 2 * N * units:
            ties.append(k)
    return ties


def beta_rule(beta, acc_rate):
    if acc_rate > 0.3:
        beta = 2.0 * beta
    elif acc_rate < 0.15:
        beta = 0.5 * beta
    return min(beta, 1.0)


def prior_draw(seed, lam, n):
    """v_n = sqrt(lambda) * z, z from Philox counter (m, n, 0, INIT)."""
    return np.sqrt(lam) * philox.normals(seed, lam.shape[0], n, 0, philox.INIT)


def move_particle(x, phi_x, mix, beta, t, seed, n, step, forward, always_accept=False):
    """One pCN-GM step (Alg. 2) for particle n; returns (x', phi', accepted, log_alpha, phi_v).

    always_accept: the SMC-GM mutation of Alg. 3 (beta = 1, a = 1): the
    mixture proposal is taken as the new state."""
    d = x.shape[0]
    Uc = float(philox.uniforms(seed, 0, n, step, philox.COMP))
    j = pcngm.choose_component(mix.w, Uc)
    z = philox.normals(seed, d, n, step, philox.NORMAL)
    v = pcngm.propose(x, j, z, mix, beta)
    phi_v = forward(v)
    if always_accept:
        return v, phi_v, True, 0.0, phi_v
    lr = pcngm.log_mixture_ratio(x, v, mix, beta)
    la = pcngm.log_alpha(t, phi_x, phi_v, lr)
    Ua = float(philox.uniforms(seed, 0, n, step, philox.ACCEPT))
    if pcngm.accept(la, Ua):
        return v, phi_v, True, la, phi_v
    return x, phi_x, False, la, phi_v


def move(X, Phi, mix, beta, t, seed, step0, steps, forward, particles=None, always_accept=False):
    """`steps` pCN-GM steps for every particle (or the listed subset).

    Step s uses the Philox step counter step0 + s.  Returns new (X, Phi),
    the accept flags (steps, N), log alphas and the proposal potentials.
    """
    X = np.array(X, dtype=np.float64, copy=True)
    Phi = np.array(Phi, dtype=np.float64, copy=True)
    ids = range(X.shape[0]) if particles is None else particles
    acc = np.zeros((steps, X.shape[0]), dtype=bool)
    la = np.zeros((steps, X.shape[0]))
    pv = np.zeros((steps, X.shape[0]))
    for s in range(steps):
        for n in ids:
            X[n], Phi[n], acc[s, n], la[s, n], pv[s, n] = move_particle(
                X[n], Phi[n], mix, beta, t, seed, n, step0 + s, forward, always_accept)
    return X, Phi, acc, la, pv


def posterior_moments(X):
    mean = np.mean(X, axis=0)
    var = np.mean((X - mean) ** 2, axis=0)
    return mean, var


def run(problem, N, K, r, L, beta0, ess_frac, seed, em_iters=50, kernel="pcn_gm",
        max_layers=1000, record=None):
    """Whole SMC-pCN-GM run (Alg. 1 with Alg. 2 as mutation).  kernel: 'pcn_gm', 'pcn', or
    'gm_indep' (SMC-GM, Alg. 3: beta = 1 and every mixture proposal accepted).

    Returns a dict with the final particles, potentials, temperatures and per-layer records.
    """
    lam = problem.lam
    d = lam.shape[0]
    S = problem.gm_modes(r)
    X = np.stack([prior_draw(seed, lam, n) for n in range(N)])
    Phi = np.array([problem.potential(x) for x in X])
    indep = kernel == "gm_indep"
    t, beta, layer, step, logZ = 0.0, 1.0 if indep else float(beta0), 0, 0, 0.0
    layers = []
    while t < 1.0 and layer < max_layers:
        h = bisect_h(Phi, t, ess_frac * N)
        logw = -h * Phi
        logZ += log_z_increment(Phi, h)
        t = 1.0 if h == 1.0 - t else t + h
        idx = systematic_indices(logw, resample_u48(seed, layer))
        X, Phi = X[idx], Phi[idx]
        if kernel == "pcn":
            mix = pcngm.Mixture.prior(lam, S, 1)
        else:
            mix, _ = gm.fit(X, S, lam, K, em_iters, seed, layer)
        X, Phi, acc, _, _ = move(X, Phi, mix, beta, t, seed, step, L, problem.potential, always_accept=indep)
        step += L
        rate = float(np.mean(acc))
        layers.append(dict(h=h, t=t, beta=beta, acc=rate, logZ=logZ))
        if not indep:
            beta = beta_rule(beta, rate)
        layer += 1
        if record is not None:
            record(layer, X, Phi, mix)
    return dict(X=X, Phi=Phi, t=t, beta=beta, layers=layers, logZ=logZ)
