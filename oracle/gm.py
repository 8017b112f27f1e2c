"""Gaussian-mixture fit of Sec. 2.4 / Alg. 3 ("estimate a Gaussian mixture by
samples").  The paper delegates the estimator to its reference Feng2018 and
prints no formula; the reading used here is the standard EM algorithm for a
mixture of diagonal Gaussians, run on the r leading KL coordinates S of the
equally weighted (resampled) particles, with the prior kept on every other
coordinate so each component stays equivalent to mu_0 (Sec. 2.3, Thm 4).

  init   : K distinct particles chosen by Philox (purpose EMINIT); the first
           pick is floor(word * N / 2^32), a collision moves to the next index
           mod N; variances start at the pooled population variance; w_j = 1/K.
  E-step : log p_nj = log w_j + sum_{i in S} [-1/2 log(2 pi lambda_ji)
                                              - (x_ni - m_ji)^2 / (2 lambda_ji)],
           responsibilities g_nj = exp(log p_nj - LSE_j log p_nj),
           log-likelihood L = sum_n LSE_j log p_nj.
  M-step : N_j = sum_n g_nj,  w_j = N_j / N,  m_j = sum_n g_nj x_n / N_j,
           lambda_ji = max(sum_n g_nj (x_ni - m_ji)^2 / N_j, floor * lambda_i).
  collapse: a component with N_j < 2 is re-seeded at the particle with the
           lowest max_j g_nj (lowest index on ties), pooled variances, and
           w_j = 1/N; the weights are then renormalised to sum 1.
A fixed number of iterations is run (no early stop); the function returns the
log-likelihood after the last E-step.
"""
import numpy as np
from . import philox
from .pcngm import Mixture


def init_indices(seed, layer, N, K):
    chosen = []
    for k in range(K):
        wd = int(philox.word32(seed, k, 0, layer, philox.EMINIT))
        c = (wd * N) >> 32
        while c in chosen:
            c = (c + 1) % N
        chosen.append(c)
    return chosen


def e_step(xs, w, m, lam):
    N = xs.shape[0]
    K = w.shape[0]
    logp = np.empty((N, K))
    for j in range(K):
        logp[:, j] = np.log(w[j]) + np.sum(-0.5 * np.log(2.0 * np.pi * lam[j])
                                           - (xs - m[j]) ** 2 / (2.0 * lam[j]), axis=1)
    mx = np.max(logp, axis=1, keepdims=True)
    lse = mx[:, 0] + np.log(np.sum(np.exp(logp - mx), axis=1))
    g = np.exp(logp - lse[:, None])
    return g, float(np.sum(lse))


def fit(X, S, lam0, K, iters, seed, layer, var_floor=1e-3):
    """EM on X[:, S]; returns (Mixture, loglik history list)."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    xs = X[:, S]
    lamS = np.asarray(lam0)[S]
    pooled_mean = np.mean(xs, axis=0)
    pooled = np.mean((xs - pooled_mean) ** 2, axis=0)
    pooled = np.maximum(pooled, var_floor * lamS)
    idx = init_indices(seed, layer, N, K)
    w = np.full(K, 1.0 / K)
    m = xs[idx].copy()
    lam = np.tile(pooled, (K, 1))
    hist = []
    for _ in range(iters):
        g, ll = e_step(xs, w, m, lam)
        hist.append(ll)
        Nj = np.sum(g, axis=0)
        for j in range(K):
            if Nj[j] < 2.0:
                n_star = int(np.argmin(np.max(g, axis=1)))
                m[j] = xs[n_star]
                lam[j] = pooled
                w[j] = 1.0 / N
                continue
            w[j] = Nj[j] / N
            m[j] = np.sum(g[:, j:j + 1] * xs, axis=0) / Nj[j]
            lam[j] = np.maximum(np.sum(g[:, j:j + 1] * (xs - m[j]) ** 2, axis=0) / Nj[j], var_floor * lamS)
        w = w / np.sum(w)
    g, ll = e_step(xs, w, m, lam)
    hist.append(ll)
    return Mixture(S, w, m, lam, lam0), hist


def e_step_full(xs, w, m, cov):
    """E-step with full covariances: log p_nj = log w_j + log N(x_n; m_j, C_j)."""
    N, r = xs.shape
    K = w.shape[0]
    logp = np.empty((N, K))
    for j in range(K):
        _, logdet = np.linalg.slogdet(cov[j])
        dev = xs - m[j]
        q = np.sum(dev * np.linalg.solve(cov[j], dev.T).T, axis=1)
        logp[:, j] = np.log(w[j]) - 0.5 * (r * np.log(2.0 * np.pi) + logdet) - 0.5 * q
    mx = np.max(logp, axis=1, keepdims=True)
    lse = mx[:, 0] + np.log(np.sum(np.exp(logp - mx), axis=1))
    return np.exp(logp - lse[:, None]), float(np.sum(lse))


def fit_full(X, S, lam0, K, iters, seed, layer, var_floor=1e-3):
    """EM with full covariances on X[:, S] (a reading beyond the paper, whose C_j
    are diagonal in the KL basis): the steps of ``fit`` with
    C_j = sum_n g_nj (x_n - m_j)(x_n - m_j)^T / N_j + floor * diag(lambda_S)
    (a ridge keeps C_j positive definite), initial and re-seeded covariances
    diag(pooled variances).  Returns (Mixture with cov, loglik history)."""
    X = np.asarray(X, dtype=np.float64)
    N = X.shape[0]
    xs = X[:, S]
    lamS = np.asarray(lam0)[S]
    pooled_mean = np.mean(xs, axis=0)
    pooled = np.maximum(np.mean((xs - pooled_mean) ** 2, axis=0), var_floor * lamS)
    idx = init_indices(seed, layer, N, K)
    w = np.full(K, 1.0 / K)
    m = xs[idx].copy()
    cov = np.stack([np.diag(pooled) for _ in range(K)])
    hist = []
    for _ in range(iters):
        g, ll = e_step_full(xs, w, m, cov)
        hist.append(ll)
        Nj = np.sum(g, axis=0)
        for j in range(K):
            if Nj[j] < 2.0:
                n_star = int(np.argmin(np.max(g, axis=1)))
                m[j] = xs[n_star]
                cov[j] = np.diag(pooled)
                w[j] = 1.0 / N
                continue
            w[j] = Nj[j] / N
            m[j] = np.sum(g[:, j:j + 1] * xs, axis=0) / Nj[j]
            dev = xs - m[j]
            cov[j] = (g[:, j:j + 1] * dev).T @ dev / Nj[j] + np.diag(var_floor * lamS)
        w = w / np.sum(w)
    g, ll = e_step_full(xs, w, m, cov)
    hist.append(ll)
    lam = np.stack([np.diag(c) for c in cov])
    return Mixture(S, w, m, lam, lam0, cov=cov), hist
