"""Whole-method pin of the oracle's SMC-pCN-GM (Alg. 1 + Alg. 2) on the
multi-modal example of Sec. 3.1: prior C = (I - 0.01 Lap)^-2 on [0, 1]
(Dirichlet sine modes), exp(-Phi(u)) = sum_{i=1..4} exp(-|u - f_i|^2 / (2 sigma^2))
with f = cos(pi x), -cos(pi x), cos(2 pi x), cos(3 pi x) (eq. example1phi).
The paper states no sigma; 0.1 is used.

In the KL coordinates x_k = <u, sqrt(2) sin(k pi x)>, |u - f_i|^2 =
|x - F_i|^2 + c_i with F_ik = <f_i, sqrt(2) sin(k pi x)> (closed form) and
c_i = |f_i|^2 - |F_i|^2 (the part of f_i outside the modes), so the
posterior is exactly a four-component Gaussian mixture: component i has mean
lambda F_i / (lambda + sigma^2), variance lambda sigma^2 / (lambda + sigma^2)
and weight proportional to exp(-c_i / (2 sigma^2)) prod_k N(F_ik; 0,
lambda_k + sigma^2).  SMC's particles, assigned to the nearest mean, must
reproduce the weights and the means within Monte Carlo error."""
import numpy as np

from oracle import prior, smc

KM = 16
SIGMA = 0.1


def _F(m, sign):
    k = np.arange(1, KM + 1)
    out = np.zeros(KM)
    nz = k != m
    out[nz] = np.sqrt(2.0) * k[nz] * (1 - (-1.0) ** (k[nz] + m)) / (np.pi * (k[nz] ** 2 - m ** 2))
    return sign * out


class Ex1:
    def __init__(self):
        self.lam = prior.eigenvalues_1d(KM, 0.01)
        self.F = [_F(1, 1.0), _F(1, -1.0), _F(2, 1.0), _F(3, 1.0)]
        self.c = [0.5 - f @ f for f in self.F]          # |cos(m pi x)|^2 = 1/2 on [0, 1]

    def gm_modes(self, r):
        return np.arange(min(r, KM))

    def potential(self, x):
        e = np.array([-((x - f) @ (x - f) + c) / (2 * SIGMA ** 2) for f, c in zip(self.F, self.c)])
        mx = e.max()
        return float(-(mx + np.log(np.sum(np.exp(e - mx)))))

    def posterior(self):
        lam, s2 = self.lam, SIGMA ** 2
        logw = np.array([-c / (2 * s2) - np.sum(f * f / (2 * (lam + s2))) - 0.5 * np.sum(np.log(lam + s2))
                         for f, c in zip(self.F, self.c)])
        w = np.exp(logw - logw.max())
        return w / w.sum(), [lam * f / (lam + s2) for f in self.F]


def test_projection_closed_form():
    x = (np.arange(100000) + 0.5) / 100000
    k = np.arange(1, KM + 1)
    B = np.sqrt(2.0) * np.sin(np.pi * np.outer(x, k))
    for m, sign, F in ((1, 1.0, _F(1, 1.0)), (2, 1.0, _F(2, 1.0)), (3, 1.0, _F(3, 1.0))):
        quad = (sign * np.cos(m * np.pi * x)) @ B / x.size
        assert np.allclose(quad, F, atol=1e-8)


def test_smc_pcn_gm_recovers_the_four_modes():
    prob = Ex1()
    w, means = prob.posterior()
    N = 2000
    out = smc.run(prob, N=N, K=4, r=KM, L=5, beta0=0.3, ess_frac=0.5, seed=31, em_iters=30)
    assert out["t"] == 1.0
    X = out["X"]
    d2 = np.stack([np.sum((X - m) ** 2, axis=1) for m in means], axis=1)
    lab = np.argmin(d2, axis=1)
    frac = np.bincount(lab, minlength=4) / N
    assert np.all(np.abs(frac - w) < 0.05), (frac, w)       # measured within 0.013
    for i in range(4):
        mi = X[lab == i].mean(axis=0)
        assert np.max(np.abs(mi - means[i])) < 0.03, (i, mi[:4], means[i][:4])   # measured <= 0.01


def test_smc_gm_finds_the_four_modes():
    """SMC-GM (Alg. 3: every particle redrawn from the fitted mixture), the method
    the paper runs on this example.  Alg. 3 does not preserve the layer targets
    (Thm 4 bounds the extra error instead), so the modal weights are not
    reproduced (measured: 0.17 / 0.38 / 0.39 / 0.05 against 0.31 / 0.31 / 0.24 / 0.15),
    nor the means of the small modes; every mode must still carry mass."""
    prob = Ex1()
    w, means = prob.posterior()
    N = 2000
    out = smc.run(prob, N=N, K=8, r=KM, L=1, beta0=1.0, ess_frac=0.5, seed=32, em_iters=50, kernel="gm_indep")
    assert out["t"] == 1.0
    assert all(lay["acc"] == 1.0 and lay["beta"] == 1.0 for lay in out["layers"])
    X = out["X"]
    lab = np.argmin(np.stack([np.sum((X - m) ** 2, axis=1) for m in means], axis=1), axis=1)
    frac = np.bincount(lab, minlength=4) / N
    assert np.all(frac > 0.02), frac
