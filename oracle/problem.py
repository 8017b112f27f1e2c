"""The inverse problem of Sec. 3 assembled from the pieces: prior (Sec. 2.1),
forward map F = observation of the Darcy solution (Sec. 3.2) and the potential
Phi (Sec. 2.1, eq. Phi)."""
import numpy as np
from . import prior, darcy, observe


class Problem:
    def __init__(self, dim, n, kl_modes, alpha, sigma, source_kind, src_amp, src_width, obs, data, **_):
        self.dim = int(dim)
        self.n = int(n)
        self.Km = int(kl_modes)
        self.alpha = float(alpha)
        self.sigma = float(sigma)
        self.obs = np.asarray(obs, dtype=np.float64)
        self.data = np.asarray(data, dtype=np.float64)
        self.src = (int(source_kind), float(src_amp), float(src_width))
        self.lam = prior.eigenvalues(self.dim, self.Km, self.alpha)
        if self.dim == 2:
            self.f = darcy.source_2d(self.n, *self.src)
        else:
            self.f = darcy.source_1d(self.n, *self.src)

    @property
    def d(self):
        return self.lam.shape[0]

    def gm_modes(self, r):
        return prior.gm_modes(self.dim, self.Km, r)

    def field(self, v):
        return prior.synthesize(self.dim, v, self.n, self.Km)

    def solve(self, v):
        u = self.field(v)
        if self.dim == 2:
            return darcy.solve_2d(u, self.f)
        return darcy.solve_1d(u, self.f)

    def observe(self, w):
        if self.dim == 2:
            return observe.observe_2d(w, self.obs)
        return observe.observe_1d(w, self.obs)

    def forward(self, v):
        return self.observe(self.solve(v))

    def potential(self, v):
        return float(observe.potential(self.forward(v), self.data, self.sigma))


def from_workload(wl):
    return Problem(obs=wl["obs"], data=wl["data"], **{k: v for k, v in wl.items() if k not in ("obs", "data")})
