"""Observation operator F(u) = (w(x_1), ..., w(x_Nd)) of Sec. 3.2 and the
potential Phi(u) = |F(u) - d|^2 / (2 sigma^2) of Sec. 2.1 (eq. Phi).

Point values of the discrete solution (a reading; the paper is silent):
* 2D: bilinear interpolation of the cell-centred w, extended past the last
  cell centre by odd reflection across the wall (w_ghost = -w_inside), so the
  interpolant vanishes on the boundary like the continuous solution.
* 1D: linear interpolation between nodes, w(0) = w(1) = 0.
"""
import numpy as np


def _ghosted(w):
    n = w.shape[-1]
    g = np.zeros(w.shape[:-2] + (n + 2, n + 2))
    g[..., 1:-1, 1:-1] = w
    g[..., 0, 1:-1] = -w[..., 0, :]
    g[..., -1, 1:-1] = -w[..., -1, :]
    g[..., 1:-1, 0] = -w[..., :, 0]
    g[..., 1:-1, -1] = -w[..., :, -1]
    g[..., 0, 0] = w[..., 0, 0]
    g[..., 0, -1] = w[..., 0, -1]
    g[..., -1, 0] = w[..., -1, 0]
    g[..., -1, -1] = w[..., -1, -1]
    return g


def observe_2d(w, obs_xy):
    """w: (..., n, n) cell-centred, row j = y, column i = x.  obs_xy: (Nd, 2) in (0,1)^2."""
    n = w.shape[-1]
    g = _ghosted(w)
    out = np.empty(w.shape[:-2] + (obs_xy.shape[0],))
    for m, (x, y) in enumerate(obs_xy):
        s = x * n - 0.5          # continuous cell-centre coordinate, centre i at s = i
        t = y * n - 0.5
        i0 = int(np.floor(s))
        j0 = int(np.floor(t))
        fx = s - i0
        fy = t - j0
        # ghosted array index = cell index + 1
        a = g[..., j0 + 1, i0 + 1]
        b = g[..., j0 + 1, i0 + 2]
        c = g[..., j0 + 2, i0 + 1]
        d = g[..., j0 + 2, i0 + 2]
        out[..., m] = (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d)
    return out


def observe_1d(w_interior, obs_x):
    n = w_interior.shape[-1] + 1
    full = np.zeros(w_interior.shape[:-1] + (n + 1,))
    full[..., 1:-1] = w_interior
    out = np.empty(w_interior.shape[:-1] + (len(obs_x),))
    for m, x in enumerate(obs_x):
        s = x * n
        i0 = min(int(np.floor(s)), n - 1)
        fx = s - i0
        out[..., m] = (1 - fx) * full[..., i0] + fx * full[..., i0 + 1]
    return out


def potential(y, data, sigma):
    """Phi = sum_m (y_m - d_m)^2 / (2 sigma^2)."""
    r = np.asarray(y) - np.asarray(data)
    return np.sum(r * r, axis=-1) / (2.0 * sigma * sigma)
