"""Gaussian prior N(0, C) with C = (I - alpha Lap)^-2 in its Karhunen-Loeve basis.

Sec. 2.1 asks for a positive, self-adjoint, trace-class C with eigenpairs
(lambda_i, phi_i); Sec. 3.1 uses C = (I - 0.01 Lap)^-2 on [0, 1] and Sec. 3.2
uses C_0 = (I - Lap)^-2 on the unit square.  The paper does not state the
boundary condition of the Laplacian.  Readings used here:

* 2D (unit square): Neumann, so phi_kl(x, y) = c_k c_l cos(k pi x) cos(l pi y)
  with c_0 = 1, c_k = sqrt(2) (k >= 1), -Lap phi_kl = pi^2 (k^2 + l^2) phi_kl and
  lambda_kl = (1 + alpha pi^2 (k^2 + l^2))^-2, 0 <= k, l < Km.  Coefficient
  storage is row-major in (k, l): index k*Km + l.  k counts along x (the
  grid column index i), l along y (the grid row index j).
* 1D ([0, 1]): Dirichlet, phi_k(x) = sqrt(2) sin(k pi x), k = 1..Km,
  lambda_k = (1 + alpha pi^2 k^2)^-2, stored at index k-1.

The field u = sum_i v_i phi_i is evaluated where the discrete forward model
needs it: 2D at cell centres x_i = (i + 1/2)/n, 1D at the midpoints
(i + 1/2)/n of the node grid.  A prior draw is v = sqrt(lambda) * z with z
standard normal (Sec. 2.3: C shares the KL basis, so it is diagonal there).
"""
import numpy as np


def eigenvalues_2d(Km, alpha):
    k = np.arange(Km, dtype=np.float64)
    lam = (1.0 + alpha * np.pi ** 2 * (k[:, None] ** 2 + k[None, :] ** 2)) ** -2.0
    return lam.reshape(-1)


def eigenvalues_1d(Km, alpha):
    k = np.arange(1, Km + 1, dtype=np.float64)
    return (1.0 + alpha * np.pi ** 2 * k ** 2) ** -2.0


def eigenvalues(dim, Km, alpha):
    return eigenvalues_2d(Km, alpha) if dim == 2 else eigenvalues_1d(Km, alpha)


def cosine_basis_1d(n, Km):
    """B[i, k] = c_k cos(k pi x_i) at cell centres x_i = (i + 1/2)/n."""
    x = (np.arange(n) + 0.5) / n
    c = np.where(np.arange(Km) == 0, 1.0, np.sqrt(2.0))
    return np.cos(np.pi * np.outer(x, np.arange(Km))) * c[None, :]


def sine_basis_midpoints(n, Km):
    """S[i, k-1] = sqrt(2) sin(k pi x_{i+1/2}), x_{i+1/2} = (i + 1/2)/n."""
    x = (np.arange(n) + 0.5) / n
    return np.sqrt(2.0) * np.sin(np.pi * np.outer(x, np.arange(1, Km + 1)))


def synthesize_2d(v, n, Km):
    """u[j, i] = sum_{k,l} v[k, l] c_k cos(k pi x_i) c_l cos(l pi y_j).

    v: (..., Km*Km); returns (..., n, n) with row index j (y) and column i (x).
    Two matrix products with the tabulated cosines: U = B V^T B^T.
    """
    v = np.asarray(v, dtype=np.float64)
    B = cosine_basis_1d(n, Km)
    V = v.reshape(v.shape[:-1] + (Km, Km))
    return np.matmul(np.matmul(B, np.swapaxes(V, -1, -2)), B.T)


def synthesize_1d(v, n, Km):
    """u at the n midpoints: u_{i+1/2} = sum_k v_k sqrt(2) sin(k pi x_{i+1/2})."""
    v = np.asarray(v, dtype=np.float64)
    return np.matmul(v, sine_basis_midpoints(n, Km).T)


def synthesize(dim, v, n, Km):
    return synthesize_2d(v, n, Km) if dim == 2 else synthesize_1d(v, n, Km)


def gm_modes(dim, Km, r):
    """Indices of the r leading KL modes (largest lambda first).

    2D: modes ordered by (k^2 + l^2, k, l); 1D: by k.  The mixture of Sec. 2.3
    is fitted on these coordinates; the rest stay at the prior (m = 0,
    lambda_j = lambda), which keeps every component equivalent to mu_0.
    """
    if dim == 1:
        return np.arange(min(r, Km))
    kk, ll = np.meshgrid(np.arange(Km), np.arange(Km), indexing="ij")
    kk = kk.ravel(); ll = ll.ravel()
    order = np.lexsort((ll, kk, kk ** 2 + ll ** 2))
    return np.sort(order[:r])
