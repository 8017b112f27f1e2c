"""Forward PDE of Sec. 3.2 (eq. example2:PDE): -div(e^u grad w) = f on (0,1)^2,
w = 0 on the boundary; and its 1D analogue (the 128-interval elliptic workload), -(e^u w')' = f on
[0, 1], w(0) = w(1) = 0.  The paper states no discretisation.  Readings:

2D, cell-centred finite volumes on an n x n grid, h = 1/n:
  coefficient k_c = exp(u_c) at cell centres;
  interior face coefficient = harmonic mean 2 k_a k_b / (k_a + k_b);
  boundary face coefficient = 2 k_c (Dirichlet 0 imposed at the wall, a
  half cell away from the centre);
  (A w)_c = sum over the four faces of K_f (w_c - w_neighbour), with
  w_neighbour = 0 across a boundary face;
  the scaled system A w = h^2 f_c, f_c the source at the cell centre.
1D, nodes x_i = i/n, unknowns w_1..w_{n-1}, K_{i+1/2} = exp(u(x_{i+1/2})):
  (A w)_i = K_{i-1/2}(w_i - w_{i-1}) + K_{i+1/2}(w_i - w_{i+1}), w_0 = w_n = 0,
  A w = h^2 f_i.

The solution is defined as w = A^{-1} b exactly; the oracle computes it with
a sparse LU factorisation (2D) or a banded solve (1D), library primitives
used as single steps.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.linalg as sla


def source_2d(n, kind, amp, width):
    """f at cell centres: kind 0 -> constant amp; kind 1 -> amp exp(-width |x - (1/2,1/2)|^2)."""
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")   # X[j, i] = x_i, Y[j, i] = y_j
    if kind == 0:
        return np.full((n, n), float(amp))
    return amp * np.exp(-width * ((X - 0.5) ** 2 + (Y - 0.5) ** 2))


def source_1d(n, kind, amp, width):
    x = np.arange(1, n) / n
    if kind == 0:
        return np.full(n - 1, float(amp))
    return amp * np.exp(-width * (x - 0.5) ** 2)


def face_coefficients(kc):
    """West/south face coefficients and diagonal of the cell-centred operator.

    Kw[j, i]: face between cells (i-1, j) and (i, j); 0 for i = 0 (the wall
    face is folded into D).  Ks[j, i]: face between (i, j-1) and (i, j); 0 for
    j = 0.  D[j, i] = sum of the four face coefficients of cell (i, j), wall
    faces counted as 2 k_c.
    """
    kc = np.asarray(kc, dtype=np.float64)
    Kw = np.zeros_like(kc)
    Ks = np.zeros_like(kc)
    Kw[..., :, 1:] = 2.0 * kc[..., :, 1:] * kc[..., :, :-1] / (kc[..., :, 1:] + kc[..., :, :-1])
    Ks[..., 1:, :] = 2.0 * kc[..., 1:, :] * kc[..., :-1, :] / (kc[..., 1:, :] + kc[..., :-1, :])
    D = Kw.copy()
    D[..., :, :-1] += Kw[..., :, 1:]
    D += Ks
    D[..., :-1, :] += Ks[..., 1:, :]
    D[..., :, 0] += 2.0 * kc[..., :, 0]
    D[..., :, -1] += 2.0 * kc[..., :, -1]
    D[..., 0, :] += 2.0 * kc[..., 0, :]
    D[..., -1, :] += 2.0 * kc[..., -1, :]
    return Kw, Ks, D


def apply_operator(Kw, Ks, D, w):
    """(A w)_c = D_c w_c - sum_{interior faces} K_f w_neighbour."""
    q = D * w
    q[..., :, 1:] -= Kw[..., :, 1:] * w[..., :, :-1]
    q[..., :, :-1] -= Kw[..., :, 1:] * w[..., :, 1:]
    q[..., 1:, :] -= Ks[..., 1:, :] * w[..., :-1, :]
    q[..., :-1, :] -= Ks[..., 1:, :] * w[..., 1:, :]
    return q


def assemble_2d(kc):
    """Sparse A (n^2 x n^2), unknown (i, j) at flat index j*n + i."""
    Kw, Ks, D = face_coefficients(kc)
    n = kc.shape[0]
    idx = np.arange(n * n).reshape(n, n)
    rows = [idx.ravel()]
    cols = [idx.ravel()]
    vals = [D.ravel()]
    a, b, v = idx[:, 1:].ravel(), idx[:, :-1].ravel(), -Kw[:, 1:].ravel()
    rows += [a, b]; cols += [b, a]; vals += [v, v]
    a, b, v = idx[1:, :].ravel(), idx[:-1, :].ravel(), -Ks[1:, :].ravel()
    rows += [a, b]; cols += [b, a]; vals += [v, v]
    return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n * n, n * n))


def solve_2d(u, f):
    """w = A(exp(u))^{-1} (h^2 f) on the n x n cell-centred grid."""
    n = u.shape[0]
    A = assemble_2d(np.exp(u))
    b = (f / (n * n)).ravel()
    return spla.splu(A).solve(b).reshape(n, n)


def solve_1d(u_mid, f_nodes):
    """1D: u at the n midpoints, f at the n-1 interior nodes; returns w_1..w_{n-1}."""
    n = u_mid.shape[0]
    K = np.exp(u_mid)                      # K_{i+1/2}, i = 0..n-1
    diag = K[:-1] + K[1:]                  # node i = 1..n-1: K_{i-1/2} + K_{i+1/2}
    off = -K[1:-1]                         # coupling between nodes i and i+1
    ab = np.zeros((3, n - 1))
    ab[0, 1:] = off
    ab[1, :] = diag
    ab[2, :-1] = off
    return sla.solve_banded((1, 1), ab, f_nodes / (n * n))
