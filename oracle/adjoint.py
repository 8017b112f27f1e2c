"""Gradient of the potential with respect to the KL coordinates, by the adjoint
of the discrete forward model.

The Langevin equation from which App. B derives the pCN-GM proposal carries a
drift -K gamma D Phi(u); the paper sets gamma = 0 there and cites the pCN
Langevin kernel (Sec. 1, Sec. 2.4) without giving it.  A gradient-based
mutation needs D Phi, which this module defines for the discrete model of
``darcy`` and ``observe``:

  Phi(x) = |O w - d|^2 / (2 sigma^2),   A(u) w = b,   u = S x,

with O the observation operator (bilinear interpolation with odd reflection),
A the cell-centred operator with harmonic face means, and S the KL synthesis.
Differentiating A w = b:

  g        = dPhi/dw = O^T (O w - d) / sigma^2
  A lam    = g                                   (A is symmetric)
  dPhi/du_c = -lam^T (dA/du_c) w
            = -sum over the faces f of cell c of (dK_f/du_c) (lam_c - lam_nb)(w_c - w_nb)

because A = sum over interior faces K_f (e_a - e_b)(e_a - e_b)^T + sum over
wall faces K_f e_c e_c^T (lam_nb = w_nb = 0 across a wall).  With k = e^u,
K_f = 2 k_a k_b / (k_a + k_b) gives dK_f/du_a = K_f k_b / (k_a + k_b), and a
wall face K_f = 2 k_c gives dK_f/du_c = K_f.  Finally dPhi/dx = S^T dPhi/du:
for u[j, i] = sum_{k,l} x[k, l] B[i, k] B[j, l], the transpose is
G[k, l] = sum_{i,j} g[j, i] B[i, k] B[j, l] = (B^T g^T B)[k, l].

Every step is a definition written out; the adjoint solve is one sparse LU
solve.  Pinned by central finite differences of the oracle's own potential
(tests/test_oracle_adjoint.py).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import darcy, observe, prior


def observation_matrix_2d(n, obs_xy):
    """O as a sparse (Nd, n*n) matrix, column index j*n + i; the same weights as
    ``observe.observe_2d`` (bilinear on the ghosted grid, ghost = -inside across
    an edge, +inside at a corner)."""
    rows, cols, vals = [], [], []

    def ghost_to_cell(gj, gi):
        # ghosted index (gj, gi) in 0..n+1 -> (cell j, cell i, sign)
        sign = 1.0
        j, i = gj - 1, gi - 1
        edge_j = j < 0 or j > n - 1
        edge_i = i < 0 or i > n - 1
        j = min(max(j, 0), n - 1)
        i = min(max(i, 0), n - 1)
        if edge_j != edge_i:      # an edge ghost (not a corner): odd reflection
            sign = -1.0
        return j, i, sign

    for m, (x, y) in enumerate(np.asarray(obs_xy, dtype=np.float64)):
        s = x * n - 0.5
        t = y * n - 0.5
        i0 = int(np.floor(s))
        j0 = int(np.floor(t))
        fx = s - i0
        fy = t - j0
        for dj, di, wgt in ((0, 0, (1 - fy) * (1 - fx)), (0, 1, (1 - fy) * fx), (1, 0, fy * (1 - fx)), (1, 1, fy * fx)):
            j, i, sign = ghost_to_cell(j0 + 1 + dj, i0 + 1 + di)
            rows.append(m)
            cols.append(j * n + i)
            vals.append(sign * wgt)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(obs_xy), n * n))


def face_derivatives(kc):
    """dK/du for the west and south face of every cell, with respect to the
    cell itself (``own``) and to its west / south neighbour (``nb``); wall
    faces (column 0 for west, row 0 for south) depend on the cell only.
    Returns (Kw, Ks, dKw_own, dKw_nb, dKs_own, dKs_nb, Ke_wall, Kn_wall), the
    last two the east / north wall faces 2 k_c of the last column / row."""
    kc = np.asarray(kc, dtype=np.float64)
    Kw, Ks, _ = darcy.face_coefficients(kc)
    Kw = Kw.copy()
    Ks = Ks.copy()
    dKw_own = np.zeros_like(kc)
    dKw_nb = np.zeros_like(kc)
    dKs_own = np.zeros_like(kc)
    dKs_nb = np.zeros_like(kc)
    a, b = kc[:, 1:], kc[:, :-1]          # west face of column i >= 1: cells i (own) and i-1 (nb)
    dKw_own[:, 1:] = Kw[:, 1:] * b / (a + b)
    dKw_nb[:, 1:] = Kw[:, 1:] * a / (a + b)
    a, b = kc[1:, :], kc[:-1, :]
    dKs_own[1:, :] = Ks[1:, :] * b / (a + b)
    dKs_nb[1:, :] = Ks[1:, :] * a / (a + b)
    Kw[:, 0] = 2.0 * kc[:, 0]             # wall faces: K = 2 k_c, dK/du_c = K
    Ks[0, :] = 2.0 * kc[0, :]
    dKw_own[:, 0] = Kw[:, 0]
    dKs_own[0, :] = Ks[0, :]
    return Kw, Ks, dKw_own, dKw_nb, dKs_own, dKs_nb, 2.0 * kc[:, -1], 2.0 * kc[-1, :]


def grad_u_from_adjoint(kc, w, lam):
    """dPhi/du on the grid from the state w and the adjoint lam (both (n, n))."""
    Kw, Ks, dWo, dWn, dSo, dSn, Ke, Kn = face_derivatives(kc)
    n = kc.shape[0]
    g = np.zeros((n, n))
    # west faces of columns i >= 1: product (lam_i - lam_{i-1})(w_i - w_{i-1}) feeds both cells
    pw = (lam[:, 1:] - lam[:, :-1]) * (w[:, 1:] - w[:, :-1])
    g[:, 1:] -= dWo[:, 1:] * pw
    g[:, :-1] -= dWn[:, 1:] * pw
    ps = (lam[1:, :] - lam[:-1, :]) * (w[1:, :] - w[:-1, :])
    g[1:, :] -= dSo[1:, :] * ps
    g[:-1, :] -= dSn[1:, :] * ps
    # wall faces: west (column 0), south (row 0), east (last column), north (last row)
    g[:, 0] -= dWo[:, 0] * lam[:, 0] * w[:, 0]
    g[0, :] -= dSo[0, :] * lam[0, :] * w[0, :]
    g[:, -1] -= Ke * lam[:, -1] * w[:, -1]
    g[-1, :] -= Kn * lam[-1, :] * w[-1, :]
    return g


def analysis_2d(g, Km):
    """S^T g: G[k, l] = sum_{i,j} g[j, i] B[i, k] B[j, l], returned flat (k*Km + l)."""
    n = g.shape[-1]
    B = prior.cosine_basis_1d(n, Km)
    return (B.T @ np.asarray(g).T @ B).reshape(-1)


def potential_and_gradient_2d(prob, x):
    """(Phi, dPhi/dx, w, lam) for one particle of a 2D problem (oracle.problem.Problem)."""
    n, Km = prob.n, prob.Km
    u = prob.field(x)
    kc = np.exp(u)
    A = darcy.assemble_2d(kc)
    lu = spla.splu(A)
    b = (prob.f / (n * n)).ravel()
    w = lu.solve(b)
    O = observation_matrix_2d(n, prob.obs)
    res = O @ w - prob.data
    phi = float(res @ res / (2.0 * prob.sigma ** 2))
    g_w = O.T @ res / prob.sigma ** 2
    lam = lu.solve(g_w)                    # A^T = A
    g_u = grad_u_from_adjoint(kc, w.reshape(n, n), lam.reshape(n, n))
    return phi, analysis_2d(g_u, Km), w.reshape(n, n), lam.reshape(n, n)
