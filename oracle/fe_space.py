"""Finite-element matrices in space (Section 1, definitions of M_h and K_h).

Omega = (0,1)^d with n interior nodes per axis, h = 1/(n+1), homogeneous
Dirichlet conditions.  In 1D the P1 hat functions are assembled element by
element with element integrals computed by Gauss quadrature.  In d = 2, 3 the
Q1 basis is the tensor product phi_(j1..jd)(x) = prod_a phi_{ja}(x_a), so the
integrals factor over the axes:

    M_h = M_1 (x) ... (x) M_1,
    K_h = sum_a M_1 (x) .. K_1 (axis a) .. (x) M_1.

Node ordering: x fastest, i.e. index j = (z*n + y)*n + x, which makes the
leftmost Kronecker factor the slowest axis.
"""
import numpy as np
import scipy.sparse as sp

from .dg_time import gauss_on


def fe_1d(n):
    """1D P1 mass and stiffness matrices (dense n x n) on n interior nodes."""
    h = 1.0 / (n + 1)
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    for e in range(n + 1):                  # element [e h, (e+1) h]
        xg, wg = gauss_on(e * h, (e + 1) * h, 3)
        phi = [((e + 1) * h - xg) / h, (xg - e * h) / h]
        dphi = [-np.ones_like(xg) / h, np.ones_like(xg) / h]
        for a in range(2):
            ia = e + a - 1                  # global interior index of local node a
            if ia < 0 or ia >= n:
                continue
            for b in range(2):
                ib = e + b - 1
                if ib < 0 or ib >= n:
                    continue
                M[ia, ib] += np.sum(wg * phi[a] * phi[b])
                K[ia, ib] += np.sum(wg * dphi[a] * dphi[b])
    return M, K


def fe_matrices(d, n):
    """Sparse (M_h, K_h) for Q1 on (0,1)^d (P1 when d = 1)."""
    M1, K1 = fe_1d(n)
    M1 = sp.csr_matrix(M1)
    K1 = sp.csr_matrix(K1)
    if d == 1:
        return M1, K1
    M = M1
    K = K1
    for _ in range(d - 1):
        # new slowest axis on the left: (M1 (x) M_prev), (K1 (x) M_prev + M1 (x) K_prev)
        K = sp.kron(K1, M, format="csr") + sp.kron(M1, K, format="csr")
        M = sp.kron(M1, M, format="csr")
    return M.tocsr(), K.tocsr()


def nodes_1d(n):
    """Interior node coordinates x_j = j h, j = 1..n."""
    return np.arange(1, n + 1) / (n + 1.0)


def quadrature_1d(n, npts=5):
    """Gauss points of all elements on (0,1) and the matrix B with
    B[j, g] = w_g * phi_j(x_g) (interior hat j at point g), so that
    int g(x) phi_j(x) dx ~= (B @ g(x_points))[j]."""
    h = 1.0 / (n + 1)
    xs = []
    ws = []
    for e in range(n + 1):
        xg, wg = gauss_on(e * h, (e + 1) * h, npts)
        xs.append(xg)
        ws.append(wg)
    x = np.concatenate(xs)
    w = np.concatenate(ws)
    B = np.zeros((n, x.size))
    for e in range(n + 1):
        sl = slice(e * npts, (e + 1) * npts)
        xg = x[sl]
        left = ((e + 1) * h - xg) / h    # hat of node e   (local node 0)
        right = (xg - e * h) / h         # hat of node e+1 (local node 1)
        if e - 1 >= 0:
            B[e - 1, sl] = w[sl] * left
        if e < n:
            B[e, sl] = w[sl] * right
    return x, B
