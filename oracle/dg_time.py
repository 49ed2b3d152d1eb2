"""DG-in-time element matrices (Section 1, definitions of K_tau, M_tau, N_tau).

Reading of the paper (the basis is left open in Section 1): on every slab
(t_{n-1}, t_n) the local basis is psi_k(t) = P_k(2 (t - t_{n-1}) / tau - 1),
k = 0..p_t, with P_k the Legendre polynomial of degree k.  The matrices are
computed from their integral definitions by Gauss-Legendre quadrature that is
exact for the polynomial degrees involved; no closed form is used.

    K_tau[k,l] = - int psi_l d/dt psi_k dt + psi_l(t_n) psi_k(t_n)
    M_tau[k,l] =   int psi_l psi_k dt
    N_tau[k,l] =   psi_l^{n-1}(t_{n-1}) psi_k^{n}(t_{n-1})

Indices: k is the test function (row), l the trial function (column).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre_basis(p_t):
    """Legendre polynomials P_0..P_{p_t} on the reference interval [-1, 1]."""
    return [npleg.Legendre.basis(k) for k in range(p_t + 1)]


def slab_basis_values(p_t, tau, t):
    """psi_k(t) for t in [0, tau] (slab-local time), shape (q, len(t))."""
    s = 2.0 * np.asarray(t, dtype=np.float64) / tau - 1.0
    return np.array([P(s) for P in legendre_basis(p_t)])


def slab_basis_derivatives(p_t, tau, t):
    """d/dt psi_k(t) for t in [0, tau], shape (q, len(t))."""
    s = 2.0 * np.asarray(t, dtype=np.float64) / tau - 1.0
    return np.array([(2.0 / tau) * P.deriv()(s) for P in legendre_basis(p_t)])


def gauss_on(a, b, npts):
    """Gauss-Legendre nodes and weights on [a, b]."""
    x, w = npleg.leggauss(npts)
    return 0.5 * (b - a) * (x + 1.0) + a, 0.5 * (b - a) * w


def time_matrices(p_t, tau):
    """(K_tau, M_tau, N_tau), each (p_t+1) x (p_t+1), Section 1."""
    q = p_t + 1
    t, w = gauss_on(0.0, tau, q + 1)           # exact up to degree 2q+1
    psi = slab_basis_values(p_t, tau, t)       # (q, nq)
    dpsi = slab_basis_derivatives(p_t, tau, t)
    end = slab_basis_values(p_t, tau, [tau])[:, 0]    # psi_k(t_n)
    start = slab_basis_values(p_t, tau, [0.0])[:, 0]  # psi_k(t_{n-1})
    K = np.zeros((q, q))
    M = np.zeros((q, q))
    Nt = np.zeros((q, q))
    for k in range(q):
        for l in range(q):
            K[k, l] = -np.sum(w * psi[l] * dpsi[k]) + end[l] * end[k]
            M[k, l] = np.sum(w * psi[l] * psi[k])
            # trial psi_l of the previous slab evaluated at its right end,
            # test psi_k of the current slab evaluated at its left end
            Nt[k, l] = end[l] * start[k]
    return K, M, Nt


def start_trace(p_t, tau):
    """psi_k(t_{n-1}^+), the value of each basis function at the slab start."""
    return slab_basis_values(p_t, tau, [0.0])[:, 0]
