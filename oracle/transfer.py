"""Restriction and prolongation (Section 2 and Section 3.2).

Time (eq. (chap4_restrictionTime)): the prolongation is the L2 projection of
a coarse DG function on (0, 2 tau) onto the two fine slabs,

    R_1^T = M_tau^{-1} Mt^1,   Mt^1[k,l] = int_0^tau     psit_l(t) psi_k(t)       dt,
    R_2^T = M_tau^{-1} Mt^2,   Mt^2[k,l] = int_tau^2tau  psit_l(t) psi_k(t - tau) dt,

with psit_l the coarse basis on (0, 2 tau).  Reading of a misprint there: the
second fine slab uses the fine basis shifted to (tau, 2 tau), psi_k(t - tau).
R_1, R_2 are the transposes; coarse step m (1-based) receives
R_1 r_{2m-1} + R_2 r_{2m}.

Space (eq. (chap4_spaceRestrictionProlongation)): 1D rows (1/2)[1 2 1] on the
fine nodes 2j-1, 2j, 2j+1 of coarse node j (reading of the dimension labels and
first row printed there, consistent with the symbol R_x = 1 + cos(theta) of
Lemma 25); P_x = R_x^T; tensor products in d dimensions.

The prolongation is the transpose of the restriction (Section 2: R = P^T).
"""
import numpy as np
import scipy.sparse as sp

from . import dg_time


def time_blocks(p_t, tau):
    """(R1, R2): q x q blocks, row = coarse dof k, column = fine dof l."""
    q = p_t + 1
    _, M, _ = dg_time.time_matrices(p_t, tau)
    t1, w1 = dg_time.gauss_on(0.0, tau, q + 1)
    t2, w2 = dg_time.gauss_on(tau, 2.0 * tau, q + 1)
    coarse1 = dg_time.slab_basis_values(p_t, 2.0 * tau, t1)   # psit_l on slab 1
    coarse2 = dg_time.slab_basis_values(p_t, 2.0 * tau, t2)   # psit_l on slab 2
    fine1 = dg_time.slab_basis_values(p_t, tau, t1)
    fine2 = dg_time.slab_basis_values(p_t, tau, t2 - tau)
    Mt1 = np.zeros((q, q))
    Mt2 = np.zeros((q, q))
    for k in range(q):
        for l in range(q):
            Mt1[k, l] = np.sum(w1 * coarse1[l] * fine1[k])
            Mt2[k, l] = np.sum(w2 * coarse2[l] * fine2[k])
    R1T = np.linalg.solve(M, Mt1)
    R2T = np.linalg.solve(M, Mt2)
    return R1T.T, R2T.T


def space_restriction_1d(n_fine):
    """R_x, shape (n_c, n_f) with n_c = (n_f - 1) / 2."""
    n_c = (n_fine - 1) // 2
    R = sp.lil_matrix((n_c, n_fine))
    for j in range(1, n_c + 1):            # 1-based coarse node j <-> fine node 2j
        R[j - 1, 2 * j - 2] = 0.5
        R[j - 1, 2 * j - 1] = 1.0
        R[j - 1, 2 * j] = 0.5
    return R.tocsr()


def space_restriction(d, n_fine):
    R1 = space_restriction_1d(n_fine)
    R = R1
    for _ in range(d - 1):
        R = sp.kron(R1, R, format="csr")
    return R


def time_restriction(N_fine, p_t, tau_fine):
    """Block matrix (N_c q) x (N_f q) of eq. (chap4_restrictionTime)."""
    R1, R2 = time_blocks(p_t, tau_fine)
    N_c = N_fine // 2
    q = p_t + 1
    Rt = sp.lil_matrix((N_c * q, N_fine * q))
    for m in range(N_c):
        Rt[m * q:(m + 1) * q, (2 * m) * q:(2 * m + 1) * q] = R1
        Rt[m * q:(m + 1) * q, (2 * m + 1) * q:(2 * m + 2) * q] = R2
    return Rt.tocsr()


def restriction(fine, full):
    """Space-time restriction from level ``fine`` (a Discretization): semi
    coarsening R_s = R^t (x) I, full coarsening R_f = R^t (x) R_x (our vector
    layout is time-major, so the time factor is on the left)."""
    Rt = time_restriction(fine.N, fine.p_t, fine.tau)
    Rs = space_restriction(fine.d, fine.n) if full else sp.identity(fine.Nx, format="csr")
    return sp.kron(Rt, Rs, format="csr")
