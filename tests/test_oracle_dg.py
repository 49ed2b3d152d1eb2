"""Pins of the oracle's DG-in-time matrices and time transfers.

Each check compares the quadrature-assembled matrices with something fixed
independently of them: numbers the paper prints, textbook closed forms, or
exact polynomial identities."""
import os

import numpy as np
import pytest

from oracle import dg_time, hierarchy, transfer


def read_mu_star(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "mu_star.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_mu_star_matches_printed_values(golden_dir):
    """Remark on the critical parameter (eq. chap4_equationOptDiscrParam):
    mu*_0..mu*_3 printed to 10 digits."""
    printed = read_mu_star(golden_dir)
    for p in range(4):
        assert abs(hierarchy.mu_star(p) - printed[str(p)]) < 1e-9, p


def test_mu_star_closed_forms_and_limit(golden_dir):
    printed = read_mu_star(golden_dir)
    # p_t = 0 and p_t = 1 closed forms printed in the same remark
    assert abs(hierarchy.mu_star(0) - np.sqrt(2.0) / 3.0) < 1e-12
    mu1 = (-3.0 - np.sqrt(2.0) + np.sqrt(11.0 + 12.0 * np.sqrt(2.0))) / 3.0
    assert abs(hierarchy.mu_star(1) - mu1) < 1e-12
    # p_t -> infinity: R -> exp, so exp(-3 mu) = sqrt(2) - 1
    assert abs(-np.log(np.sqrt(2.0) - 1.0) / 3.0 - printed["inf"]) < 1e-9
    # and the high-degree Pade roots approach it
    assert abs(hierarchy.mu_star(8) - printed["inf"]) < 1e-9


def test_mu_star_from_assembled_dg_matrices(golden_dir):
    """mu* recomputed from the eigenvalue of the oracle's own
    (K_tau + lambda M_tau)^{-1} N_tau reproduces the printed constants; this
    pins K_tau, M_tau and N_tau (Lemma chap4_theorem2 + the remark)."""
    printed = read_mu_star(golden_dir)
    tau = 1.0
    for p in range(4):
        K, M, N = dg_time.time_matrices(p, tau)

        def R(z):   # z = -lambda tau
            lam = -z / tau
            ev = np.linalg.eigvals(np.linalg.solve(K + lam * M, N))
            return ev[np.argmax(np.abs(ev))].real

        lo, hi, target = 0.0, 1.0, np.sqrt(2.0) - 1.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if R(-3.0 * mid) > target:
                lo = mid
            else:
                hi = mid
        assert abs(0.5 * (lo + hi) - printed[str(p)]) < 1e-9, p


@pytest.mark.parametrize("p", range(6))
def test_dg_stability_function_is_pade(p):
    """sigma((K + lambda M)^{-1} N) = {0, R(-lambda tau)} (Lemma chap4_theorem2,
    with the sign reading R(-lambda tau))."""
    tau = 0.37
    K, M, N = dg_time.time_matrices(p, tau)
    for lam in [0.0, 0.3, 2.0, 17.0, 400.0, 0.5 + 3.0j]:
        ev = np.linalg.eigvals(np.linalg.solve(K + lam * M, N))
        ev = ev[np.argsort(np.abs(ev))]
        assert np.all(np.abs(ev[:-1]) < 1e-10)
        assert abs(ev[-1] - hierarchy.pade_R(p, -lam * tau)) < 1e-11


def test_pade_textbook_properties():
    # (0,1) Pade of exp is 1/(1-z): DG degree 0 is backward Euler (Section 1)
    for z in [-0.1, -2.0, -30.0]:
        assert abs(hierarchy.pade_R(0, z) - 1.0 / (1.0 - z)) < 1e-15
    # (p,p+1) Pade approximates exp to order 2p+1: error ~ z^{2p+2}
    for p in range(4):
        e1 = abs(hierarchy.pade_R(p, -1e-2) - np.exp(-1e-2))
        e2 = abs(hierarchy.pade_R(p, -5e-3) - np.exp(-5e-3))
        if e1 > 1e-15:
            assert abs(np.log2(e1 / e2) - (2 * p + 2)) < 0.1
    # L-stable: R(z) -> 0 as z -> -inf
    for p in range(4):
        assert abs(hierarchy.pade_R(p, -1e8)) < 1e-7


def test_dg0_is_backward_euler():
    """p_t = 0: K = 1, M = tau, N = 1, i.e. (M_h + tau K_h) u_n = M_h u_{n-1} + f_n."""
    K, M, N = dg_time.time_matrices(0, 0.25)
    assert np.allclose(K, [[1.0]]) and np.allclose(M, [[0.25]]) and np.allclose(N, [[1.0]])


def test_dg_matrices_integration_by_parts():
    """K + K^T = psi(t_n) psi(t_n)^T + psi(t_{n-1}) psi(t_{n-1})^T and N is the
    rank-one product of the end trace (trial) and the start trace (test)."""
    for p in range(5):
        K, M, N = dg_time.time_matrices(p, 0.7)
        end = dg_time.slab_basis_values(p, 0.7, [0.7])[:, 0]
        start = dg_time.slab_basis_values(p, 0.7, [0.0])[:, 0]
        assert np.allclose(K + K.T, np.outer(end, end) + np.outer(start, start), atol=1e-13)
        assert np.allclose(N, np.outer(start, end), atol=1e-14)
        assert np.allclose(M, M.T) and np.all(np.linalg.eigvalsh(M) > 0)


def test_time_restriction_legendre_p1():
    """Hand derivation for the Legendre basis, p_t = 1: on the first fine slab
    the coarse P_1 equals (P_0 ... ) -> R_1^T = [[1, -1/2], [0, 1/2]],
    R_2^T = [[1, 1/2], [0, 1/2]] (rows fine, columns coarse)."""
    R1, R2 = transfer.time_blocks(1, 0.3)
    assert np.allclose(R1.T, [[1.0, -0.5], [0.0, 0.5]], atol=1e-14)
    assert np.allclose(R2.T, [[1.0, 0.5], [0.0, 0.5]], atol=1e-14)


@pytest.mark.parametrize("p", range(5))
def test_prolongation_reproduces_coarse_functions(p):
    """P = R^T is the exact injection of coarse DG polynomials into the fine
    slabs (nested spaces, eq. chap4_restrictionTime)."""
    tau = 0.2
    R1, R2 = transfer.time_blocks(p, tau)
    rng = np.random.default_rng(p)
    c = rng.standard_normal(p + 1)                     # coarse coefficients on (0, 2 tau)
    t1 = np.linspace(0.0, tau, 7)
    t2 = np.linspace(tau, 2 * tau, 7)
    coarse1 = c @ dg_time.slab_basis_values(p, 2 * tau, t1)
    coarse2 = c @ dg_time.slab_basis_values(p, 2 * tau, t2)
    fine1 = (R1.T @ c) @ dg_time.slab_basis_values(p, tau, t1)
    fine2 = (R2.T @ c) @ dg_time.slab_basis_values(p, tau, t2 - tau)
    assert np.allclose(fine1, coarse1, atol=1e-13)
    assert np.allclose(fine2, coarse2, atol=1e-13)
