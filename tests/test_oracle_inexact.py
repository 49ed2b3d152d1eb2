"""Pins of the oracle's inexact block inverse (Remark on the V-cycle
approximation in space): one spatial multigrid V-cycle per time step with
damped point-block Jacobi (omega_x = 2/3, nu_x = 2), and its Fourier analysis."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import hierarchy, lfa, multigrid, spacetime, transfer
from paper_1411_0519_gb300 import workloads


@pytest.mark.parametrize("d,n,p,mu", [(1, 63, 1, 1e-2), (1, 63, 0, 30.0), (2, 15, 1, 1.0), (2, 31, 2, 100.0)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_spatial_vcycle_is_a_convergent_approximate_inverse(d, n, p, mu, adjoint):
    """x <- x + V(b - A x) converges to A^{-1} b (A^{-T} b) at a textbook
    multigrid rate; this pins the point-block Jacobi blocks, the spatial
    transfers and the re-discretised coarse operators."""
    h = 1.0 / (n + 1)
    tau = mu * h * h
    V = multigrid.SpatialVCycle(d, n, p, tau)
    disc = spacetime.Discretization(d, n, p, 1, tau)
    A = disc.A.T.tocsc() if adjoint else disc.A.tocsc()
    b = np.random.default_rng(0).standard_normal((A.shape[0], 3))
    x_ref = spla.spsolve(A, b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(12):
        x = x + V.apply(b - A @ x, adjoint)
        errs.append(np.abs(x - x_ref).max() / np.abs(x_ref).max())
    rates = np.array(errs[1:]) / np.array(errs[:-1])
    assert errs[-1] < 1e-8
    assert rates[:6].max() < 0.3


@pytest.mark.parametrize("d,n", [(1, 31), (2, 15)])
def test_spatial_coarse_operator_is_galerkin(d, n):
    """(R_x (x) I) A_{tau,h} (R_x (x) I)^T = A_{tau,2h}: the coarse blocks of the
    spatial V-cycle equal the Galerkin products (nested Q1 spaces)."""
    tau = 0.013
    for p in [0, 1, 2]:
        fine = spacetime.Discretization(d, n, p, 1, tau)
        coarse = spacetime.Discretization(d, (n - 1) // 2, p, 1, tau)
        R = sp.kron(sp.identity(p + 1), transfer.space_restriction(d, n))
        G = (R @ fine.A @ R.T).toarray()
        assert np.abs(G - coarse.A.toarray()).max() < 1e-13 * np.abs(coarse.A.toarray()).max()


@pytest.mark.parametrize("p", [0, 1])
def test_inexact_lfa_tends_to_exact_lfa(p):
    """With many spatial smoothing steps the spatial iteration matrix vanishes and
    the two-grid factor of the inexact smoother equals the exact one; with
    nu_x = 2 it is a little larger for small mu (as the Remark states)."""
    for mu in [0.01, 1.0, 100.0]:
        a = lfa.two_grid_factor_batch(p, mu, 2, False, Nx=128, Nt=32)
        b = lfa.two_grid_factor_inexact_batch(p, mu, 2, False, Nx=128, Nt=32, nu_x=40)
        assert abs(a - b) < 1e-3
    a = lfa.two_grid_factor_batch(p, 0.01, 2, False, Nx=128, Nt=32)
    c = lfa.two_grid_factor_inexact_batch(p, 0.01, 2, False, Nx=128, Nt=32)
    assert c > a


def measured_inexact(p, mu, full, n=127, N=32, iters=25):
    h = 1.0 / (n + 1)
    T = mu * h * h * N
    H = multigrid.Hierarchy(1, n, p, N, T, coarsening="full" if full else "semi", coarsest_steps=N // 2,
                            smoother="vcycle")
    u = workloads.uniform_iterate(1, n, p, N, seed=0).reshape(H.finest.disc.shape())
    f = np.zeros_like(u)
    rs = [np.linalg.norm(H.finest.residual(u, f))]
    for _ in range(iters):
        u = multigrid.two_grid(H, u, f, 2, 2, 0.5)
        rs.append(np.linalg.norm(H.finest.residual(u, f)))
    rs = np.array(rs)
    return float(np.max(rs[1:] / rs[:-1]))


@pytest.mark.parametrize("p", [0, 1])
def test_inexact_two_grid_agrees_with_its_lfa(p):
    """Figures of the Remark (data not printed): measured two-grid factors with the
    inexact smoother agree with the LFA of eq. (chap4_twoGridIterationMatrixApprox)
    within 0.05 and stay <= 1/2 for semi coarsening and for full coarsening at mu >= mu*."""
    ms = hierarchy.mu_star(p)
    for mu, full in [(1e-3, False), (1.0, False), (100.0, False), (ms, True), (10.0, True)]:
        meas = measured_inexact(p, mu, full)
        th = lfa.two_grid_factor_inexact_batch(p, mu, 2, full, Nx=128, Nt=32)
        assert abs(meas - th) < 0.05, (mu, full, meas, th)
        assert meas <= 0.5 and th <= 0.5


@pytest.mark.parametrize("d,n,N,p", [(1, 15, 8, 1), (2, 7, 8, 1), (2, 7, 4, 2)])
def test_inexact_mg_fixed_point_equals_direct_solve(d, n, N, p):
    H = multigrid.Hierarchy(d, n, p, N, 0.5, smoother="vcycle")
    disc = H.finest.disc
    f = np.random.default_rng(1).uniform(-1, 1, disc.shape())
    u, it, _ = multigrid.solve(H, f, rtol=1e-14, maxit=80)
    ud = spla.spsolve(spacetime.global_matrix(disc), f.reshape(-1)).reshape(disc.shape())
    assert np.abs(u - ud).max() <= 1e-12 * np.abs(ud).max()


@pytest.mark.parametrize("d,n,N,p,T", [(1, 63, 64, 1, 1.0), (2, 31, 64, 1, 1.0), (2, 31, 32, 0, 1.0),
                                       (2, 15, 16, 2, 16.0)])
def test_inexact_iteration_counts_in_the_tables_band(d, n, N, p, T):
    """Tables 1-2 use this smoother (nu_x = 2, omega_x = 2/3) and report 4-9
    V-cycles to eps = 1e-8 with f = 0 and a random initial iterate."""
    H = multigrid.Hierarchy(d, n, p, N, T, smoother="vcycle")
    disc = H.finest.disc
    u0 = workloads.uniform_iterate(d, n, p, N, seed=0).reshape(disc.shape())
    _, it, _ = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=30)
    assert 4 <= it <= 9
