"""Pins of the oracle's spatial FE matrices and the space-time transfers."""
import numpy as np
import pytest

from oracle import fe_space, spacetime, transfer


@pytest.mark.parametrize("n", [1, 3, 7, 31])
def test_fe_1d_matches_printed_stencils_and_eigenvalues(n):
    """Section 3 prints M_h = h/6 tridiag(1,4,1), K_h = 1/h tridiag(-1,2,-1); the
    eigenvectors are sin(j k pi h) with eigenvalues h/3 (2 + cos k pi h) and
    2/h (1 - cos k pi h) (the symbols of Lemma 17)."""
    M, K = fe_space.fe_1d(n)
    h = 1.0 / (n + 1)
    Mref = h / 6.0 * (4 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1))
    Kref = 1.0 / h * (2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))
    assert np.allclose(M, Mref, atol=1e-15)
    assert np.allclose(K, Kref, atol=1e-12)
    j = np.arange(1, n + 1)
    for k in range(1, n + 1):
        v = np.sin(j * k * np.pi * h)
        th = k * np.pi * h
        assert np.allclose(M @ v, h / 3.0 * (2 + np.cos(th)) * v, atol=1e-13)
        assert np.allclose(K @ v, 2.0 / h * (1 - np.cos(th)) * v, atol=1e-10)


def test_q1_2d_against_direct_element_assembly():
    """Brute force: assemble the 2D Q1 mass and stiffness matrices element by
    element with a 2D Gauss rule on the bilinear basis (no Kronecker identity)
    and compare with the tensor-product construction of fe_space."""
    n = 5
    h = 1.0 / (n + 1)
    M, K = fe_space.fe_matrices(2, n)
    g, w = np.polynomial.legendre.leggauss(3)
    Md = np.zeros((n * n, n * n))
    Kd = np.zeros((n * n, n * n))
    for ey in range(n + 1):
        for ex in range(n + 1):
            loc = [(ex + a, ey + b) for b in range(2) for a in range(2)]   # global node coords
            for gy, wy in zip(g, w):
                for gx, wx in zip(g, w):
                    sx, sy = 0.5 * (gx + 1), 0.5 * (gy + 1)              # in [0,1]^2
                    wgt = wx * wy * 0.25 * h * h
                    phi, dx, dy = [], [], []
                    for b in range(2):
                        for a in range(2):
                            fx = (1 - sx) if a == 0 else sx
                            fy = (1 - sy) if b == 0 else sy
                            phi.append(fx * fy)
                            dx.append(((-1.0 if a == 0 else 1.0) / h) * fy)
                            dy.append(fx * ((-1.0 if b == 0 else 1.0) / h))
                    for i, (ix, iy) in enumerate(loc):
                        if not (1 <= ix <= n and 1 <= iy <= n):
                            continue
                        I = (iy - 1) * n + (ix - 1)
                        for j, (jx, jy) in enumerate(loc):
                            if not (1 <= jx <= n and 1 <= jy <= n):
                                continue
                            J = (jy - 1) * n + (jx - 1)
                            Md[I, J] += wgt * phi[i] * phi[j]
                            Kd[I, J] += wgt * (dx[i] * dx[j] + dy[i] * dy[j])
    assert np.allclose(M.toarray(), Md, atol=1e-15)
    assert np.allclose(K.toarray(), Kd, atol=1e-13)


def galerkin_case(d, n, p, N, full):
    tau = 0.013
    fine = spacetime.Discretization(d, n, p, N, tau)
    R = transfer.restriction(fine, full)
    Lf = spacetime.global_matrix(fine)
    nc = (n - 1) // 2 if full else n
    coarse = spacetime.Discretization(d, nc, p, N // 2, 2 * tau)
    Lc = spacetime.global_matrix(coarse).toarray()
    G = (R @ Lf @ R.T).toarray()
    return np.abs(G - Lc).max() / np.abs(Lc).max()


@pytest.mark.parametrize("d,n,N", [(1, 15, 8), (2, 7, 4), (3, 3, 4)])
@pytest.mark.parametrize("p", [0, 1, 2])
@pytest.mark.parametrize("full", [False, True])
def test_galerkin_identity(d, n, N, p, full):
    """R L_{tau,h} P = L_{2tau,h} (semi) and L_{2tau,2h} (full): the re-discretised
    coarse operators of Section 3.2 equal the Galerkin products, because the
    spaces are nested and R = P^T (Section 2)."""
    assert galerkin_case(d, n, p, N, full) < 1e-13


def test_space_restriction_rows():
    """1D rows (1/2)[1 2 1] at fine nodes 2j-1, 2j, 2j+1; symbol R_x(theta) = 1 + cos(theta)
    (Lemma 25): applied to a fine Fourier mode it returns (1 + cos theta) times the
    coarse mode at frequency 2 theta (away from the boundary)."""
    n = 31
    R = transfer.space_restriction_1d(n).toarray()
    j = np.arange(1, n + 1)
    th = 0.4
    fine = np.exp(1j * j * th)
    coarse = R @ fine
    jc = np.arange(1, (n - 1) // 2 + 1)
    assert np.allclose(coarse, (1 + np.cos(th)) * np.exp(1j * 2 * jc * th))


def test_load_vector_of_constant():
    """int f phi_j psi_l for f = 1: h^d in space (interior hats have integral h),
    tau for l = 0 and 0 for l >= 1 (Legendre orthogonality)."""
    d, n, p, N, T = 2, 7, 2, 4, 2.0
    disc = spacetime.Discretization(d, n, p, N, T / N)
    f = spacetime.load_vector(disc, lambda c, t: np.ones_like(c[0]), T)
    f = f.reshape(N, p + 1, -1)
    h = 1.0 / (n + 1)
    assert np.allclose(f[:, 0], (T / N) * h ** d)
    assert np.allclose(f[:, 1:], 0.0, atol=1e-15)
