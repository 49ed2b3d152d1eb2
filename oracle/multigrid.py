"""Space-time multigrid (Section 2) on the hierarchy of ``hierarchy.build_levels``.

* damped block-Jacobi smoother, eq. (chap4_smoother), with the exact block
  inverse D^{-1} = diag(A)^{-1} used throughout Section 3 (one sparse LU of A
  per level, applied to all time steps), or the inexact D~^{-1} of the Remark
  on the V-cycle approximation (one spatial V-cycle per time step);
* coarse operators re-discretised on (tau_L, h_L) (Section 3.2);
* restriction / prolongation of ``transfer`` with P = R^T (Section 2);
* coarsest level solved exactly (Section 2): one time step with the LU of A,
  several steps by forward substitution;
* V-cycle (gamma = 1) repeated until ||r_k|| / ||r_0|| <= eps (Section 2),
  reading: l2 norm of the residual coefficient vector;
* forward substitution in time (Section 1), the sequential reference solve;
* the adjoint: the same cycle on L^T (a block upper-bidiagonal system solved
  backward in time), with the same transfers since (R L P)^T = R L^T P when
  R = P^T.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import hierarchy, spacetime, transfer


class SpatialVCycle:
    """Inexact block inverse of the Remark on the V-cycle approximation in space
    (eq. chap4_smootherApprox): one multigrid V-cycle in space for
    A_{tau,h} = K_tau (x) M_h + M_tau (x) K_h with zero initial guess, damped
    point-block Jacobi smoothing with D^x = diag{(M_h)_jj K_tau + (K_h)_jj M_tau}
    (in 1D: 2h/3 K_tau + 2/h M_tau), nu_x pre- and post-smoothing steps,
    restriction R_x (x) I, prolongation its transpose, coarse operators
    A_{tau,2h} re-discretised, and an exact solve on one node."""

    def __init__(self, d, n, p_t, tau, nu_x=2, omega_x=2.0 / 3.0):
        self.nu_x, self.omega_x = nu_x, omega_x
        self.q = p_t + 1
        self.levels = []
        nl = n
        while True:
            disc = spacetime.Discretization(d, nl, p_t, 1, tau)
            A = disc.A.tocsr()
            Nx = disc.Nx
            # point blocks A[(l, j), (l', j)] of every node j, shape (Nx, q, q)
            blocks = np.zeros((Nx, self.q, self.q))
            for a in range(self.q):
                for b in range(self.q):
                    blocks[:, a, b] = A[a * Nx:(a + 1) * Nx, b * Nx:(b + 1) * Nx].diagonal()
            lvl = {"n": nl, "Nx": Nx, "A": A, "blocks": blocks, "R": None, "lu": None}
            self.levels.append(lvl)
            if nl == 1:
                lvl["lu"] = spla.splu(A.tocsc())
                break
            Rx = transfer.space_restriction(d, nl)
            lvl["R"] = sp.kron(sp.identity(self.q), Rx, format="csr")
            nl = (nl - 1) // 2

    def _jacobi(self, lvl, x, b, adjoint):
        A = lvl["A"].T if adjoint else lvl["A"]
        blocks = np.transpose(lvl["blocks"], (0, 2, 1)) if adjoint else lvl["blocks"]
        r = b - A @ x                                   # (q Nx, m)
        q, Nx = self.q, lvl["Nx"]
        rn = r.reshape(q, Nx, -1).transpose(1, 0, 2)     # (Nx, q, m)
        dn = np.linalg.solve(blocks, rn)
        return x + self.omega_x * dn.transpose(1, 0, 2).reshape(q * Nx, -1)

    def apply(self, b, adjoint=False, i=0):
        """Approximate A^{-1} b for the columns of b (shape (q Nx, m))."""
        lvl = self.levels[i]
        if lvl["lu"] is not None:
            return (lvl["lu"].solve(b, trans="T") if adjoint else lvl["lu"].solve(b))
        A = lvl["A"].T if adjoint else lvl["A"]
        x = np.zeros_like(b)
        for _ in range(self.nu_x):
            x = self._jacobi(lvl, x, b, adjoint)
        bc = lvl["R"] @ (b - A @ x)
        x = x + lvl["R"].T @ self.apply(bc, adjoint, i + 1)
        for _ in range(self.nu_x):
            x = self._jacobi(lvl, x, b, adjoint)
        return x


class Level:
    def __init__(self, d, lv, p_t, smoother="exact", nu_x=2, omega_x=2.0 / 3.0):
        self.disc = spacetime.Discretization(d, lv["n"], p_t, lv["N"], lv["tau"])
        self.full = lv["full"]
        self.mu = lv["mu"]
        self.lu = spla.splu(self.disc.A.tocsc())
        self._luT = None       # LU of A^T, built on first adjoint use
        self.R = None          # restriction to the next coarser level
        self.inexact = SpatialVCycle(d, lv["n"], p_t, lv["tau"], nu_x, omega_x) if smoother == "vcycle" else None

    @property
    def luT(self):
        if self._luT is None:
            self._luT = spla.splu(self.disc.A.T.tocsc())
        return self._luT

    def block_solve(self, r, adjoint=False):
        """D^{-1} r: A^{-1} (or A^{-T}) applied to every time block of r, or its
        approximation by one spatial V-cycle when the level smoother is 'vcycle'."""
        if self.inexact is not None:
            return self.inexact.apply(np.ascontiguousarray(r.T), adjoint).T
        lu = self.luT if adjoint else self.lu
        return lu.solve(np.ascontiguousarray(r.T)).T

    def exact_block_solve(self, r, adjoint=False):
        lu = self.luT if adjoint else self.lu
        return lu.solve(np.ascontiguousarray(r.T)).T

    def residual(self, u, f, adjoint=False):
        if adjoint:
            return f - spacetime.apply_LT(self.disc, u)
        return f - spacetime.apply_L(self.disc, u)


class Hierarchy:
    """Levels finest-first (index 0 is the finest, the paper's M_L)."""

    def __init__(self, d, n, p_t, N, T, coarsening="auto", coarsest_steps=1, smoother="exact", nu_x=2,
                 omega_x=2.0 / 3.0):
        self.params = hierarchy.build_levels(d, n, p_t, N, T, coarsening, coarsest_steps)
        self.levels = [Level(d, lv, p_t, smoother, nu_x, omega_x) for lv in self.params]
        for i in range(len(self.levels) - 1):
            self.levels[i].R = transfer.restriction(self.levels[i].disc, self.levels[i].full)

    @property
    def finest(self):
        return self.levels[0]


def smooth(level, u, f, nu, omega, adjoint=False):
    """nu steps of u <- u + omega D^{-1} (f - L u), eq. (chap4_smoother)."""
    for _ in range(nu):
        u = u + omega * level.block_solve(level.residual(u, f, adjoint), adjoint)
    return u


def coarsest_solve(level, f, adjoint=False):
    """Exact solve on the coarsest level (Section 2), whatever the smoother."""
    if level.disc.N == 1:
        return level.exact_block_solve(f, adjoint)
    return backward_substitution(level, f) if adjoint else forward_substitution(level, f)


def forward_substitution(level, f):
    """A u_1 = f_1, A u_n = f_n - B u_{n-1} (Section 1)."""
    disc = level.disc
    u = np.zeros_like(f)
    for s in range(disc.N):
        rhs = f[s].copy()
        if s > 0:
            rhs -= disc.B @ u[s - 1]
        u[s] = level.lu.solve(rhs)
    return u


def backward_substitution(level, g):
    """A^T lam_N = g_N, A^T lam_n = g_n - B^T lam_{n+1}: the transposed system."""
    disc = level.disc
    lam = np.zeros_like(g)
    for s in range(disc.N - 1, -1, -1):
        rhs = g[s].copy()
        if s < disc.N - 1:
            rhs -= disc.B.T @ lam[s + 1]
        lam[s] = level.luT.solve(rhs)
    return lam


def vcycle(H, i, u, f, nu1=2, nu2=2, omega=0.5, adjoint=False, gamma=1):
    """One multigrid cycle on level i (0 = finest) for L u = f (or L^T u = f),
    Section 2: pre-smoothing, restriction of the residual, gamma applications of
    the cycle on the coarse level to the correction equation (from zero; gamma = 1
    V-cycle, 2 W-cycle; the coarsest level is solved exactly), prolongation of
    the correction, post-smoothing."""
    lv = H.levels[i]
    if i == len(H.levels) - 1:
        return coarsest_solve(lv, f, adjoint)
    u = smooth(lv, u, f, nu1, omega, adjoint)
    r = lv.residual(u, f, adjoint)
    coarse = H.levels[i + 1]
    fc = (lv.R @ r.reshape(-1)).reshape(coarse.disc.shape())
    ec = np.zeros_like(fc)
    for _ in range(gamma):
        ec = vcycle(H, i + 1, ec, fc, nu1, nu2, omega, adjoint, gamma)
    u = u + (lv.R.T @ ec.reshape(-1)).reshape(lv.disc.shape())
    u = smooth(lv, u, f, nu2, omega, adjoint)
    return u


def solve(H, f, u=None, rtol=1e-8, maxit=100, nu1=2, nu2=2, omega=0.5, adjoint=False, gamma=1):
    """Repeat cycles (gamma = 1: V, 2: W) until ||f - L u||_2 <= rtol ||f - L u^0||_2.

    Returns (u, iterations, history of residual norms)."""
    lv = H.finest
    f = np.asarray(f, dtype=np.float64).reshape(lv.disc.shape())
    u = np.zeros_like(f) if u is None else np.array(u, dtype=np.float64).reshape(lv.disc.shape())
    r0 = np.linalg.norm(lv.residual(u, f, adjoint))
    hist = [r0]
    it = 0
    while hist[-1] > rtol * r0 and it < maxit and r0 > 0:
        u = vcycle(H, 0, u, f, nu1, nu2, omega, adjoint, gamma)
        it += 1
        hist.append(np.linalg.norm(lv.residual(u, f, adjoint)))
    return u, it, hist


def two_grid(H, u, f, nu1, nu2, omega):
    """Two-grid cycle: smoothing on level 0, exact solve on level 1 (Section 3.2)."""
    lv = H.levels[0]
    u = smooth(lv, u, f, nu1, omega)
    r = lv.residual(u, f)
    coarse = H.levels[1]
    fc = (lv.R @ r.reshape(-1)).reshape(coarse.disc.shape())
    ec = forward_substitution(coarse, fc)
    u = u + (lv.R.T @ ec.reshape(-1)).reshape(lv.disc.shape())
    return smooth(lv, u, f, nu2, omega)


def tracking_gradients(H, u_d, f, u0_ic, rtol=1e-12, maxit=100):
    """Loss J = 0.5 ||u - u_d||^2 over the space-time coefficient vector.

    Forward: L u = f + IC term.  Adjoint: L^T lam = u - u_d.  Then
    dJ/df = lam and dJ/du0_ic = M_h sum_k psi_k(t_0^+) lam_{1,k}
    (the derivative of the block-1 initial-value term)."""
    disc = H.finest.disc
    g = spacetime.add_ic(disc, f, u0_ic)
    u, _, _ = solve(H, g, rtol=rtol, maxit=maxit)
    lam, _, _ = solve(H, u - u_d.reshape(disc.shape()), rtol=rtol, maxit=maxit, adjoint=True)
    start = spacetime.dg_time.start_trace(disc.p_t, disc.tau)
    lam1 = lam[0].reshape(disc.q, disc.Nx)
    grad_u0 = disc.Mh @ (start @ lam1)
    J = 0.5 * np.sum((u - u_d.reshape(disc.shape())) ** 2)
    return J, u, lam, grad_u0
