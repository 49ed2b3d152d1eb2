"""The space-time block system (Section 1).

    A_{tau,h} = K_tau (x) M_h + M_tau (x) K_h,      B_{tau,h} = - N_tau (x) M_h,

and the block lower-bidiagonal system (chap4_generalLinearSystem)

    A u_1 = f_1,   B u_{n-1} + A u_n = f_n  (n = 2..N).

A space-time vector is stored as an array of shape (N, q * Nx): row n-1 holds
the block u_n of the paper, itself time-dof-major, u_n[l * Nx + j]
(Section 1, definition of f_{n+1}).  The load vector follows the same layout;
reading of the garbled index offset there: f_n integrates over
(t_{n-1}, t_n) with 1-based n.

The initial value enters through the n = 0 term of system (equation1):
f_1 <- f_1 + (N_tau (x) M_h) u_0, where the previous-slab trace of u_0 is the
nodal interpolant u0_ic of the initial value, i.e.
f_1[k, :] += psi_k(t_0^+) * (M_h u0_ic).
"""
import numpy as np
import scipy.sparse as sp

from . import dg_time, fe_space


class Discretization:
    """One space-time level: d, n, p_t, N, tau and its assembled matrices."""

    def __init__(self, d, n, p_t, N, tau):
        self.d, self.n, self.p_t, self.N, self.tau = d, n, p_t, N, float(tau)
        self.q = p_t + 1
        self.h = 1.0 / (n + 1)
        self.Nx = n ** d
        self.Kt, self.Mt, self.Nt = dg_time.time_matrices(p_t, self.tau)
        self.Mh, self.Kh = fe_space.fe_matrices(d, n)
        self.A = (sp.kron(self.Kt, self.Mh) + sp.kron(self.Mt, self.Kh)).tocsc()
        self.B = (-sp.kron(self.Nt, self.Mh)).tocsr()

    @property
    def mu(self):
        """Discretization parameter mu = tau / h^2 (Lemma 20)."""
        return self.tau / self.h ** 2

    @property
    def ndof(self):
        return self.N * self.q * self.Nx

    def shape(self):
        return (self.N, self.q * self.Nx)


def apply_L(disc, u):
    """(L u)_n = A u_n + B u_{n-1}, with u_0 = 0 (system (chap4_generalLinearSystem))."""
    out = (disc.A @ u.T).T
    out[1:] += (disc.B @ u[:-1].T).T
    return out


def apply_LT(disc, lam):
    """(L^T lam)_n = A^T lam_n + B^T lam_{n+1}, with lam_{N+1} = 0."""
    out = (disc.A.T @ lam.T).T
    out[:-1] += (disc.B.T @ lam[1:].T).T
    return out


def global_matrix(disc):
    """The whole N q Nx square matrix L as one sparse matrix (small cases only)."""
    N = disc.N
    diag = sp.kron(sp.identity(N), disc.A)
    sub = sp.kron(sp.diags([np.ones(N - 1)], [-1], shape=(N, N)), disc.B)
    return (diag + sub).tocsc()


def ic_term(disc, u0_ic):
    """Block-1 contribution of the initial value: psi_k(t_0^+) * (M_h u0_ic)."""
    start = dg_time.start_trace(disc.p_t, disc.tau)
    mu0 = disc.Mh @ np.asarray(u0_ic, dtype=np.float64).reshape(-1)
    return np.concatenate([start[k] * mu0 for k in range(disc.q)])


def add_ic(disc, f, u0_ic):
    """Right-hand side with the initial value folded into block 1."""
    g = np.array(f, dtype=np.float64, copy=True).reshape(disc.shape())
    g[0] += ic_term(disc, u0_ic)
    return g


def load_vector(disc, func, T, npts=5):
    """f_n[l Nx + j] = int_{t_{n-1}}^{t_n} int_Omega f(x,t) phi_j(x) psi_l(t) dx dt
    (Section 1), by tensor Gauss quadrature with ``npts`` points per element
    and per slab.  ``func(coords, t)`` takes a list of d coordinate arrays
    (broadcastable, axis order as ``numpy.meshgrid(..., indexing='ij')`` with
    the slowest axis first) and a scalar t."""
    d, n, q, N = disc.d, disc.n, disc.q, disc.N
    tau = T / N
    xg, Bm = fe_space.quadrature_1d(n, npts)
    tg, wt = dg_time.gauss_on(0.0, tau, npts)
    psi = dg_time.slab_basis_values(disc.p_t, tau, tg)       # (q, npts)
    grids = np.meshgrid(*([xg] * d), indexing="ij")            # slowest axis first
    out = np.zeros((N, q * disc.Nx))
    for s in range(N):
        acc = np.zeros((q,) + (n,) * d)
        for g in range(npts):
            vals = func(grids[::-1], s * tau + tg[g])            # coords passed as (x, y, z)
            proj = vals
            for ax in range(d):
                proj = np.tensordot(Bm, proj, axes=([1], [ax]))  # contracts axis ax
                proj = np.moveaxis(proj, 0, ax)
            for k in range(q):
                acc[k] += wt[g] * psi[k, g] * proj
        out[s] = acc.reshape(-1)
    return out


def _space_values(n, d, npts, coeffs):
    """Values of sum_j coeffs[j] phi_j at all element Gauss points; coeffs has
    shape (..., n, ..., n) with the last d axes spatial (x last)."""
    xg, Bm = fe_space.quadrature_1d(n, npts)
    # unweighted basis values: Bm holds w_g phi_j(x_g); recover phi by dividing the weights
    w = np.concatenate([dg_time.gauss_on(e / (n + 1.0), (e + 1) / (n + 1.0), npts)[1] for e in range(n + 1)])
    Phi = Bm / w[None, :]
    vals = coeffs
    lead = coeffs.ndim - d
    for ax in range(d):
        vals = np.tensordot(vals, Phi, axes=([lead + ax], [0]))   # new axis appended
        vals = np.moveaxis(vals, -1, lead + ax)
    return xg, w, vals


def l2_error(disc, u, exact, T, npts=5):
    """|| u_h - u ||_{L2(Omega x (0,T))} by tensor Gauss quadrature; ``exact``
    takes (coords list (x, y, z order), t)."""
    d, n, q, N = disc.d, disc.n, disc.q, disc.N
    tau = T / N
    tg, wt = dg_time.gauss_on(0.0, tau, npts)
    psi = dg_time.slab_basis_values(disc.p_t, tau, tg)
    total = 0.0
    for s in range(N):
        coeffs = u[s].reshape((q,) + (n,) * d)
        xg, w, vals = _space_values(n, d, npts, coeffs)        # (q, G, ..., G)
        grids = np.meshgrid(*([xg] * d), indexing="ij")
        W = np.ones((xg.size,) * d)
        for ax in range(d):
            W = W * w.reshape((1,) * ax + (-1,) + (1,) * (d - ax - 1))
        for g in range(npts):
            uh = np.tensordot(psi[:, g], vals, axes=([0], [0]))
            ue = exact(grids[::-1], s * tau + tg[g])
            total += wt[g] * np.sum(W * (uh - ue) ** 2)
    return np.sqrt(total)


def end_error(disc, u, exact, T, npts=5):
    """|| u_h(., T^-) - u(., T) ||_{L2(Omega)}."""
    d, n, q, N = disc.d, disc.n, disc.q, disc.N
    tau = T / N
    end = dg_time.slab_basis_values(disc.p_t, tau, [tau])[:, 0]
    coeffs = np.tensordot(end, u[N - 1].reshape((q,) + (n,) * d), axes=([0], [0]))
    xg, w, vals = _space_values(n, d, npts, coeffs[None])
    grids = np.meshgrid(*([xg] * d), indexing="ij")
    W = np.ones((xg.size,) * d)
    for ax in range(d):
        W = W * w.reshape((1,) * ax + (-1,) + (1,) * (d - ax - 1))
    return np.sqrt(np.sum(W * (vals[0] - exact(grids[::-1], T)) ** 2))
