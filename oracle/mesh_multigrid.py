"""Space-time multigrid on the simplicial mesh families of ``simplex``
(Section 4, Examples 1 and 2): the same damped block-Jacobi cycle as
``multigrid`` (its smooth / vcycle / solve / forward_substitution functions
run unchanged on these levels), with

* the space-time system of Section 1 on P1 of a refined mesh,
  A = K_tau (x) M_h + M_tau (x) K_h, B = -N_tau (x) M_h;
* the coarsening rule of Section 4 with h_L the longest edge of the level's
  mesh: full space-time coarsening to the next coarser mesh iff
  mu_L = tau_L / h_L^2 >= mu* (1 - 1e-12) and a coarser mesh exists, else
  semi coarsening in time, down to N_L = coarsest_steps;
* restriction R = R^t (x) P^T with the nested-space prolongation P of the
  mesh family (full) or R^t (x) I (semi), prolongation R^T (Section 2);
* the smoother's block inverse exact (sparse LU of A) or the paper's inexact
  D~^{-1} (Remark on the V-cycle approximation in space): one spatial V-cycle
  with damped point-block Jacobi smoothing, D^x_j = (M_h)_jj K_tau +
  (K_h)_jj M_tau, nu_x pre- and post-steps, restriction I (x) P^T, coarse
  operators of the coarser meshes (equal to the Galerkin products of nested
  spaces), exact solve on the initial mesh.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import dg_time, hierarchy, simplex, transfer


class MeshDiscretization:
    """One space-time level on a MeshSpace: the attributes of
    spacetime.Discretization that the cycle uses."""

    def __init__(self, space, p_t, N, tau):
        self.space = space
        self.d, self.p_t, self.N, self.tau = space.d, p_t, N, float(tau)
        self.q = p_t + 1
        self.h = space.h
        self.Nx = space.Nx
        self.Kt, self.Mt, self.Nt = dg_time.time_matrices(p_t, self.tau)
        self.Mh, self.Kh = space.Mh, space.Kh
        self.A = (sp.kron(self.Kt, self.Mh) + sp.kron(self.Mt, self.Kh)).tocsc()
        self.B = (-sp.kron(self.Nt, self.Mh)).tocsr()

    @property
    def mu(self):
        return self.tau / self.h ** 2

    @property
    def ndof(self):
        return self.N * self.q * self.Nx

    def shape(self):
        return (self.N, self.q * self.Nx)


def apply_L(disc, u):
    out = (disc.A @ u.T).T
    out[1:] += (disc.B @ u[:-1].T).T
    return out


def apply_LT(disc, lam):
    out = (disc.A.T @ lam.T).T
    out[:-1] += (disc.B.T @ lam[1:].T).T
    return out


def ic_term(disc, u0_ic):
    start = dg_time.start_trace(disc.p_t, disc.tau)
    mu0 = disc.Mh @ np.asarray(u0_ic, dtype=np.float64).reshape(-1)
    return np.concatenate([start[k] * mu0 for k in range(disc.q)])


def add_ic(disc, f, u0_ic):
    g = np.array(f, dtype=np.float64, copy=True).reshape(disc.shape())
    g[0] += ic_term(disc, u0_ic)
    return g


def build_levels(family, level, p_t, N, T, coarsening="auto", coarsest_steps=1):
    """Level parameters finest first: N, spatial level l, tau, h, mu, and 'full'
    (how the level is coarsened to the next; None on the coarsest)."""
    ms = hierarchy.mu_star(p_t)
    out = []
    Nl, l, tau = N, level, T / N
    while True:
        h = family.spaces[l].h
        mu = tau / h ** 2
        lv = {"N": Nl, "l": l, "tau": tau, "h": h, "mu": mu, "full": None}
        out.append(lv)
        if Nl <= coarsest_steps:
            break
        if coarsening == "semi":
            full = False
        elif coarsening == "full":
            full = l >= 1
        else:
            full = bool(mu >= ms * (1.0 - 1e-12)) and l >= 1
        lv["full"] = full
        Nl //= 2
        tau *= 2.0
        if full:
            l -= 1
    return out


class MeshSpatialVCycle:
    """D~^{-1}: one spatial V-cycle for A_{tau,h} on mesh levels l, l-1, ..., 0
    from a zero guess (the Remark on the V-cycle approximation in space)."""

    def __init__(self, family, l, p_t, tau, nu_x=2, omega_x=2.0 / 3.0):
        self.nu_x, self.omega_x = nu_x, omega_x
        self.q = p_t + 1
        self.levels = []
        for k in range(l, -1, -1):
            disc = MeshDiscretization(family.spaces[k], p_t, 1, tau)
            A = disc.A.tocsr()
            Nx = disc.Nx
            blocks = np.zeros((Nx, self.q, self.q))
            for a in range(self.q):
                for b in range(self.q):
                    blocks[:, a, b] = A[a * Nx:(a + 1) * Nx, b * Nx:(b + 1) * Nx].diagonal()
            lvl = {"Nx": Nx, "A": A, "blocks": blocks, "R": None, "lu": None}
            if k == 0:
                lvl["lu"] = spla.splu(A.tocsc())
            else:
                lvl["R"] = sp.kron(sp.identity(self.q), family.P[k].T, format="csr")
            self.levels.append(lvl)

    def _jacobi(self, lvl, x, b, adjoint):
        A = lvl["A"].T if adjoint else lvl["A"]
        blocks = np.transpose(lvl["blocks"], (0, 2, 1)) if adjoint else lvl["blocks"]
        r = b - A @ x
        q, Nx = self.q, lvl["Nx"]
        rn = r.reshape(q, Nx, -1).transpose(1, 0, 2)
        dn = np.linalg.solve(blocks, rn)
        return x + self.omega_x * dn.transpose(1, 0, 2).reshape(q * Nx, -1)

    def apply(self, b, adjoint=False, i=0):
        lvl = self.levels[i]
        if lvl["lu"] is not None:
            return lvl["lu"].solve(b, trans="T") if adjoint else lvl["lu"].solve(b)
        A = lvl["A"].T if adjoint else lvl["A"]
        x = np.zeros_like(b)
        for _ in range(self.nu_x):
            x = self._jacobi(lvl, x, b, adjoint)
        bc = lvl["R"] @ (b - A @ x)
        x = x + lvl["R"].T @ self.apply(bc, adjoint, i + 1)
        for _ in range(self.nu_x):
            x = self._jacobi(lvl, x, b, adjoint)
        return x


class MeshLevel:
    """A level of the space-time hierarchy with the interface of multigrid.Level."""

    def __init__(self, family, lv, p_t, smoother="vcycle", nu_x=2, omega_x=2.0 / 3.0):
        self.disc = MeshDiscretization(family.spaces[lv["l"]], p_t, lv["N"], lv["tau"])
        self.l = lv["l"]
        self.full = lv["full"]
        self.mu = lv["mu"]
        self.lu = spla.splu(self.disc.A.tocsc())
        self._luT = None
        self.R = None
        self.inexact = (MeshSpatialVCycle(family, lv["l"], p_t, lv["tau"], nu_x, omega_x)
                        if smoother == "vcycle" else None)

    @property
    def luT(self):
        if self._luT is None:
            self._luT = spla.splu(self.disc.A.T.tocsc())
        return self._luT

    def block_solve(self, r, adjoint=False):
        if self.inexact is not None:
            return self.inexact.apply(np.ascontiguousarray(r.T), adjoint).T
        return self.exact_block_solve(r, adjoint)

    def exact_block_solve(self, r, adjoint=False):
        lu = self.luT if adjoint else self.lu
        return lu.solve(np.ascontiguousarray(r.T)).T

    def residual(self, u, f, adjoint=False):
        return f - (apply_LT(self.disc, u) if adjoint else apply_L(self.disc, u))


class MeshHierarchy:
    """Space-time levels finest first on `refinements` uniform refinements of
    `initial` (a simplex.Mesh), N time steps on (0, T)."""

    def __init__(self, initial, refinements, p_t, N, T, coarsening="auto", coarsest_steps=1,
                 smoother="vcycle", nu_x=2, omega_x=2.0 / 3.0, family=None):
        self.family = family or simplex.MeshFamily(initial, refinements)
        self.params = build_levels(self.family, refinements, p_t, N, T, coarsening, coarsest_steps)
        self.levels = [MeshLevel(self.family, lv, p_t, smoother, nu_x, omega_x) for lv in self.params]
        for i in range(len(self.levels) - 1):
            fine = self.levels[i]
            Rt = transfer.time_restriction(fine.disc.N, p_t, fine.disc.tau)
            Rs = (self.family.P[fine.l].T.tocsr() if fine.full else sp.identity(fine.disc.Nx, format="csr"))
            fine.R = sp.kron(Rt, Rs, format="csr")

    @property
    def finest(self):
        return self.levels[0]
