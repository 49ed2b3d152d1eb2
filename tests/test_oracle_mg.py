"""Pins of the oracle's multigrid solver against direct solves, forward
substitution, the adjoint identity and textbook convergence orders."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import hierarchy, multigrid, spacetime
from paper_1411_0519_gb300 import workloads


def direct(disc, f, adjoint=False):
    L = spacetime.global_matrix(disc)
    if adjoint:
        L = L.T.tocsc()
    return spla.spsolve(L, f.reshape(-1)).reshape(disc.shape())


@pytest.mark.parametrize("d,n,N,p", [(1, 7, 8, 0), (1, 7, 8, 1), (1, 7, 8, 2),
                                     (2, 7, 4, 1), (2, 7, 8, 0), (3, 3, 4, 1)])
def test_mg_fixed_point_equals_direct_solve(d, n, N, p):
    """The V-cycle iteration converges to the unique solution of system
    (chap4_generalLinearSystem): compare with a sparse direct solve of the
    whole space-time matrix on tiny grids."""
    H = multigrid.Hierarchy(d, n, p, N, 0.5)
    disc = H.finest.disc
    f = np.random.default_rng(1).uniform(-1, 1, disc.shape())
    u, it, hist = multigrid.solve(H, f, rtol=1e-14, maxit=60)
    ud = direct(disc, f)
    assert np.abs(u - ud).max() <= 1e-12 * np.abs(ud).max()


@pytest.mark.parametrize("d,n,N,p,T", [(1, 31, 32, 1, 1.0), (2, 15, 16, 1, 1.0), (2, 15, 8, 2, 0.05)])
def test_mg_equals_forward_substitution(d, n, N, p, T):
    """Section 1: forward substitution in time gives the same discrete solution."""
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    f = np.random.default_rng(2).uniform(-1, 1, disc.shape())
    u, _, _ = multigrid.solve(H, f, rtol=1e-13, maxit=60)
    uf = multigrid.forward_substitution(H.finest, f)
    assert np.abs(u - uf).max() <= 1e-11 * np.abs(uf).max()


def test_adjoint_dot_product_and_solve():
    """<L u, l> = <u, L^T l>; the adjoint V-cycle converges to the solution of L^T l = g."""
    H = multigrid.Hierarchy(2, 7, 1, 8, 1.0)
    disc = H.finest.disc
    rng = np.random.default_rng(3)
    u = rng.standard_normal(disc.shape())
    lam = rng.standard_normal(disc.shape())
    lhs = np.sum(spacetime.apply_L(disc, u) * lam)
    rhs = np.sum(u * spacetime.apply_LT(disc, lam))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    g = rng.uniform(-1, 1, disc.shape())
    lam, it, _ = multigrid.solve(H, g, rtol=1e-14, maxit=60, adjoint=True)
    ld = direct(disc, g, adjoint=True)
    assert np.abs(lam - ld).max() <= 1e-12 * np.abs(ld).max()
    lb = multigrid.backward_substitution(H.finest, g)
    assert np.abs(lb - ld).max() <= 1e-12 * np.abs(ld).max()


def _exact(c, t):
    out = np.cos(t) * np.ones_like(c[0])
    for x in c:
        out = out * np.sin(np.pi * x)
    return out


def _source(c, t):
    d = len(c)
    s = np.ones_like(c[0])
    for x in c:
        s = s * np.sin(np.pi * x)
    return s * (-np.sin(t) + d * np.pi ** 2 * np.cos(t))


def _orders(d, p, ks, T=1.0):
    errs, ends = [], []
    for k in ks:
        n, N = 2 ** k - 1, 2 ** k            # tau proportional to h
        H = multigrid.Hierarchy(d, n, p, N, T)
        disc = H.finest.disc
        f = spacetime.load_vector(disc, _source, T)
        u0 = workloads.sine_ic(d, n)
        g = spacetime.add_ic(disc, f, u0)
        u, _, _ = multigrid.solve(H, g, rtol=1e-13, maxit=60)
        errs.append(spacetime.l2_error(disc, u, _exact, T))
        ends.append(spacetime.end_error(disc, u, _exact, T))
    errs, ends = np.array(errs), np.array(ends)
    return np.log2(errs[:-1] / errs[1:]), np.log2(ends[:-1] / ends[1:])


@pytest.mark.parametrize("d,p,ks", [(1, 0, [4, 5, 6]), (1, 1, [3, 4, 5]), (1, 2, [3, 4, 5]), (2, 1, [3, 4, 5])])
def test_manufactured_convergence_orders(d, p, ks):
    """Manufactured u = prod sin(pi x_a) cos t with tau ~ h: the L2(Q) error
    decays at order min(p_t + 1, 2) (DG in time, P1/Q1 in space; standard
    a-priori theory, cf. the reference to Thomee in Section 1), the error at
    t = T at order 2 for p_t >= 1 and 1 for p_t = 0."""
    l2, end = _orders(d, p, ks)
    expect = min(p + 1, 2)
    assert abs(l2[-1] - expect) < 0.15, l2
    assert abs(end[-1] - expect) < 0.15, end


def test_coarsening_rule_heat2d_255():
    """Section 4 rule on the 255^2, N = 1024, T = 1 workload: mu = 64 halves
    under full coarsening down to 0.5 on n = 1, then semi coarsening doubles it:
    7 full levels, then 3 semi levels down to one time step."""
    lv = hierarchy.build_levels(2, 255, 1, 1024, 1.0)
    assert [l["full"] for l in lv] == [True] * 7 + [False] * 3 + [None]
    assert [l["N"] for l in lv] == [1024 >> i for i in range(11)]
    assert [l["n"] for l in lv] == [255, 127, 63, 31, 15, 7, 3, 1, 1, 1, 1]
    for a, b in zip(lv[:-1], lv[1:]):
        assert np.isclose(b["mu"], a["mu"] / 2 if a["full"] else 2 * a["mu"])


def test_coarsening_rule_switches_at_mu_star():
    ms = hierarchy.mu_star(1)
    n = 63
    h = 1.0 / (n + 1)
    for mu, first in [(ms * 1.01, True), (ms * 0.99, False)]:
        N = 16
        T = mu * h * h * N
        lv = hierarchy.build_levels(1, n, 1, N, T)
        assert lv[0]["full"] is first


@pytest.mark.parametrize("d,n,N,p,T", [(1, 63, 64, 1, 1.0), (1, 255, 256, 1, 1.0), (2, 31, 64, 1, 1.0),
                                       (2, 31, 32, 0, 1.0), (1, 63, 64, 2, 64.0)])
def test_iteration_counts_bounded(d, n, N, p, T):
    """Tables 1-2 report 4-9 V-cycles to eps = 1e-8 with f = 0 and a random
    initial iterate in [0, 1] (Section 4 protocol); the exact-block-inverse
    Q1 variant here must stay in that band."""
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    u0 = workloads.uniform_iterate(d, n, p, N, seed=0).reshape(disc.shape())
    _, it, _ = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=30)
    assert 2 <= it <= 10
