"""CUDA path (through the C ABI) against the CPU oracle, element by element,
on seeded inputs: every step of the V-cycle on every level, then whole
cycles, solves and adjoint solves.

Tolerances (FP64): single steps 1e-12 relative to the largest entry (the
block inverse by sine transforms rounds differently from the oracle's sparse
LU; its error is a few ulps times the block condition number), whole cycles
and solves 1e-10 relative, iteration counts within 1."""
import numpy as np
import pytest
import torch

from oracle import multigrid, spacetime
from paper_1411_0519_gb300 import workloads
from tests.gpu_util import Case, rel_err, require_gpu, to_gpu, to_np

pytestmark = pytest.mark.gpu

# (d, n, p_t, N, T): several tiles and ragged tails, every (d, q) family
SMALL = [
    (1, 63, 1, 64, 1.0),
    (1, 31, 0, 16, 0.3),
    (1, 15, 3, 16, 2.0),
    (2, 31, 1, 32, 1.0),
    (2, 15, 2, 8, 0.05),
    (2, 7, 0, 8, 1.0),
    (3, 7, 1, 8, 1.0),
    (3, 7, 2, 4, 0.02),
]


@pytest.fixture(params=SMALL, ids=lambda c: "d%d-n%d-p%d-N%d" % c[:4])
def case(request):
    require_gpu()
    c = Case(*request.param)
    yield c
    c.close()


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=shape)


def test_hierarchy_matches_oracle(case):
    s = case.solver
    assert s.num_levels == len(case.H.params)
    for L in range(s.num_levels):
        info = s.level_info(L)
        p = case.H.params[s.num_levels - 1 - L]
        assert info["N"] == p["N"] and info["n"] == p["n"]
        assert abs(info["mu"] - p["mu"]) <= 1e-12 * p["mu"]
        if L < s.num_levels - 1:
            assert bool(info["full"]) == bool(case.H.params[s.num_levels - 2 - L]["full"])


@pytest.mark.parametrize("adjoint", [False, True])
def test_residual_every_level(case, adjoint):
    s = case.solver
    for L in range(s.num_levels):
        lv = case.level(L)
        shp = lv.disc.shape()
        u, f = rand(shp, 1 + L), rand(shp, 100 + L)
        r = s.level_residual(L, to_gpu(f), to_gpu(u), adjoint=adjoint)
        ro = lv.residual(u, f, adjoint)
        assert rel_err(to_np(r), ro) < 1e-13, L


def test_residual_with_initial_value(case):
    s = case.solver
    disc = case.H.finest.disc
    u, f = rand(disc.shape(), 5), rand(disc.shape(), 6)
    u0 = workloads.smooth_ic(case.d, case.n, seed=7)
    r = s.residual(to_gpu(f), to_gpu(u), to_gpu(u0))
    ro = case.H.finest.residual(u, spacetime.add_ic(disc, f, u0))
    assert rel_err(to_np(r), ro) < 1e-13


@pytest.mark.parametrize("adjoint", [False, True])
def test_block_inverse_every_level(case, adjoint):
    s = case.solver
    for L in range(s.num_levels):
        lv = case.level(L)
        r = rand(lv.disc.shape(), 10 + L)
        d = s.level_block_solve(L, to_gpu(r), adjoint=adjoint)
        do = lv.block_solve(r, adjoint)
        assert rel_err(to_np(d), do) < 1e-12, L


@pytest.mark.parametrize("adjoint", [False, True])
def test_smoothing_steps(case, adjoint):
    s = case.solver
    L = s.num_levels - 1
    lv = case.level(L)
    u, f = rand(lv.disc.shape(), 20), rand(lv.disc.shape(), 21)
    ug = to_gpu(u)
    s.level_smooth(L, to_gpu(f), ug, nu=2, adjoint=adjoint)
    uo = multigrid.smooth(lv, u, f, 2, 0.5, adjoint)
    assert rel_err(to_np(ug), uo) < 1e-12


def test_restriction_and_prolongation_every_level(case):
    s = case.solver
    for L in range(1, s.num_levels):
        fine = case.level(L)
        coarse = case.level(L - 1)
        r = rand(fine.disc.shape(), 30 + L)
        fc = s.level_restrict(L, to_gpu(r))
        fco = (fine.R @ r.reshape(-1)).reshape(coarse.disc.shape())
        assert rel_err(to_np(fc), fco) < 1e-14, L
        e = rand(coarse.disc.shape(), 40 + L)
        u = rand(fine.disc.shape(), 50 + L)
        ug = to_gpu(u)
        s.level_prolong(L, to_gpu(e), ug)
        uo = u + (fine.R.T @ e.reshape(-1)).reshape(fine.disc.shape())
        assert rel_err(to_np(ug), uo) < 1e-14, L


@pytest.mark.parametrize("adjoint", [False, True])
def test_coarsest_solve(case, adjoint):
    s = case.solver
    lv = case.level(0)
    f = rand(lv.disc.shape(), 60)
    u = s.coarsest_solve(to_gpu(f), adjoint=adjoint)
    uo = multigrid.coarsest_solve(lv, f, adjoint)
    assert rel_err(to_np(u), uo) < 1e-12


def test_one_vcycle_from_same_iterate(case):
    s = case.solver
    disc = case.H.finest.disc
    u, f = rand(disc.shape(), 70), rand(disc.shape(), 71)
    ug = to_gpu(u)
    s.vcycle(ug, to_gpu(f))
    uo = multigrid.vcycle(case.H, 0, u, f)
    assert rel_err(to_np(ug), uo) < 1e-10


def test_solve_parity(case):
    disc = case.H.finest.disc
    f = rand(disc.shape(), 80)
    u0 = workloads.smooth_ic(case.d, case.n, seed=81)
    from paper_1411_0519_gb300 import stmg
    s2 = stmg.Solver(case.d, case.n, case.p_t, case.N, case.T, rtol=1e-10, maxit=60)
    u, it, rr = s2.solve(to_gpu(f), to_gpu(u0))
    s2.close()
    g = spacetime.add_ic(disc, f, u0)
    uo, ito, hist = multigrid.solve(case.H, g, rtol=1e-10, maxit=60)
    assert abs(it - ito) <= 1, (it, ito)
    assert rr <= 1e-10
    assert rel_err(to_np(u), uo) < 1e-10


def test_adjoint_solve_parity(case):
    from paper_1411_0519_gb300 import stmg
    disc = case.H.finest.disc
    g = rand(disc.shape(), 90)
    s2 = stmg.Solver(case.d, case.n, case.p_t, case.N, case.T, rtol=1e-10, maxit=60)
    lam, gu0, it, rr = s2.adjoint_solve(to_gpu(g))
    s2.close()
    lo, ito, _ = multigrid.solve(case.H, g, rtol=1e-10, maxit=60, adjoint=True)
    assert abs(it - ito) <= 1, (it, ito)
    assert rel_err(to_np(lam), lo) < 1e-10
    start = (-1.0) ** np.arange(disc.q)
    go = disc.Mh @ (start @ lo[0].reshape(disc.q, disc.Nx))
    assert rel_err(to_np(gu0), go) < 1e-10


def test_wcycle_step_and_solve_parity(case):
    """Cycle index gamma = 2 (W-cycle, Section 2): one cycle from the same
    iterate, and a solve, against the oracle's W-cycle."""
    from paper_1411_0519_gb300 import stmg
    disc = case.H.finest.disc
    s2 = stmg.Solver(case.d, case.n, case.p_t, case.N, case.T, rtol=1e-10, maxit=60, gamma=2)
    try:
        u, f = rand(disc.shape(), 72), rand(disc.shape(), 73)
        ug = to_gpu(u)
        s2.vcycle(ug, to_gpu(f))
        assert rel_err(to_np(ug), multigrid.vcycle(case.H, 0, u, f, gamma=2)) < 1e-10
        uw, it, rr = s2.solve(to_gpu(f))
        uo, ito, _ = multigrid.solve(case.H, f, rtol=1e-10, maxit=60, gamma=2)
        assert abs(it - ito) <= 1, (it, ito)
        assert rr <= 1e-10 and rel_err(to_np(uw), uo) < 1e-10
    finally:
        s2.close()


@pytest.mark.parametrize("coarsening,coarsest_steps", [("semi", 1), ("full", 1), ("auto", 4)])
def test_coarsening_options_and_coarsest_substitution(coarsening, coarsest_steps):
    require_gpu()
    d, n, p, N, T = 2, 15, 1, 16, 1.0
    c = Case(d, n, p, N, T, coarsening=coarsening, coarsest_steps=coarsest_steps, rtol=1e-10, maxit=80)
    try:
        disc = c.H.finest.disc
        f = rand(disc.shape(), 3)
        u, it, rr = c.solver.solve(to_gpu(f))
        uo, ito, _ = multigrid.solve(c.H, f, rtol=1e-10, maxit=80)
        assert abs(it - ito) <= 1
        assert rel_err(to_np(u), uo) < 1e-10
    finally:
        c.close()


def test_manufactured_heat1d_63():
    """The 1D workload: u = sin(pi x) cos t, P1, p_t = 1, N = 64, T = 1, to 1e-10."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    w = workloads.WORKLOADS["heat1d_63"]
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc

    def src(cc, t):
        return np.sin(np.pi * cc[0]) * (-np.sin(t) + np.pi ** 2 * np.cos(t))
    f = spacetime.load_vector(disc, src, T)
    u0 = workloads.sine_ic(d, n)
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=60)
    u, it, rr = s.solve(to_gpu(f), to_gpu(u0))
    s.close()
    uo, ito, _ = multigrid.solve(H, spacetime.add_ic(disc, f, u0), rtol=1e-10, maxit=60)
    assert abs(it - ito) <= 1 and rr <= 1e-10
    assert rel_err(to_np(u), uo) < 1e-10
    ue = lambda cc, t: np.sin(np.pi * cc[0]) * np.cos(t)
    assert spacetime.l2_error(disc, to_np(u).reshape(disc.shape()), ue, T) < 2e-4


@pytest.mark.parametrize("d,n,p,N,cs", [(2, 7, 1, 1, 1), (1, 15, 2, 4, 4), (3, 3, 0, 2, 2), (2, 1, 1, 8, 1)])
def test_single_level_and_tiny_grids(d, n, p, N, cs):
    """Edge cases of the hierarchy: one level (N <= coarsest_steps: the exact
    coarsest solve must carry the initial value) and a one-node grid."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    T = 0.5
    c = Case(d, n, p, N, T, coarsest_steps=cs, rtol=1e-12, maxit=40)
    try:
        disc = c.H.finest.disc
        f = rand(disc.shape(), 7)
        u0 = workloads.smooth_ic(d, n, seed=8) if n > 1 else np.array([0.7])
        u, it, rr = c.solver.solve(to_gpu(f), to_gpu(u0))
        g = spacetime.add_ic(disc, f, u0)
        uo, ito, _ = multigrid.solve(c.H, g, rtol=1e-12, maxit=40)
        assert abs(it - ito) <= 1 and rr <= 1e-12
        assert rel_err(to_np(u), uo) < 1e-10
        lam, gu0, ita, rra = c.solver.adjoint_solve(to_gpu(f))
        lo, _, _ = multigrid.solve(c.H, f, rtol=1e-12, maxit=40, adjoint=True)
        assert rel_err(to_np(lam), lo) < 1e-10
    finally:
        c.close()


@pytest.mark.parametrize("nu1,nu2,omega,gamma,adjoint", [
    (0, 2, 0.5, 1, False),
    (1, 0, 0.5, 1, False),
    (3, 1, 1.0, 1, True),
    (0, 1, 0.5, 2, False),
    (2, 0, 0.7, 2, True),
])
@pytest.mark.parametrize("shape", [(2, 15, 1, 16, 1.0), (1, 15, 5, 8, 0.5)], ids=["d2-q2", "d1-q6"])
def test_smoothing_counts_and_damping(shape, nu1, nu2, omega, gamma, adjoint):
    """Damped steps run on the tabulated w A^{-1} f, formed by the first step of a
    level visit and reused by the later ones (the other half of the smoothing,
    the second visit of a W-cycle, the next cycle of a solve): pre- or
    post-smoothing alone, an odd count, omega = 1, the transposed problem, and
    the generic-q kernels (q = 6) — one cycle and a solve against the oracle."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = shape
    H = multigrid.Hierarchy(d, n, p, N, T)
    s = stmg.Solver(d, n, p, N, T, nu1=nu1, nu2=nu2, omega=omega, gamma=gamma, rtol=1e-10, maxit=200)
    try:
        disc = H.finest.disc
        u, f = rand(disc.shape(), 81), rand(disc.shape(), 82)
        if not adjoint:
            ug = to_gpu(u)
            s.vcycle(ug, to_gpu(f))
            ref = multigrid.vcycle(H, 0, u, f, nu1, nu2, omega, gamma=gamma)
            assert rel_err(to_np(ug), ref) < 1e-10
            uw, it, rr = s.solve(to_gpu(f))
        else:
            uw, _, it, rr = s.adjoint_solve(to_gpu(f))
        uo, ito, _ = multigrid.solve(H, f, rtol=1e-10, maxit=200, nu1=nu1, nu2=nu2, omega=omega,
                                     adjoint=adjoint, gamma=gamma)
        assert abs(it - ito) <= 1, (it, ito)
        assert rr <= 1e-10 and rel_err(to_np(uw), uo) < 1e-10
    finally:
        s.close()
