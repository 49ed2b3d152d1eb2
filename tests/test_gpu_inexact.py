"""The inexact block inverse (one spatial V-cycle per time step, Remark on the
V-cycle approximation in space) through the C ABI against the oracle: the
block inverse on every level, smoothing steps, one V-cycle, solves and
adjoint solves; mixed precision with this smoother; the iteration count of
the 2D workload inside the band of Tables 1-2."""
import numpy as np
import pytest
import torch

from oracle import multigrid
from paper_1411_0519_gb300 import workloads
from tests.gpu_util import rel_err, require_gpu, to_gpu, to_np

pytestmark = pytest.mark.gpu

SMALL = [(1, 63, 1, 16, 1.0), (1, 31, 0, 8, 0.05), (2, 31, 1, 16, 1.0), (2, 15, 2, 8, 0.2), (3, 7, 1, 4, 1.0)]


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=shape)


@pytest.fixture(params=SMALL, ids=lambda c: "d%d-n%d-p%d-N%d" % c[:4])
def case(request):
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = request.param
    s = stmg.Solver(d, n, p, N, T, smoother="vcycle", rtol=1e-10, maxit=80)
    H = multigrid.Hierarchy(d, n, p, N, T, smoother="vcycle")
    yield s, H
    s.close()


@pytest.mark.parametrize("adjoint", [False, True])
def test_inexact_block_inverse_every_level(case, adjoint):
    s, H = case
    for L in range(s.num_levels):
        lv = H.levels[s.num_levels - 1 - L]
        r = rand(lv.disc.shape(), 10 + L)
        d = s.level_block_solve(L, to_gpu(r), adjoint=adjoint)
        do = lv.block_solve(r, adjoint)
        assert rel_err(to_np(d), do) < 1e-12, L


@pytest.mark.parametrize("adjoint", [False, True])
def test_inexact_smoothing_steps(case, adjoint):
    s, H = case
    L = s.num_levels - 1
    lv = H.finest
    u, f = rand(lv.disc.shape(), 20), rand(lv.disc.shape(), 21)
    ug = to_gpu(u)
    s.level_smooth(L, to_gpu(f), ug, nu=2, adjoint=adjoint)
    uo = multigrid.smooth(lv, u, f, 2, 0.5, adjoint)
    assert rel_err(to_np(ug), uo) < 1e-12


def test_inexact_vcycle_and_solves(case):
    s, H = case
    disc = H.finest.disc
    u, f = rand(disc.shape(), 70), rand(disc.shape(), 71)
    ug = to_gpu(u)
    s.vcycle(ug, to_gpu(f))
    assert rel_err(to_np(ug), multigrid.vcycle(H, 0, u, f)) < 1e-10
    uu, it, rr = s.solve(to_gpu(f))
    uo, ito, _ = multigrid.solve(H, f, rtol=1e-10, maxit=80)
    assert abs(it - ito) <= 1 and rr <= 1e-10
    assert rel_err(to_np(uu), uo) < 1e-10
    lam, gu0, ita, rra = s.adjoint_solve(to_gpu(f))
    lo, itoa, _ = multigrid.solve(H, f, rtol=1e-10, maxit=80, adjoint=True)
    assert abs(ita - itoa) <= 1
    assert rel_err(to_np(lam), lo) < 1e-10


def test_inexact_heat2d_255_iterations_and_mixed():
    """The 2D workload with the paper's practical smoother: V-cycles to 1e-8 in
    the 4-9 band of Tables 1-2; mixed precision reaches the same tolerance and
    agrees with FP64."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    w = workloads.WORKLOADS["heat2d_255"]
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=0))
    u0 = to_gpu(workloads.sine_ic(d, n))
    s = stmg.Solver(d, n, p, N, T, smoother="vcycle", rtol=1e-8, maxit=40)
    u, it, rr = s.solve(f, u0)
    s.close()
    assert 4 <= it <= 9 and rr <= 1e-8
    torch.cuda.empty_cache()
    sm = stmg.Solver(d, n, p, N, T, smoother="vcycle", precision="mixed", inner_cycles=4, rtol=1e-8, maxit=40)
    um, itm, rrm = sm.solve(f, u0)
    sm.close()
    assert rrm <= 1e-8
    err = ((um - u).norm() / u.norm()).item()
    print(f"heat2d_255 inexact smoother: fp64 {it} V-cycles, mixed {itm} refinements, difference {err:.2e}")
    assert err < 1e-5
