"""High time degree on the GPU (Example 2 of the paper sweeps p_t to 45):
the generic-q kernels through the C ABI against the oracle -- every step on
every level, solves and adjoint solves -- and the Example 2 protocol
(tau = 1, f = 0, u^0 ~ U[0, 1], eps = 1e-8) against the oracle's counts and
the printed table.

Tolerances: single steps 1e-11; solves 1e-10 relative to the largest entry at
every degree, as in the FP64 parity tests (the q x q blocks at q = 46 have
condition numbers near 1e4 and the oracle's quadrature K_tau matches the
library's closed form to about 1e-13, so a few 1e-10 would be the worst case;
the measured differences stay below 1e-12).  The residual of a solve is
recomputed on nodes by st_residual (stencils, no sine transform) and by the
oracle's operator."""
import os

import numpy as np
import pytest
import torch

from oracle import multigrid, spacetime
from tests.gpu_util import Case, rel_err, require_gpu, to_gpu, to_np

pytestmark = pytest.mark.gpu

CASES = [(2, 7, 4, 8, 1.0), (1, 15, 10, 16, 16.0), (2, 7, 45, 4, 4.0), (3, 3, 6, 4, 1.0), (2, 15, 20, 8, 0.1)]


@pytest.fixture(params=CASES, ids=lambda c: "d%d-n%d-p%d-N%d" % c[:4])
def case(request):
    require_gpu()
    c = Case(*request.param, rtol=1e-10, maxit=60)
    yield c
    c.close()


def rand(shape, seed):
    return np.random.default_rng(seed).uniform(-1, 1, size=shape)


@pytest.mark.parametrize("adjoint", [False, True])
def test_steps_every_level(case, adjoint):
    s = case.solver
    for L in range(s.num_levels):
        lv = case.level(L)
        shp = lv.disc.shape()
        u, f = rand(shp, 1 + L), rand(shp, 100 + L)
        r = s.level_residual(L, to_gpu(f), to_gpu(u), adjoint=adjoint)
        assert rel_err(to_np(r), lv.residual(u, f, adjoint)) < 1e-11, ("residual", L)
        d = s.level_block_solve(L, to_gpu(f), adjoint=adjoint)
        assert rel_err(to_np(d), lv.block_solve(f, adjoint)) < 1e-11, ("block inverse", L)
        ug = to_gpu(u)
        s.level_smooth(L, to_gpu(f), ug, nu=2, adjoint=adjoint)
        assert rel_err(to_np(ug), multigrid.smooth(lv, u, f, 2, 0.5, adjoint)) < 1e-11, ("smooth", L)
    for L in range(1, s.num_levels):
        fine, coarse = case.level(L), case.level(L - 1)
        r = rand(fine.disc.shape(), 30 + L)
        fc = s.level_restrict(L, to_gpu(r))
        assert rel_err(to_np(fc), (fine.R @ r.reshape(-1)).reshape(coarse.disc.shape())) < 1e-11, ("restrict", L)
        e, u = rand(coarse.disc.shape(), 40 + L), rand(fine.disc.shape(), 50 + L)
        ug = to_gpu(u)
        s.level_prolong(L, to_gpu(e), ug)
        uo = u + (fine.R.T @ e.reshape(-1)).reshape(fine.disc.shape())
        assert rel_err(to_np(ug), uo) < 1e-11, ("prolong", L)
    lv = case.level(0)
    f = rand(lv.disc.shape(), 60)
    u = s.coarsest_solve(to_gpu(f), adjoint=adjoint)
    assert rel_err(to_np(u), multigrid.coarsest_solve(lv, f, adjoint)) < 1e-11


def test_solves_and_gradients(case):
    from paper_1411_0519_gb300 import workloads
    s = case.solver
    disc = case.H.finest.disc
    f = rand(disc.shape(), 80)
    u0 = workloads.smooth_ic(case.d, case.n, seed=81)
    tol = 1e-10
    u, it, rr = s.solve(to_gpu(f), to_gpu(u0))
    uo, ito, _ = multigrid.solve(case.H, spacetime.add_ic(disc, f, u0), rtol=1e-10, maxit=60)
    assert abs(it - ito) <= 1 and rr <= 1e-10
    err = rel_err(to_np(u), uo)
    print(f"p_t={case.p_t}: solve against the oracle {err:.2e} (tolerance {tol:g})")
    assert err < tol
    r = s.residual(to_gpu(f), u, to_gpu(u0))      # on nodes, independent of the sine basis
    ro = case.H.finest.residual(to_np(u).reshape(disc.shape()), spacetime.add_ic(disc, f, u0))
    assert np.abs(to_np(r).reshape(ro.shape) - ro).max() <= 1e-11 * np.abs(f).max()
    g = spacetime.add_ic(disc, f, u0)
    assert np.linalg.norm(ro) <= 1.5e-10 * np.linalg.norm(g)
    lam, gu0, ita, rra = s.adjoint_solve(to_gpu(f))
    lo, itoa, _ = multigrid.solve(case.H, f, rtol=1e-10, maxit=60, adjoint=True)
    assert abs(ita - itoa) <= 1 and rel_err(to_np(lam), lo) < tol
    start = (-1.0) ** np.arange(disc.q)
    go = disc.Mh @ (start @ lo[0].reshape(disc.q, disc.Nx))
    assert rel_err(to_np(gu0), go) < tol


def test_high_order_mixed_precision_against_fp64():
    require_gpu()
    from paper_1411_0519_gb300 import stmg, workloads
    d, n, p, N, T = 2, 31, 10, 32, 32.0
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=0))
    s64 = stmg.Solver(d, n, p, N, T, rtol=1e-8, maxit=60)
    u64, it64, rr64 = s64.solve(f)
    s64.close()
    smx = stmg.Solver(d, n, p, N, T, rtol=1e-8, maxit=60, precision="mixed", inner_cycles=4)
    umx, itm, rrm = smx.solve(f)
    smx.close()
    assert rr64 <= 1e-8 and rrm <= 1e-8
    err = ((umx - u64).norm() / u64.norm()).item()
    print(f"p_t = 10 mixed against FP64: {err:.2e} ({it64} cycles / {itm} refinements)")
    assert err < 1e-5


def _paper_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "example2_iterations.txt")
    rows = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        vals = [int(v) for v in line.split()]
        rows[vals[0]] = vals[1:]
    return [0, 1, 2, 3, 4, 5, 10, 15, 20, 25, 30, 35, 40, 45], rows


def test_example2_protocol_every_degree():
    """tau = 1, f = 0, u^0 ~ U[0, 1], eps = 1e-8 on the 15^2 grid (N = 32): the
    GPU count equals the oracle's within one and the printed count of the
    refined levels (7) within one, for every degree of the table."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    degrees, rows = _paper_rows()
    d, n, N = 2, 15, 32
    got = []
    for p, ref in zip(degrees, rows[3]):
        H = multigrid.Hierarchy(d, n, p, N, float(N))
        disc = H.finest.disc
        u0 = np.random.default_rng(0).uniform(0.0, 1.0, disc.shape())
        _, ito, _ = multigrid.solve(H, np.zeros(disc.shape()), u=u0, rtol=1e-8, maxit=40)
        s = stmg.Solver(d, n, p, N, float(N), rtol=1e-8, maxit=40)
        ug = to_gpu(u0)
        _, it, rr = s.solve(torch.zeros_like(ug), u=ug, initial_guess=True)
        s.close()
        got.append(it)
        assert rr <= 1e-8 and abs(it - ito) <= 1 and abs(it - ref) <= 1, (p, it, ito, ref)
    print("Example 2 protocol, 15^2 x 32, V-cycles per p_t:", dict(zip(degrees, got)))
