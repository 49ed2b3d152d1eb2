"""The mixed-precision form (FP32 V-cycles inside FP64 iterative refinement)
against the FP64 oracle, element by element.

The mixed form does not follow the oracle's iterate sequence (its inner cycles
round to FP32), so its result is compared with the discrete solution itself.
The error of any iterate with residual r is e = L^{-1} r, hence

    ||u_mixed - u*||_2 <= ||L^{-1}||_2 ||f + IC - L u_mixed||_2          (1)

with u* the exact discrete solution (the oracle's forward substitution in
time, Section 1), ||L^{-1}||_2 from the oracle by power iteration on
L^{-T} L^{-1} (exact solves), and the residual recomputed by the oracle's own
operator.  Each test prints the error and the bound (1) and asserts:

* the oracle's residual of u_mixed is within the requested tolerance (the
  mixed solution solves the oracle's system, not only the GPU's);
* the error obeys (1), and the largest elementwise difference to the oracle's
  multigrid solution (multigrid.solve at the same tolerance) is at most
  ||L^{-1}||_2 (||r_mixed||_2 + ||r_oracle||_2), the sum of both bounds.

One FP32 inner cycle is also compared with the oracle's FP64 cycle from the
same iterate: the difference is FP32 rounding only, bounded relative to the
size of the correction (tolerance derived in the test)."""
import numpy as np
import pytest

from oracle import multigrid, spacetime
from paper_1411_0519_gb300 import workloads
from tests.gpu_util import require_gpu, to_gpu, to_np

pytestmark = pytest.mark.gpu

# the SMALL cases of the FP64 parity tests: every (d, q) family, several tiles, ragged tails
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


def _linv_norm(lv, shape, iters=40, seed=0):
    """||L^{-1}||_2 by power iteration on L^{-T} L^{-1} with the oracle's exact
    forward / backward substitution (converges from below; the tests allow 5 %)."""
    x = np.random.default_rng(seed).standard_normal(shape)
    lam = 0.0
    for _ in range(iters):
        x /= np.linalg.norm(x)
        y = multigrid.backward_substitution(lv, multigrid.forward_substitution(lv, x))
        lam = np.linalg.norm(y)
        x = y
    return np.sqrt(lam)


def _check_against_oracle(H, g, u_mixed, rtol, label):
    """Assertions (1) and the oracle-residual check for a mixed result u_mixed
    of L u = g on hierarchy H; returns the relative 2-norm error."""
    lv = H.finest
    shape = lv.disc.shape()
    u_mixed = np.asarray(u_mixed).reshape(shape)
    ustar = multigrid.forward_substitution(lv, g)
    r_m = np.linalg.norm(lv.residual(u_mixed, g))
    uo, ito, hist = multigrid.solve(H, g, rtol=rtol, maxit=80)
    r_o = hist[-1]
    linv = 1.05 * _linv_norm(lv, shape)
    err2 = np.linalg.norm(u_mixed - ustar) / np.linalg.norm(ustar)
    bound2 = linv * r_m / np.linalg.norm(ustar)
    dmax = np.abs(u_mixed - uo).max()
    bmax = linv * (r_m + r_o)
    print(f"{label}: oracle residual of the mixed solution {r_m / np.linalg.norm(g):.2e}, "
          f"||u_mixed - u*||/||u*|| = {err2:.2e} (bound {bound2:.2e}), "
          f"max |u_mixed - u_oracle_mg| / max |u_oracle_mg| = {dmax / np.abs(uo).max():.2e} "
          f"(bound {bmax / np.abs(uo).max():.2e})")
    assert r_m <= 1.5 * rtol * np.linalg.norm(g), (r_m, np.linalg.norm(g))
    assert err2 <= bound2, (err2, bound2)
    assert dmax <= bmax, (dmax, bmax)
    return err2


@pytest.mark.parametrize("shape", SMALL, ids=lambda c: "d%d-n%d-p%d-N%d" % c[:4])
@pytest.mark.parametrize("inner", [1, 4])
def test_mixed_solve_against_oracle(shape, inner):
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = shape
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    f = np.random.default_rng(80).uniform(-1, 1, disc.shape())
    u0 = workloads.smooth_ic(d, n, seed=81)
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=80, precision="mixed", inner_cycles=inner)
    try:
        u, it, rr = s.solve(to_gpu(f), to_gpu(u0))
    finally:
        s.close()
    assert rr <= 1e-10
    _check_against_oracle(H, spacetime.add_ic(disc, f, u0), to_np(u), 1e-10,
                          f"mixed d={d} n={n} p_t={p} N={N} inner={inner} ({it} refinements)")


def test_mixed_manufactured_heat1d_63_against_oracle():
    """The 1D workload (u = sin(pi x) cos t, P1, p_t = 1, N = 64) in the mixed form to 1e-10."""
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
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=60, precision="mixed", inner_cycles=4)
    try:
        u, it, rr = s.solve(to_gpu(f), to_gpu(u0))
    finally:
        s.close()
    assert rr <= 1e-10
    _check_against_oracle(H, spacetime.add_ic(disc, f, u0), to_np(u), 1e-10, f"mixed heat1d_63 ({it} refinements)")
    ue = lambda cc, t: np.sin(np.pi * cc[0]) * np.cos(t)
    assert spacetime.l2_error(disc, to_np(u).reshape(disc.shape()), ue, T) < 2e-4


@pytest.mark.parametrize("shape", SMALL, ids=lambda c: "d%d-n%d-p%d-N%d" % c[:4])
def test_one_fp32_inner_cycle_against_oracle_cycle(shape):
    """st_vcycle in the mixed form with one inner cycle from a given iterate u:
    u + s V32(r / s) against the oracle's FP64 cycle u + V(r) (the cycle is
    linear in r).  Every operation of the FP32 cycle rounds to 2^-24 relative to
    its operands; along the cycle the rounding errors of about
    m = levels x (nu1 + nu2 + 3) passes add up, each amplified by at most the
    norm of the rest of the cycle (below 4 for these damped, stable smoothers),
    so the difference is bounded by 4 m 2^-24 of the correction's size."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = shape
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    rng = np.random.default_rng(70)
    u, f = rng.uniform(-1, 1, disc.shape()), rng.uniform(-1, 1, disc.shape())
    s = stmg.Solver(d, n, p, N, T, precision="mixed", inner_cycles=1)
    try:
        ug = to_gpu(u)
        s.vcycle(ug, to_gpu(f))
        got = to_np(ug).reshape(disc.shape())
        levels = s.num_levels
    finally:
        s.close()
    ref = multigrid.vcycle(H, 0, u, f)
    corr = np.linalg.norm(ref - u)
    diff = np.linalg.norm(got - ref)
    tol = 4.0 * levels * (2 + 2 + 3) * 2.0 ** -24
    print(f"one FP32 inner cycle d={d} n={n} p_t={p} N={N}: ||u32 - u64|| / ||correction|| = "
          f"{diff / corr:.2e} (tolerance {tol:.2e}, {levels} levels)")
    assert diff <= tol * corr


def test_mixed_inexact_block_inverse_against_oracle():
    """The mixed form with the paper's practical smoother (one spatial V-cycle per
    step) against the oracle's discrete solution."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = 2, 31, 1, 16, 1.0
    H = multigrid.Hierarchy(d, n, p, N, T, smoother="vcycle")
    disc = H.finest.disc
    f = np.random.default_rng(90).uniform(-1, 1, disc.shape())
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=80, precision="mixed", inner_cycles=4, smoother="vcycle")
    try:
        u, it, rr = s.solve(to_gpu(f))
    finally:
        s.close()
    assert rr <= 1e-10
    _check_against_oracle(H, f, to_np(u), 1e-10, f"mixed inexact d={d} n={n} ({it} refinements)")


def test_mixed_high_degree_against_oracle():
    """p_t = 10 (generic-q kernels) in the mixed form against the oracle."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = 2, 15, 10, 16, 16.0
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    f = np.random.default_rng(91).uniform(-1, 1, disc.shape())
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=80, precision="mixed", inner_cycles=4)
    try:
        u, it, rr = s.solve(to_gpu(f))
    finally:
        s.close()
    assert rr <= 1e-10
    _check_against_oracle(H, f, to_np(u), 1e-10, f"mixed p_t={p} d={d} n={n} ({it} refinements)")


@pytest.mark.parametrize("scale", [1e-40, 1e40, 1e-200, 1e200])
def test_mixed_data_beyond_the_fp32_range_against_oracle(scale):
    """Data whose magnitude lies outside the FP32 range enter the double-float
    transforms scaled by an exact power of two: the mixed solution of f * scale
    is scale times the solution of f, and matches the oracle's discrete solution."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = 2, 63, 1, 16, 1.0
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    f = np.random.default_rng(6).uniform(-1, 1, disc.shape())
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=60, precision="mixed", inner_cycles=4)
    try:
        u1, it1, rr1 = s.solve(to_gpu(f))
        us, its, rrs = s.solve(to_gpu(f * scale))
    finally:
        s.close()
    assert rr1 <= 1e-10 and rrs <= 1e-10 and abs(its - it1) <= 1
    a, b = to_np(us) / scale, to_np(u1)
    assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()
    _check_against_oracle(H, f, to_np(us) / scale, 1e-10, f"mixed, data x {scale:g}")
