"""The paper's two-grid experiment (Section 3.2, figures of the semi and full
coarsening factors) run on the GPU at the paper's size: 1D, N_x = 1023
interior nodes, N_t = 256 time steps, f = 0, a random initial iterate in
[0, 1], omega = 1/2, nu1 = nu2 = nu; the convergence factor is
max_k ||r_{k+1}|| / ||r_k||.  A two-grid cycle is the library's V-cycle with a
two-level hierarchy whose coarse level (128 steps) is solved exactly by
forward substitution (coarsest_steps = N/2).  The measured factors are
compared with the oracle's local Fourier analysis on the full frequency grid
(|difference| <= 0.05; <= 1/2 where the paper bounds them).  The curve values
themselves are not printed in the paper (parity unpinned for them)."""
import numpy as np
import pytest
import torch

from oracle import hierarchy, lfa
from paper_1411_0519_gb300 import workloads
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu

NX, NT = 1023, 256


def measured_factor(p, mu, nu, full, iters=250, eps=1e-140):
    """The paper's protocol: two-grid cycles until ||r_k|| <= 1e-140 ||r_0|| (at
    most 250), factor = max_k ||r_{k+1}|| / ||r_k||."""
    from paper_1411_0519_gb300 import stmg
    h = 1.0 / (NX + 1)
    T = mu * h * h * NT
    s = stmg.Solver(1, NX, p, NT, T, nu1=nu, nu2=nu, coarsening="full" if full else "semi",
                    coarsest_steps=NT // 2, rtol=0.0, maxit=1)
    assert s.num_levels == 2
    u = torch.from_numpy(workloads.uniform_iterate(1, NX, p, NT, seed=0)).cuda()
    f = torch.zeros_like(u)
    r = s.residual(f, u)
    norms = [s.norm2(r)]
    for _ in range(iters):
        s.vcycle(u, f)
        s.residual(f, u, out=r)
        norms.append(s.norm2(r))
        if norms[-1] <= eps * norms[0]:
            break
    s.close()
    norms = np.array(norms)
    return float(np.max(norms[1:] / norms[:-1]))


CASES = [(p, nu, mu, False) for p in (0, 1) for nu in (1, 2, 5) for mu in (1e-2, 1.0, 1e2)]
CASES += [(p, nu, "star", True) for p in (0, 1) for nu in (1, 2)]
CASES += [(p, 2, 10.0, True) for p in (0, 1)]


@pytest.mark.parametrize("p,nu,mu,full", CASES)
def test_two_grid_factor_matches_lfa(p, nu, mu, full):
    require_gpu()
    mu = hierarchy.mu_star(p) if mu == "star" else mu
    meas = measured_factor(p, mu, nu, full)
    th = lfa.two_grid_factor_batch(p, mu, nu, full, Nx=NX + 1, Nt=NT)
    print(f"p_t={p} nu={nu} mu={mu:.4g} {'full' if full else 'semi'}: GPU {meas:.4f}  LFA {th:.4f}")
    assert abs(meas - th) <= 0.05
    # the paper's bound 1/2 is attained by the LFA for nu = 1 (semi, and full at mu = mu*)
    assert meas <= 0.5 and th <= 0.5 + 1e-3


SWEEP_MU = [1e-6, 1e-3, 1e-1, 1.0, 10.0, 1e3, 1e4, 1e6]


@pytest.mark.parametrize("full", [False, True], ids=["semi", "full"])
@pytest.mark.parametrize("p", [0, 1])
def test_two_grid_sweep_against_lfa(p, full):
    """A thinned version of the paper's sweep (mu from 1e-6 to 1e6, nu = 1, 2, 5),
    the paper's protocol (until 1e-140 or 250 cycles).  Section 3.2 bounds the
    factor by 1/2 for semi coarsening at every mu and for full coarsening at
    mu >= mu*: asserted for the measured and the LFA factors.  Agreement with
    the LFA (which Section 3.2 notes is not rigorous for the Dirichlet problem
    measured): |GPU - LFA| <= 0.05 for 1e-2 <= mu <= 1e2; outside that range the
    finite problem's slowest modes separate from the periodic analysis (at
    p_t = 0 and mu ~ 1e3 ... 1e5 the measured factor settles above the LFA
    value after about a hundred cycles, by up to 0.17; below mu* with full
    coarsening, and at mu = 1e6, by about 0.05), so there |GPU - LFA| <= 0.2;
    the GPU equals the oracle's own measurement there (next test)."""
    require_gpu()
    ms = hierarchy.mu_star(p)
    rows = []
    for nu in (1, 2, 5):
        for mu in SWEEP_MU:
            meas = measured_factor(p, mu, nu, full)
            th = lfa.two_grid_factor_batch(p, mu, nu, full, Nx=NX + 1, Nt=NT)
            rows.append((nu, mu, meas, th))
    print(f"p_t={p} {'full' if full else 'semi'}: " + "; ".join(
        f"nu={nu} mu={mu:.0e} GPU {m:.3f} LFA {t:.3f}" for nu, mu, m, t in rows))
    for nu, mu, meas, th in rows:
        assert abs(meas - th) <= (0.05 if 1e-2 <= mu <= 1e2 else 0.2), (nu, mu, meas, th)
        if not full or mu >= ms:
            assert meas <= 0.5 and th <= 0.5 + 1e-3, (nu, mu, meas, th)


def test_two_grid_factor_equals_the_oracle_measurement_where_lfa_departs():
    """p_t = 0, nu = 1, semi coarsening, mu = 10^3.75: the measured factor (0.43)
    lies well above the LFA value (0.26); the oracle's two-grid cycle on the same
    1023-node, 256-step problem from the same iterate gives the same factor."""
    require_gpu()
    from oracle import multigrid
    p, mu, nu = 0, 10.0 ** 3.75, 1
    meas = measured_factor(p, mu, nu, False)
    h = 1.0 / (NX + 1)
    H = multigrid.Hierarchy(1, NX, p, NT, mu * h * h * NT, coarsening="semi", coarsest_steps=NT // 2)
    u = workloads.uniform_iterate(1, NX, p, NT, seed=0).reshape(H.finest.disc.shape())
    f = np.zeros_like(u)
    r0 = prev = np.linalg.norm(H.finest.residual(u, f))
    worst = 0.0
    for _ in range(250):
        u = multigrid.two_grid(H, u, f, nu, nu, 0.5)
        rn = np.linalg.norm(H.finest.residual(u, f))
        worst = max(worst, rn / prev)
        prev = rn
        if rn <= 1e-140 * r0:
            break
    th = lfa.two_grid_factor_batch(p, mu, nu, False, Nx=NX + 1, Nt=NT)
    print(f"p_t=0 nu=1 mu={mu:.4g} semi: GPU {meas:.6f}  oracle {worst:.6f}  LFA {th:.4f}")
    assert abs(meas - worst) <= 1e-6 and meas > th + 0.1


@pytest.mark.parametrize("p", [0, 1])
def test_full_coarsening_below_mu_star_does_not_smooth(p):
    require_gpu()
    meas = measured_factor(p, 1e-2, 2, True, iters=20)
    th = lfa.two_grid_factor_batch(p, 1e-2, 2, True, Nx=NX + 1, Nt=NT)
    print(f"p_t={p} mu=0.01 full: GPU {meas:.4f}  LFA {th:.4f}")
    assert meas > 0.5 and th > 0.5
