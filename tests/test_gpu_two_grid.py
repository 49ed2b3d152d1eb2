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


def measured_factor(p, mu, nu, full, iters=40):
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
        if norms[-1] < 1e-250:
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


@pytest.mark.parametrize("p", [0, 1])
def test_full_coarsening_below_mu_star_does_not_smooth(p):
    require_gpu()
    meas = measured_factor(p, 1e-2, 2, True, iters=20)
    th = lfa.two_grid_factor_batch(p, 1e-2, 2, True, Nx=NX + 1, Nt=NT)
    print(f"p_t={p} mu=0.01 full: GPU {meas:.4f}  LFA {th:.4f}")
    assert meas > 0.5 and th > 0.5
