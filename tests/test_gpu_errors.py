"""Failure handling through the C ABI, without faulting the GPU: statuses for
non-convergence, NaN input, workspace limits and bad arguments, and resuming
a stopped solve from its last iterate."""
import numpy as np
import pytest
import torch

from paper_1411_0519_gb300 import workloads
from tests.gpu_util import require_gpu, to_gpu

pytestmark = pytest.mark.gpu


def _stmg():
    from paper_1411_0519_gb300 import stmg
    return stmg


def test_maxit_reached_reports_enotconv_and_resume_continues():
    require_gpu()
    stmg = _stmg()
    d, n, p, N = 2, 31, 1, 32
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=0))
    full = stmg.Solver(d, n, p, N, 1.0, rtol=1e-10, maxit=60)
    uref, itref, _ = full.solve(f)
    stop = stmg.Solver(d, n, p, N, 1.0, rtol=1e-10, maxit=3)
    u, it, rr = stop.solve(f, raise_on_failure=False)
    assert stop.last_status == stmg.ST_ENOTCONV and it == 3 and rr > 1e-10
    # resume: the iterate is the only state; pass it back in
    u2, it2, rr2 = full.solve(f, u=u.clone(), initial_guess=True)
    assert rr2 <= 1e-10                  # relative to the resumed start
    assert ((u2 - uref).norm() / uref.norm()).item() < 1e-8
    assert it2 < itref + 3
    with pytest.raises(stmg.StmgError) as e:
        stop.solve(f)
    assert e.value.code == stmg.ST_ENOTCONV


def test_nan_input_reports_enan():
    require_gpu()
    stmg = _stmg()
    d, n, p, N = 2, 15, 1, 8
    fh = workloads.uniform_load(d, n, p, N, seed=0)
    fh[3, 1, 4, 5] = np.nan
    s = stmg.Solver(d, n, p, N, 1.0)
    u, it, rr = s.solve(to_gpu(fh), raise_on_failure=False)
    assert s.last_status == stmg.ST_ENAN


def test_workspace_cap_reports_enomem():
    require_gpu()
    stmg = _stmg()
    with pytest.raises(stmg.StmgError) as e:
        stmg.Solver(2, 63, 1, 64, 1.0, max_workspace_bytes=1 << 20)
    assert e.value.code == stmg.ST_ENOMEM


def test_bad_tensors_are_rejected_before_any_launch():
    require_gpu()
    stmg = _stmg()
    s = stmg.Solver(2, 7, 1, 4, 1.0)
    good = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        s.solve(torch.zeros(10, dtype=torch.float64, device="cuda"))
    with pytest.raises(TypeError):
        s.solve(good.float())
    with pytest.raises(TypeError):
        s.solve(good.cpu())
    with pytest.raises(stmg.StmgError) as e:
        s.level_residual(99, good, good)
    assert e.value.code == stmg.ST_EINVAL
    # a zero right-hand side is already solved: zero iterations, zero iterate
    u, it, rr = s.solve(good)
    assert it == 0 and float(u.abs().max()) == 0.0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_without_guess_returns_zero_when_no_cycle_runs(precision):
    """Without an initial guess the FP64 form starts from u = 0 without storing
    it; when no cycle runs (zero data, or maxit = 0) the output buffer still
    holds that zero iterate, whatever it held before."""
    require_gpu()
    stmg = _stmg()
    d, n, p, N = 2, 15, 1, 8
    s = stmg.Solver(d, n, p, N, 1.0, precision=precision)
    u = torch.full(s.shape, 7.0, dtype=torch.float64, device="cuda")
    out, it, rr = s.solve(torch.zeros(s.shape, dtype=torch.float64, device="cuda"), u=u, initial_guess=False)
    assert it == 0 and rr == 0.0 and torch.count_nonzero(out).item() == 0
    s0 = stmg.Solver(d, n, p, N, 1.0, precision=precision, maxit=0)
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=0))
    u.fill_(7.0)
    out, it, rr = s0.solve(f, u=u, initial_guess=False, raise_on_failure=False)
    assert s0.last_status == stmg.ST_ENOTCONV and it == 0 and rr == 1.0
    assert torch.count_nonzero(out).item() == 0
    # a given initial guess is kept as the iterate
    g = to_gpu(np.random.default_rng(5).uniform(-1, 1, size=s.shape))
    out, it, rr = s0.solve(f, u=g.clone(), initial_guess=True, raise_on_failure=False)
    assert it == 0 and torch.allclose(out, g, rtol=1e-12, atol=1e-12)
    s.close()
    s0.close()
