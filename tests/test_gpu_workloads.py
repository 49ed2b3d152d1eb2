"""GPU tests at the sizes of the benchmark workloads, through the C ABI.

* heat2d_255 (133M unknowns): the oracle cannot run this size whole, so it
  recomputes sampled time steps one by one from the GPU's vectors: the
  residual of the solution, one damped block-Jacobi step, restriction and
  prolongation on sampled coarse / fine steps.
* adjoint2d_127: gradients of 0.5 ||u - u_d||^2 through the autograd
  Function against central finite differences along 8 seeded directions
  (rel 1e-6), and the adjoint solution checked by the oracle's transposed
  operator on sampled steps; the full oracle adjoint on a reduced grid.
* heat3d_63 (384M unknowns, p_t = 2) and heat2d_511 (1.07B unknowns, mu
  sweep across mu*): mixed precision against plain FP64 on the GPU, forward
  and adjoint, and the mixed solution's residual recomputed by the oracle's
  operators A, B on sampled time steps (each sampled step's residual must lie
  within the solve's global tolerance); the errors are printed and bounded.
"""
import numpy as np
import pytest
import torch

from oracle import multigrid, spacetime, transfer
from paper_1411_0519_gb300 import workloads
from tests.gpu_util import rel_err, require_gpu, to_gpu, to_np

pytestmark = pytest.mark.gpu


def _solver(w, **kw):
    from paper_1411_0519_gb300 import stmg
    return stmg.Solver(w["d"], w["n"], w["p_t"], w["N"], w["T"], **kw)


def _steps(x, idx, shape):
    """Time steps `idx` of a GPU space-time vector as (len(idx), q*Nx) arrays."""
    t = x.view(shape[0], -1)[list(idx)]
    return to_np(t)


def test_heat2d_255_sampled_parity():
    require_gpu()
    w = workloads.WORKLOADS["heat2d_255"]
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    s = _solver(w, rtol=1e-8, maxit=60)
    f = workloads.uniform_load(d, n, p, N, seed=0)
    u0 = workloads.sine_ic(d, n)
    fg, u0g = to_gpu(f), to_gpu(u0)
    u, it, rr = s.solve(fg, u0g)
    assert rr <= 1e-8 and it <= 12
    r = s.residual(fg, u, u0g)
    tau = T / N
    disc = spacetime.Discretization(d, n, p, 1, tau)
    f2 = f.reshape(N, -1)
    samples = [0, 1, 511, 1023]
    need = sorted(set(samples + [k - 1 for k in samples if k > 0]))
    Ud = dict(zip(need, _steps(u, need, s.shape)))
    R = _steps(r, samples, s.shape)
    ic = spacetime.ic_term(disc, u0)
    for row, k in zip(R, samples):
        ro = f2[k] - disc.A @ Ud[k]
        ro = ro + (ic if k == 0 else -(disc.B @ Ud[k - 1]))
        scale = np.abs(f2[k]).max()
        assert np.abs(row - ro).max() <= 1e-12 * scale, k
    # one damped block-Jacobi step on the finest level, recomputed per sampled step
    L = s.num_levels - 1
    rng = np.random.default_rng(5)
    useed = torch.from_numpy(rng.uniform(-1, 1, s.shape)).cuda()
    v = useed.clone()
    s.level_smooth(L, fg, v, nu=1)
    lv = multigrid.Level(d, {"N": 1, "n": n, "tau": tau, "full": None, "mu": 0.0}, p)
    Vs = _steps(v, samples, s.shape)
    Us = _steps(useed, samples, s.shape)
    Up = _steps(useed, [max(k - 1, 0) for k in samples], s.shape)
    for row, k, uk, up in zip(Vs, samples, Us, Up):
        rk = f2[k] - disc.A @ uk - (disc.B @ up if k > 0 else 0.0)
        ref = uk + 0.5 * lv.lu.solve(rk)
        assert np.abs(row - ref).max() <= 1e-11 * np.abs(ref).max(), k
    # restriction to level L-1 (full coarsening) on sampled coarse steps
    info = s.level_info(L - 1)
    assert info["full"] == 1
    fc = s.level_restrict(L, useed)
    R1, R2 = transfer.time_blocks(p, tau)
    Rx = transfer.space_restriction(d, n)
    nc = info["n"]
    for m in [0, 300, 511]:
        Us_pair = _steps(useed, [2 * m, 2 * m + 1], s.shape)
        ref = np.zeros((p + 1, nc ** d))
        for sl, Rb in enumerate([R1, R2]):
            fine = Us_pair[sl].reshape(p + 1, -1)
            ref += Rb @ np.stack([Rx @ fine[l] for l in range(p + 1)])
        got = _steps(fc, [m], s.level_shape(L - 1))[0].reshape(p + 1, -1)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), m
    # prolongation on sampled fine steps
    e = torch.from_numpy(rng.uniform(-1, 1, s.level_shape(L - 1))).cuda()
    z = torch.zeros(s.shape, dtype=torch.float64, device="cuda")
    s.level_prolong(L, e, z)
    for k in [0, 1, 777]:
        m, sl = k // 2, k % 2
        ec = _steps(e, [m], s.level_shape(L - 1))[0].reshape(p + 1, -1)
        Rb = R1 if sl == 0 else R2
        ref = Rb.T @ np.stack([Rx.T @ ec[l] for l in range(p + 1)])
        got = _steps(z, [k], s.shape)[0].reshape(p + 1, -1)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), k
    s.close()


def _loss_and_grads(s, f, u0, ud):
    from paper_1411_0519_gb300 import stmg
    fg = f.clone().requires_grad_(True)
    u0g = u0.clone().requires_grad_(True)
    u = stmg.solve(fg, u0g, s)
    J = 0.5 * ((u - ud) ** 2).sum()
    J.backward()
    return J.item(), fg.grad.detach(), u0g.grad.detach()


def test_adjoint2d_127_finite_differences_and_adjoint_residual():
    require_gpu()
    w = workloads.WORKLOADS["adjoint2d_127"]
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    s = _solver(w, rtol=1e-12, maxit=80)
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=1))
    u0 = to_gpu(workloads.smooth_ic(d, n, seed=2))
    ud = to_gpu(workloads.smooth_target(d, n, p, N, T, seed=0))
    J, gf, gu0 = _loss_and_grads(s, f, u0, ud)
    dirs_f = workloads.random_directions(s.shape, 8, seed=3)
    dirs_u = workloads.random_directions((n,) * d, 8, seed=4)
    for vf, vu in zip(dirs_f, dirs_u):
        vf, vu = to_gpu(vf), to_gpu(vu)
        eps_f = 1e-4 * f.norm().item()
        eps_u = 1e-4 * u0.norm().item()
        # central differences of the quadratic loss along (vf, vu), scaled steps per block
        def J_at(t):
            u, _, _ = s.solve(f + t * eps_f * vf, u0 + t * eps_u * vu)
            return 0.5 * ((u - ud) ** 2).sum().item()
        fd = (J_at(1.0) - J_at(-1.0)) / 2.0
        an = eps_f * (gf * vf).sum().item() + eps_u * (gu0 * vu).sum().item()
        assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-300), (fd, an)
    # the adjoint solution satisfies L^T lam = u - u_d on sampled steps (oracle operator)
    u, _, _ = s.solve(f, u0)
    g = (u - ud).contiguous()
    lam, gu0b, it, rr = s.adjoint_solve(g)
    assert rr <= 1e-12
    tau = T / N
    disc = spacetime.Discretization(d, n, p, 1, tau)
    G = g.view(N, -1)
    Lm = lam.view(N, -1)
    for k in [0, 100, N - 1]:
        lk = to_np(Lm[k])
        ref = to_np(G[k]) - disc.A.T @ lk
        if k < N - 1:
            ref = ref - disc.B.T @ to_np(Lm[k + 1])
        assert np.abs(ref).max() <= 1e-9 * np.abs(to_np(G[k])).max(), k
    s.close()


def test_adjoint_gradients_match_oracle_reduced_grid():
    """The oracle's tracking-loss gradients on a reduced grid (31^2, N = 32)."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = 2, 31, 1, 32, 1.0
    f = workloads.uniform_load(d, n, p, N, seed=1)
    u0 = workloads.smooth_ic(d, n, seed=2)
    ud = workloads.smooth_target(d, n, p, N, T, seed=0)
    H = multigrid.Hierarchy(d, n, p, N, T)
    disc = H.finest.disc
    Jo, uo, lo, go = multigrid.tracking_gradients(H, ud.reshape(disc.shape()), f.reshape(disc.shape()), u0,
                                                  rtol=1e-13)
    s = stmg.Solver(d, n, p, N, T, rtol=1e-13, maxit=80)
    J, gf, gu0 = _loss_and_grads(s, to_gpu(f), to_gpu(u0), to_gpu(ud))
    assert abs(J - Jo) <= 1e-9 * abs(Jo)
    assert rel_err(to_np(gf), lo) < 1e-9
    assert rel_err(to_np(gu0), go) < 1e-9
    s.close()


def _sampled_oracle_residuals(w, f_np, u, samples, rtol, adjoint=False):
    """Oracle residuals f_k - A u_k - B u_{k-1} (adjoint: f_k - A^T u_k - B^T u_{k+1})
    of the GPU vector u on sampled steps k (u0 = 0); each must satisfy
    ||r_k|| <= rtol ||f|| (the whole residual does).  Returns the relative values."""
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    disc = spacetime.Discretization(d, n, p, 1, T / N)
    f2 = f_np.reshape(N, -1)
    fn = np.linalg.norm(f2)
    shape = (N, p + 1) + (n,) * d
    out = []
    for k in samples:
        nb = k + 1 if adjoint else k - 1
        idx = [k] + ([nb] if 0 <= nb < N else [])
        rows = _steps(u, idx, shape)
        if adjoint:
            rk = f2[k] - disc.A.T @ rows[0] - (disc.B.T @ rows[1] if len(idx) > 1 else 0.0)
        else:
            rk = f2[k] - disc.A @ rows[0] - (disc.B @ rows[1] if len(idx) > 1 else 0.0)
        out.append(np.linalg.norm(rk) / fn)
        assert np.linalg.norm(rk) <= rtol * fn, (k, np.linalg.norm(rk) / fn)
    return out


def test_heat3d_63_mixed_against_fp64():
    require_gpu()
    w = workloads.WORKLOADS["heat3d_63"]
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    f_np = workloads.gaussian_load(d, n, p, N, T, seed=0)
    f = to_gpu(f_np)
    s64 = _solver(w, rtol=1e-8, maxit=60, precision="fp64")
    u64, it64, rr64 = s64.solve(f)
    s64.close()
    smx = _solver(w, rtol=1e-8, maxit=60, precision="mixed", inner_cycles=4)
    umx, itm, rrm = smx.solve(f)
    smx.close()
    assert rr64 <= 1e-8 and rrm <= 1e-8
    err = ((umx - u64).norm() / u64.norm()).item()
    rs = _sampled_oracle_residuals(w, f_np, umx, [0, 1, N // 2, N - 1], 1e-8)
    print(f"heat3d_63: fp64 {it64} cycles, mixed {itm} refinement steps, ||u_mixed - u_fp64|| / ||u_fp64|| = "
          f"{err:.2e}; oracle residual of the mixed solution on sampled steps / ||f||: "
          + ", ".join(f"{v:.1e}" for v in rs))
    assert err < 1e-5


@pytest.mark.parametrize("mu", [1.0 / 16, 0.25, 1.0, 16.0])
def test_heat2d_511_mu_sweep_mixed_forward_and_adjoint(mu):
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    w = dict(workloads.WORKLOADS["heat2d_511"])
    w["T"] = mu / 128.0                      # mu = tau / h^2 = 128 T on the finest level
    d, n, p, N, T = w["d"], w["n"], w["p_t"], w["N"], w["T"]
    f_np = workloads.uniform_load(d, n, p, N, seed=0)
    f = to_gpu(f_np)
    s64 = _solver(w, rtol=1e-8, maxit=80, precision="fp64")
    kinds = [s64.level_info(L)["full"] for L in range(s64.num_levels - 1)]
    u64, it64, rr64 = s64.solve(f)
    lam64, g64, ita64, rra64 = s64.adjoint_solve(u64)
    s64.close()
    torch.cuda.empty_cache()
    smx = _solver(w, rtol=1e-8, maxit=80, precision="mixed", inner_cycles=4)
    umx, itm, rrm = smx.solve(f)
    lammx, gmx, itam, rram = smx.adjoint_solve(u64)
    smx.close()
    assert max(rr64, rra64, rrm, rram) <= 1e-8
    eu = ((umx - u64).norm() / u64.norm()).item()
    el = ((lammx - lam64).norm() / lam64.norm()).item()
    samples = [0, 1, N // 2, N - 1]
    rs = _sampled_oracle_residuals(w, f_np, umx, samples, 1e-8)
    ra = _sampled_oracle_residuals(w, to_np(u64).reshape(-1), lammx, samples, 1e-8, adjoint=True)
    print(f"heat2d_511 mu={mu}: levels full/semi {kinds}; fp64 {it64}/{ita64}, mixed {itm}/{itam}; "
          f"forward err {eu:.2e}, adjoint err {el:.2e}; oracle residuals on sampled steps / ||rhs||: forward "
          + ", ".join(f"{v:.1e}" for v in rs) + "; adjoint " + ", ".join(f"{v:.1e}" for v in ra))
    assert eu < 1e-5 and el < 1e-5
    del u64, lam64, umx, lammx
    torch.cuda.empty_cache()


@pytest.mark.parametrize("d,n,p,N", [(2, 1023, 1, 4), (3, 127, 1, 2), (1, 1023, 3, 8)])
def test_largest_lines_converge_checked_by_the_node_residual(d, n, p, N):
    """Line lengths at the top of the supported range (the sine transforms of
    1024-point lines run in the shared-memory kernels, 128-point 3D lines in the
    register kernels): the solve in the sine basis reaches 1e-10, and the
    residual recomputed by the node-basis stencil kernel (independent of the
    sine path) confirms it."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    T = 1.0
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=3))
    u0 = to_gpu(workloads.sine_ic(d, n))
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=60)
    u, it, rr = s.solve(f, u0)
    assert rr <= 1e-10 and it <= 15
    r = s.residual(f, u, u0)
    r0 = s.residual(f, torch.zeros_like(u), u0)
    ratio = (r.norm() / r0.norm()).item()
    print(f"d={d} n={n} p_t={p} N={N}: {it} V-cycles, node-basis relative residual {ratio:.2e}")
    assert ratio <= 2e-10
    s.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("d,n,p,N", [(2, 255, 1, 64), (2, 63, 2, 32), (3, 127, 1, 4), (2, 511, 1, 8)])
def test_mixed_boundary_transforms_keep_the_fp64_residual(d, n, p, N):
    """The mixed form transforms f and u in double-float arithmetic (register
    kernels, n + 1 = 64 ... 512).  Its solve stops on the relative residual in
    the sine basis; the residual recomputed on nodes by the independent stencil
    kernel must reach the same 1e-8, which an FP32-accurate transform (about
    1e-7) would not."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    T = 1.0
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=4))
    u0 = to_gpu(workloads.sine_ic(d, n))
    s = stmg.Solver(d, n, p, N, T, rtol=1e-9, maxit=60, precision="mixed", inner_cycles=4)
    u, it, rr = s.solve(f, u0)
    s.close()
    assert rr <= 1e-9
    s64 = stmg.Solver(d, n, p, N, T, rtol=1e-9, maxit=60)
    r = s64.residual(f, u, u0)
    r0 = s64.residual(f, torch.zeros_like(u), u0)
    s64.close()
    ratio = (r.norm() / r0.norm()).item()
    print(f"mixed d={d} n={n} p_t={p} N={N}: {it} refinements, sine-basis {rr:.2e}, node-basis {ratio:.2e}")
    assert ratio <= 3e-9
    torch.cuda.empty_cache()


@pytest.mark.parametrize("precision,given", [("fp64", False), ("mixed", False), ("fp64", True)])
def test_solve_host_matches_device_solve(precision, given):
    """st_solve_host (host buffers, chunked copies overlapped with the
    transforms) returns the same solution as st_solve on device buffers."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = 2, 63, 1, 32, 1.0
    f_np = workloads.uniform_load(d, n, p, N, seed=5)
    u0_np = workloads.sine_ic(d, n)
    s = stmg.Solver(d, n, p, N, T, rtol=1e-10, maxit=60, precision=precision, inner_cycles=4)
    guess = np.random.default_rng(9).uniform(-1, 1, s.shape) if given else None
    ud = to_gpu(guess) if given else None
    u_dev, it_d, rr_d = s.solve(to_gpu(f_np), to_gpu(u0_np), u=ud, initial_guess=given)
    fh = torch.from_numpy(f_np).pin_memory()
    u0h = torch.from_numpy(u0_np).pin_memory()
    uh = torch.from_numpy(guess.copy()).pin_memory() if given else None
    u_host, it_h, rr_h = s.solve_host(fh, u0h, uh, initial_guess=given)
    s.close()
    assert it_h == it_d and rr_h <= 1e-10
    assert rel_err(u_host.numpy(), to_np(u_dev)) < 1e-13


@pytest.mark.parametrize("scale", [1e-30, 1.0, 1e30])
def test_mixed_refinement_is_scale_invariant(scale):
    """The mixed form takes the FP32 residual unscaled as the right-hand side of
    its FP32 cycles while its entries are far from the FP32 range limits, and
    falls back to the FP64 residual divided by its norm otherwise (entries of
    1e-30 and 1e30 here).  Either way the refinement sees the same problem: the
    same number of refinements, the same relative residual, and a solution that
    scales with the data."""
    require_gpu()
    from paper_1411_0519_gb300 import stmg
    d, n, p, N, T = 2, 63, 1, 32, 1.0
    f = to_gpu(workloads.uniform_load(d, n, p, N, seed=6))
    s = stmg.Solver(d, n, p, N, T, rtol=1e-9, maxit=60, precision="mixed", inner_cycles=4)
    u1, it1, rr1 = s.solve(f)
    us, its, rrs = s.solve(f * scale)
    s.close()
    assert abs(its - it1) <= 1 and rrs <= 1e-9 and rr1 <= 1e-9
    assert rel_err(to_np(us) / scale, to_np(u1)) < 1e-7
