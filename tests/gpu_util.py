"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs."""
import numpy as np
import pytest
import torch

from oracle import hierarchy, multigrid, spacetime


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def to_np(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_err(a, b):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    scale = max(np.abs(b).max(), 1e-300)
    return float(np.abs(a - b).max() / scale)


def oracle_index(solver, L):
    """API levels count from the coarsest (0); the oracle lists finest first."""
    return solver.num_levels - 1 - L


class Case:
    """A problem with both the GPU solver and the oracle hierarchy."""

    def __init__(self, d, n, p_t, N, T, coarsening="auto", coarsest_steps=1, precision="fp64", **kw):
        self.d, self.n, self.p_t, self.N, self.T = d, n, p_t, N, T
        from paper_1411_0519_gb300 import stmg
        self.solver = stmg.Solver(d, n, p_t, N, T, coarsening=coarsening, coarsest_steps=coarsest_steps,
                                  precision=precision, **kw)
        self.H = multigrid.Hierarchy(d, n, p_t, N, T, coarsening=coarsening, coarsest_steps=coarsest_steps)

    def level(self, L):
        return self.H.levels[oracle_index(self.solver, L)]

    def close(self):
        self.solver.close()
