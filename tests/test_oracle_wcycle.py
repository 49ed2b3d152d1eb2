"""Pins of the oracle's W-cycle (cycle index gamma = 2, Section 2)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import multigrid, spacetime


@pytest.mark.parametrize("d,n,N,p", [(1, 15, 16, 1), (1, 7, 8, 2), (2, 7, 8, 1), (2, 7, 4, 0)])
def test_wcycle_fixed_point_equals_direct_solve(d, n, N, p):
    H = multigrid.Hierarchy(d, n, p, N, 0.5)
    disc = H.finest.disc
    f = np.random.default_rng(2).uniform(-1, 1, disc.shape())
    u, it, _ = multigrid.solve(H, f, rtol=1e-14, maxit=80, gamma=2)
    ud = spla.spsolve(spacetime.global_matrix(disc), f.reshape(-1)).reshape(disc.shape())
    assert np.abs(u - ud).max() <= 1e-12 * np.abs(ud).max()


def test_two_level_wcycle_equals_vcycle():
    """With two levels the coarse problem is solved exactly, so a second coarse
    cycle has nothing left to correct: W and V give the same iterate."""
    H = multigrid.Hierarchy(1, 31, 1, 16, 1.0, coarsest_steps=8)
    assert len(H.levels) == 2
    rng = np.random.default_rng(3)
    u, f = rng.uniform(-1, 1, H.finest.disc.shape()), rng.uniform(-1, 1, H.finest.disc.shape())
    v = multigrid.vcycle(H, 0, u, f)
    w = multigrid.vcycle(H, 0, u, f, gamma=2)
    assert np.abs(v - w).max() <= 1e-13 * np.abs(v).max()


@pytest.mark.parametrize("d,n,N,p,T", [(1, 63, 64, 1, 1.0), (2, 15, 32, 1, 1.0), (1, 31, 64, 0, 0.01)])
def test_wcycle_contracts_at_least_as_fast_as_vcycle(d, n, N, p, T):
    """Three or more levels: the W-cycle treats the coarse correction equation
    by two cycles, so its error reduction per cycle is at least that of the
    V-cycle (and it needs at most as many cycles to 1e-8)."""
    H = multigrid.Hierarchy(d, n, p, N, T)
    assert len(H.levels) >= 3
    disc = H.finest.disc
    f = np.random.default_rng(4).uniform(-1, 1, disc.shape())
    _, itv, hv = multigrid.solve(H, f, rtol=1e-8, maxit=60)
    _, itw, hw = multigrid.solve(H, f, rtol=1e-8, maxit=60, gamma=2)
    assert itw <= itv
    assert hw[2] / hw[0] <= hv[2] / hv[0] * (1 + 1e-9)


def test_wcycle_on_three_levels_differs_from_vcycle():
    """A dropped gamma (W treated as V) fails here."""
    H = multigrid.Hierarchy(1, 31, 1, 16, 1.0, coarsest_steps=4)
    assert len(H.levels) == 3
    rng = np.random.default_rng(5)
    u, f = rng.uniform(-1, 1, H.finest.disc.shape()), rng.uniform(-1, 1, H.finest.disc.shape())
    v = multigrid.vcycle(H, 0, u, f)
    w = multigrid.vcycle(H, 0, u, f, gamma=2)
    assert np.abs(v - w).max() > 1e-6 * np.abs(v).max()
