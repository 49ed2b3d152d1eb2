"""Pins of the oracle's local Fourier analysis and of the smoother / two-grid
cycle against the paper's lemmas and bounds (Section 3)."""
import numpy as np
import pytest

from oracle import hierarchy, lfa, multigrid
from paper_1411_0519_gb300 import workloads


def lemma20_radius(p, mu, tx, tt, omega):
    """Lemma 20; for p_t = 0 the symbol is a scalar and the |1 - w| branch (the
    zero eigenvalue of the rank-one N_tau) does not exist."""
    alpha = hierarchy.pade_R(p, -mu * lfa.beta(tx))
    s2 = (1 - omega) ** 2 + 2 * omega * (1 - omega) * alpha * np.cos(tt) + alpha ** 2 * omega ** 2
    return np.sqrt(s2) if p == 0 else max(abs(1 - omega), np.sqrt(s2))


@pytest.mark.parametrize("p", [0, 1, 2, 3])
@pytest.mark.parametrize("omega", [0.5, 1.0, 0.8])
def test_smoother_symbol_spectral_radius_lemma20(p, omega):
    """rho(Shat) = max{|1-w|, sqrt((1-w)^2 + 2w(1-w) alpha cos tt + alpha^2 w^2)},
    alpha = R(-mu beta(tx)) (Lemma 20), with Shat built from the assembled matrices."""
    rng = np.random.default_rng(p)
    for _ in range(20):
        mu = 10 ** rng.uniform(-3, 3)
        h = 1.0 / 64
        sym = lfa.Symbols(p, mu * h * h, h, omega)
        tx, tt = rng.uniform(-np.pi, np.pi, 2)
        rho = lfa.spectral_radius(sym.S(tx, tt))
        assert abs(rho - lemma20_radius(p, mu, tx, tt, omega)) < 1e-12


@pytest.mark.parametrize("p", [0, 1, 2, 3])
def test_semi_smoothing_factor_bound(p):
    """mu_S^s <= 1/sqrt(2) at omega = 1/2 for all mu (Lemma 21b)."""
    for mu in [1e-3, 0.1, 1.0, 10.0, 1e3]:
        assert lfa.smoothing_factor(p, mu, full=False, Nx=64, Nt=32) <= 1 / np.sqrt(2) + 1e-12


@pytest.mark.parametrize("p", [0, 2])
def test_full_smoothing_factor_lemma23(p):
    """Even p_t: sup over theta_t in [0, pi], theta_x in [pi/2, pi] equals
    (1 + R(-3 mu)) / 2 (Lemma 23); at mu = mu* this is 1/sqrt(2).  The proof
    assumes R(-mu beta) decreasing in beta on [3, 12]; for p_t = 2 the Pade
    function has a minimum near z = -11, so the identity is checked only for
    mu up to mu* there (for p_t = 0, R = 1/(1-z) is monotone for all mu)."""
    mus = [0.05, hierarchy.mu_star(p), 3.0] if p == 0 else [0.05, 0.2, hierarchy.mu_star(p)]
    for mu in mus:
        h = 1.0 / 64
        sym = lfa.Symbols(p, mu * h * h, h, 0.5)
        best = 0.0
        for tx in np.linspace(np.pi / 2, np.pi, 33):
            for tt in np.linspace(0, np.pi, 33):
                best = max(best, lfa.spectral_radius(sym.S(tx, tt)))
        assert abs(best - 0.5 * (1 + hierarchy.pade_R(p, -3 * mu))) < 1e-12
    assert abs(0.5 * (1 + hierarchy.pade_R(p, -3 * hierarchy.mu_star(p))) - 1 / np.sqrt(2)) < 1e-12


@pytest.mark.parametrize("p", [0, 1, 2])
def test_symbol_galerkin_identity(p):
    """Rtilde Ltilde Ptilde = coarse symbol for both coarsenings: the transfer
    symbols of Lemmas 12, 13, 25-29 are consistent with the re-discretised
    coarse operator (the symbol form of R L P = L_c)."""
    h = 1.0 / 128
    sym = lfa.Symbols(p, 0.7 * h * h, h)
    rng = np.random.default_rng(p)
    for _ in range(10):
        tx, tt = rng.uniform(-np.pi / 2, np.pi / 2, 2)
        G = sym.R_semi(tt) @ sym.Ltilde(tx, tt) @ sym.P_semi(tt)
        assert np.allclose(G, sym.Lc_semi(tx, tt), atol=1e-14)
        G = sym.R_full(tx, tt) @ sym.Ltilde(tx, tt) @ sym.P_full(tx, tt)
        assert np.allclose(G, sym.Lc_full(tx, tt), atol=1e-14)


def measured_two_grid(p, mu, full, n=127, N=32, iters=25):
    """Section 3.2 protocol: f = 0, random u0 in [0, 1], max_k ||r_{k+1}|| / ||r_k||."""
    h = 1.0 / (n + 1)
    T = mu * h * h * N
    H = multigrid.Hierarchy(1, n, p, N, T, coarsening="full" if full else "semi", coarsest_steps=N // 2)
    disc = H.finest.disc
    u = workloads.uniform_iterate(1, n, p, N, seed=0).reshape(disc.shape())
    f = np.zeros_like(u)
    rs = [np.linalg.norm(H.finest.residual(u, f))]
    for _ in range(iters):
        u = multigrid.two_grid(H, u, f, 2, 2, 0.5)
        rs.append(np.linalg.norm(H.finest.residual(u, f)))
    rs = np.array(rs)
    return float(np.max(rs[1:] / rs[:-1]))


@pytest.mark.parametrize("p", [0, 1])
def test_two_grid_contraction_agrees_with_lfa(p):
    """Figures of Section 3.2 (data not printed): the measured two-grid factor
    agrees with the LFA factor; semi coarsening <= 1/2 for every mu, full
    coarsening <= 1/2 for mu >= mu*, and full coarsening above 1/2 well below mu*.
    Tolerance 0.05 on the agreement (the curves themselves are unpinned)."""
    ms = hierarchy.mu_star(p)
    for mu, full in [(0.01, False), (1.0, False), (100.0, False), (ms, True), (10.0, True)]:
        meas = measured_two_grid(p, mu, full)
        th = lfa.two_grid_factor(p, mu, 2, full, Nx=128, Nt=32)
        assert abs(meas - th) < 0.05, (mu, full, meas, th)
        assert meas <= 0.5 and th <= 0.5
    meas = measured_two_grid(p, 0.01, True)
    th = lfa.two_grid_factor(p, 0.01, 2, True, Nx=128, Nt=32)
    assert meas > 0.5 and th > 0.5


@pytest.mark.parametrize("p", [0, 1])
@pytest.mark.parametrize("full", [False, True])
def test_batched_two_grid_factor_equals_loop(p, full):
    """The vectorised LFA used for the paper-size comparison equals the
    frequency-by-frequency evaluation of Theorems 5-6."""
    for mu in [0.01, hierarchy.mu_star(p), 30.0]:
        a = lfa.two_grid_factor(p, mu, 2, full, Nx=64, Nt=16)
        b = lfa.two_grid_factor_batch(p, mu, 2, full, Nx=64, Nt=16)
        assert abs(a - b) < 1e-12
