"""Stability function, critical parameter mu* and the coarsening rule.

Lemma (chap4_theorem2): the nonzero eigenvalue of (K_tau + lambda M_tau)^{-1} N_tau
is the A-stability function of the DG scheme, the (p_t, p_t+1) subdiagonal
Pade approximation of exp.  Reading of a sign slip there (compare Lemma 20,
alpha = R(-mu beta)): the eigenvalue is R(-lambda tau).

Remark (chap4_remarkCriticalDiscretizationParameter), eq.
(chap4_equationOptDiscrParam): mu*_{p_t} solves R(-3 mu*) = sqrt(2) - 1.

Section 4: full space-time coarsening is applied on level L iff
mu_L = tau_L / h_L^2 >= mu*, otherwise semi coarsening in time; semi doubles
mu, full halves it.  Readings where the paper is silent: the comparison uses
mu_L >= mu* (1 - 1e-12); full coarsening also needs at least 3 interior nodes
per axis; the same 1D mu* is used in d = 2, 3; coarsening stops at the
requested number of coarsest time steps (one by default, Section 2).
"""
from math import factorial

import numpy as np


def pade_coefficients(p):
    """Numerator / denominator coefficients (ascending powers) of the
    (p, p+1) Pade approximation of exp(z) (textbook closed form for the
    [m/k] Pade approximant with m = p, k = p + 1)."""
    m, k = p, p + 1
    num = [factorial(m + k - j) * factorial(m) / (factorial(m + k) * factorial(j) * factorial(m - j))
           for j in range(m + 1)]
    den = [factorial(m + k - j) * factorial(k) / (factorial(m + k) * factorial(j) * factorial(k - j)) * (-1) ** j
           for j in range(k + 1)]
    return np.array(num), np.array(den)


def pade_R(p, z):
    num, den = pade_coefficients(p)
    z = np.asarray(z, dtype=np.complex128)
    P = sum(c * z ** j for j, c in enumerate(num))
    Q = sum(c * z ** j for j, c in enumerate(den))
    r = P / Q
    return r.real if np.all(np.abs(r.imag) == 0) else r


def mu_star(p, tol=1e-15):
    """Root of R(-3 mu) = sqrt(2) - 1 by bisection on (0, 1]."""
    target = np.sqrt(2.0) - 1.0
    lo, hi = 0.0, 1.0
    assert float(pade_R(p, -3.0 * hi)) < target < float(pade_R(p, -3.0 * lo))
    while hi - lo > tol:
        mid = 0.5 * (lo + hi)
        if float(pade_R(p, -3.0 * mid)) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def build_levels(d, n, p_t, N, T, coarsening="auto", coarsest_steps=1):
    """Level parameters from the finest to the coarsest.

    Returns a list of dicts (finest first) with keys N, n, tau, h, mu and
    'full' telling how this level is coarsened to the next one (None on the
    coarsest level).  coarsening: 'auto' (paper's rule), 'semi' (never
    coarsen space) or 'full' (coarsen space whenever n >= 3)."""
    ms = mu_star(p_t)
    levels = []
    Nl, nl, tau = N, n, T / N
    while True:
        h = 1.0 / (nl + 1)
        mu = tau / h ** 2
        lv = {"N": Nl, "n": nl, "tau": tau, "h": h, "mu": mu, "full": None}
        levels.append(lv)
        if Nl <= coarsest_steps:
            break
        if coarsening == "semi":
            full = False
        elif coarsening == "full":
            full = nl >= 3
        else:
            full = (mu >= ms * (1.0 - 1e-12)) and nl >= 3
        lv["full"] = full
        Nl //= 2
        tau *= 2.0
        if full:
            nl = (nl - 1) // 2
    return levels
