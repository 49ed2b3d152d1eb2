"""Local Fourier mode analysis for d = 1 (Section 3).

Symbols, built from the oracle's own quadrature matrices (K_tau, M_tau, N_tau):

  Lemma 17   Lhat(tx, tt) = h/3 (2 + cos tx) [K + h^-2 beta(tx) M - e^{-i tt} N],
             beta(t) = 6 (1 - cos t) / (2 + cos t)
  Lemma 18   Shat(tx, tt) = (1 - w) I + w e^{-i tt} (K + h^-2 beta M)^{-1} N
  Lemma 12   Rhat(tt) = e^{-i tt} R_1 + R_2
  Lemma 13   Phat(tt) = 1/2 [e^{i tt} R_1^T + R_2^T]
  Lemma 25   Rhat_x(tx) = 1 + cos tx,  Phat_x = Rhat_x / 2
  Thms 5, 6  two-grid symbols on the harmonics
             (tx, tt), (g(tx), tt), (tx, g(tt)), (g(tx), g(tt)), g(t) = t - sign(t) pi.

Reading of two misprints in the coarse-grid inverse for semi coarsening
(mapping (chap4_mappinginvLs)): the second block is Lhat_{2tau,h}(g(tx), 2 tt).
Smoothing order (Theorems 5, 6): S^{nu2} K S^{nu1}.  gamma(0) = pi (the paper's
sign(0) would map the frequency 0 onto itself).

Frequencies (Definition of the asymptotic two-grid factors): low frequencies
(tx, tt) in (-pi/2, pi/2]^2 on a periodic grid of Nx x Nt points, tx != 0.
"""
import numpy as np

from . import dg_time, transfer


def gam(t):
    """gamma(t) = t - sign(t) pi (Lemma chap4_lemma9); reading: gamma(0) = pi,
    so that gamma maps the low set (-pi/2, pi/2] one to one onto the high set."""
    return t - np.pi if t > 0 else t + np.pi


def beta(tx):
    return 6.0 * (1.0 - np.cos(tx)) / (2.0 + np.cos(tx))


class Symbols:
    def __init__(self, p_t, tau, h, omega=0.5):
        self.p_t, self.tau, self.h, self.omega = p_t, tau, h, omega
        self.q = p_t + 1
        self.K, self.M, self.N = dg_time.time_matrices(p_t, tau)
        self.R1, self.R2 = transfer.time_blocks(p_t, tau)

    def L(self, tx, tt, tau=None, h=None):
        tau = self.tau if tau is None else tau
        h = self.h if h is None else h
        K, M, N = dg_time.time_matrices(self.p_t, tau)
        return h / 3.0 * (2.0 + np.cos(tx)) * (K + beta(tx) / h ** 2 * M - np.exp(-1j * tt) * N)

    def S(self, tx, tt):
        inner = np.linalg.solve(self.K + beta(tx) / self.h ** 2 * self.M, self.N)
        return (1.0 - self.omega) * np.eye(self.q) + self.omega * np.exp(-1j * tt) * inner

    def Rt(self, tt):
        return np.exp(-1j * tt) * self.R1 + self.R2

    def Pt(self, tt):
        return 0.5 * (np.exp(1j * tt) * self.R1.T + self.R2.T)

    @staticmethod
    def Rx(tx):
        return 1.0 + np.cos(tx)

    @staticmethod
    def Px(tx):
        return 0.5 * (1.0 + np.cos(tx))

    def harmonics(self, tx, tt):
        return [(tx, tt), (gam(tx), tt), (tx, gam(tt)), (gam(tx), gam(tt))]

    def Ltilde(self, tx, tt):
        q = self.q
        out = np.zeros((4 * q, 4 * q), dtype=complex)
        for i, (a, b) in enumerate(self.harmonics(tx, tt)):
            out[i * q:(i + 1) * q, i * q:(i + 1) * q] = self.L(a, b)
        return out

    def Stilde(self, tx, tt):
        q = self.q
        out = np.zeros((4 * q, 4 * q), dtype=complex)
        for i, (a, b) in enumerate(self.harmonics(tx, tt)):
            out[i * q:(i + 1) * q, i * q:(i + 1) * q] = self.S(a, b)
        return out

    def R_semi(self, tt):
        q = self.q
        Z = np.zeros((q, q))
        return np.block([[self.Rt(tt), Z, self.Rt(gam(tt)), Z],
                         [Z, self.Rt(tt), Z, self.Rt(gam(tt))]])

    def P_semi(self, tt):
        q = self.q
        Z = np.zeros((q, q))
        return np.block([[self.Pt(tt), Z], [Z, self.Pt(tt)],
                         [self.Pt(gam(tt)), Z], [Z, self.Pt(gam(tt))]])

    def Lc_semi(self, tx, tt):
        q = self.q
        out = np.zeros((2 * q, 2 * q), dtype=complex)
        out[:q, :q] = self.L(tx, 2 * tt, tau=2 * self.tau)
        out[q:, q:] = self.L(gam(tx), 2 * tt, tau=2 * self.tau)
        return out

    def R_full(self, tx, tt):
        return np.hstack([self.Rx(a) * self.Rt(b) for (a, b) in self.harmonics(tx, tt)])

    def P_full(self, tx, tt):
        return np.vstack([self.Px(a) * self.Pt(b) for (a, b) in self.harmonics(tx, tt)])

    def Lc_full(self, tx, tt):
        return self.L(2 * tx, 2 * tt, tau=2 * self.tau, h=2 * self.h)

    def two_grid(self, tx, tt, nu1, nu2, full):
        """Mtilde^s or Mtilde^f (Theorems 5, 6), a 4q x 4q matrix."""
        Lt = self.Ltilde(tx, tt)
        St = self.Stilde(tx, tt)
        if full:
            Kt = np.eye(4 * self.q) - self.P_full(tx, tt) @ np.linalg.solve(
                self.Lc_full(tx, tt), self.R_full(tx, tt) @ Lt)
        else:
            Kt = np.eye(4 * self.q) - self.P_semi(tt) @ np.linalg.solve(
                self.Lc_semi(tx, tt), self.R_semi(tt) @ Lt)
        return np.linalg.matrix_power(St, nu2) @ Kt @ np.linalg.matrix_power(St, nu1)


def spectral_radius(A):
    return float(np.max(np.abs(np.linalg.eigvals(A))))


def low_frequencies(Nx, Nt):
    tx = 2.0 * np.pi * np.arange(1 - Nx // 2, Nx // 2 + 1) / Nx
    tt = 2.0 * np.pi * np.arange(1 - Nt // 2, Nt // 2 + 1) / Nt
    tx = tx[(tx > -np.pi / 2) & (tx <= np.pi / 2) & (tx != 0.0)]
    tt = tt[(tt > -np.pi / 2) & (tt <= np.pi / 2)]
    return tx, tt


def two_grid_factor(p_t, mu, nu, full, Nx=1024, Nt=256, omega=0.5, stride=1):
    """rho(Mhat_mu^{s|f}): max spectral radius over the low frequencies with
    tx != 0 (Definition of the asymptotic two-grid factors).  ``stride``
    subsamples the frequency grid (for quick tests)."""
    h = 1.0 / Nx
    tau = mu * h ** 2
    sym = Symbols(p_t, tau, h, omega)
    txs, tts = low_frequencies(Nx, Nt)
    best = 0.0
    for tx in txs[::stride]:
        for tt in tts[::stride]:
            best = max(best, spectral_radius(sym.two_grid(tx, tt, nu, nu, full)))
    return best


def smoothing_factor(p_t, mu, full, Nx=1024, Nt=256, omega=0.5):
    """mu_S^{s|f}: max rho(Shat) over the high frequencies (Definition of the
    asymptotic smoothing factors)."""
    h = 1.0 / Nx
    tau = mu * h ** 2
    sym = Symbols(p_t, tau, h, omega)
    tx = 2.0 * np.pi * np.arange(1 - Nx // 2, Nx // 2 + 1) / Nx
    tt = 2.0 * np.pi * np.arange(1 - Nt // 2, Nt // 2 + 1) / Nt
    best = 0.0
    for a in tx:
        for b in tt:
            low_t = -np.pi / 2 < b <= np.pi / 2
            low_x = -np.pi / 2 < a <= np.pi / 2
            high = (not low_t) if not full else not (low_t and low_x)
            if high:
                best = max(best, spectral_radius(sym.S(a, b)))
    return best
