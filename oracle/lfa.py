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


# ---------------------------------------------------------------------------
# Batched evaluation over many frequencies (same formulas as Symbols, written
# with numpy broadcasting so that the full frequency grid of the paper's
# experiments, N_x = 1024 and N_t = 256, takes seconds).
# ---------------------------------------------------------------------------
def _L_batch(K, M, N, tx, tt, tau, h):
    """Lhat for arrays tx, tt (Lemma 17): shape (F, q, q)."""
    pref = (h / 3.0 * (2.0 + np.cos(tx)))[:, None, None]
    b = (beta(tx) / h ** 2)[:, None, None]
    ph = np.exp(-1j * tt)[:, None, None]
    return pref * (K[None] + b * M[None] - ph * N[None])


def _S_batch(K, M, N, tx, tt, h, omega):
    q = K.shape[0]
    A = K[None] + (beta(tx) / h ** 2)[:, None, None] * M[None]
    inner = np.linalg.solve(A, np.broadcast_to(N, A.shape))
    return (1.0 - omega) * np.eye(q)[None] + omega * np.exp(-1j * tt)[:, None, None] * inner


def _gam_arr(t):
    return np.where(t > 0, t - np.pi, t + np.pi)


def two_grid_factor_batch(p_t, mu, nu, full, Nx=1024, Nt=256, omega=0.5):
    """rho(Mhat_mu^{s|f}) over all low frequencies with tx != 0, vectorised;
    equal to two_grid_factor (checked by a test)."""
    h = 1.0 / Nx
    tau = mu * h ** 2
    q = p_t + 1
    K, M, N = dg_time.time_matrices(p_t, tau)
    K2, M2, N2 = dg_time.time_matrices(p_t, 2 * tau)
    R1, R2 = transfer.time_blocks(p_t, tau)
    txs, tts = low_frequencies(Nx, Nt)
    TX, TT = np.meshgrid(txs, tts, indexing="ij")
    tx, tt = TX.ravel(), TT.ravel()
    F = tx.size
    harm = [(tx, tt), (_gam_arr(tx), tt), (tx, _gam_arr(tt)), (_gam_arr(tx), _gam_arr(tt))]
    Lt = np.zeros((F, 4 * q, 4 * q), dtype=complex)
    St = np.zeros((F, 4 * q, 4 * q), dtype=complex)
    for i, (a, b) in enumerate(harm):
        Lt[:, i * q:(i + 1) * q, i * q:(i + 1) * q] = _L_batch(K, M, N, a, b, tau, h)
        St[:, i * q:(i + 1) * q, i * q:(i + 1) * q] = _S_batch(K, M, N, a, b, h, omega)

    def Rt(t):
        return np.exp(-1j * t)[:, None, None] * R1[None] + R2[None]

    def Pt(t):
        return 0.5 * (np.exp(1j * t)[:, None, None] * R1.T[None] + R2.T[None])

    if full:
        Rf = np.concatenate([(1.0 + np.cos(a))[:, None, None] * Rt(b) for (a, b) in harm], axis=2)
        Pf = np.concatenate([(0.5 * (1.0 + np.cos(a)))[:, None, None] * Pt(b) for (a, b) in harm], axis=1)
        K4, M4, N4 = dg_time.time_matrices(p_t, 2 * tau)
        Lc = _L_batch(K4, M4, N4, 2 * tx, 2 * tt, 2 * tau, 2 * h)
        Kt = np.eye(4 * q)[None] - Pf @ np.linalg.solve(Lc, Rf @ Lt)
    else:
        Z = np.zeros((F, q, q), dtype=complex)
        Rs = np.concatenate([np.concatenate([Rt(tt), Z, Rt(_gam_arr(tt)), Z], axis=2),
                             np.concatenate([Z, Rt(tt), Z, Rt(_gam_arr(tt))], axis=2)], axis=1)
        Ps = np.concatenate([np.concatenate([Pt(tt), Z], axis=2), np.concatenate([Z, Pt(tt)], axis=2),
                             np.concatenate([Pt(_gam_arr(tt)), Z], axis=2),
                             np.concatenate([Z, Pt(_gam_arr(tt))], axis=2)], axis=1)
        Lc = np.zeros((F, 2 * q, 2 * q), dtype=complex)
        Lc[:, :q, :q] = _L_batch(K2, M2, N2, tx, 2 * tt, 2 * tau, h)
        Lc[:, q:, q:] = _L_batch(K2, M2, N2, _gam_arr(tx), 2 * tt, 2 * tau, h)
        Kt = np.eye(4 * q)[None] - Ps @ np.linalg.solve(Lc, Rs @ Lt)
    Mt = np.linalg.matrix_power(St, nu) @ Kt @ np.linalg.matrix_power(St, nu)
    return float(np.max(np.abs(np.linalg.eigvals(Mt))))


def _Ahat_batch(K, M, tx, h):
    """Ahat(tx) = h/3 (2 + cos tx) K + 2/h (1 - cos tx) M (proof of Lemma 18)."""
    return (h / 3.0 * (2.0 + np.cos(tx)))[:, None, None] * K[None] + \
        (2.0 / h * (1.0 - np.cos(tx)))[:, None, None] * M[None]


def spatial_iteration_symbol(K, M, tx, h, nu_x=2, omega_x=2.0 / 3.0):
    """Mtilde(tx), 2q x 2q (Remark on the V-cycle approximation in space): the
    spatial two-grid iteration matrix on the harmonics (tx, gamma(tx)) with
    damped point-block Jacobi D^x = 2h/3 K + 2/h M, R_x = 1 + cos, P_x = R_x / 2,
    coarse Ahat on 2h; smoothing order S^{nu2} K S^{nu1} (nu1 = nu2 = nu_x)."""
    q = K.shape[0]
    F = tx.size
    gx = _gam_arr(tx)
    A1, A2 = _Ahat_batch(K, M, tx, h), _Ahat_batch(K, M, gx, h)
    Dx = 2.0 * h / 3.0 * K + 2.0 / h * M
    Dinv = np.linalg.inv(Dx)
    S1 = np.eye(q)[None] - omega_x * (Dinv[None] @ A1)
    S2 = np.eye(q)[None] - omega_x * (Dinv[None] @ A2)
    At = np.zeros((F, 2 * q, 2 * q), dtype=complex)
    St = np.zeros((F, 2 * q, 2 * q), dtype=complex)
    At[:, :q, :q], At[:, q:, q:] = A1, A2
    St[:, :q, :q], St[:, q:, q:] = S1, S2
    Rx = np.concatenate([(1.0 + np.cos(tx))[:, None, None] * np.eye(q)[None],
                         (1.0 + np.cos(gx))[:, None, None] * np.eye(q)[None]], axis=2)
    Px = np.concatenate([(0.5 * (1.0 + np.cos(tx)))[:, None, None] * np.eye(q)[None],
                         (0.5 * (1.0 + np.cos(gx)))[:, None, None] * np.eye(q)[None]], axis=1)
    Ac = _Ahat_batch(K, M, 2 * tx, 2 * h)
    Kx = np.eye(2 * q)[None] - Px @ np.linalg.solve(Ac, Rx @ At)
    Sn = np.linalg.matrix_power(St, nu_x)
    return Sn @ Kx @ Sn


def two_grid_factor_inexact_batch(p_t, mu, nu, full, Nx=1024, Nt=256, omega=0.5, nu_x=2, omega_x=2.0 / 3.0):
    """rho(Mbar_mu^{s|f}) (eq. chap4_twoGridIterationMatrixApprox): the two-grid
    factor with the inexact smoother Sbar = I - w (I - M) D^{-1} L, M acting as
    Mtilde(tx) on the two space harmonics of each time harmonic (mapping
    (chap4_mappingPropertyApprox)); otherwise as two_grid_factor_batch."""
    h = 1.0 / Nx
    tau = mu * h ** 2
    q = p_t + 1
    K, M, N = dg_time.time_matrices(p_t, tau)
    K2, M2, N2 = dg_time.time_matrices(p_t, 2 * tau)
    R1, R2 = transfer.time_blocks(p_t, tau)
    txs, tts = low_frequencies(Nx, Nt)
    TX, TT = np.meshgrid(txs, tts, indexing="ij")
    tx, tt = TX.ravel(), TT.ravel()
    F = tx.size
    harm = [(tx, tt), (_gam_arr(tx), tt), (tx, _gam_arr(tt)), (_gam_arr(tx), _gam_arr(tt))]
    Lt = np.zeros((F, 4 * q, 4 * q), dtype=complex)
    DL = np.zeros((F, 4 * q, 4 * q), dtype=complex)
    for i, (a, b) in enumerate(harm):
        Lab = _L_batch(K, M, N, a, b, tau, h)
        Lt[:, i * q:(i + 1) * q, i * q:(i + 1) * q] = Lab
        DL[:, i * q:(i + 1) * q, i * q:(i + 1) * q] = np.linalg.solve(_Ahat_batch(K, M, a, h), Lab)
    Mx = spatial_iteration_symbol(K, M, tx, h, nu_x, omega_x)
    Mbig = np.zeros((F, 4 * q, 4 * q), dtype=complex)
    Mbig[:, :2 * q, :2 * q] = Mx
    Mbig[:, 2 * q:, 2 * q:] = Mx
    Sbar = np.eye(4 * q)[None] - omega * (np.eye(4 * q)[None] - Mbig) @ DL

    def Rt(t):
        return np.exp(-1j * t)[:, None, None] * R1[None] + R2[None]

    def Pt(t):
        return 0.5 * (np.exp(1j * t)[:, None, None] * R1.T[None] + R2.T[None])

    if full:
        Rf = np.concatenate([(1.0 + np.cos(a))[:, None, None] * Rt(b) for (a, b) in harm], axis=2)
        Pf = np.concatenate([(0.5 * (1.0 + np.cos(a)))[:, None, None] * Pt(b) for (a, b) in harm], axis=1)
        Lc = _L_batch(K2, M2, N2, 2 * tx, 2 * tt, 2 * tau, 2 * h)
        Kt = np.eye(4 * q)[None] - Pf @ np.linalg.solve(Lc, Rf @ Lt)
    else:
        Z = np.zeros((F, q, q), dtype=complex)
        Rs = np.concatenate([np.concatenate([Rt(tt), Z, Rt(_gam_arr(tt)), Z], axis=2),
                             np.concatenate([Z, Rt(tt), Z, Rt(_gam_arr(tt))], axis=2)], axis=1)
        Ps = np.concatenate([np.concatenate([Pt(tt), Z], axis=2), np.concatenate([Z, Pt(tt)], axis=2),
                             np.concatenate([Pt(_gam_arr(tt)), Z], axis=2),
                             np.concatenate([Z, Pt(_gam_arr(tt))], axis=2)], axis=1)
        Lc = np.zeros((F, 2 * q, 2 * q), dtype=complex)
        Lc[:, :q, :q] = _L_batch(K2, M2, N2, tx, 2 * tt, 2 * tau, h)
        Lc[:, q:, q:] = _L_batch(K2, M2, N2, _gam_arr(tx), 2 * tt, 2 * tau, h)
        Kt = np.eye(4 * q)[None] - Ps @ np.linalg.solve(Lc, Rs @ Lt)
    Mt = np.linalg.matrix_power(Sbar, nu) @ Kt @ np.linalg.matrix_power(Sbar, nu)
    return float(np.max(np.abs(np.linalg.eigvals(Mt))))
