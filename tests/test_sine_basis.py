"""The sine-basis identities behind the CUDA cycle (Section 3.1 symbols),
checked on the CPU against the oracle's assembled matrices: with S the
unnormalised DST-I along every axis (S[j, k] = sin(jk pi / Nf)),

* S M_h S^-1 and S K_h S^-1 are diagonal with lamM_i = prod_a m(k_a) and
  lamK_i = sum_a kappa(k_a) prod_{b != a} m(k_b), m(k) = h/3 (2 + cos(k pi/Nf)),
  kappa(k) = 2/h (1 - cos(k pi/Nf)) (d = 1, 2, 3);
* the full-coarsening restriction in the sine basis takes, per axis, the fine
  modes k and Nf - k of coarse mode k with weights (1 + c_k)/2 and -(1 - c_k)/2
  (c_k = cos(k pi / Nf)), mode Nf/2 has no coarse partner, and the
  prolongation P = R^T has the same weights doubled;
* the Legendre time blocks: the damped step on the tabulated w A^-1 f equals
  the damped block-Jacobi step for every mode (the form the FP64 smoother uses).
These are the formulas the library tabulates on the host; the test pins them
to the oracle's element-by-element assembly, not to the library."""
import numpy as np
import pytest

from oracle import dg_time, fe_space, transfer


def dst_matrix(n):
    Nf = n + 1
    j = np.arange(1, n + 1)
    return np.sin(np.outer(j, j) * np.pi / Nf)


def dst_nd(d, n):
    S1 = dst_matrix(n)
    S = S1
    for _ in range(d - 1):
        S = np.kron(S1, S)
    return S


def mode_symbols(d, n):
    """lamM, lamK per mode in the node ordering (first axis fastest)."""
    h = 1.0 / (n + 1)
    c = np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    m = h / 3.0 * (2.0 + c)
    kap = 2.0 / h * (1.0 - c)
    lamM = np.ones(1)
    lamK = np.zeros(1)
    for _ in range(d):   # new slowest axis on the left, as the Kronecker factors
        lamK = np.kron(kap, lamM) + np.kron(m, lamK)
        lamM = np.kron(m, lamM)
    return lamM, lamK


@pytest.mark.parametrize("d,n", [(1, 15), (1, 31), (2, 7), (2, 15), (3, 7)])
def test_sine_basis_diagonalises_mass_and_stiffness(d, n):
    M, K = fe_space.fe_matrices(d, n)
    S = dst_nd(d, n)
    Si = np.linalg.inv(S)
    lamM, lamK = mode_symbols(d, n)
    for A, lam in ((M.toarray(), lamM), (K.toarray(), lamK)):
        D = S @ A @ Si
        scale = np.abs(lam).max()
        assert np.abs(D - np.diag(np.diag(D))).max() < 1e-11 * scale
        assert np.allclose(np.diag(D), lam, rtol=1e-12, atol=1e-13 * scale)


def pair_weights_1d(nf):
    """Restriction in the sine basis along one axis, from the stated weights."""
    Nf = nf + 1
    nc = (nf - 1) // 2
    W = np.zeros((nc, nf))
    for k in range(1, nc + 1):
        ck = np.cos(k * np.pi / Nf)
        W[k - 1, k - 1] = 0.5 * (1.0 + ck)
        W[k - 1, Nf - k - 1] = -0.5 * (1.0 - ck)
    return W


@pytest.mark.parametrize("d,nf", [(1, 15), (1, 63), (2, 15), (3, 7)])
def test_restriction_and_prolongation_pair_modes(d, nf):
    nc = (nf - 1) // 2
    R = transfer.space_restriction(d, nf).toarray()
    Sf, Sc = dst_nd(d, nf), dst_nd(d, nc)
    Rs = Sc @ R @ np.linalg.inv(Sf)                    # restriction acting on sine coefficients
    W1 = pair_weights_1d(nf)
    W = W1
    for _ in range(d - 1):
        W = np.kron(W1, W)
    assert np.abs(Rs - W).max() < 1e-12
    # mode Nf/2 of an axis has no coarse partner: its column is zero
    assert np.abs(pair_weights_1d(nf)[:, (nf + 1) // 2 - 1]).max() == 0.0
    Ps = Sf @ R.T @ np.linalg.inv(Sc)                  # P = R^T on sine coefficients
    assert np.abs(Ps - (2 ** d) * W.T).max() < 1e-12


@pytest.mark.parametrize("p_t", [0, 1, 3, 6])
@pytest.mark.parametrize("adjoint", [False, True])
def test_damped_step_on_tabulated_right_hand_side(p_t, adjoint):
    """out = w A^-1 (f + lamM sigma t) + (1 - w) u, with sigma the coupling
    vector of B = -lamM N_tau (forward: rows (-1)^k times the plain trace;
    adjoint: all rows times the alternating trace), equals wf + ws t + (1 - w) u
    with wf = w A^-1 f and ws = lamM w A^-1 sigma, for A = lamM K_tau + lamK M_tau."""
    tau, w = 0.25, 0.5
    Kt, Mt, Nt = dg_time.time_matrices(p_t, tau)
    q = p_t + 1
    rng = np.random.default_rng(7 + p_t)
    for lamM, lamK in ((0.3, 5.0), (1e-3, 200.0), (2.0, 0.01)):
        A = lamM * Kt + lamK * Mt
        if adjoint:
            A = A.T
        f, u, uprev = rng.uniform(-1, 1, (3, q))
        # the coupling of the block row: -B u_prev (forward) or -B^T u_next (adjoint)
        Bt = (-lamM * Nt).T if adjoint else -lamM * Nt
        g = f - Bt @ uprev
        ref = w * np.linalg.solve(A, g) + (1 - w) * u
        sigma = np.ones(q) if adjoint else (-1.0) ** np.arange(q)
        t = (((-1.0) ** np.arange(q)) @ uprev) if adjoint else uprev.sum()
        Wm = w * np.linalg.inv(A)
        out = Wm @ f + (lamM * (Wm @ sigma)) * t + (1 - w) * u
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n", [63, 127, 255, 511])
def test_dst_through_half_length_fft_equals_the_dense_transform(n):
    """The steps of the register sine transform, restated with numpy's FFT:
    pre-processing y_j = x_j (s_j + 1/2) + x_{Nf-j} (s_j - 1/2) (s_j = sin(j pi/Nf),
    y_0 = 0), the half-length complex FFT Z of z_m = y_{2m} + i y_{2m+1}, the
    even/odd split Y_k = 1/2 [A + (w_i - i w_r) B] (A = Z_k + conj Z_{H-k},
    B = Z_k - conj Z_{H-k}, W^k = w_r + i w_i = e^{-2 pi i k / Nf}) and the
    outputs X_{2k} = -Im Y_k, X_{2k+1} = sum_{c <= k} Re Y_c - Re Y_0 / 2, against
    the dense unnormalised DST-I; also with the split's 1/2 moved into the
    pre-processing weights, as the kernels do."""
    Nf = n + 1
    H = Nf // 2
    x = np.zeros(Nf)
    x[1:] = np.random.default_rng(n).uniform(-1, 1, n)
    j = np.arange(Nf)
    s = np.sin(j * np.pi / Nf)
    xr = x[(Nf - j) % Nf]                    # x_{Nf - j}, with x_Nf = x_0 = 0
    for half_in_pre in (False, True):
        scale = 0.5 if half_in_pre else 1.0
        y = x * scale * (s + 0.5) + xr * scale * (s - 0.5)
        y[0] = 0.0
        Z = np.fft.fft(y[0::2] + 1j * y[1::2])
        k = np.arange(H)
        Zc = np.conj(Z[(H - k) % H])
        A, B = Z + Zc, Z - Zc
        W = np.exp(-2j * np.pi * k / Nf)
        Y = (0.5 if not half_in_pre else 1.0) * (A + (W.imag - 1j * W.real) * B)
        X = np.zeros(Nf)
        X[0::2] = -Y.imag
        X[1::2] = np.cumsum(Y.real) - 0.5 * Y.real[0]
        ref = dst_matrix(n) @ x[1:]
        assert np.abs(X[1:] - ref).max() < 1e-12 * np.abs(ref).max()
