"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each test patches one plausible error into an oracle function and checks that
the pin guarding that function fails; this shows the pins are not vacuous."""
import numpy as np
import pytest

from oracle import dg_time, hierarchy, multigrid, spacetime, transfer
from tests import test_oracle_mg as mg_pins
from tests import test_oracle_space as space_pins


def test_transposed_n_tau_breaks_pade_pin(monkeypatch):
    orig = dg_time.time_matrices

    def bad(p_t, tau):
        K, M, N = orig(p_t, tau)
        return K, M, N.T
    monkeypatch.setattr(dg_time, "time_matrices", bad)
    K, M, N = dg_time.time_matrices(1, 0.5)
    ev = np.linalg.eigvals(np.linalg.solve(K + 2.0 * M, N))
    assert abs(ev[np.argmax(np.abs(ev))] - hierarchy.pade_R(1, -1.0)) > 1e-3


def test_sign_error_in_k_tau_breaks_pade_pin(monkeypatch):
    orig = dg_time.time_matrices

    def bad(p_t, tau):
        K, M, N = orig(p_t, tau)
        return K.T, M, N            # transposed K_tau (test/trial swapped)
    monkeypatch.setattr(dg_time, "time_matrices", bad)
    K, M, N = dg_time.time_matrices(1, 0.5)
    ev = np.linalg.eigvals(np.linalg.solve(K + 2.0 * M, N))
    assert abs(ev[np.argmax(np.abs(ev))] - hierarchy.pade_R(1, -1.0)) > 1e-3


def test_swapped_time_blocks_break_galerkin_pin(monkeypatch):
    orig = transfer.time_blocks
    monkeypatch.setattr(transfer, "time_blocks", lambda p, tau: orig(p, tau)[::-1])
    assert space_pins.galerkin_case(1, 15, 1, 8, False) > 1e-3


def test_quarter_weighting_breaks_galerkin_pin(monkeypatch):
    orig = transfer.space_restriction_1d
    monkeypatch.setattr(transfer, "space_restriction_1d", lambda n: 0.5 * orig(n))
    assert space_pins.galerkin_case(1, 15, 1, 8, True) > 1e-3


def test_dropped_coupling_breaks_forward_substitution_pin(monkeypatch):
    def bad_apply(disc, u):
        return (disc.A @ u.T).T               # B u_{n-1} term dropped
    monkeypatch.setattr(spacetime, "apply_L", bad_apply)
    with pytest.raises(AssertionError):
        mg_pins.test_mg_equals_forward_substitution(1, 31, 32, 1, 1.0)


def test_wrong_stiffness_scaling_breaks_convergence_pin(monkeypatch):
    orig = dg_time.time_matrices

    def bad(p_t, tau):
        K, M, N = orig(p_t, tau)
        return K, 0.5 * M, N                  # halved M_tau: wrong diffusion rate
    monkeypatch.setattr(dg_time, "time_matrices", bad)
    with pytest.raises(AssertionError):
        mg_pins.test_manufactured_convergence_orders(1, 1, [3, 4, 5])


def test_wrong_damping_breaks_contraction_pin(monkeypatch):
    orig = multigrid.smooth
    monkeypatch.setattr(multigrid, "smooth", lambda lv, u, f, nu, omega, adjoint=False:
                        orig(lv, u, f, nu, 1.6, adjoint))
    from tests import test_oracle_lfa as lfa_pins
    meas = lfa_pins.measured_two_grid(1, 1.0, False, n=63, N=16, iters=12)
    assert meas > 0.2     # the LFA value at omega = 1/2 is about 0.115


def test_dropped_cycle_index_breaks_wcycle_pin(monkeypatch):
    """gamma ignored (every W-cycle run as a V-cycle, recursion included)."""
    from tests import test_oracle_wcycle as w_pins
    orig = multigrid.vcycle
    monkeypatch.setattr(multigrid, "vcycle", lambda H, i, u, f, nu1=2, nu2=2, omega=0.5, adjoint=False, gamma=1:
                        orig(H, i, u, f, nu1, nu2, omega, adjoint, 1))
    with pytest.raises(AssertionError):
        w_pins.test_wcycle_on_three_levels_differs_from_vcycle()


def test_wrong_spatial_damping_breaks_inexact_inverse_pin(monkeypatch):
    """The spatial V-cycle of the inexact block inverse with omega_x = 1.6
    instead of 2/3 no longer contracts at a multigrid rate."""
    from tests import test_oracle_inexact as inexact_pins
    orig = multigrid.SpatialVCycle

    class Bad(orig):
        def __init__(self, d, n, p_t, tau, nu_x=2, omega_x=2.0 / 3.0):
            super().__init__(d, n, p_t, tau, nu_x, 1.6)
    monkeypatch.setattr(multigrid, "SpatialVCycle", Bad)
    with pytest.raises(AssertionError):
        inexact_pins.test_spatial_vcycle_is_a_convergent_approximate_inverse(2, 15, 1, 1.0, False)


def test_quarter_weighting_breaks_inexact_galerkin_pin(monkeypatch):
    from tests import test_oracle_inexact as inexact_pins
    orig = transfer.space_restriction_1d
    monkeypatch.setattr(transfer, "space_restriction_1d", lambda n: 0.5 * orig(n))
    with pytest.raises(AssertionError):
        inexact_pins.test_spatial_coarse_operator_is_galerkin(1, 31)


def test_transposed_time_restriction_breaks_high_degree_pin(monkeypatch):
    """Coarse and fine degrees swapped in the time blocks at p_t = 10."""
    from tests import test_oracle_high_order as hi_pins
    orig = transfer.time_blocks
    monkeypatch.setattr(transfer, "time_blocks", lambda p, tau: tuple(R.T for R in orig(p, tau)))
    with pytest.raises(AssertionError):
        hi_pins.test_time_restriction_is_lower_triangular_and_exact_on_polynomials(10)
