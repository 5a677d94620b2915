"""Pins of the oracle's temporal autocorrelation C(t) = (1/t) int_0^t P (Sec. 4).

The oracle evaluates the integral in closed form from a full eigendecomposition; it is
pinned here by a two-level closed form, the empty sector, the short-time law and direct
numerical quadrature of P(t).
"""
import numpy as np

from oracle import dense
import workloads


def _system(L, N, J, Delta, h, pbc, state):
    H = dense.hamiltonian_kron(L, J, Delta, h, pbc, N)
    states = list(dense.sector_states(L, N))
    psi0 = np.zeros(len(states))
    psi0[states.index(state)] = 1.0
    return H, psi0


def test_two_level_closed_form():
    """L = 2, N = 1: P = 1 - A/2 + (A/2) cos(W t), so C = 1 - A/2 + (A/2) sin(W t)/(W t)."""
    J, h = 1.3, [0.8, -0.3]
    H, psi0 = _system(2, 1, J, 0.4, h, False, 0b01)
    times = np.array([1e-3, 0.3, 1.7, 5.0, 23.0])
    d = h[0] - h[1]
    W = np.sqrt(J * J + d * d)
    A = J * J / (W * W)
    want = 1.0 - A / 2.0 + (A / 2.0) * np.sin(W * times) / (W * times)
    assert np.max(np.abs(dense.autocorrelation_dense(H, psi0, times) - want)) < 1e-13


def test_empty_sector_and_zero_time():
    H, psi0 = _system(6, 0, 1.0, 1.0, workloads.quasiperiodic_field(6, 2.0, 0.3), True, 0)
    assert np.allclose(dense.autocorrelation_dense(H, psi0, [0.0, 0.5, 40.0]), 1.0, atol=1e-14)
    H, psi0 = _system(8, 4, 1.0, 1.0, workloads.quasiperiodic_field(8, 1.0, 0.3), True, workloads.neel_state(8))
    assert dense.autocorrelation_dense(H, psi0, [0.0])[0] == 1.0


def test_short_time_law():
    """1 - P = (L J^2/4) t^2 + O(t^4) for the Neel state on a ring, so
    1 - C = (L J^2/12) t^2 + O(t^4)."""
    L = 10
    H, psi0 = _system(L, 5, 1.0, 1.0, workloads.quasiperiodic_field(L, 2.0, 0.4), True, workloads.neel_state(L))
    for t in (1e-3, 2e-3):
        c = dense.autocorrelation_dense(H, psi0, [t])[0]
        assert abs((1.0 - c) / t**2 - L / 12.0) < 1e-3 * L


def test_equals_quadrature_of_P():
    """C(t) against composite Simpson quadrature of the dense P(t') on a fine grid."""
    L = 10
    H, psi0 = _system(L, 5, 1.0, 0.8, workloads.quasiperiodic_field(L, 1.5, 1.1), True, workloads.neel_state(L))
    for t in (0.7, 6.0, 31.0):
        n = 20000
        x = np.linspace(0.0, t, n + 1)
        P = dense.return_probability_dense(H, psi0, x)
        integral = (x[1] - x[0]) / 3.0 * (P[0] + P[-1] + 4.0 * P[1:-1:2].sum() + 2.0 * P[2:-1:2].sum())
        assert abs(dense.autocorrelation_dense(H, psi0, [t])[0] - integral / t) < 1e-9
