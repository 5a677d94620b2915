"""Device small exponential (kry_tridiag_expv) against the oracle's Pade exponential.

y = exp(-i tau T) e_1 must match to 1e-13; the error estimate err = h |e_m^T tau
phi_1(-i tau (T - c)) e_1| is checked against the last first-column entry of the Pade
exponential of the augmented matrix [[-i tau (T - c), 0], [tau e_m^T, 0]].
"""
import numpy as np
import pytest

from oracle import pade

pytestmark = pytest.mark.gpu


def _gershgorin_centre(a, b):
    m = a.size
    lo, hi = np.inf, -np.inf
    for j in range(m):
        off = (abs(b[j - 1]) if j >= 1 else 0.0) + (abs(b[j]) if j + 1 < m else 0.0)
        lo, hi = min(lo, a[j] - off), max(hi, a[j] + off)
    return 0.5 * (lo + hi)


def _reference(a, b, h, tau):
    m = a.size
    T = np.diag(a) + np.diag(b[: m - 1], 1) + np.diag(b[: m - 1], -1)
    y = pade.expm(-1j * tau * T)[:, 0]
    c = _gershgorin_centre(a, b)
    M = np.zeros((m + 1, m + 1), complex)
    M[:m, :m] = -1j * tau * (T - c * np.eye(m))
    M[m, m - 1] = tau
    err = abs(h) * abs(pade.expm(M)[m, 0])
    return y, err


@pytest.mark.parametrize("m", [1, 2, 5, 17, 30, 32])
@pytest.mark.parametrize("tau", [0.0, 1e-9, 0.05, 0.7, 3.0])
def test_expv_matches_pade(kry, m, tau):
    rng = np.random.default_rng(m * 13 + int(tau * 100))
    a = rng.normal(size=m) * 3.0 + 1.5
    b = np.abs(rng.normal(size=max(m - 1, 1))) * 2.0 + 0.1
    h = 1.7
    y, err = kry.tridiag_expv(a, b[: m - 1], h, tau)
    yr, er = _reference(a, b, h, tau)
    assert np.max(np.abs(y - yr)) < 1e-13
    assert abs(err - er) <= 1e-11 * er + 1e-20


def test_expv_large_argument(kry):
    """tau * half-width near the per-step cap (50) still matches."""
    m = 30
    rng = np.random.default_rng(9)
    a = rng.normal(size=m) * 4.0
    b = np.abs(rng.normal(size=m - 1)) * 3.0 + 0.5
    lo = np.min(a - np.r_[0, np.abs(b)] - np.r_[np.abs(b), 0])
    hi = np.max(a + np.r_[0, np.abs(b)] + np.r_[np.abs(b), 0])
    tau = 48.0 / (0.5 * (hi - lo))
    y, err = kry.tridiag_expv(a, b, 0.9, tau)
    yr, er = _reference(a, np.r_[b, 0.0], 0.9, tau)
    assert np.max(np.abs(y - yr)) < 1e-12
    assert abs(err - er) <= 1e-10 * er + 1e-15
    assert abs(np.linalg.norm(y) - 1.0) < 1e-12


def test_expv_rejects_bad_arguments(kry):
    with pytest.raises(kry.KryError):
        kry.tridiag_expv(np.zeros(33), np.zeros(32), 1.0, 1.0)
    with pytest.raises(kry.KryError):
        kry.tridiag_expv(np.zeros(3), np.zeros(2), 1.0, -1.0)
