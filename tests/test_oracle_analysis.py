"""Pins of the power-law exponent fit (oracle.analysis) and the library's own fit against it.

The library's kry_decay_exponent is host arithmetic, so it runs here without a GPU."""
import ctypes

import numpy as np
import pytest

from oracle import analysis, dense


@pytest.mark.parametrize("gamma,a", [(0.97, 1.0), (0.27, 0.3), (0.83, 2.5), (0.0, 0.7), (1.6, 1e-3)])
def test_exact_power_law(gamma, a):
    t = np.logspace(-1, 3, 50)
    C = a * t ** (-gamma)
    g, la = analysis.decay_exponent(t, C, 1.0, 1e3)
    assert abs(g - gamma) < 1e-12 and abs(la - np.log(a)) < 1e-11


def test_window_excludes_the_other_branch():
    """A broken power law: t^-0.2 before t = 10, t^-0.9 after; the window [20, 1000] sees only
    the second branch, [0.1, 5] only the first."""
    t = np.logspace(-1, 3, 81)
    C = np.where(t < 10.0, t ** -0.2, 10.0 ** 0.7 * t ** -0.9)
    assert abs(analysis.decay_exponent(t, C, 20.0, 1e3)[0] - 0.9) < 1e-12
    assert abs(analysis.decay_exponent(t, C, 0.1, 5.0)[0] - 0.2) < 1e-12


def test_two_level_autocorrelation_saturates():
    """L = 2: C(t) = 1 - A/2 + (A/2) sin(W t)/(W t) tends to 1 - A/2, so gamma -> 0; the fitted
    slope over [1e3, 1e4] is bounded by the oscillating term, |gamma| <= A/((2 - A) W t_min) x 4."""
    J, h = 1.0, [0.3, -0.4]
    d = h[0] - h[1]
    W = np.hypot(J, d)
    A = J * J / (W * W)
    t = np.logspace(3, 4, 200)
    H = np.array([[h[0] / 2 - h[1] / 2, J / 2], [J / 2, -h[0] / 2 + h[1] / 2]])
    C = dense.autocorrelation_dense(H, np.array([1.0, 0.0], complex), t)
    g, la = analysis.decay_exponent(t, C, 1e3, 1e4)
    assert abs(g) <= 4.0 * A / ((2.0 - A) * W * 1e3)
    assert abs(la - np.log(1.0 - A / 2.0)) < 1e-3


def test_scale_invariance():
    rng = np.random.default_rng(3)
    t = np.logspace(0, 2, 40)
    C = t ** -0.5 * (1.0 + 0.05 * rng.standard_normal(t.size))
    g1, _ = analysis.decay_exponent(t, C, 1.0, 100.0)
    g2, _ = analysis.decay_exponent(3.0 * t, 5.0 * C, 3.0, 300.0)
    assert abs(g1 - g2) < 1e-12


def test_too_few_points():
    with pytest.raises(ValueError):
        analysis.decay_exponent([1.0, 2.0], [1.0, 0.5], 1.5, 3.0)


def test_library_fit_matches_oracle():
    import paper_1704_02770_gb300 as k
    k.load()
    rng = np.random.default_rng(5)
    t = np.logspace(-1, 2, 40)
    C = 0.8 * t ** -0.6 * np.exp(0.1 * rng.standard_normal(t.size))
    for lo, hi in [(1.0, 100.0), (0.1, 100.0), (0.5, 3.0)]:
        g, la = k.decay_exponent(t, C, lo, hi)
        go, lao = analysis.decay_exponent(t, C, lo, hi)
        assert abs(g - go) < 1e-12 and abs(la - lao) < 1e-11
    with pytest.raises(k.KryError):
        k.decay_exponent([1.0, 2.0], [1.0, 0.5], 1.5, 3.0)
    with pytest.raises(k.KryError):
        k.decay_exponent([1.0, 2.0], [1.0, -0.5], 0.5, 3.0)
