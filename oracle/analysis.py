"""Power-law decay exponent of the survival observables (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 4 characterises the long-time decay of P(t) and of the temporal autocorrelation C(t)
by an exponent gamma, C(t) ~ a t^(-gamma).  The paper does not say how gamma is fitted;
the reading taken here is the ordinary least-squares line through (log t, log C) over the
output times inside a window [t_min, t_max], gamma = -slope.

Pinned by (tests/test_oracle_analysis.py): exact power laws for several gamma and
amplitudes; a broken power law whose other branch lies outside the window; the two-level
C(t), which tends to a constant (gamma -> 0 at long times, with the closed-form residual
slope); invariance of gamma under C -> cC and t -> st.
"""
from __future__ import annotations

import numpy as np


def decay_exponent(times, C, t_min: float, t_max: float) -> tuple[float, float]:
    """(gamma, log a) of the least-squares fit log C = log a - gamma log t over the points with
    t_min <= t <= t_max.  Needs at least two distinct times there and C > 0."""
    t = np.asarray(times, dtype=np.float64)
    c = np.asarray(C, dtype=np.float64)
    sel = (t >= t_min) & (t <= t_max)
    x, y = np.log(t[sel]), np.log(c[sel])
    if x.size < 2 or np.ptp(x) == 0.0:
        raise ValueError("need two distinct times in the window")
    slope, intercept = np.polyfit(x, y, 1)
    return float(-slope), float(intercept)
