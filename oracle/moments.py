"""Return probability at early times from the moments of H (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definition followed: P(t) = |A(t)|^2, A(t) = <psi0| exp(-iHt) |psi0> (Eq. SP of Sec. 4), with
the exponential written as its power series.  For a basis state psi0 = |s0> and any shift c,
    A(t) = exp(-ict) sum_n (-it)^n mu_n / n!,   mu_n = <s0| (H - c)^n |s0>,
and the moments mu_0 .. mu_{2K} need only the states within K hops of s0 (basis.c,
orc_moments), so sectors far too large for the CSR oracle (L = 30, D = 155,117,520) are
reachable at early times.  c is the diagonal element of s0.

Error bound (rigorous, no assumption on convergence): with the spectral measure of psi0,
A(t) = int exp(-iEt) dmu(E), and |exp(-ix) - sum_{n<N} (-ix)^n / n!| <= |x|^N / N!, so the
series truncated after n = 2K - 1 differs from A by at most t^(2K) mu_{2K} / (2K)!
(mu_{2K} = ||(H - c)^K psi0||^2 is the 2K-th absolute moment).  Since |A| <= 1,
|P_series - P| <= (2 + dA) dA.

Pinned by (tests/test_oracle_moments.py): dense eigendecomposition (Kronecker-product H) for
L <= 12 with the bound checked; the moments against dense matrix powers on sectors larger
than the ball; mu_1 = 0 and mu_2 = (J/2)^2 n_anti(s0) (closed form of the energy variance);
the two-level formula at L = 2; the size of the one-hop ball (1 + n_anti) and of the two-hop
ball against a brute-force search.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import basis as ob


_bound = False


def _lib():
    global _bound
    L = ob.lib()
    if not _bound:
        L.orc_moments.restype = ctypes.c_int
        L.orc_moments.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_uint64,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64)]
        _bound = True
    return L


def moments(L: int, J: float, Delta: float, h, pbc: bool, state: int, hops: int):
    """(mu[0 .. 2*hops], number of states within `hops` hops of `state`)."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    assert h.size == L
    mu = np.zeros(2 * hops + 1)
    nball = ctypes.c_int64(0)
    rc = _lib().orc_moments(L, float(J), float(Delta), h.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            int(pbc), ctypes.c_uint64(state), hops,
                            mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(nball))
    if rc != 0:
        raise RuntimeError(f"orc_moments failed ({rc})")
    return mu, int(nball.value)


def amplitude(mu, t: float):
    """(A(t) exp(+ict) from the series through mu_{2K-1}, bound on its error)."""
    n2 = mu.size - 1
    A = 0j
    for n in range(n2):
        A += (-1j * t) ** n * mu[n] / math.factorial(n)
    dA = t ** n2 * mu[n2] / math.factorial(n2)
    return A, dA


def return_probability(mu, t: float):
    """(P(t), rigorous bound on |P - P_exact|)."""
    A, dA = amplitude(mu, t)
    return abs(A) ** 2, (2.0 + dA) * dA
