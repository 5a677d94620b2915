"""Small dense matrix exponential by diagonal Pade approximation with scaling and squaring.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2 ("Krylov subspace methods") evaluates the small Krylov exponential with
irreducible Pade approximants.  The diagonal (q, q) approximant of e^X is
N_q(X) / N_q(-X) with N_q(X) = sum_k c_k X^k, c_k = (2q-k)! q! / ((2q)! k! (q-k)!);
it is irreducible.  Following Moler & Van Loan, "Nineteen dubious ways to compute the
exponential of a matrix, twenty-five years later" (SIAM Review 45, 2003, Sec. 3), the
argument is scaled by 2^-s until its infinity norm is <= 1/2, where q = 6 has a
relative backward error below 1e-15, and the result is squared s times.

Pinned by: scipy.linalg.expm on random complex matrices of several norms, and the
eigendecomposition formula for Hermitian arguments (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np


def pade_coefficients(q: int) -> list[float]:
    return [math.factorial(2 * q - k) * math.factorial(q)
            / (math.factorial(2 * q) * math.factorial(k) * math.factorial(q - k))
            for k in range(q + 1)]


def expm(A: np.ndarray, q: int = 6) -> np.ndarray:
    A = np.asarray(A, dtype=np.complex128)
    n = A.shape[0]
    nrm = np.max(np.sum(np.abs(A), axis=1)) if n else 0.0
    s = 0
    if nrm > 0.5:
        s = int(math.ceil(math.log2(nrm / 0.5)))
    X = A / (2.0 ** s)
    c = pade_coefficients(q)
    I = np.eye(n, dtype=np.complex128)
    Num = c[0] * I
    Den = c[0] * I
    P = I
    for k in range(1, q + 1):
        P = P @ X
        Num = Num + c[k] * P
        Den = Den + ((-1) ** k) * c[k] * P
    E = np.linalg.solve(Den, Num)
    for _ in range(s):
        E = E @ E
    return E
