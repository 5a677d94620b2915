"""Gradient of the return probability with respect to h_i and Delta (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper computes P(t) only;
its derivative is defined here from P(t) = |<psi0|exp(-iHt)|psi0>|^2 (Eq. SP) with
H(theta) of Eq. 1 (XXZ form), dH/dh_i = Sz_i and dH/dDelta = J sum_b Sz_i Sz_j.

  * daleckii_krein: with H = U diag(E) U^H and c = U^H psi0,
        dA/dtheta = sum_ab conj(c_a) (U^H dH U)_ab c_b f_ab,
        f_ab = -i t exp(-i t (E_a + E_b)/2) sinc(t (E_a - E_b)/2),
    the divided difference of exp(-i t x) written so that it stays exact at E_a = E_b
    (Daleckii-Krein formula for the Frechet derivative of a matrix function); then
    dP/dtheta = 2 Re(conj(A) dA/dtheta).
  * central_fd: (P(theta + eps) - P(theta - eps)) / (2 eps) with any P evaluator.

Pinned by: sum_i dP/dh_i = 0 (Sz_total is conserved in the sector), the small-t law
dP/dtheta = O(t^4), and agreement of the two independent formulas above
(tests/test_oracle_gradient.py).
"""
from __future__ import annotations

import numpy as np

from . import dense


def sz_diag(L: int, N: int, i: int) -> np.ndarray:
    st = dense.sector_states(L, N)
    return np.where((st >> np.uint64(i)) & np.uint64(1), 0.5, -0.5)


def zz_diag(L: int, N: int, J: float, pbc: bool) -> np.ndarray:
    st = dense.sector_states(L, N)
    out = np.zeros(st.size)
    for (i, j) in dense.bonds(L, pbc):
        zi = np.where((st >> np.uint64(i)) & np.uint64(1), 0.5, -0.5)
        zj = np.where((st >> np.uint64(j)) & np.uint64(1), 0.5, -0.5)
        out += J * zi * zj
    return out


def daleckii_krein(H: np.ndarray, dH_list, psi0: np.ndarray, t: float):
    """Return (P, [dP/dtheta for each dH in dH_list]); dH given as dense or diagonal arrays."""
    E, U = np.linalg.eigh(H)
    c = U.conj().T @ psi0
    A = np.sum(np.abs(c) ** 2 * np.exp(-1j * E * t))
    Ea, Eb = np.meshgrid(E, E, indexing="ij")
    x = t * (Ea - Eb) / 2.0
    f = -1j * t * np.exp(-1j * t * (Ea + Eb) / 2.0) * np.sinc(x / np.pi)
    out = []
    for dH in dH_list:
        dH = np.diag(dH) if dH.ndim == 1 else dH
        M = U.conj().T @ dH @ U
        dA = np.sum(np.conj(c)[:, None] * M * c[None, :] * f)
        out.append(2.0 * np.real(np.conj(A) * dA))
    return float(abs(A) ** 2), out


def central_fd(P_of_theta, theta: float, eps: float = 1e-5) -> float:
    return (P_of_theta(theta + eps) - P_of_theta(theta - eps)) / (2.0 * eps)
