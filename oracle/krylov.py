"""Krylov time evolution and the return probability, FP64 (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 2 ("Krylov subspace methods") and Eq. SP of Sec. 4:
  * Krylov space K_m = span{psi, H psi, ..., H^(m-1) psi}, built by Arnoldi.  The paper
    writes the projection as V^T H V; for complex vectors it is V^H H V.  Arnoldi
    orthogonalises every new vector against all previous ones; here by classical
    Gram-Schmidt applied twice (CGS2), so the basis is orthonormal to working precision.
  * psi(t + tau) ~ beta V_m exp(-i tau H_m) e_1, the small exponential by diagonal Pade
    (oracle.pade) applied to the augmented matrix
        [[-i tau H_m, 0], [-i tau h_{m+1,m} e_m^T, 0]]
    whose last first-column entry is the leading term of the Krylov error expansion
    (Saad, SIAM J. Numer. Anal. 29, 1992), used as the local error estimate as in the
    time-stepping scheme of Sidje, ACM TOMS 24 (1998) (the paper's "expokit").
  * Steps are accepted when  err <= tol/2 * tau / t_end  (tol read as the absolute error
    budget of P over the whole run, since |dP| <= 2 ||d psi||) and shrunk otherwise by
    0.9 (tol_loc/err)^(1/m); every step is truncated at the next output time, where
    P(t_k) = |<psi0|psi(t_k)>|^2 is read.
  * An Arnoldi breakdown (h_{j+1,j} <= 1e-13 ||H||) stops the basis early; the error
    estimate still uses that tiny h, so nothing is assumed exact.

Pinned by: dense eigendecomposition for L <= 10, the free-fermion determinant at
Delta = 0, the two-level formula at L = 2, P = 1 for N = 0 or N = L, the short-time
expansion P = 1 - Var(H) t^2, conservation of norm and energy, and forward-then-backward
unitarity (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math

import numpy as np

from . import pade


def arnoldi_cgs2(matvec, v1: np.ndarray, m: int, anorm: float):
    """Arnoldi with full reorthogonalisation by CGS2.

    Returns (V, Hbar, m_eff): V has m_eff (+1 when no breakdown) orthonormal rows,
    Hbar is the (m_eff+1) x m_eff Hessenberg matrix with H V_m = V_{m+1} Hbar.
    """
    D = v1.size
    V = np.zeros((m + 1, D), dtype=np.complex128)
    Hb = np.zeros((m + 1, m), dtype=np.complex128)
    V[0] = v1
    for j in range(m):
        w = matvec(V[j])
        for _ in range(2):
            c = V[: j + 1].conj() @ w
            w = w - c @ V[: j + 1]
            Hb[: j + 1, j] += c
        b = float(np.linalg.norm(w))
        Hb[j + 1, j] = b
        if b <= 1e-13 * anorm or j + 1 == m:
            if b > 1e-13 * anorm:
                V[j + 1] = w / b
            return V[: j + 2], Hb[: j + 2, : j + 1], j + 1
        V[j + 1] = w / b
    raise AssertionError("unreachable")


def first_step(anorm: float, m: int, tol: float, t_end: float) -> float:
    """First step size from the a-priori behaviour (tau ||H|| / m)^m of the Krylov error
    quoted in Sec. 2; only a starting guess, the error control adapts it."""
    if anorm <= 0.0:
        return t_end
    return min(t_end, (m / math.e) * (0.01 * tol) ** (1.0 / m) / anorm)


def evolve(matvec, anorm: float, psi0: np.ndarray, times, m: int = 30, tol: float = 1e-12,
           max_reject: int = 200):
    """Evolve psi0 under exp(-iHt) and return (P[times], psi(t_last), stats)."""
    times = np.asarray(times, dtype=np.float64)
    if np.any(times < 0) or np.any(np.diff(times) < 0):
        raise ValueError("times must be non-negative and non-decreasing")
    psi0 = np.asarray(psi0, dtype=np.complex128)
    psi = psi0.copy()
    P = np.zeros(times.size)
    stats = dict(steps=0, rejects=0, hv=0, err_sum=0.0)
    t_end = float(times[-1]) if times.size else 0.0
    t = 0.0
    tau = first_step(anorm, m, tol, t_end) if t_end > 0 else 0.0
    for k, tk in enumerate(times):
        while tk - t > 1e-14 * max(1.0, t_end):
            beta = float(np.linalg.norm(psi))
            V, Hb, me = arnoldi_cgs2(matvec, psi / beta, m, anorm)
            stats["hv"] += me
            while True:
                step = min(tau, tk - t)
                A = np.zeros((me + 1, me + 1), dtype=np.complex128)
                A[:me, :me] = -1j * step * Hb[:me, :me]
                A[me, me - 1] = -1j * step * Hb[me, me - 1]
                E = pade.expm(A)
                err = beta * abs(E[me, 0])
                tol_loc = 0.5 * tol * step / t_end
                if err <= tol_loc:
                    break
                stats["rejects"] += 1
                if stats["rejects"] > max_reject:
                    raise RuntimeError("tolerance not reachable")
                tau = 0.9 * step * (tol_loc / err) ** (1.0 / me)
            psi = beta * (E[:me, 0] @ V[:me])
            t += step
            stats["steps"] += 1
            stats["err_sum"] += err
            if step >= tau:   # not truncated by an output time: adapt the step size
                grow = 0.9 * (tol_loc / max(err, 1e-300)) ** (1.0 / me)
                tau = step * min(5.0, max(0.2, grow))
        P[k] = abs(np.vdot(psi0, psi)) ** 2
    return P, psi, stats


def basis_vector(D: int, r: int) -> np.ndarray:
    e = np.zeros(D, dtype=np.complex128)
    e[r] = 1.0
    return e


def return_probability(H, state_index: int, times, m: int = 30, tol: float = 1e-12):
    """P(t) for psi0 = e_{state_index} under the CSR Hamiltonian H (oracle.basis.CSR)."""
    psi0 = basis_vector(H.D, state_index)
    P, _, stats = evolve(H.matvec, H.norm_inf(), psi0, times, m=m, tol=tol)
    return P, stats
