"""Dense references for small sectors (oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).

These are independent of the CSR construction in oracle.basis:
  * sector_states: brute-force list of all L-bit integers with N set bits, in order.
  * hamiltonian_kron: Eq. 1 in its XXZ form assembled in the full 2^L space from
    Kronecker products of single-site operators (Sz = diag(-1/2, 1/2), S+ = |1><0|,
    bit i <-> site i+1), then restricted to the sector rows and columns.
  * return_probability_dense: P(t) = |sum_a |<a|psi0>|^2 exp(-i E_a t)|^2 from a full
    eigendecomposition (Eq. SP of Sec. 4).
  * free_fermion_P: the Delta = 0 limit of Eq. 1 ("V = 0 corresponding to the case of
    free particles", Sec. 2).  By the Jordan-Wigner map the sector is N free fermions
    with single-particle matrix h1 (hopping J/2, on-site h_i); on a ring the wrap hop
    picks up the sign (-1)^(N-1).  For a product initial state the return amplitude is
    det[(exp(-i h1 t))_{occ, occ}].
  * two_level_P: L = 2, N = 1 is a two-level system with coupling J/2 and detuning
    h_1 - h_2: P = 1 - J^2/(J^2+d^2) sin^2(sqrt(J^2+d^2) t / 2).
  * autocorrelation_dense: the temporal autocorrelation function of Sec. 4,
    C(t) = (1/t) int_0^t P(t') dt', from the same eigendecomposition.  With
    p_a = |<a|psi0>|^2, P(t') = sum_{a,b} p_a p_b cos((E_a - E_b) t'), so
    int_0^t P = sum_{a,b} p_a p_b sin((E_a - E_b) t) / (E_a - E_b)   (= t when E_a = E_b).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def sector_states(L: int, N: int) -> np.ndarray:
    s = np.arange(1 << L, dtype=np.uint64)
    pc = np.zeros(s.size, dtype=np.int64)
    for b in range(L):
        pc += ((s >> np.uint64(b)) & np.uint64(1)).astype(np.int64)
    return s[pc == N]


def bonds(L: int, pbc: bool):
    bl = [(i, i + 1) for i in range(L - 1)]
    if pbc and L >= 3:
        bl.append((L - 1, 0))
    return bl


def _site_op(op, i, L):
    return sp.kron(sp.kron(sp.identity(1 << (L - 1 - i), format="csr"), sp.csr_matrix(op)),
                   sp.identity(1 << i, format="csr"), format="csr")


def hamiltonian_kron(L: int, J: float, Delta: float, h, pbc: bool = True, N: int | None = None):
    """Sector (or full, N=None) Hamiltonian as a dense real array."""
    Sz = np.array([[-0.5, 0.0], [0.0, 0.5]])
    Sp = np.array([[0.0, 0.0], [1.0, 0.0]])
    Sm = Sp.T
    dim = 1 << L
    H = sp.csr_matrix((dim, dim))
    for (i, j) in bonds(L, pbc):
        H = H + J * 0.5 * (_site_op(Sp, i, L) @ _site_op(Sm, j, L)
                           + _site_op(Sm, i, L) @ _site_op(Sp, j, L))
        H = H + J * Delta * (_site_op(Sz, i, L) @ _site_op(Sz, j, L))
    for i in range(L):
        H = H + h[i] * _site_op(Sz, i, L)
    H = H.toarray()
    if N is None:
        return H
    st = sector_states(L, N).astype(np.int64)
    return H[np.ix_(st, st)]


def return_probability_dense(H: np.ndarray, psi0: np.ndarray, times) -> np.ndarray:
    E, U = np.linalg.eigh(H)
    c = U.conj().T @ psi0
    w = np.abs(c) ** 2
    t = np.asarray(times, dtype=np.float64)
    A = (w[None, :] * np.exp(-1j * np.outer(t, E))).sum(axis=1)
    return np.abs(A) ** 2


def autocorrelation_dense(H: np.ndarray, psi0: np.ndarray, times) -> np.ndarray:
    """C(t) = (1/t) int_0^t P(t') dt' (Sec. 4, temporal autocorrelation), exactly from the
    eigendecomposition; C(0) = 1.  O(D^2) memory per time: meant for small sectors."""
    E, U = np.linalg.eigh(H)
    w = np.abs(U.conj().T @ psi0) ** 2
    om = E[:, None] - E[None, :]
    ww = w[:, None] * w[None, :]
    out = []
    for t in np.asarray(times, dtype=np.float64):
        if t == 0.0:
            out.append(1.0)
            continue
        # sin(om t)/om, with its limit t where om = 0 (np.sinc(x) = sin(pi x)/(pi x))
        s = t * np.sinc(om * t / np.pi)
        out.append(float((ww * s).sum()) / t)
    return np.array(out)


def evolve_dense(H: np.ndarray, psi0: np.ndarray, t: float) -> np.ndarray:
    E, U = np.linalg.eigh(H)
    return U @ (np.exp(-1j * E * t) * (U.conj().T @ psi0))


def free_fermion_P(L: int, J: float, h, pbc: bool, state: int, times) -> np.ndarray:
    occ = [i for i in range(L) if (state >> i) & 1]
    N = len(occ)
    h1 = np.diag(np.asarray(h, dtype=np.float64))
    for i in range(L - 1):
        h1[i, i + 1] = h1[i + 1, i] = 0.5 * J
    if pbc and L >= 3:
        sgn = (-1.0) ** (N - 1)
        h1[L - 1, 0] = h1[0, L - 1] = sgn * 0.5 * J
    E, U = np.linalg.eigh(h1)
    out = []
    for t in np.asarray(times, dtype=np.float64):
        G = U @ np.diag(np.exp(-1j * E * t)) @ U.conj().T
        out.append(abs(np.linalg.det(G[np.ix_(occ, occ)])) ** 2)
    return np.array(out)


def two_level_P(J: float, h, times) -> np.ndarray:
    d = h[0] - h[1]
    W = np.sqrt(J * J + d * d)
    t = np.asarray(times, dtype=np.float64)
    return 1.0 - (J * J / (W * W)) * np.sin(W * t / 2.0) ** 2
