"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test names the passage or the independent fact it checks.  A plausible slip in the
oracle (dropped Delta or field term, wrong hop sign or bond, transposed projection,
wrong Pade coefficient, wrong step acceptance) fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.linalg

from conftest import read_rows
from oracle import basis as ob
from oracle import dense, krylov, pade
import workloads


# ---------------------------------------------------------------- basis (Sec. 2, Alg. 2)

def test_worked_example_L4_N2():
    """Sec. 2 basis representation: L=4, N=2 -> 3, 5, 6, 9, 10, 12 in sorted order."""
    want = [int(x) for x in read_rows("basis_L4_N2.txt")[0]]
    assert ob.basis(4, 2).tolist() == want


def test_printed_dimensions():
    """D = L!/(N!(L-N)!) against the dimensions printed in Fig. 5, Sec. 5 and Table I."""
    for L, N, D, rel, *_ in read_rows("dimensions.txt"):
        L, N, D, rel = int(L), int(N), float(D), float(rel)
        got = ob.binom(L, N)
        assert got == math.comb(L, N)
        assert abs(got - D) <= rel * D + 0.5, (L, got, D)


def test_table1_basis_memory():
    for L, gb in read_rows("basis_memory_GB.txt"):
        got = 8 * ob.binom(int(L), int(L) // 2) / 1e9
        assert abs(got / float(gb) - 1.0) < 0.01


@pytest.mark.parametrize("L", range(1, 13))
def test_gosper_equals_bruteforce(L):
    """Algorithm 2 reproduces the sorted list of all L-bit integers with N set bits."""
    for N in range(0, L + 1):
        assert np.array_equal(ob.basis(L, N), dense.sector_states(L, N)), (L, N)


def test_gosper_bruteforce_L18():
    for N in (1, 5, 9, 17):
        assert np.array_equal(ob.basis(18, N), dense.sector_states(18, N))


def test_lookup():
    b = ob.basis(10, 4)
    for i in range(0, b.size, 7):
        assert ob.lookup(b, int(b[i])) == i
    assert ob.lookup(b, 0b111) == -1          # wrong particle number
    assert ob.lookup(b, 1 << 11 | 0b111) == -1  # outside the chain


# ---------------------------------------------------------------- Hamiltonian (Eq. 1)

@pytest.mark.parametrize("L,N,pbc", [(2, 1, False), (3, 1, True), (4, 2, True), (5, 2, True),
                                     (6, 3, False), (8, 4, True), (9, 4, True), (10, 5, True),
                                     (10, 3, False)])
def test_csr_equals_kronecker(L, N, pbc):
    """CSR from bit operations + binary lookup equals Eq. 1 built from Kronecker products."""
    rng = np.random.default_rng(L * 31 + N)
    J, Delta = 0.7 + rng.random(), rng.normal()
    h = rng.normal(size=L)
    H = ob.CSR(L, N, J, Delta, h, pbc)
    Hk = dense.hamiltonian_kron(L, J, Delta, h, pbc, N)
    assert np.allclose(H.dense(), Hk, atol=1e-14, rtol=0)


def test_csr_symmetric_and_row_structure():
    L, N = 12, 6
    h = workloads.quasiperiodic_field(L, 2.0, 0.3)
    H = ob.CSR(L, N, 1.0, 1.0, h, True)
    A = H.dense()
    assert np.array_equal(A, A.T)
    # off-diagonal row sums = (J/2) * number of antiparallel bonds (Eq. 1 hopping term)
    off = np.abs(A - np.diag(np.diag(A))).sum(axis=1)
    st = H.basis
    n_anti = np.zeros(st.size)
    for (i, j) in dense.bonds(L, True):
        n_anti += ((st >> np.uint64(i)) & np.uint64(1)) != ((st >> np.uint64(j)) & np.uint64(1))
    assert np.allclose(off, 0.5 * n_anti)


# ---------------------------------------------------------------- Pade exponential

@pytest.mark.parametrize("scale", [1e-3, 0.4, 3.0, 40.0])
def test_pade_matches_library_expm(scale):
    rng = np.random.default_rng(int(scale * 1000))
    A = scale * (rng.normal(size=(12, 12)) + 1j * rng.normal(size=(12, 12))) / 12
    assert np.allclose(pade.expm(A), scipy.linalg.expm(A), rtol=1e-12, atol=1e-13)


def test_pade_hermitian_eigen_formula():
    rng = np.random.default_rng(5)
    B = rng.normal(size=(20, 20))
    Hm = (B + B.T) / 2
    E, U = np.linalg.eigh(Hm)
    for t in (0.1, 2.0, 17.0):
        ref = U @ np.diag(np.exp(-1j * E * t)) @ U.T
        assert np.allclose(pade.expm(-1j * t * Hm), ref, atol=1e-12)


# ---------------------------------------------------------------- Krylov P(t)

def _krylov_P(L, N, J, Delta, h, pbc, state, times, m=30, tol=1e-12):
    H = ob.CSR(L, N, J, Delta, h, pbc)
    r0 = ob.lookup(H.basis, state)
    P, stats = krylov.return_probability(H, r0, times, m=m, tol=tol)
    return P, H, r0, stats


@pytest.mark.parametrize("L,pbc,hh", [(10, True, 2.0), (10, False, 1.0), (8, True, 0.0)])
def test_krylov_equals_dense_eigh(L, pbc, hh):
    """Krylov P(t) (Sec. 2) equals full diagonalisation to 1e-11 at 40 log-spaced t."""
    N = L // 2
    h = workloads.quasiperiodic_field(L, hh, 1.1)
    times = workloads.log_times(40, 0.1, 100.0)
    P, H, r0, _ = _krylov_P(L, N, 1.0, 1.0, h, pbc, workloads.neel_state(L), times)
    Pd = dense.return_probability_dense(dense.hamiltonian_kron(L, 1.0, 1.0, h, pbc, N),
                                        krylov.basis_vector(H.D, r0), times)
    assert np.max(np.abs(P - Pd)) < 1e-11


def test_krylov_small_m_and_tiny_sector():
    """m larger than D (Arnoldi breakdown) and a small m = 8 both reproduce eigh."""
    times = [0.0, 0.3, 1.0, 7.0, 30.0]
    h = [0.3, -0.2, 0.5, 0.1]
    P, H, r0, _ = _krylov_P(4, 2, 1.0, 0.5, h, True, 0b0101, times, m=30)
    Pd = dense.return_probability_dense(dense.hamiltonian_kron(4, 1.0, 0.5, h, True, 2),
                                        krylov.basis_vector(H.D, r0), times)
    assert np.max(np.abs(P - Pd)) < 1e-12
    L = 10
    hq = workloads.quasiperiodic_field(L, 1.0, 0.2)
    P4, H, r0, st = _krylov_P(L, 5, 1.0, 1.0, hq, True, workloads.neel_state(L), times, m=8,
                              tol=1e-10)
    Pd = dense.return_probability_dense(dense.hamiltonian_kron(L, 1.0, 1.0, hq, True, 5),
                                        krylov.basis_vector(H.D, r0), times)
    assert np.max(np.abs(P4 - Pd)) < 1e-10
    assert st["steps"] > 10


@pytest.mark.parametrize("pbc", [True, False])
def test_free_fermion_determinant(pbc):
    """Delta = 0 is free particles (Sec. 2): Krylov P equals the single-particle determinant."""
    L, N = 12, 6
    h = workloads.quasiperiodic_field(L, 1.5, 0.7)
    times = workloads.log_times(12, 0.1, 50.0)
    state = workloads.neel_state(L)
    P, *_ = _krylov_P(L, N, 1.0, 0.0, h, pbc, state, times)
    Pf = dense.free_fermion_P(L, 1.0, h, pbc, state, times)
    assert np.max(np.abs(P - Pf)) < 1e-11


def test_two_level_formula():
    h = [0.8, -0.3]
    times = np.linspace(0.0, 20.0, 15)
    P, *_ = _krylov_P(2, 1, 1.3, 0.4, h, False, 0b01, times)
    assert np.max(np.abs(P - dense.two_level_P(1.3, h, times))) < 1e-12


@pytest.mark.parametrize("N", [0, 8])
def test_empty_and_full_sector(N):
    times = [0.5, 5.0, 50.0]
    P, *_ = _krylov_P(8, N, 1.0, 1.0, workloads.quasiperiodic_field(8, 2.0, 0.0), True,
                      (1 << N) - 1, times)
    assert np.allclose(P, 1.0, atol=1e-14)


def test_short_time_expansion():
    """P(t) = 1 - Var(H) t^2 + O(t^4); for the Neel state on a ring Var = L J^2 / 4."""
    L = 12
    h = workloads.quasiperiodic_field(L, 2.0, 0.4)
    times = [1e-3, 2e-3, 4e-3]
    P, *_ = _krylov_P(L, 6, 1.0, 1.0, h, True, workloads.neel_state(L), times)
    for t, p in zip(times, P):
        assert abs((1 - p) / t**2 - L / 4.0) < 5 * t**2 * L**2


def test_symmetries_of_P():
    """P is unchanged by J -> -J (sublattice gauge on an even ring) and by H -> -H (P(t)=P(-t))."""
    L = 10
    h = np.array(workloads.quasiperiodic_field(L, 1.0, 0.9))
    times = workloads.log_times(8, 0.1, 30.0)
    st = workloads.neel_state(L)
    P1, *_ = _krylov_P(L, 5, 1.0, 0.7, h, True, st, times)
    P2, *_ = _krylov_P(L, 5, -1.0, -0.7, h, True, st, times)     # J -> -J at fixed J*Delta
    P3, *_ = _krylov_P(L, 5, -1.0, 0.7, -h, True, st, times)     # H -> -H
    assert np.max(np.abs(P1 - P2)) < 1e-11
    assert np.max(np.abs(P1 - P3)) < 1e-11


def test_norm_energy_and_unitarity():
    L, N = 12, 6
    h = workloads.quasiperiodic_field(L, 1.5, 2.0)
    H = ob.CSR(L, N, 1.0, 1.0, h, True)
    rng = np.random.default_rng(3)
    psi0 = rng.normal(size=H.D) + 1j * rng.normal(size=H.D)
    psi0 /= np.linalg.norm(psi0)
    E0 = np.vdot(psi0, H.matvec(psi0)).real
    _, psi, _ = krylov.evolve(H.matvec, H.norm_inf(), psi0, [7.5], m=30, tol=1e-12)
    assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
    assert abs(np.vdot(psi, H.matvec(psi)).real - E0) < 1e-11
    back, back_psi, _ = krylov.evolve(lambda x: -H.matvec(x), H.norm_inf(), psi, [7.5],
                                      m=30, tol=1e-12)
    assert np.linalg.norm(back_psi - psi0) < 1e-11


def test_arnoldi_is_orthonormal_and_tridiagonal():
    L, N = 12, 6
    H = ob.CSR(L, N, 1.0, 1.0, workloads.quasiperiodic_field(L, 1.5, 2.0), True)
    v = krylov.basis_vector(H.D, ob.lookup(H.basis, workloads.neel_state(L)))
    V, Hb, me = krylov.arnoldi_cgs2(H.matvec, v, 30, H.norm_inf())
    G = V[: me + 1].conj() @ V[: me + 1].T
    assert np.max(np.abs(G - np.eye(me + 1))) < 1e-13
    # Hermitian H: the Arnoldi Hessenberg matrix is tridiagonal (Lanczos) up to rounding
    T = Hb[:me, :me]
    assert np.max(np.abs(np.triu(T, 2))) < 1e-12
    assert np.max(np.abs(T - T.conj().T)) < 1e-12


@pytest.mark.parametrize("pbc", [True, False])
def test_single_particle_ring_L55(pbc):
    """N = 1 on L = 55 (the Fibonacci ring of Sec. 2 and Sec. 4): the oracle's sector matrix is
    the tight-binding chain written out by hand, hopping J/2 between neighbouring sites (and
    across the ring bond with PBC), diagonal h_i - sum(h)/2 + (J Delta/4)(n_bonds - 2 n_anti)
    with n_anti = 2 antiparallel bonds inside the chain (1 at an open end)."""
    import workloads
    L, J, Delta = 55, 1.3, 0.7
    h = np.asarray(workloads.aubry_andre_field(L, 2.0, J, 0.4))
    Hc = ob.CSR(L, 1, J, Delta, h, pbc).dense()
    nb = L if pbc else L - 1
    T = np.zeros((L, L))
    for i in range(L):
        nanti = 2 if (pbc or 0 < i < L - 1) else 1
        T[i, i] = h[i] - 0.5 * h.sum() + 0.25 * J * Delta * (nb - 2 * nanti)
    for i in range(L - 1):
        T[i, i + 1] = T[i + 1, i] = 0.5 * J
    if pbc:
        T[0, L - 1] = T[L - 1, 0] = 0.5 * J
    assert np.max(np.abs(Hc - T)) < 1e-12   # sums of 55 bond terms in another order
