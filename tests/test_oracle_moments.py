"""Pins of oracle.moments (early-time P from the moments of H) and of oracle.basis.row_apply
(single rows of H x), against dense references and closed forms (no GPU).

oracle.moments is the L = 30 oracle: it evaluates Eq. SP's amplitude as the power series of
the exponential, from the moments mu_n = <s0|(H - c)^n|s0>, which need only the states a
few hops from s0.  oracle.basis.row_apply is the row-sampled H.v oracle for sectors whose
CSR matrix does not fit in host memory (L = 30, and L > 32 on the sorted-list basis).
"""
import numpy as np
import pytest

from oracle import basis as ob
from oracle import dense, moments
import workloads


def _psi0(L, N, state):
    b = dense.sector_states(L, N)
    e = np.zeros(b.size)
    e[int(np.searchsorted(b, state))] = 1.0
    return e


def _n_anti(state, L, pbc):
    return sum(((state >> i) & 1) != ((state >> j) & 1) for i, j in dense.bonds(L, pbc))


# ---------------------------------------------------------------- moments

@pytest.mark.parametrize("L,N,pbc,hh,Delta,hops", [(10, 5, True, 1.5, 1.0, 8), (12, 6, False, 1.0, 0.5, 7),
                                                   (11, 5, True, 2.0, 1.3, 6), (12, 6, True, 0.0, 1.0, 9)])
def test_series_matches_eigh_within_its_bound(L, N, pbc, hh, Delta, hops):
    """P from the truncated series against dense eigh of the Kronecker-product H (Eq. 1):
    the difference never exceeds the series' rigorous bound, and where the bound is tiny the
    two agree to rounding."""
    h = workloads.quasiperiodic_field(L, hh, 0.7)
    state = workloads.neel_state(L) if L % 2 == 0 else workloads.neel_state(L - 1)
    mu, nball = moments.moments(L, 1.0, Delta, h, pbc, state, hops)
    Hd = dense.hamiltonian_kron(L, 1.0, Delta, h, pbc, N)
    times = [0.02, 0.1, 0.2, 0.3, 0.45]
    Pd = dense.return_probability_dense(Hd, _psi0(L, N, state), times)
    for t, pd in zip(times, Pd):
        P, bound = moments.return_probability(mu, t)
        assert abs(P - pd) <= bound + 2e-15, (t, P - pd, bound)
        if bound < 1e-13:
            assert abs(P - pd) <= 1e-13


def test_moments_equal_dense_matrix_powers_beyond_the_ball():
    """L = 14 (D = 3432): with 4 hops the ball holds a small part of the sector, yet every
    moment mu_0..mu_8 equals <s0|(H - c)^n|s0> from dense matrix powers."""
    L, N, hops = 14, 7, 4
    h = workloads.quasiperiodic_field(L, 1.5, 2.1)
    state = workloads.neel_state(L)
    mu, nball = moments.moments(L, 1.0, 1.0, h, True, state, hops)
    Hd = dense.hamiltonian_kron(L, 1.0, 1.0, h, True, N)
    e = _psi0(L, N, state)
    c = float(e @ Hd @ e)
    A = Hd - c * np.eye(Hd.shape[0])
    v = e.copy()
    assert nball < Hd.shape[0] // 2
    for n in range(2 * hops + 1):
        want = float(e @ v)
        assert abs(mu[n] - want) <= 1e-12 * max(1.0, abs(want)), (n, mu[n], want)
        v = A @ v


@pytest.mark.parametrize("L,pbc", [(8, True), (9, False), (30, True), (31, True), (16, False)])
def test_variance_closed_form(L, pbc):
    """mu_0 = 1, mu_1 = 0 (the shift is the diagonal element), and the energy variance
    mu_2 = (J/2)^2 n_anti(s0): each antiparallel bond couples s0 to one state by J/2."""
    J = 1.3
    state = workloads.neel_state(L)
    h = workloads.quasiperiodic_field(L, 1.2, 0.4)
    mu, nball = moments.moments(L, J, 0.8, h, pbc, state, 1)
    na = _n_anti(state, L, pbc)
    assert mu[0] == 1.0 and mu[1] == 0.0
    assert abs(mu[2] - 0.25 * J * J * na) <= 1e-14 * na
    assert nball == 1 + na
    if pbc and L % 2 == 0:
        assert na == L   # the Neel state on an even ring: every bond antiparallel


def _ball_bruteforce(L, pbc, state, hops):
    ball, front = {state}, {state}
    for _ in range(hops):
        nxt = set()
        for s in front:
            for i, j in dense.bonds(L, pbc):
                if ((s >> i) & 1) != ((s >> j) & 1):
                    nxt.add(s ^ ((1 << i) | (1 << j)))
        front = nxt - ball
        ball |= nxt
    return ball


@pytest.mark.parametrize("L,pbc,hops", [(12, True, 3), (30, True, 2), (17, False, 3)])
def test_ball_size_bruteforce(L, pbc, hops):
    state = workloads.neel_state(L)
    _, nball = moments.moments(L, 1.0, 1.0, [0.0] * L, pbc, state, hops)
    assert nball == len(_ball_bruteforce(L, pbc, state, hops))


def test_two_level_formula():
    J, h = 1.3, [0.8, -0.3]
    mu, _ = moments.moments(2, J, 0.4, h, False, 0b01, 12)
    for t in (0.1, 0.5, 1.0):
        P, bound = moments.return_probability(mu, t)
        assert abs(P - dense.two_level_P(J, h, [t])[0]) <= bound + 1e-15


def test_planted_moment_slips_are_caught():
    """Dropping the odd moments (the imaginary part of the series) or scaling the hop alone
    moves P by far more than the bound."""
    L, N = 10, 5
    h = workloads.quasiperiodic_field(L, 1.5, 0.3)
    state = workloads.neel_state(L)
    Hd = dense.hamiltonian_kron(L, 1.0, 1.0, h, True, N)
    t = 0.3
    Pd = dense.return_probability_dense(Hd, _psi0(L, N, state), [t])[0]
    mu, _ = moments.moments(L, 1.0, 1.0, h, True, state, 8)
    odd = mu.copy()
    odd[1::2] = 0.0
    P, bound = moments.return_probability(mu, t)
    assert abs(P - Pd) <= bound + 1e-15
    assert abs(moments.return_probability(odd, t)[0] - Pd) > 1e3 * bound
    # hop J/2 -> 1.05 J/2 with the Delta term kept at J Delta: J' = 1.05, Delta' = 1/1.05
    mu_hop, _ = moments.moments(L, 1.05, 1.0 / 1.05, h, True, state, 8)
    assert abs(moments.return_probability(mu_hop, t)[0] - Pd) > 1e3 * bound


# ---------------------------------------------------------------- row_apply

@pytest.mark.parametrize("L,N,pbc", [(10, 5, True), (11, 4, False), (12, 6, True), (13, 6, False),
                                     (14, 7, True), (14, 3, True), (6, 0, True), (6, 6, False)])
def test_row_apply_equals_csr_matvec(L, N, pbc):
    """row_apply (one row at a time, by bit operations and binary lookup) equals the CSR
    matrix-vector product on every row, for a random complex x."""
    h = workloads.quasiperiodic_field(L, 1.7, 0.9)
    H = ob.CSR(L, N, 1.0, 0.7, h, pbc)
    rng = np.random.default_rng(L * 100 + N)
    x = rng.normal(size=H.D) + 1j * rng.normal(size=H.D)
    rows = np.arange(H.D)
    got = ob.row_apply(L, 1.0, 0.7, h, pbc, H.basis, x, rows)
    want = H.matvec(x)
    assert np.max(np.abs(got - want)) <= 1e-13 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("L,pbc,Delta", [(8, True, 1.0), (9, False, 0.4), (10, True, 2.0)])
def test_row_apply_equals_kronecker_hamiltonian(L, pbc, Delta):
    """row_apply against H of Eq. 1 assembled from Kronecker products in the full 2^L space
    (oracle.dense), independent of the CSR construction; sampled rows, all N."""
    h = workloads.quasiperiodic_field(L, 1.1, 2.3)
    for N in range(L + 1):
        b = ob.basis(L, N)
        Hd = dense.hamiltonian_kron(L, 0.9, Delta, h, pbc, N)
        rng = np.random.default_rng(N)
        x = rng.normal(size=b.size) + 1j * rng.normal(size=b.size)
        rows = np.unique(rng.integers(0, b.size, size=min(b.size, 25)))
        got = ob.row_apply(L, 0.9, Delta, h, pbc, b, x, rows)
        assert np.max(np.abs(got - (Hd @ x)[rows])) <= 1e-13 * max(1.0, np.max(np.abs(got)))


def test_row_apply_planted_bond_slip_is_caught():
    """A row_apply that forgets the ring bond differs from the Kronecker H on a ring."""
    L, N = 8, 4
    h = workloads.quasiperiodic_field(L, 1.0, 0.2)
    b = ob.basis(L, N)
    x = np.random.default_rng(1).normal(size=b.size) + 0j
    rows = np.arange(b.size)
    Hd = dense.hamiltonian_kron(L, 1.0, 1.0, h, True, N)
    slip = ob.row_apply(L, 1.0, 1.0, h, False, b, x, rows)
    assert np.max(np.abs(slip - Hd @ x)) > 0.1
