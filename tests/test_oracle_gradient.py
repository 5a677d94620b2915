"""Pins of the oracle gradient dP(t)/dh_i, dP/dDelta (no GPU)."""
import numpy as np

from oracle import basis as ob
from oracle import dense, gradient, krylov
import workloads


def _setup(L=10, hh=1.0, Delta=1.0, phi=0.4):
    N = L // 2
    h = np.array(workloads.quasiperiodic_field(L, hh, phi))
    st = workloads.neel_state(L)
    b = dense.sector_states(L, N)
    r0 = int(np.searchsorted(b, st))
    psi0 = np.zeros(b.size, complex)
    psi0[r0] = 1.0
    return L, N, h, Delta, psi0


def _dk(L, N, h, Delta, psi0, t):
    H = dense.hamiltonian_kron(L, 1.0, Delta, h, True, N)
    dHs = [gradient.sz_diag(L, N, i) for i in range(L)] + [gradient.zz_diag(L, N, 1.0, True)]
    return gradient.daleckii_krein(H, dHs, psi0, t)


def test_dk_matches_dense_finite_differences():
    L, N, h, Delta, psi0 = _setup()
    t = 3.0
    P, g = _dk(L, N, h, Delta, psi0, t)

    def P_of_hi(i):
        def f(x):
            hh = h.copy()
            hh[i] = x
            return dense.return_probability_dense(
                dense.hamiltonian_kron(L, 1.0, Delta, hh, True, N), psi0, [t])[0]
        return f

    for i in (0, 3, 7):
        fd = gradient.central_fd(P_of_hi(i), h[i], 1e-5)
        assert abs(fd - g[i]) < 1e-8
    fdD = gradient.central_fd(lambda d: dense.return_probability_dense(
        dense.hamiltonian_kron(L, 1.0, d, h, True, N), psi0, [t])[0], Delta, 1e-5)
    assert abs(fdD - g[L]) < 1e-8


def test_field_gradient_sums_to_zero():
    """sum_i Sz_i is conserved in the sector, so sum_i dP/dh_i = 0."""
    L, N, h, Delta, psi0 = _setup(L=8, hh=2.0)
    for t in (0.7, 10.0):
        _, g = _dk(L, N, h, Delta, psi0, t)
        assert abs(sum(g[:L])) < 1e-11


def test_gradient_small_t_is_fourth_order():
    """P = 1 - Var t^2 + O(t^4) and Var does not depend on h or Delta for a product state."""
    L, N, h, Delta, psi0 = _setup(L=8)
    _, g1 = _dk(L, N, h, Delta, psi0, 1e-2)
    _, g2 = _dk(L, N, h, Delta, psi0, 2e-2)
    for a, b in zip(g1, g2):
        if abs(b) > 1e-14:
            assert 12.0 < b / a < 20.0     # ratio 2^4 = 16 for an O(t^4) quantity


def test_dk_matches_krylov_finite_differences():
    """Two independent evaluators: dense DK gradient vs central FD of the Krylov oracle."""
    L, N, h, Delta, psi0 = _setup(L=10, hh=1.0)
    t = 10.0
    _, g = _dk(L, N, h, Delta, psi0, t)
    st = workloads.neel_state(L)

    def P_kry(hv, d):
        H = ob.CSR(L, N, 1.0, d, hv, True)
        P, _ = krylov.return_probability(H, ob.lookup(H.basis, st), [t], m=30, tol=1e-13)
        return P[0]

    i = 4
    fd = gradient.central_fd(lambda x: P_kry(np.where(np.arange(L) == i, x, h), Delta), h[i], 1e-5)
    assert abs(fd - g[i]) < 1e-7
    fdD = gradient.central_fd(lambda d: P_kry(h, d), Delta, 1e-5)
    assert abs(fdD - g[L]) < 1e-7
