"""Planted mistakes in the oracle (on the CPU) are caught by its pins.

Each test perturbs one oracle ingredient the way a plausible slip would, and checks
that the corresponding independent reference disagrees.  This shows the pins are
sharp enough to fail when the oracle is wrong.
"""
import numpy as np
import scipy.linalg

from oracle import basis as ob
from oracle import dense, krylov, pade
import workloads


def _P_vs_dense(matvec_factory, L=10, pbc=True):
    N = L // 2
    h = workloads.quasiperiodic_field(L, 2.0, 1.1)
    H = ob.CSR(L, N, 1.0, 1.0, h, pbc)
    r0 = ob.lookup(H.basis, workloads.neel_state(L))
    times = workloads.log_times(10, 0.1, 30.0)
    psi0 = krylov.basis_vector(H.D, r0)
    P, _, _ = krylov.evolve(matvec_factory(H), H.norm_inf(), psi0, times, m=30, tol=1e-12)
    Pd = dense.return_probability_dense(dense.hamiltonian_kron(L, 1.0, 1.0, h, pbc, N),
                                        psi0, times)
    return np.max(np.abs(P - Pd))


def test_dropped_field_term_is_caught():
    L = 8
    h = np.array(workloads.quasiperiodic_field(L, 2.0, 0.3))
    good = ob.CSR(L, 4, 1.0, 1.0, h, True).dense()
    bad = ob.CSR(L, 4, 1.0, 1.0, 0 * h, True).dense()
    ref = dense.hamiltonian_kron(L, 1.0, 1.0, h, True, 4)
    assert np.allclose(good, ref) and not np.allclose(bad, ref)


def test_missing_ring_bond_is_caught():
    L = 8
    h = np.array(workloads.quasiperiodic_field(L, 2.0, 0.3))
    bad = ob.CSR(L, 4, 1.0, 1.0, h, False).dense()
    assert not np.allclose(bad, dense.hamiltonian_kron(L, 1.0, 1.0, h, True, 4))


def test_wrong_pade_coefficient_is_caught(monkeypatch):
    orig = pade.pade_coefficients
    monkeypatch.setattr(pade, "pade_coefficients",
                        lambda q: [c * (1.0 + (1e-3 if k == 3 else 0.0))
                                   for k, c in enumerate(orig(q))])
    A = 0.4 * np.random.default_rng(0).normal(size=(8, 8))
    assert not np.allclose(pade.expm(A), scipy.linalg.expm(A), rtol=1e-10, atol=1e-12)


def test_transposed_projection_is_caught():
    """V^T w instead of V^H w (the garbled 'V^T H V' read literally) loses orthonormality.

    The recurrence H V = V Hbar still holds for the planted variant, so P(t) stays
    right; the orthonormality pin of the Arnoldi basis is what catches it.
    """
    L, N = 10, 5
    H = ob.CSR(L, N, 1.0, 1.0, workloads.quasiperiodic_field(L, 1.5, 2.0), True)
    rng = np.random.default_rng(1)
    psi0 = rng.normal(size=H.D) + 1j * rng.normal(size=H.D)
    psi0 /= np.linalg.norm(psi0)
    m = 12
    V = np.zeros((m + 1, H.D), complex)
    V[0] = psi0
    for j in range(m):
        w = H.matvec(V[j])
        for _ in range(2):
            c = V[: j + 1] @ w               # planted: missing conjugate
            w = w - c @ V[: j + 1]
        V[j + 1] = w / np.linalg.norm(w)
    G = V.conj() @ V.T
    assert np.max(np.abs(G - np.eye(m + 1))) > 1e-3
    Vg, _, me = krylov.arnoldi_cgs2(H.matvec, psi0, m, H.norm_inf())
    Gg = Vg[: me + 1].conj() @ Vg[: me + 1].T
    assert np.max(np.abs(Gg - np.eye(me + 1))) < 1e-13


def test_wrong_hop_amplitude_is_caught():
    """The hop J/2 scaled by 1.05 alone; the diagonal of Eq. 1 (bond and field terms) kept."""
    def factory(H):
        rows = np.repeat(np.arange(H.D), np.diff(H.rowptr))
        on = H.col == rows
        diag = np.zeros(H.D)
        diag[rows[on]] = H.val[on]
        return lambda x: H.matvec(x) + 0.05 * (H.matvec(x) - diag * x)
    err = _P_vs_dense(factory)
    assert err > 1e-6


# ---- temporal autocorrelation and its exponent (Sec. 4)

def _two_level_C_want(J, h, times):
    d = h[0] - h[1]
    W = np.sqrt(J * J + d * d)
    A = J * J / (W * W)
    return 1.0 - A / 2.0 + (A / 2.0) * np.sin(W * times) / (W * times)


def _C_variant(H, psi0, times, slip):
    """The oracle's spectral form of C(t) with one planted slip."""
    E, U = np.linalg.eigh(H)
    w = np.abs(U.conj().T @ psi0) ** 2
    om = E[:, None] - E[None, :]
    ww = w[:, None] * w[None, :]
    out = []
    for t in times:
        if slip == "no_average":        # P(t) instead of its time average
            out.append(float((ww * np.cos(om * t)).sum()))
        elif slip == "no_division":     # the integral without the 1/t
            out.append(float((ww * t * np.sinc(om * t / np.pi)).sum()))
        elif slip == "half_frequency":  # sin(om t / 2) / (om t / 2)
            out.append(float((ww * np.sinc(om * t / (2 * np.pi))).sum()))
    return np.array(out)


def test_planted_autocorrelation_slips_are_caught():
    J, h = 1.3, [0.8, -0.3]
    H = dense.hamiltonian_kron(2, J, 0.4, h, False, 1)
    psi0 = np.array([1.0, 0.0])   # either site: P is the same for both
    times = np.array([0.3, 1.7, 5.0, 23.0])
    want = _two_level_C_want(J, h, times)
    assert np.max(np.abs(dense.autocorrelation_dense(H, psi0, times) - want)) < 1e-13
    for slip in ("no_average", "no_division", "half_frequency"):
        assert np.max(np.abs(_C_variant(H, psi0, times, slip) - want)) > 1e-3, slip


def test_planted_exponent_slips_are_caught():
    from oracle import analysis
    t = np.logspace(0, 3, 30)
    C = 0.5 * t ** -0.83
    assert abs(analysis.decay_exponent(t, C, 1.0, 1e3)[0] - 0.83) < 1e-12
    slope = np.polyfit(np.log(t), np.log(C), 1)[0]
    assert abs(slope - 0.83) > 1.0                     # the sign slip (gamma = +slope)
    mixed = np.polyfit(np.log10(t), np.log(C), 1)[0]
    assert abs(-mixed - 0.83) > 0.5                    # log10 t against ln C
