"""GPU temporal autocorrelation C(t) = (1/t) int_0^t P (Sec. 4) against the oracle.

The oracle is the exact spectral form of the integral (eigendecomposition of the dense
sector Hamiltonian, pinned on the CPU).  C is an average of P, so its error is bounded by
P's error plus the per-step quadrature error: the bars are P's own, complex128 1e-10 and
complex64 (mixed precision) 1e-5.  At the full L=24 size, where no dense oracle exists, C is
checked against a fine composite Simpson rule of P computed by the same call, against the
bounds 0 <= tC(t) nondecreasing, and P is checked to be the return-probability call's P.
"""
import numpy as np
import pytest

from oracle import dense
import workloads

pytestmark = pytest.mark.gpu


def _dense_C(L, N, J, Delta, h, pbc, state, times):
    b = dense.sector_states(L, N)
    psi0 = np.zeros(b.size, complex)
    psi0[int(np.searchsorted(b, state))] = 1.0
    Hd = dense.hamiltonian_kron(L, J, Delta, h, pbc, N)
    return dense.autocorrelation_dense(Hd, psi0, times), dense.return_probability_dense(Hd, psi0, times)


@pytest.mark.parametrize("L,pbc,hh,Delta,dtype,tol,bar", [
    (12, True, 1.0, 1.0, "c128", 1e-10, 1e-10),
    (14, True, 2.0, 1.0, "c128", 1e-10, 1e-10),
    (13, False, 0.5, 0.3, "c128", 1e-10, 1e-10),
    (14, True, 2.0, 1.0, "c64", 1e-7, 1e-5),
])
def test_autocorrelation_vs_spectral(kry, L, pbc, hh, Delta, dtype, tol, bar):
    N = L // 2
    h = workloads.quasiperiodic_field(L, hh, 0.4)
    st = workloads.neel_state(L) if L % 2 == 0 else workloads.neel_state(L - 1)
    times = [0.0] + list(workloads.log_times(40, 0.1, 100.0))
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, Delta, h, pbc=pbc)
    C, P, stats = H.autocorrelation(st, times, tol=tol, dtype=dtype)
    Cd, Pd = _dense_C(L, N, 1.0, Delta, h, pbc, st, times)
    err = float(np.max(np.abs(C - Cd)))
    print(f"[parity] C(t) L{L} {dtype}: max|dC| = {err:.3e}, max|dP| = {np.max(np.abs(P - Pd)):.3e}")
    assert C[0] == 1.0
    assert err <= bar
    assert np.max(np.abs(P - Pd)) <= bar
    assert stats["n_krylov_steps"] > 0


def test_P_is_the_return_probability(kry):
    """Computing C adds work to the small exponential only: P is bit-identical."""
    L = 14
    h = workloads.quasiperiodic_field(L, 1.5, 0.4)
    st = workloads.neel_state(L)
    times = workloads.log_times(30, 0.1, 50.0)
    H = kry.Hamiltonian(kry.Basis(L, L // 2), 1.0, 1.0, h)
    for dtype in ("c128", "c64"):
        C, P, _ = H.autocorrelation(st, times, dtype=dtype, tol=1e-10 if dtype == "c128" else 1e-7)
        P2, _ = H.return_probability(st, times, dtype=dtype, tol=1e-10 if dtype == "c128" else 1e-7)
        assert np.array_equal(P, P2)
        C3, P3, _ = H.autocorrelation(st, times, dtype=dtype, tol=1e-10 if dtype == "c128" else 1e-7)
        assert np.array_equal(C, C3) and np.array_equal(P, P3)   # deterministic


def test_repeated_and_zero_times(kry):
    L = 12
    h = workloads.quasiperiodic_field(L, 1.0, 0.4)
    st = workloads.neel_state(L)
    times = [0.0, 0.0, 0.5, 0.5, 0.5, 3.0, 3.0]
    H = kry.Hamiltonian(kry.Basis(L, L // 2), 1.0, 1.0, h)
    C, _, _ = H.autocorrelation(st, times)
    Cd, _ = _dense_C(L, L // 2, 1.0, 1.0, h, True, st, times)
    assert C[0] == 1.0 and C[1] == 1.0
    assert C[2] == C[3] == C[4] and C[5] == C[6]
    assert np.max(np.abs(C - Cd)) <= 1e-10


def test_rejects_bad_arguments(kry):
    L = 10
    B = kry.Basis(L, 5)
    h = workloads.quasiperiodic_field(L, 1.0, 0.4)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    with pytest.raises(kry.KryError):
        H.autocorrelation(0b111, [1.0])
    with pytest.raises(kry.KryError):
        H.autocorrelation(workloads.neel_state(L), [2.0, 1.0])
    HK = kry.Hamiltonian(B, 1.0, 1.0, [h, h, h])
    good = workloads.random_basis_states(L, 5, 7, 3)
    with pytest.raises(ValueError):
        HK.return_probability_states(good[:2], [1.0])
    with pytest.raises(kry.KryError) as e:
        HK.return_probability_states([good[0], 0b1111, good[2]], [1.0])
    assert e.value.code == kry.KRY_EINVAL and "realisation 1" in str(e.value)


def _ensemble_case(L, K, seed):
    N = L // 2
    hs = [workloads.quasiperiodic_field(L, 1.5, p) for p in workloads.phases(seed, K)]
    states = workloads.random_basis_states(L, N, seed + 100, K)
    return N, hs, states


@pytest.mark.parametrize("dtype,tol,bar", [("c128", 1e-10, 1e-10), ("c64", 1e-7, 1e-5)])
def test_random_state_ensemble_vs_spectral(kry, dtype, tol, bar):
    """K = 6 realisations, each with its own phase and its own random basis state (batched
    path): P and C of every realisation against the dense spectral oracle."""
    L, K = 12, 6
    N, hs, states = _ensemble_case(L, K, 21)
    times = [0.0] + list(workloads.log_times(30, 0.1, 100.0))
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs)
    P, C, _ = H.return_probability_states(states, times, tol=tol, dtype=dtype, autocorrelation=True)
    P2, _ = H.return_probability_states(states, times, tol=tol, dtype=dtype)
    assert np.array_equal(P, P2)   # computing C changes nothing in P
    worst_c = worst_p = 0.0
    for k in range(K):
        Cd, Pd = _dense_C(L, N, 1.0, 1.0, hs[k], True, states[k], times)
        worst_c = max(worst_c, float(np.max(np.abs(C[:, k] - Cd))))
        worst_p = max(worst_p, float(np.max(np.abs(P[:, k] - Pd))))
    print(f"[parity] ensemble L{L} K{K} {dtype}: max|dC| = {worst_c:.3e}, max|dP| = {worst_p:.3e}")
    assert np.all(C[0] == 1.0) and np.all(P[0] == 1.0)
    assert worst_c <= bar and worst_p <= bar


def test_batched_autocorrelation_common_state(kry):
    L, K = 14, 4
    N, hs, _ = _ensemble_case(L, K, 22)
    st = workloads.neel_state(L)
    times = workloads.log_times(20, 0.1, 50.0)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs)
    C, P, _ = H.autocorrelation(st, times)
    assert C.shape == (len(times), K)
    for k in range(K):
        Cd, _ = _dense_C(L, N, 1.0, 1.0, hs[k], True, st, times)
        assert np.max(np.abs(C[:, k] - Cd)) <= 1e-10
    Pr, _ = H.return_probability(st, times)
    assert np.array_equal(P, Pr)


def test_ensemble_full_size_L22(kry):
    """L=22 (D = 705,432), K = 16 random basis states: per-realisation C against Simpson of the
    call's own P on a grid of step 1/200 to t = 1, and 0 <= C <= 1, C(0) = 1."""
    L, K = 22, 16
    N, hs, states = _ensemble_case(L, K, 23)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs)
    grid = np.linspace(0.0, 1.0, 201)
    P, C, st = H.return_probability_states(states, grid, tol=1e-10, autocorrelation=True)
    hstep = grid[1] - grid[0]
    w = np.ones(201)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    simpson = hstep / 3.0 * (w @ P)
    err = float(np.max(np.abs(C[-1] - simpson)))
    print(f"[parity] ensemble L22 K16: max|C(1) - Simpson| = {err:.3e}")
    assert err <= 2e-7
    assert np.all(C[0] == 1.0) and np.all((C >= -1e-12) & (C <= 1.0 + 1e-12))
    assert st["n_krylov_steps"] > 0


@pytest.mark.parametrize("dtype,bar", [("c128", 2e-7), ("c64", 2e-5)])
def test_full_size_L24_against_simpson(kry, dtype, bar):
    """L=24 (D = 2,704,156): t C(t) against composite Simpson of the call's own P on a grid
    of step 1/200 up to t = 2 (Simpson error h^4/180 * t * max|P''''| stays below 1e-7 for the
    energy scale of this chain), and tC nondecreasing with 0 <= C <= 1 on a log grid."""
    c = workloads.config("L24_mixed")
    H = kry.Hamiltonian(kry.Basis(c["L"], c["n_up"]), c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
    tol = c["tol"] if dtype == "c128" else 1e-7
    grid = np.linspace(0.0, 2.0, 401)
    C, P, _ = H.autocorrelation(c["state"], grid, dtype=dtype, tol=tol)
    hstep = grid[1] - grid[0]
    for o in (40, 100, 200, 400):
        w = np.ones(o + 1)
        w[1:-1:2] = 4.0
        w[2:-1:2] = 2.0
        simpson = hstep / 3.0 * float(np.dot(w, P[: o + 1]))
        err = abs(grid[o] * C[o] - simpson) / grid[o]
        print(f"[parity] C(t) L24 {dtype} t={grid[o]:.2f}: |C - Simpson/t| = {err:.3e}")
        assert err <= bar
    times = np.asarray(c["times"])
    C, P, _ = H.autocorrelation(c["state"], times, dtype=dtype, tol=tol)
    P2, _ = H.return_probability(c["state"], times, dtype=dtype, tol=tol)
    assert np.array_equal(P, P2)
    assert np.all((C >= -1e-12) & (C <= 1.0 + 1e-12))
    tc = times * C
    assert np.all(np.diff(tc) >= -1e-9 * np.maximum(tc[1:], 1.0))
