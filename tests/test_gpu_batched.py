"""Batched realisations ([state][K] interleaved, one H.v / Lanczos pass for all K) against
single runs and the oracle.

Bars: complex128 |dP| <= 1e-10 against the oracle, complex64 <= 1e-5; a batch of K equal
copies reproduces the single run to 1e-12 (same arithmetic, different reduction order).
"""
import numpy as np
import pytest
import torch

from oracle import basis as ob
from oracle import krylov
import workloads

pytestmark = pytest.mark.gpu


def _fields(L, hh, seed, K):
    return np.array([workloads.quasiperiodic_field(L, hh, p) for p in workloads.phases(seed, K)])


@pytest.mark.parametrize("K,dtype", [(3, torch.complex128), (64, torch.complex64), (40, torch.complex128),
                                     (100, torch.complex64)])
def test_apply_batched_vs_oracle(kry, K, dtype):
    L, N = 12, 6
    h = _fields(L, 2.0, 7, K)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 0.8, h)
    g = torch.Generator().manual_seed(K)
    x = torch.randn(B.dim, K, dtype=torch.complex128, generator=g)
    y = H.apply(x.to(dtype).cuda().contiguous()).cpu().numpy().astype(np.complex128).reshape(B.dim, K)
    xn = x.to(dtype).numpy().astype(np.complex128)
    tol = 1e-13 if dtype == torch.complex128 else 2e-6
    for k in (0, K // 2, K - 1):
        yo = ob.CSR(L, N, 1.0, 0.8, h[k], True).matvec(np.ascontiguousarray(xn[:, k]))
        assert np.max(np.abs(y[:, k] - yo)) <= tol * np.max(np.abs(yo))


def test_identical_copies_equal_single_run(kry):
    c = workloads.config("L16_fp64")
    L, N, h = c["L"], c["n_up"], np.array(c["h"][0])
    B = kry.Basis(L, N)
    times = c["times"][:30]
    P1, _ = kry.Hamiltonian(B, 1.0, 1.0, h).return_probability(c["state"], times, tol=1e-10)
    PK, st = kry.Hamiltonian(B, 1.0, 1.0, np.tile(h, (5, 1))).return_probability(c["state"], times, tol=1e-10)
    assert PK.shape == (len(times), 5)
    for k in range(5):
        assert np.max(np.abs(PK[:, k] - P1)) <= 1e-12


@pytest.mark.parametrize("dtype,bar", [("c128", 1e-10), ("c64", 1e-5), ("c128e", 1e-10)])
def test_each_realisation_matches_oracle(kry, dtype, bar):
    L, N, K = 14, 7, 6
    h = _fields(L, 1.5, 3, K)
    times = workloads.log_times(20, 0.1, 60.0)
    st = workloads.neel_state(L)
    B = kry.Basis(L, N)
    P, _ = kry.Hamiltonian(B, 1.0, 1.0, h).return_probability(
        st, times, tol=1e-7 if dtype == "c64" else 1e-10, dtype=dtype)
    worst = 0.0
    for k in range(K):
        Hc = ob.CSR(L, N, 1.0, 1.0, h[k], True)
        Po, _ = krylov.return_probability(Hc, ob.lookup(Hc.basis, st), times, m=30, tol=1e-12)
        worst = max(worst, float(np.max(np.abs(P[:, k] - Po))))
    print(f"[parity] batched L14 K=6 {dtype}: max|dP| = {worst:.3e}")
    assert worst <= bar


@pytest.mark.parametrize("dtype,bound", [("c128", 1e-12), ("c64", 2e-5), ("c128e", 1e-12)])
def test_orthogonality_check_batched(kry, dtype, bound):
    """Every realisation of a batch keeps each new Lanczos vector orthogonal to the previous
    ones after one classical Gram-Schmidt pass: measured after every update with orth_check
    on (every realisation takes the dots of pass C1), and the results agree with the default
    run."""
    L, N, K = 14, 7, 6
    h = _fields(L, 1.5, 3, K)
    times = workloads.log_times(12, 0.1, 30.0)
    st = workloads.neel_state(L)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, h)
    tol = 1e-7 if dtype == "c64" else 1e-10
    P0, _ = H.return_probability(st, times, tol=tol, dtype=dtype)
    H.orth_check(True)
    P1, st1 = H.return_probability(st, times, tol=tol, dtype=dtype)
    H.orth_check(False)
    print(f"[orth] batched L14 K=6 {dtype}: max |<v_i, w>|/||w|| = {st1['max_orth_loss']:.2e}")
    assert 0.0 < st1["max_orth_loss"] <= bound
    assert np.max(np.abs(P1 - P0)) <= (1e-6 if dtype == "c64" else 1e-12)


@pytest.mark.parametrize("emulated", [False, True])
def test_general_initial_states_batched(kry, emulated):
    """Dense complex128 initial vectors [D][K] and psi(t) out, in FP64 and with float-float
    vectors inside (complex128 in and out)."""
    L, N, K = 10, 5, 4
    h = _fields(L, 1.0, 9, K)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    rng = np.random.default_rng(2)
    psi0 = rng.normal(size=(B.dim, K)) + 1j * rng.normal(size=(B.dim, K))
    psi0 /= np.linalg.norm(psi0, axis=0)
    times = [0.0, 0.4, 3.0]
    x = torch.from_numpy(np.ascontiguousarray(psi0)).cuda()
    out = torch.empty_like(x)
    P, _ = H.evolve(x, times, tol=1e-10, psi_out=out, emulated=emulated)
    out = out.cpu().numpy()
    for k in range(K):
        Hc = ob.CSR(L, N, 1.0, 1.0, h[k], True)
        Po, psio, _ = krylov.evolve(Hc.matvec, Hc.norm_inf(), psi0[:, k].copy(), times, m=30, tol=1e-12)
        assert np.max(np.abs(P[:, k] - Po)) <= 1e-10
        assert np.linalg.norm(out[:, k] - psio) <= 1e-10


def test_float_float_batch_against_fp64_batch(kry):
    """The K = 16 phase ensemble of L = 16 in float-float against the FP64 batch: the same
    recurrences to rounding (about 1e-14), and a batch of identical copies reproduces the
    single float-float run."""
    L, N, K = 16, 8, 16
    h = _fields(L, 1.5, 3, K)
    times = workloads.log_times(20, 0.1, 30.0)
    st = workloads.neel_state(L)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, h)
    Pe, ste = H.return_probability(st, times, dtype="c128e")
    P8, st8 = H.return_probability(st, times, dtype="c128")
    d = float(np.max(np.abs(Pe - P8)))
    print(f"[parity] batched L16 K=16 c128e vs c128: max|dP| = {d:.3e}")
    assert d <= 1e-12 and ste["n_second_pass"] == 0
    H1 = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, h[0])
    P1, _ = H1.return_probability(st, times, dtype="c128e")
    Hc = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, np.tile(h[0], (3, 1)))
    Pc, _ = Hc.return_probability(st, times, dtype="c128e")
    assert np.max(np.abs(Pc - P1[:, None])) <= 1e-12


def test_launch_count_batched(kry):
    """Per Lanczos index the batched step launches ten kernels (the H.v, the dots, the update,
    the two of the second pass, four partial-sum reductions and the refresh of the running
    Krylov dimension over the realisations);
    then the two of the small exponential, the combine, its reduction and the step
    bookkeeping: 10 m + 5 per replay, plus the initial basis state."""
    L, N, K, m = 12, 6, 8, 30
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, _fields(L, 1.5, 3, K))
    st = workloads.neel_state(L)
    H.return_probability(st, [0.1])   # capture
    H.profile(True)
    _, s = H.return_probability(st, [0.5, 2.0, 5.0], m=m, tol=1e-10)
    steps = H.profile_read()["smallexp"]["launches"]
    H.profile(False)
    assert steps >= s["n_krylov_steps"] > 0
    assert s["n_launches"] == steps * (10 * m + 5) + 1
