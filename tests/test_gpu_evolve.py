"""GPU return probability / evolution against the oracle (the parity tests proper).

Bars (from the workloads' accuracy targets): complex128 |P_gpu - P_oracle| <= 1e-10 at
every output time; complex64 (mixed precision) <= 1e-5.  The oracle runs at tol = 1e-12,
so its own error is far below either bar.  The measured error is printed for every case.
"""
import numpy as np
import pytest
import torch

from oracle import basis as ob
from oracle import dense, krylov
import workloads

pytestmark = pytest.mark.gpu


def _oracle_P(L, N, J, Delta, h, pbc, state, times, tol=1e-12):
    H = ob.CSR(L, N, J, Delta, h, pbc)
    P, _ = krylov.return_probability(H, ob.lookup(H.basis, state), times, m=30, tol=tol)
    return P


def _gpu_P(kry, L, N, J, Delta, h, pbc, state, times, m=30, tol=1e-10, dtype="c128"):
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, J, Delta, h, pbc=pbc)
    return H.return_probability(state, times, m=m, tol=tol, dtype=dtype)


def _report(name, err):
    print(f"[parity] {name}: max|dP| = {err:.3e}")


def test_config_L16_fp64(kry):
    c = workloads.config("L16_fp64")
    P, st = _gpu_P(kry, c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"],
                   c["times"], m=c["m"], tol=c["tol"])
    Po = _oracle_P(c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"], c["times"])
    err = float(np.max(np.abs(P - Po)))
    _report("L16 c128", err)
    assert err <= 1e-10
    assert st["n_krylov_steps"] > 10 and st["n_hv"] >= 30 * st["n_krylov_steps"] - 30
    assert st["max_orth_loss"] < 1e-10   # measured only when a second pass was triggered


def test_config_L16_mixed(kry):
    c = workloads.config("L16_fp64")
    P, st = _gpu_P(kry, c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"],
                   c["times"], m=c["m"], tol=1e-7, dtype="c64")
    Po = _oracle_P(c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"], c["times"])
    err = float(np.max(np.abs(P - Po)))
    _report("L16 c64", err)
    assert err <= 1e-5


@pytest.mark.parametrize("L,pbc,hh,Delta", [(10, True, 2.0, 1.0), (10, False, 1.0, 0.5),
                                            (12, True, 0.0, 1.0), (13, True, 1.0, 0.3)])
def test_small_sectors_vs_dense(kry, L, pbc, hh, Delta):
    N = L // 2
    h = workloads.quasiperiodic_field(L, hh, 0.4)
    st = workloads.neel_state(L) if L % 2 == 0 else workloads.neel_state(L - 1)
    times = workloads.log_times(40, 0.1, 100.0)
    P, _ = _gpu_P(kry, L, N, 1.0, Delta, h, pbc, st, times)
    b = dense.sector_states(L, N)
    psi0 = np.zeros(b.size, complex)
    psi0[int(np.searchsorted(b, st))] = 1.0
    Pd = dense.return_probability_dense(dense.hamiltonian_kron(L, 1.0, Delta, h, pbc, N), psi0, times)
    err = float(np.max(np.abs(P - Pd)))
    _report(f"L{L} vs eigh", err)
    assert err <= 1e-10


def test_free_fermions(kry):
    L, N = 14, 7
    h = workloads.quasiperiodic_field(L, 1.0, 2.2)
    times = workloads.log_times(20, 0.1, 50.0)
    st = workloads.neel_state(L)
    P, _ = _gpu_P(kry, L, N, 1.0, 0.0, h, True, st, times)
    err = float(np.max(np.abs(P - dense.free_fermion_P(L, 1.0, h, True, st, times))))
    _report("free fermions L14", err)
    assert err <= 1e-10


@pytest.mark.parametrize("dtype,bar", [("c128", 1e-12), ("c128e", 1e-12), ("c64", 1e-6)])
def test_edge_cases(kry, dtype, bar):
    """Degenerate cases in every precision: a sector smaller than the Krylov dimension
    (breakdown), the empty and the full sector (D = 1, P = 1), the two-level system, t = 0,
    and a Krylov dimension of 4."""
    tol = 1e-7 if dtype == "c64" else 1e-10
    times = [0.0, 0.0, 0.3, 1.0, 7.0, 30.0]
    h4 = [0.3, -0.2, 0.5, 0.1]
    # D = 6 < m: the Krylov space becomes invariant (breakdown)
    P, st = _gpu_P(kry, 4, 2, 1.0, 0.5, h4, True, 0b0101, times, tol=tol, dtype=dtype)
    assert np.max(np.abs(P - _oracle_P(4, 2, 1.0, 0.5, h4, True, 0b0101, times))) <= bar
    assert st["n_breakdowns"] >= 1
    assert P[0] == pytest.approx(1.0, abs=1e-15) and P[1] == pytest.approx(1.0, abs=1e-15)
    # empty and full sectors: P = 1
    for N in (0, 6):
        P, _ = _gpu_P(kry, 6, N, 1.0, 1.0, [0.1] * 6, True, (1 << N) - 1, times, tol=tol, dtype=dtype)
        assert np.max(np.abs(P - 1.0)) <= 1e-13
    # two-level system
    tt = np.linspace(0.0, 20.0, 9)
    P, _ = _gpu_P(kry, 2, 1, 1.3, 0.4, [0.8, -0.3], False, 0b01, tt, tol=tol, dtype=dtype)
    assert np.max(np.abs(P - dense.two_level_P(1.3, [0.8, -0.3], tt))) <= max(bar, 1e-11)
    # small Krylov dimension, loose tolerance
    L = 10
    hq = workloads.quasiperiodic_field(L, 1.0, 0.2)
    tt = [0.05, 0.2, 0.5]
    P, st = _gpu_P(kry, L, 5, 1.0, 1.0, hq, True, workloads.neel_state(L), tt, m=4, tol=1e-6, dtype=dtype)
    err = np.max(np.abs(P - _oracle_P(L, 5, 1.0, 1.0, hq, True, workloads.neel_state(L), tt)))
    assert err <= (1e-5 if dtype == "c64" else 1e-6)
    assert st["n_krylov_steps"] > 3


def test_general_initial_state_and_psi_out(kry):
    L, N = 12, 6
    h = workloads.quasiperiodic_field(L, 1.5, 2.0)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h, pbc=True)
    rng = np.random.default_rng(3)
    psi0 = rng.normal(size=B.dim) + 1j * rng.normal(size=B.dim)
    psi0 /= np.linalg.norm(psi0)
    times = [0.0, 0.5, 2.0, 7.5]
    x = torch.from_numpy(psi0).cuda()
    out = torch.empty_like(x)
    P, _ = H.evolve(x, times, m=30, tol=1e-10, psi_out=out)
    Hc = ob.CSR(L, N, 1.0, 1.0, h, True)
    Po, psio, _ = krylov.evolve(Hc.matvec, Hc.norm_inf(), psi0, times, m=30, tol=1e-12)
    assert np.max(np.abs(P - Po)) <= 1e-10
    assert np.linalg.norm(out.cpu().numpy() - psio) <= 1e-10
    # complex64 input
    P64, _ = H.evolve(x.to(torch.complex64), times, m=30, tol=1e-7)
    assert np.max(np.abs(P64 - Po)) <= 1e-5


def test_unitarity_forward_backward(kry):
    L, N = 14, 7
    h = np.array(workloads.quasiperiodic_field(L, 2.0, 0.9))
    B = kry.Basis(L, N)
    Hf = kry.Hamiltonian(B, 1.0, 1.0, h)
    Hb = kry.Hamiltonian(B, -1.0, 1.0, -h)   # -H: J -> -J at fixed Delta flips every term
    rng = np.random.default_rng(5)
    psi0 = rng.normal(size=B.dim) + 1j * rng.normal(size=B.dim)
    psi0 /= np.linalg.norm(psi0)
    x = torch.from_numpy(psi0).cuda()
    mid, back = torch.empty_like(x), torch.empty_like(x)
    Hf.evolve(x, [5.0], psi_out=mid)
    Hb.evolve(mid, [5.0], psi_out=back)
    assert abs(torch.linalg.vector_norm(mid).item() - 1.0) <= 1e-11
    assert torch.linalg.vector_norm(back - x).item() <= 1e-10


def test_deterministic(kry):
    c = workloads.config("L16_fp64")
    a, _ = _gpu_P(kry, c["L"], c["n_up"], 1.0, 1.0, c["h"][0], True, c["state"], c["times"][:20])
    b, _ = _gpu_P(kry, c["L"], c["n_up"], 1.0, 1.0, c["h"][0], True, c["state"], c["times"][:20])
    assert np.array_equal(a, b)


def test_profiling_changes_nothing_and_counts_every_kernel(kry):
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    P0, st0 = H.return_probability(c["state"], c["times"][:25], tol=1e-10)
    H.profile(True)
    P1, st1 = H.return_probability(c["state"], c["times"][:25], tol=1e-10)
    prof = H.profile_read()
    H.profile(False)
    assert np.array_equal(P0, P1)
    m = 30
    steps = prof["smallexp"]["launches"]
    assert steps >= st1["n_krylov_steps"]
    for k in ("hv", "dots", "update", "passC"):
        assert prof[k]["launches"] == m * steps
    assert min(prof[k]["ms"] for k in ("hv", "dots", "update")) > 0.0 and prof["passC"]["ms"] >= 0.0
    assert prof["combine"]["launches"] == steps
    # algorithmic bytes: the H.v reads v_j and writes u (2 vectors); the dots read u and
    # v_0..v_j (j + 2 vectors); the update reads u and v_0..v_j and writes w (j + 3); all
    # complex128 of length D
    n, vec = st1["n_krylov_steps"], B.dim * 16
    assert prof["hv"]["bytes"] == pytest.approx(n * 2 * m * vec, rel=1e-12)
    assert prof["dots"]["bytes"] == pytest.approx(n * sum(j + 2 for j in range(m)) * vec, rel=1e-12)
    assert prof["update"]["bytes"] == pytest.approx(n * sum(j + 3 for j in range(m)) * vec, rel=1e-12)
    # three kernels per Lanczos index (H.v, dots, update) and the two of the second
    # Gram-Schmidt pass (no-ops unless flagged), then exponential and combine
    assert st1["n_launches"] == steps * (5 * m + 2) + 1
    # as a conditional node, the second pass launches only where it runs: the same bits
    H.second_pass_node(True)
    H.profile(True)
    P2, st2 = H.return_probability(c["state"], c["times"][:25], tol=1e-10)
    steps2 = H.profile_read()["smallexp"]["launches"]
    H.profile(False)
    H.second_pass_node(False)
    assert np.array_equal(P2, P0)
    assert st2["n_launches"] == steps2 * (3 * m + 2) + 2 * st2["n_second_dots"] + 1
    with pytest.raises(kry.KryError):
        H.second_pass_node(2)


@pytest.mark.parametrize("dtype,bound", [("c128", 1e-12), ("c64", 1e-5)])
def test_orthogonality_check(kry, dtype, bound):
    """One classical Gram-Schmidt pass keeps every new Lanczos vector orthogonal to the
    previous ones: measured after every update with orth_check on, and the results agree
    with the default run."""
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    tol = 1e-10 if dtype == "c128" else 1e-7
    P0, st0 = H.return_probability(c["state"], c["times"], tol=tol, dtype=dtype)
    H.orth_check(True)
    P1, st1 = H.return_probability(c["state"], c["times"], tol=tol, dtype=dtype)
    H.orth_check(False)
    print(f"[orth] L16 {dtype}: max |<v_i, w>|/||w|| = {st1['max_orth_loss']:.2e}, "
          f"second passes {st1['n_second_pass']} of {st1['n_hv']} updates")
    assert 0.0 < st1["max_orth_loss"] <= bound
    assert np.max(np.abs(P1 - P0)) <= (1e-12 if dtype == "c128" else 1e-6)


@pytest.mark.parametrize("node", [False, True])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_second_pass_on_every_vector(kry, dtype, node):
    """orth_check(2): the second Gram-Schmidt pass (plain launches, or a conditional node's
    body) runs and subtracts after every update; the results equal the single-pass run to
    rounding, and the L16 evolution still matches the oracle."""
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    H.second_pass_node(node)
    tol = 1e-10 if dtype == "c128" else 1e-7
    P0, st0 = H.return_probability(c["state"], c["times"], tol=tol, dtype=dtype)
    H.orth_check(2)
    P2, st2 = H.return_probability(c["state"], c["times"], tol=tol, dtype=dtype)
    H.orth_check(False)
    # every update takes the dots; all but those whose dots are exactly zero subtract them
    assert st2["n_second_dots"] == st2["n_hv"] and st2["n_second_pass"] >= 0.99 * st2["n_hv"]
    assert st0["n_second_pass"] == 0
    assert np.max(np.abs(P2 - P0)) <= (1e-12 if dtype == "c128" else 1e-6)
    Po = _oracle_P(c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"], c["times"])
    assert np.max(np.abs(P2 - Po)) <= (1e-10 if dtype == "c128" else 1e-5)
    with pytest.raises(kry.KryError):
        H.orth_check(3)


def test_unreachable_tolerance_reports_etol(kry):
    with pytest.raises(kry.KryError) as e:
        _gpu_P(kry, 10, 5, 1.0, 1.0, [0.5] * 10, True, workloads.neel_state(10), [1.0, 5.0], tol=1e-300)
    assert e.value.code == kry.KRY_ETOL


def test_bad_state_is_rejected(kry):
    B = kry.Basis(10, 5)
    H = kry.Hamiltonian(B, 1.0, 1.0, [0.0] * 10)
    with pytest.raises(kry.KryError):
        H.return_probability(0b111, [1.0])
    with pytest.raises(kry.KryError):
        H.return_probability(workloads.neel_state(10), [2.0, 1.0])


def test_config_L24_mixed_vs_fp64(kry):
    c = workloads.config("L24_mixed")
    args = (kry, c["L"], c["n_up"], 1.0, 1.0, c["h"][0], True, c["state"], c["times"])
    P128, _ = _gpu_P(*args, tol=1e-10, dtype="c128")
    P64, _ = _gpu_P(*args, tol=1e-7, dtype="c64")
    err = float(np.max(np.abs(P128 - P64)))
    _report("L24 c64 vs c128, 40 times to t=100", err)
    assert err <= 1e-5


def test_config_L30_full_size(kry):
    """Full-size L=30 sector: short-time law P = 1 - (L J^2/4) t^2 + O(t^4) for the Neel
    state on a ring, and complex64 against complex128 over the early output times."""
    c = workloads.config("L30_qp")
    L, N = c["L"], c["n_up"]
    tt = [1e-3, 2e-3]
    P, _ = _gpu_P(kry, L, N, 1.0, 1.0, c["h"][0], True, c["state"], tt, tol=1e-10, dtype="c128")
    for t, p in zip(tt, P):
        assert abs((1.0 - p) / t**2 - L / 4.0) < 1e-3 * L
    times = c["times"][:10]
    P128, st = _gpu_P(kry, L, N, 1.0, 1.0, c["h"][0], True, c["state"], times, tol=1e-10, dtype="c128")
    torch.cuda.empty_cache()
    P64, _ = _gpu_P(kry, L, N, 1.0, 1.0, c["h"][0], True, c["state"], times, tol=1e-7, dtype="c64")
    err = float(np.max(np.abs(P128 - P64)))
    _report("L30 c64 vs c128 (t <= 0.5)", err)
    assert err <= 1e-5


@pytest.mark.parametrize("K", [1, 3])
def test_caller_owned_workspace(kry, K):
    """kry_set_workspace: a torch buffer of kry_workspace_bytes gives the same P as the
    library's own workspace; a smaller one is refused; None returns to library memory."""
    L, N = 14, 7
    hs = [workloads.quasiperiodic_field(L, 1.0, p) for p in workloads.phases(12, K)]
    times = workloads.log_times(12, 0.1, 20.0)
    st = workloads.neel_state(L)
    ref, _ = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs if K > 1 else hs[0]).return_probability(st, times)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs if K > 1 else hs[0])
    nb = H.workspace_size("c128", 30, n_times=len(times))
    assert nb > 0
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    H.set_workspace(buf)
    P, _ = H.return_probability(st, times)
    assert np.array_equal(np.asarray(P), np.asarray(ref))
    H.set_workspace(buf[: nb // 2])
    with pytest.raises(kry.KryError) as e:
        H.return_probability(st, times)
    assert e.value.code == kry.KRY_EINVAL
    H.set_workspace(None)
    P2, _ = H.return_probability(st, times)
    assert np.array_equal(np.asarray(P2), np.asarray(ref))
