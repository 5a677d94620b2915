"""KRY_C128E: complex128 in and out, float-float Krylov vectors and vector arithmetic (H.v
sums, dots, updates) on the FP32 pipe inside, against the oracle at the FP64 bar (|dP| <=
1e-10) and against the FP64-arithmetic form.  Storage and arithmetic carry about 47-48
significant bits, so its results differ from the FP64 form's by rounding at the 1e-13 level,
far inside the bar.
"""
import itertools

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


def test_config_L16_against_oracle_and_fp64(kry):
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
    Pe, st = H.return_probability(c["state"], c["times"], m=c["m"], tol=c["tol"], dtype="c128e")
    P128, _ = H.return_probability(c["state"], c["times"], m=c["m"], tol=c["tol"], dtype="c128")
    Po = _oracle_P(c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"], c["times"])
    err, d128 = float(np.max(np.abs(Pe - Po))), float(np.max(np.abs(Pe - P128)))
    print(f"[parity] L16 c128e: max|dP| = {err:.3e} vs oracle, {d128:.3e} vs c128 "
          f"({st['n_krylov_steps']} Krylov steps)")
    assert err <= 1e-10 and d128 <= 1e-11
    assert st["n_krylov_steps"] > 10


@pytest.mark.parametrize("L,pbc,hh,Delta", [(10, True, 2.0, 1.0), (10, False, 1.0, 0.5),
                                            (12, True, 0.0, 1.0), (13, True, 1.0, 0.3)])
def test_small_sectors_vs_dense(kry, L, pbc, hh, Delta):
    N = L // 2
    h = workloads.quasiperiodic_field(L, hh, 0.4)
    st = workloads.neel_state(L) if L % 2 == 0 else workloads.neel_state(L - 1)
    times = workloads.log_times(40, 0.1, 100.0)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, Delta, h, pbc=pbc)
    P, _ = H.return_probability(st, times, dtype="c128e")
    b = dense.sector_states(L, N)
    psi0 = np.zeros(b.size, complex)
    psi0[int(np.searchsorted(b, st))] = 1.0
    Pd = dense.return_probability_dense(dense.hamiltonian_kron(L, 1.0, Delta, h, pbc, N), psi0, times)
    err = float(np.max(np.abs(P - Pd)))
    print(f"[parity] L{L} c128e vs eigh: max|dP| = {err:.3e}")
    assert err <= 1e-10


def test_free_fermions(kry):
    L, N = 14, 7
    h = workloads.quasiperiodic_field(L, 1.0, 2.2)
    times = workloads.log_times(20, 0.1, 50.0)
    st = workloads.neel_state(L)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 0.0, h)
    P, _ = H.return_probability(st, times, dtype="c128e")
    err = float(np.max(np.abs(P - dense.free_fermion_P(L, 1.0, h, True, st, times))))
    print(f"[parity] free fermions L14 c128e: max|dP| = {err:.3e}")
    assert err <= 1e-10


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
    P, _ = H.evolve(x, times, m=30, tol=1e-10, psi_out=out, emulated=True)
    Hc = ob.CSR(L, N, 1.0, 1.0, h, True)
    Po, psio, _ = krylov.evolve(Hc.matvec, Hc.norm_inf(), psi0, times, m=30, tol=1e-12)
    assert np.max(np.abs(P - Po)) <= 1e-10
    assert np.linalg.norm(out.cpu().numpy() - psio) <= 1e-10


@pytest.mark.parametrize("dtype", ["c128e"])
def test_every_shape_gives_the_same_bits(kry, dtype):
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    times = workloads.log_times(20, 0.1, 30.0)
    for grid, rows in itertools.product((0, 304), (1, 2, 4)):
        base = None
        for hvf, dots in itertools.product((0, 1, 2, 3), (0, 1)):
            H.set_shape([grid, hvf, dots, rows, 0], dtype)
            P, _ = H.return_probability(c["state"], times, dtype=dtype)
            if base is None:
                base = P
            assert np.array_equal(P, base), (grid, hvf, dots, rows)
    Po = _oracle_P(c["L"], c["n_up"], 1.0, 1.0, c["h"][0], True, c["state"], times)
    assert np.max(np.abs(base - Po)) <= 1e-10


def test_orthogonality_and_forced_second_pass(kry):
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    P0, _ = H.return_probability(c["state"], c["times"], dtype="c128e")
    H.orth_check(True)
    P1, st1 = H.return_probability(c["state"], c["times"], dtype="c128e")
    H.orth_check(2)
    P2, st2 = H.return_probability(c["state"], c["times"], dtype="c128e")
    H.orth_check(False)
    print(f"[orth] L16 c128e: max |<v_i, w>|/||w|| = {st1['max_orth_loss']:.2e}")
    assert 0.0 < st1["max_orth_loss"] <= 1e-12
    assert st2["n_second_dots"] == st2["n_hv"]
    assert np.max(np.abs(P1 - P0)) <= 1e-12 and np.max(np.abs(P2 - P0)) <= 1e-12


@pytest.mark.parametrize("dtype,bound", [("c128e", 5e-13), ("c128", 5e-14)])
def test_orthogonality_at_L26(kry, dtype, bound):
    """The loss of orthogonality of one Gram-Schmidt pass at L = 26 (D = 10.4 million, about
    1,000 rows per thread in the dots): the float-float accumulators fold their compensation
    back every tile, so the loss stays near the storage precision (7e-14 to 2e-13 measured in
    c128e, where an accumulator left to grow its compensation over the rows gave 1.1e-12),
    and no second pass is needed."""
    L = 26
    H = kry.Hamiltonian(kry.Basis(L, L // 2), 1.0, 1.0, workloads.quasiperiodic_field(L, 1.5, 0.4))
    H.orth_check(True)
    P, st = H.return_probability(workloads.neel_state(L), [0.5, 2.0], dtype=dtype)
    H.orth_check(False)
    P0, st0 = H.return_probability(workloads.neel_state(L), [0.5, 2.0], dtype=dtype)
    print(f"[orth] L26 {dtype}: max |<v_i, w>|/||w|| = {st['max_orth_loss']:.2e}")
    assert 0.0 < st["max_orth_loss"] <= bound
    assert st0["n_second_pass"] == 0


def test_autocorrelation_matches_fp64(kry):
    L, N = 14, 7
    h = workloads.quasiperiodic_field(L, 1.0, 0.6)
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, h)
    times = workloads.log_times(20, 0.1, 50.0)
    st = workloads.neel_state(L)
    Ce, Pe, _ = H.autocorrelation(st, times, dtype="c128e")
    C8, P8, _ = H.autocorrelation(st, times, dtype="c128")
    assert np.max(np.abs(Ce - C8)) <= 1e-11 and np.max(np.abs(Pe - P8)) <= 1e-11


def test_batched_and_list_bases(kry):
    """The float-float form serves batched realisations and the sorted-list basis like the
    other dtypes (same workspace as complex128): against the FP64 form on a K = 3 batch of
    L = 10 and on the sorted-list basis of L = 10 and L = 40 (N = 2)."""
    L, N = 10, 5
    hs = [workloads.quasiperiodic_field(L, 1.0, p) for p in workloads.phases(3, 3)]
    times = workloads.log_times(12, 0.1, 20.0)
    Hb = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs)
    Pb, _ = Hb.return_probability(workloads.neel_state(L), times, dtype="c128e")
    Pb8, _ = Hb.return_probability(workloads.neel_state(L), times, dtype="c128")
    assert Pb.shape == (len(times), 3) and np.max(np.abs(Pb - Pb8)) <= 1e-12
    assert Hb.workspace_size("c128e") == Hb.workspace_size("c128")
    for LL, NN, st in ((L, N, workloads.neel_state(L)), (40, 2, (1 << 0) | (1 << 20))):
        h = workloads.quasiperiodic_field(LL, 1.0, 0.3)
        Hl = kry.Hamiltonian(kry.Basis(LL, NN, list=True), 1.0, 1.0, h)
        Pl, _ = Hl.return_probability(st, times, dtype="c128e")
        Pl8, _ = Hl.return_probability(st, times, dtype="c128")
        d = float(np.max(np.abs(Pl - Pl8)))
        print(f"[parity] list basis L{LL} N{NN} c128e vs c128: max|dP| = {d:.3e}")
        assert d <= 1e-12