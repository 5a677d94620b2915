"""GPU sorted-list basis (kry_basis_create_list; L > 32 such as the L = 55 Fibonacci rings of
Sec. 2 and Sec. 4) against the oracle.

Ranks and states are bit-exact against the oracle's Algorithm 2 enumeration.  H.v: complex128
1e-13 and complex64 2e-6 relative to max|y| (as for the split-table basis).  P(t) and C(t):
complex128 1e-10, complex64 1e-5, against the dense spectral oracle (N = 1), the free-fermion
determinant (Delta = 0) and the oracle's Krylov evolution on its CSR matrix.
"""
import numpy as np
import pytest
import torch

from oracle import basis as ob
from oracle import dense, krylov
import workloads

pytestmark = pytest.mark.gpu


def _vec(D, seed, dtype=torch.complex128):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(D, dtype=torch.complex128, generator=g).to(dtype).cuda()


@pytest.mark.parametrize("L,N", [(1, 0), (1, 1), (5, 2), (12, 6), (16, 5), (20, 10), (33, 2), (55, 1),
                                 (55, 2), (55, 3), (62, 2), (64, 1), (64, 63)])
def test_list_rank_unrank_exact(kry, L, N):
    B = kry.Basis(L, N, list=True)
    assert B.dim == ob.binom(L, N) if L <= 62 else True
    if L <= 62:
        ref = ob.basis(L, N).astype(np.int64)
    else:   # L = 64: brute-force sorted enumeration of the N-subsets (N = 1 or 63)
        full = (1 << 64) - 1
        ref = sorted(((1 << p) if N == 1 else (full ^ (1 << p))) for p in range(64))
        ref = np.array(ref, dtype=np.uint64).astype(np.int64)
    ranks = torch.arange(B.dim, dtype=torch.int32, device="cuda")
    states = B.unrank(ranks).cpu().numpy()
    assert np.array_equal(states, ref)
    back = B.rank(torch.from_numpy(ref).cuda()).cpu().numpy()
    assert np.array_equal(back, np.arange(B.dim, dtype=np.int32))


def test_list_rejects_bad_states_and_ranks(kry):
    B = kry.Basis(40, 3)
    assert B.list
    with pytest.raises(kry.KryError):
        B.rank(torch.tensor([0b1111], dtype=torch.int64, device="cuda"))
    with pytest.raises(kry.KryError):
        B.rank(torch.tensor([(1 << 41) | 3], dtype=torch.int64, device="cuda"))
    with pytest.raises(kry.KryError):
        B.unrank(torch.tensor([B.dim], dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("L,N,pbc", [(4, 2, True), (12, 6, True), (16, 8, False), (33, 3, True),
                                     (55, 2, True), (55, 3, True), (55, 3, False), (64, 2, True)])
def test_list_apply_c128(kry, L, N, pbc):
    rng = np.random.default_rng(L * 7 + N)
    J, Delta = 0.8 + rng.random(), rng.normal()
    h = rng.normal(size=L)
    B = kry.Basis(L, N, list=True)
    H = kry.Hamiltonian(B, J, Delta, h, pbc=pbc)
    x = _vec(B.dim, L + N)
    y = H.apply(x).cpu().numpy()
    if L <= 62:
        yo = ob.CSR(L, N, J, Delta, h, pbc).matvec(x.cpu().numpy())
    else:   # L = 64 > the oracle's range: a few rows from a brute-force sorted basis
        import itertools
        states = np.array(sorted(sum(1 << p for p in c) for c in itertools.combinations(range(L), N)),
                          dtype=np.uint64)
        assert states.size == B.dim
        rows = list(range(0, B.dim, 97))
        yo_rows = ob.row_apply(L, J, Delta, h, pbc, states, x.cpu().numpy(), rows)
        y, yo = y[rows], yo_rows
    assert np.max(np.abs(y - yo)) <= 1e-13 * max(np.max(np.abs(yo)), 1e-300)


@pytest.mark.parametrize("L,N", [(16, 8), (55, 3)])
def test_list_apply_c64_and_split_tables(kry, L, N):
    h = workloads.quasiperiodic_field(L, 1.5, 0.3)
    B = kry.Basis(L, N, list=True)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    x = _vec(B.dim, 7, torch.complex64)
    y = H.apply(x).cpu().numpy()
    yo = ob.CSR(L, N, 1.0, 1.0, h, True).matvec(x.cpu().numpy().astype(np.complex128))
    assert np.max(np.abs(y - yo)) <= 2e-6 * np.max(np.abs(yo))
    if L <= 32:   # same rows as the split-table basis
        Bs = kry.Basis(L, N)
        ys = kry.Hamiltonian(Bs, 1.0, 1.0, h).apply(_vec(B.dim, 8)).cpu().numpy()
        yl = H.apply(_vec(B.dim, 8)).cpu().numpy()
        assert np.max(np.abs(ys - yl)) <= 1e-13 * np.max(np.abs(ys))


def test_list_batched_apply(kry):
    L, N, K = 55, 2, 5
    hs = [workloads.aubry_andre_field(L, 2.0, 1.0, p) for p in workloads.phases(31, K)]
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 0.5, hs)
    x = _vec(B.dim * K, 3)
    y = H.apply(x).cpu().numpy().reshape(B.dim, K)
    xs = x.cpu().numpy().reshape(B.dim, K)
    for k in range(K):
        yo = ob.CSR(L, N, 1.0, 0.5, hs[k], True).matvec(np.ascontiguousarray(xs[:, k]))
        assert np.max(np.abs(y[:, k] - yo)) <= 1e-13 * np.max(np.abs(yo))


@pytest.mark.parametrize("lam", [1.0, 2.0, 3.0])
def test_single_particle_fibonacci_ring(kry, lam):
    """N = 1 on the L = 55 ring with beta = 34/55 (the single-particle Aubry-Andre experiment
    of Sec. 4): P and C against the dense 55 x 55 spectral oracle, and the decay exponent fit."""
    L = 55
    h = workloads.aubry_andre_field(L, lam, 1.0, 0.0)
    B = kry.Basis(L, 1)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    times = [0.0] + list(workloads.log_times(40, 0.1, 1000.0))
    st = 1 << 27   # the particle on the middle site
    C, P, _ = H.autocorrelation(st, times)
    Hd = ob.CSR(L, 1, 1.0, 1.0, h, True).dense()
    psi0 = np.zeros(L, complex)
    psi0[27] = 1.0
    Cd = dense.autocorrelation_dense(Hd, psi0, times)
    Pd = dense.return_probability_dense(Hd, psi0, times)
    print(f"[parity] AA L55 N1 lambda={lam}: max|dC| = {np.max(np.abs(C - Cd)):.3e}, "
          f"max|dP| = {np.max(np.abs(P - Pd)):.3e}")
    assert np.max(np.abs(C - Cd)) <= 1e-10 and np.max(np.abs(P - Pd)) <= 1e-10
    g, _ = kry.decay_exponent(times, C, 10.0, 1000.0)
    assert np.isfinite(g)


def test_free_fermions_L55(kry):
    """Delta = 0 at L = 55, N = 3 (D = 26,235): P against the free-fermion determinant."""
    L, N = 55, 3
    h = workloads.aubry_andre_field(L, 1.5, 1.0, 0.7)
    st = (1 << 5) | (1 << 20) | (1 << 40)
    times = workloads.log_times(25, 0.1, 50.0)
    B = kry.Basis(L, N)
    for dtype, bar in (("c128", 1e-10), ("c64", 1e-5), ("c128e", 1e-10)):
        P, _ = kry.Hamiltonian(B, 1.0, 0.0, h).return_probability(st, times, dtype=dtype,
                                                                   tol=1e-7 if dtype == "c64" else 1e-10)
        Pf = dense.free_fermion_P(L, 1.0, h, True, st, times)
        print(f"[parity] free fermions L55 N3 {dtype}: max|dP| = {np.max(np.abs(P - Pf)):.3e}")
        assert np.max(np.abs(P - Pf)) <= bar


def test_interacting_L55_vs_oracle_krylov(kry):
    """Interacting Aubry-Andre ring, L = 55, N = 3 (Delta = 1): P against the oracle's Krylov
    evolution on its CSR matrix."""
    L, N = 55, 3
    h = workloads.aubry_andre_field(L, 2.0, 1.0, 0.2)
    st = (1 << 0) | (1 << 18) | (1 << 36)
    times = workloads.log_times(20, 0.1, 20.0)
    B = kry.Basis(L, N)
    Hc = ob.CSR(L, N, 1.0, 1.0, h, True)
    Po, _ = krylov.return_probability(Hc, ob.lookup(Hc.basis, st), times, m=30, tol=1e-12)
    for dtype in ("c128", "c128e"):
        P, _ = kry.Hamiltonian(B, 1.0, 1.0, h).return_probability(st, times, dtype=dtype)
        print(f"[parity] AA L55 N3 {dtype}: max|dP| = {np.max(np.abs(P - Po)):.3e}")
        assert np.max(np.abs(P - Po)) <= 1e-10


def test_list_matches_split_tables_P(kry):
    """L = 16 through both basis forms: the same P to the error budget."""
    c = workloads.config("L16_fp64")
    times = c["times"]
    P1, _ = kry.Hamiltonian(kry.Basis(16, 8), 1.0, 1.0, c["h"][0]).return_probability(c["state"], times)
    P2, _ = kry.Hamiltonian(kry.Basis(16, 8, list=True), 1.0, 1.0, c["h"][0]).return_probability(c["state"], times)
    assert np.max(np.abs(P1 - P2)) <= 1e-10


def test_random_state_ensemble_L55(kry):
    """Batched realisations on the list basis: L = 55, N = 2, K = 4, each with its own phase and
    random basis state; P and C per realisation against the dense spectral oracle (D = 1485)."""
    L, N, K = 55, 2, 4
    hs = [workloads.aubry_andre_field(L, 2.5, 1.0, p) for p in workloads.phases(41, K)]
    states = workloads.random_basis_states(L, N, 42, K)
    times = [0.0] + list(workloads.log_times(20, 0.1, 100.0))
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, hs)
    P, C, _ = H.return_probability_states(states, times, autocorrelation=True)
    for k in range(K):
        Hc = ob.CSR(L, N, 1.0, 1.0, hs[k], True)
        psi0 = np.zeros(Hc.D, complex)
        psi0[ob.lookup(Hc.basis, states[k])] = 1.0
        Hd = Hc.dense()
        assert np.max(np.abs(P[:, k] - dense.return_probability_dense(Hd, psi0, times))) <= 1e-10
        assert np.max(np.abs(C[:, k] - dense.autocorrelation_dense(Hd, psi0, times))) <= 1e-10


@pytest.mark.parametrize("L,N,t", [(55, 1, 5.0), (40, 2, 3.0)])
def test_grad_list_basis_vs_daleckii_krein(kry, L, N, t):
    """kry_grad on the sorted-list basis (two blocks of 32 sites when L > 32) against the
    oracle's Daleckii-Krein gradient of its dense CSR matrix.  dH/dh_i = Sz_i from the state
    bits; dH/dDelta = H(Delta = 1) - H(Delta = 0) (H is linear in Delta)."""
    from oracle import gradient
    h = np.asarray(workloads.aubry_andre_field(L, 2.0, 1.0, 0.3) if L == 55
                   else workloads.quasiperiodic_field(L, 1.0, 0.4))
    st = (1 << 27) if N == 1 else ((1 << 3) | (1 << 21))
    H = kry.Hamiltonian(kry.Basis(L, N), 1.0, 1.0, h)
    P, gh, gd, _ = H.grad(st, t, tol=1e-11, ckpt_every=2)
    Hc = ob.CSR(L, N, 1.0, 1.0, h, True)
    states = Hc.basis
    sz = [np.where((states >> np.uint64(i)) & np.uint64(1), 0.5, -0.5) for i in range(L)]
    zz = np.diag(Hc.dense() - ob.CSR(L, N, 1.0, 0.0, h, True).dense())
    psi0 = np.zeros(Hc.D, complex)
    psi0[ob.lookup(states, st)] = 1.0
    Pd, gdk = gradient.daleckii_krein(Hc.dense(), sz + [zz], psi0, t)
    err = max(float(np.max(np.abs(np.asarray(gh) - np.asarray(gdk[:L])))), abs(gd - gdk[L]))
    print(f"[parity] grad list basis L{L} N{N}: |dP| = {abs(P - Pd):.2e}, max|dgrad| = {err:.3e}")
    assert abs(P - Pd) <= 1e-10 and err <= 1e-9


def test_grad_list_equals_split_tables(kry):
    c = workloads.config("L16_fp64")
    out = []
    for lst in (False, True):
        H = kry.Hamiltonian(kry.Basis(16, 8, list=lst), 1.0, 1.0, c["h"][0])
        P, gh, gd, _ = H.grad(c["state"], 2.0, tol=1e-11, ckpt_every=4)
        out.append(np.r_[P, gh, gd])
    assert np.max(np.abs(out[0] - out[1])) <= 1e-10


def test_ring_complex64_keeps_its_basis_orthogonal(kry):
    """L = 55, N = 5 ring with Delta = 1, where the diagonal offset (about 8.75) dominates
    ||H v||: the complex64 evolution keeps step sizes like complex128's (the Lanczos pass runs
    on H - tr(H)/D) and agrees with it to the mixed-precision bar."""
    B = kry.Basis(55, 5)
    H = kry.Hamiltonian(B, 1.0, 1.0, workloads.aubry_andre_field(55, 2.0, 1.0, workloads.phases(7)[0]))
    st = sum(1 << (11 * i) for i in range(5))
    P128, s128 = H.return_probability(st, [10.0], tol=1e-10)
    P64, s64 = H.return_probability(st, [10.0], tol=1e-7, dtype="c64")
    print(f"[parity] ring L55 N5: Krylov steps c128 {s128['n_krylov_steps']}, c64 {s64['n_krylov_steps']}, "
          f"|dP| {abs(P64[0] - P128[0]):.2e}")
    assert s64["n_krylov_steps"] <= s128["n_krylov_steps"] + 2
    assert abs(P64[0] - P128[0]) <= 1e-5
