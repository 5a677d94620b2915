"""Adjoint gradient (kry_grad, autograd.Function) against the oracle's dense Daleckii-Krein
gradient, finite differences and its invariants.

Bars: dense DK (L <= 10) 1e-9; central differences of P with step 1e-5 have truncation and
rounding errors near 1e-7, so the FD comparisons use 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import basis as ob
from oracle import dense, gradient, krylov
import workloads

pytestmark = pytest.mark.gpu


def _dk(L, N, J, Delta, h, pbc, state, t):
    b = dense.sector_states(L, N)
    psi0 = np.zeros(b.size, complex)
    psi0[int(np.searchsorted(b, state))] = 1.0
    H = dense.hamiltonian_kron(L, J, Delta, h, pbc, N)
    dHs = [gradient.sz_diag(L, N, i) for i in range(L)] + [gradient.zz_diag(L, N, J, pbc)]
    return gradient.daleckii_krein(H, dHs, psi0, t)


@pytest.mark.parametrize("L,pbc,t,Delta", [(8, True, 3.0, 1.0), (10, True, 10.0, 1.0),
                                           (10, False, 4.0, 0.6)])
def test_grad_matches_dense_daleckii_krein(kry, L, pbc, t, Delta):
    N = L // 2
    h = np.array(workloads.quasiperiodic_field(L, 1.0, 0.4))
    st = workloads.neel_state(L)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, Delta, h, pbc=pbc)
    P, gh, gd, stats = H.grad(st, t, tol=1e-11, ckpt_every=2)
    Pd, gdk = _dk(L, N, 1.0, Delta, h, pbc, st, t)
    err = max(float(np.max(np.abs(gh - np.array(gdk[:L])))), abs(gd - gdk[L]))
    print(f"[parity] grad L{L} t={t}: |P-P_dense| = {abs(P - Pd):.2e}, max|dgrad| = {err:.3e}")
    assert abs(P - Pd) <= 1e-10
    assert err <= 1e-9


def test_grad_independent_of_checkpoint_spacing(kry):
    L, N, t = 10, 5, 8.0
    h = workloads.quasiperiodic_field(L, 1.5, 0.9)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    ref = None
    for every in (1, 3, 8, 1000):
        P, gh, gd, _ = H.grad(workloads.neel_state(L), t, tol=1e-11, ckpt_every=every)
        v = np.r_[gh, gd]
        if ref is None:
            ref = v
        assert np.max(np.abs(v - ref)) <= 1e-10


def test_grad_with_more_checkpoints_than_the_initial_buffer(kry):
    """ckpt_every = 1 with a small Krylov space: far more than 64 Krylov steps, so the
    checkpoint buffer grows (and the forward sweep is repeated); the gradient still matches
    the oracle's dense Daleckii-Krein formula."""
    L, N, t, m = 10, 5, 10.0, 8
    h = np.array(workloads.quasiperiodic_field(L, 1.0, 1.3))
    st = workloads.neel_state(L)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    _, steps = H.return_probability(st, [t], m=m, tol=1e-10)
    assert steps["n_krylov_steps"] > 64
    P, gh, gd, stats = H.grad(st, t, m=m, tol=1e-10, ckpt_every=1)
    Pd, gdk = _dk(L, N, 1.0, 1.0, h, True, st, t)
    err = max(float(np.max(np.abs(gh - np.array(gdk[:L])))), abs(gd - gdk[L]))
    print(f"[parity] grad L10 t=10 m=8 every step checkpointed ({steps['n_krylov_steps']} steps): "
          f"max|dgrad| = {err:.3e}")
    assert abs(P - Pd) <= 1e-10
    assert err <= 1e-8


def test_costate_is_conjugate_forward_state(kry):
    """For real H and a real psi0, lambda(s) = exp(iH(t-s)) psi0 = conj(psi(t-s)): the
    evolution under -H equals the conjugated evolution under H."""
    L, N = 12, 6
    h = np.array(workloads.quasiperiodic_field(L, 2.0, 0.3))
    B = kry.Basis(L, N)
    Hf, Hn = kry.Hamiltonian(B, 1.0, 1.0, h), kry.Hamiltonian(B, -1.0, 1.0, -h)
    x = torch.zeros(B.dim, dtype=torch.complex128, device="cuda")
    r0 = B.rank(torch.tensor([workloads.neel_state(L)], dtype=torch.int64, device="cuda")).item()
    x[r0] = 1.0
    a, c = torch.empty_like(x), torch.empty_like(x)
    Hf.evolve(x, [3.7], psi_out=a)
    Hn.evolve(x, [3.7], psi_out=c)
    assert torch.linalg.vector_norm(c - a.conj()).item() <= 1e-10


def test_config_L20_grad_full_size(kry):
    """dP(t=10)/dh_i (20 sites) and dP/dDelta at L = 20 (D = 184,756) with checkpoints every
    8 steps: sum rule, central differences of P on the GPU, and one component against
    central differences of the CPU oracle."""
    c = workloads.config("L20_grad")
    L, N, t = c["L"], c["n_up"], c["times"][0]
    h = np.array(c["h"][0])
    st = c["state"]
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    P, gh, gd, stats = H.grad(st, t, tol=1e-10, ckpt_every=c["ckpt_every"])
    assert abs(np.sum(gh)) <= 1e-9          # sum_i Sz_i is conserved in the sector
    eps = 1e-5

    def P_gpu(hv, d):
        Hx = kry.Hamiltonian(B, 1.0, d, hv)
        p, _ = Hx.return_probability(st, [t], tol=1e-12)
        return p[0]

    worst = 0.0
    for i in (0, 7, 13):
        fd = gradient.central_fd(lambda x: P_gpu(np.where(np.arange(L) == i, x, h), 1.0), h[i], eps)
        worst = max(worst, abs(fd - gh[i]))
    fdD = gradient.central_fd(lambda d: P_gpu(h, d), 1.0, eps)
    worst = max(worst, abs(fdD - gd))
    print(f"[parity] grad L20 vs GPU central FD: max|d| = {worst:.3e}")
    assert worst <= 1e-6

    Hp = ob.CSR(L, N, 1.0, 1.0, h + eps * (np.arange(L) == 0), True)
    Hm = ob.CSR(L, N, 1.0, 1.0, h - eps * (np.arange(L) == 0), True)
    r0 = ob.lookup(Hp.basis, st)
    Pp, _ = krylov.return_probability(Hp, r0, [t], m=30, tol=1e-12)
    Pm, _ = krylov.return_probability(Hm, r0, [t], m=30, tol=1e-12)
    fd_or = (Pp[0] - Pm[0]) / (2 * eps)
    print(f"[parity] grad L20 dP/dh_0 vs oracle FD: {abs(fd_or - gh[0]):.3e}")
    assert abs(fd_or - gh[0]) <= 1e-6


def test_autograd_function(kry):
    L, N, t = 8, 4, 2.5
    B = kry.Basis(L, N)
    h = torch.tensor(workloads.quasiperiodic_field(L, 1.0, 0.2), dtype=torch.float64, requires_grad=True)
    Delta = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    P = kry.return_probability(h, Delta, B, 1.0, workloads.neel_state(L), t, tol=1e-11)
    (3.0 * P).backward()
    Pd, gdk = _dk(L, N, 1.0, 0.8, h.detach().numpy(), True, workloads.neel_state(L), t)
    assert abs(P.item() - Pd) <= 1e-10
    assert np.max(np.abs(h.grad.numpy() - 3.0 * np.array(gdk[:L]))) <= 3e-9
    assert abs(Delta.grad.item() - 3.0 * gdk[L]) <= 3e-9


def test_autograd_without_gradient_and_on_cuda_tensors(kry):
    """Under no_grad only P is evolved (no adjoint); with CUDA inputs the gradients come back
    on the inputs' device."""
    L, N, t = 8, 4, 2.5
    B = kry.Basis(L, N)
    hv = workloads.quasiperiodic_field(L, 1.0, 0.2)
    Pd, gdk = _dk(L, N, 1.0, 0.8, np.array(hv), True, workloads.neel_state(L), t)
    with torch.no_grad():
        P0 = kry.return_probability(torch.tensor(hv, dtype=torch.float64), torch.tensor(0.8, dtype=torch.float64),
                                    B, 1.0, workloads.neel_state(L), t, tol=1e-11)
    assert abs(P0.item() - Pd) <= 1e-10
    h = torch.tensor(hv, dtype=torch.float64, device="cuda", requires_grad=True)
    Delta = torch.tensor(0.8, dtype=torch.float64, device="cuda", requires_grad=True)
    P = kry.return_probability(h, Delta, B, 1.0, workloads.neel_state(L), t, tol=1e-11)
    P.backward()
    assert h.grad.is_cuda and Delta.grad.is_cuda
    assert np.max(np.abs(h.grad.cpu().numpy() - np.array(gdk[:L]))) <= 1e-9
    assert abs(Delta.grad.item() - gdk[L]) <= 1e-9


def test_grad_rejects_bad_arguments(kry):
    B = kry.Basis(8, 4)
    H = kry.Hamiltonian(B, 1.0, 1.0, [0.1] * 8)
    with pytest.raises(kry.KryError):
        H.grad(0b111, 1.0)
    with pytest.raises(kry.KryError):
        H.grad(workloads.neel_state(8), -1.0)
    with pytest.raises(kry.KryError):
        H.grad(workloads.neel_state(8), 1.0, ckpt_every=0)
