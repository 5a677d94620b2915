"""GPU matrix-free H.v (kry_apply) against the oracle CSR SpMV.

Tolerances: complex128, 1e-13 relative to max|y| (FP64 sums of at most L+1 terms in a
different order); complex64, 2e-6 relative (FP32 rounding of the same sums).
"""
import numpy as np
import pytest
import torch

from oracle import basis as ob
import workloads

pytestmark = pytest.mark.gpu

CASES = [(1, 0, True), (1, 1, True), (2, 1, False), (2, 1, True), (3, 1, True), (4, 2, True),
         (5, 2, False), (10, 3, False), (12, 6, True), (16, 8, True), (17, 5, True),
         (20, 10, True), (22, 11, True), (24, 12, True)]


def _vec(D, seed, dtype=torch.complex128):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(D, dtype=torch.complex128, generator=g)
    return x.to(dtype).cuda()


@pytest.mark.parametrize("L,N,pbc", CASES)
def test_apply_c128(kry, L, N, pbc):
    rng = np.random.default_rng(L * 100 + N)
    J, Delta = 0.8 + rng.random(), rng.normal()
    h = rng.normal(size=L)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, J, Delta, h, pbc=pbc)
    x = _vec(B.dim, L + N)
    y = H.apply(x).cpu().numpy()
    yo = ob.CSR(L, N, J, Delta, h, pbc).matvec(x.cpu().numpy())
    scale = max(np.max(np.abs(yo)), 1e-300)
    assert np.max(np.abs(y - yo)) <= 1e-13 * scale


@pytest.mark.parametrize("L,N,pbc", [(12, 6, True), (16, 8, True), (24, 12, True)])
def test_apply_c64(kry, L, N, pbc):
    h = workloads.quasiperiodic_field(L, 1.5, 0.3)
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h, pbc=pbc)
    x = _vec(B.dim, 7, torch.complex64)
    y = H.apply(x).cpu().numpy()
    yo = ob.CSR(L, N, 1.0, 1.0, h, pbc).matvec(x.cpu().numpy().astype(np.complex128))
    assert np.max(np.abs(y - yo)) <= 2e-6 * np.max(np.abs(yo))


def test_apply_is_hermitian(kry):
    L, N = 18, 9
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 0.7, workloads.quasiperiodic_field(L, 2.0, 1.0), pbc=True)
    x, y = _vec(B.dim, 1), _vec(B.dim, 2)
    lhs = torch.vdot(x, H.apply(y)).item()
    rhs = torch.vdot(H.apply(x), y).item()
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_apply_L30_sampled_rows(kry):
    """Full-size sector of the L=30 workload: sampled rows against the oracle row builder."""
    L, N = 30, 15
    h = workloads.quasiperiodic_field(L, 1.5, workloads.phases(5)[0])
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h, pbc=True)
    x = _vec(B.dim, 30)
    y = H.apply(x)
    b = ob.basis(L, N)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.integers(0, B.dim, 2000), [0, B.dim - 1]]))
    xs = x.cpu().numpy()
    yo = ob.row_apply(L, 1.0, 1.0, h, True, b, xs, rows)
    yg = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.max(np.abs(yg - yo)) <= 1e-13 * np.max(np.abs(yo))


def test_apply_rejects_bad_arguments(kry):
    B = kry.Basis(8, 4)
    H = kry.Hamiltonian(B, 1.0, 1.0, [0.0] * 8)
    x = _vec(B.dim, 0)
    with pytest.raises(ValueError):
        H.apply(x[:-1])
    assert kry.load().kry_apply(H._h, 0, x.data_ptr(), x.data_ptr(), None) == kry.KRY_EINVAL
