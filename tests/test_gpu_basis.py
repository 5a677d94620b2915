"""GPU rank/unrank against the oracle's Gosper list (Algorithm 2): bit-exact."""
import numpy as np
import pytest
import torch

from oracle import basis as ob

pytestmark = pytest.mark.gpu


def _rank_unrank(kry, L, N, states_np):
    B = kry.Basis(L, N)
    st = torch.from_numpy(states_np.astype(np.int64)).cuda()
    r = B.rank(st)
    s2 = B.unrank(r)
    return B, r.cpu().numpy().astype(np.int64), s2.cpu().numpy().astype(np.uint64)


def test_exhaustive_all_sectors_up_to_L20(kry):
    for L in range(1, 21):
        for N in range(0, L + 1):
            b = ob.basis(L, N)
            B, r, s2 = _rank_unrank(kry, L, N, b)
            assert B.dim == b.size
            assert np.array_equal(r, np.arange(b.size)), (L, N)
            assert np.array_equal(s2, b), (L, N)


def test_worked_example(kry):
    B, r, s2 = _rank_unrank(kry, 4, 2, np.array([3, 5, 6, 9, 10, 12], dtype=np.uint64))
    assert r.tolist() == [0, 1, 2, 3, 4, 5]


@pytest.mark.parametrize("L,N", [(30, 15), (32, 16), (31, 7)])
def test_full_size_sampled(kry, L, N):
    """Large sectors: sampled ranks against the oracle list where it fits, else round trips."""
    B = kry.Basis(L, N)
    D = B.dim
    rng = np.random.default_rng(L)
    ranks = np.unique(np.concatenate([rng.integers(0, D, 1 << 20), [0, 1, D - 2, D - 1]]))
    st = B.unrank(torch.from_numpy(ranks.astype(np.int32)).cuda()).cpu().numpy().astype(np.uint64)
    if L == 30:
        b = ob.basis(L, N)
        assert np.array_equal(st, b[ranks])
    # sorted ranks give increasing states with N particles below bit L; rank inverts unrank
    assert np.all(np.diff(st.astype(np.int64)) > 0)
    pc = np.zeros(st.size, dtype=np.int64)
    for k in range(L):
        pc += ((st >> np.uint64(k)) & np.uint64(1)).astype(np.int64)
    assert np.all(pc == N) and np.all(st >> np.uint64(L) == 0)
    r2 = B.rank(torch.from_numpy(st.astype(np.int64)).cuda()).cpu().numpy().astype(np.int64)
    assert np.array_equal(r2, ranks)


def test_invalid_inputs_are_reported(kry):
    B = kry.Basis(10, 4)
    with pytest.raises(kry.KryError) as e:
        B.rank(torch.tensor([0b111, 0b1111], dtype=torch.int64, device="cuda"))
    assert e.value.code == kry.KRY_EINVAL
    with pytest.raises(kry.KryError):
        B.rank(torch.tensor([(1 << 10) | 0b111], dtype=torch.int64, device="cuda"))
    with pytest.raises(kry.KryError):
        B.unrank(torch.tensor([B.dim], dtype=torch.int32, device="cuda"))
    empty = B.rank(torch.zeros(0, dtype=torch.int64, device="cuda"))
    assert empty.numel() == 0
