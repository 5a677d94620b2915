"""Launch shapes and the autotuner.

The shape parts that only reorder independent loads (the H.v gather form, the dots prefetch)
must give bitwise the same P; the CTA count and the update rows per thread change which rows a
thread sums into its partial norms, so P agrees to rounding.  The autotuner picks the fastest of
the shapes it measured, restores nothing it should not, and round-trips through its cache."""
import itertools
import json

import numpy as np
import pytest

from oracle import basis as ob
from oracle import krylov
import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_every_shape_gives_the_same_bits(kry, dtype):
    """All combinations of parts 1-3 on the L = 16 workload (and on an open L = 13 chain,
    whose lower and upper parts differ in size), at two grids."""
    c = workloads.config("L16_fp64")
    tol = 1e-10 if dtype == "c128" else 1e-7
    for L, N, pbc, hv in ((16, 8, True, c["h"][0]), (13, 6, False, workloads.quasiperiodic_field(13, 1.0, 0.7))):
        state = workloads.neel_state(L) if L % 2 == 0 else workloads.neel_state(L - 1)
        times = workloads.log_times(25, 0.1, 30.0)
        B = kry.Basis(L, N)
        H = kry.Hamiltonian(B, 1.0, 1.0, hv, pbc=pbc)
        assert H.get_shape(dtype) == [0, 0, 0, 2, 0]
        ref, _ = H.return_probability(state, times, tol=tol, dtype=dtype)
        for grid, rows in itertools.product((0, 152), (1, 2, 4)):
            base = None
            for hvf, dots in itertools.product((0, 1, 2, 3), (0, 1)):
                H.set_shape([grid, hvf, dots, rows, 0], dtype)
                P, _ = H.return_probability(state, times, tol=tol, dtype=dtype)
                if base is None:
                    base = P
                    assert np.max(np.abs(P - ref)) <= (1e-12 if dtype == "c128" else 1e-6)
                assert np.array_equal(P, base), (grid, hvf, dots, rows)
        Hc = ob.CSR(L, N, 1.0, 1.0, hv, pbc)
        Po, _ = krylov.return_probability(Hc, ob.lookup(Hc.basis, state), times, m=30, tol=1e-12)
        assert np.max(np.abs(base - Po)) <= (1e-10 if dtype == "c128" else 1e-5)


def test_hv_forms_equal_bitwise_on_apply_sizes(kry):
    """The chunked and the one-at-a-time gathers inside the Lanczos pass at L = 22 and 24 (upper
    and lower parts of 11/12 sites): one Krylov step, P bitwise equal."""
    for L in (22, 24):
        B = kry.Basis(L, L // 2)
        H = kry.Hamiltonian(B, 1.0, 1.0, workloads.quasiperiodic_field(L, 1.5, 0.2))
        out = []
        for hvf in (0, 1, 2, 3):
            H.set_shape([0, hvf, 0, 2, 0], "c64")
            P, st = H.return_probability(workloads.neel_state(L), [0.05, 0.3], tol=1e-7, dtype="c64")
            out.append(P)
        assert all(np.array_equal(out[0], o) for o in out[1:])


@pytest.mark.parametrize("dtype", ["c64", "c128e"])
def test_dots_forms_equal_bitwise_on_apply_sizes(kry, dtype):
    """The dots with the next vector prefetched into registers and without prefetch, at L = 22
    and 24 over several Krylov steps to t = 8 (every Lanczos index, so every split of the
    vectors over the groups, and a ragged last tile): P bitwise equal."""
    for L in (22, 24):
        B = kry.Basis(L, L // 2)
        H = kry.Hamiltonian(B, 1.0, 1.0, workloads.quasiperiodic_field(L, 1.5, 0.2))
        out = []
        for dots in (0, 1):
            H.set_shape([0, 0, dots, 2, 0], dtype)
            P, st = H.return_probability(workloads.neel_state(L), [0.05, 0.3, 1.0, 4.0, 8.0], tol=1e-7, dtype=dtype)
            out.append(P)
        assert st["n_krylov_steps"] >= 2
        assert all(np.array_equal(out[0], o) for o in out[1:])


def test_autotune_single(kry, tmp_path):
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    times = c["times"][:25]
    P0, _ = H.return_probability(c["state"], times)
    res = H.autotune(c["state"], 1.0, dtype="c128", reps=2)
    shapes = [tuple(s) for s, _ in res["candidates"]]
    assert tuple(res["shape"]) in shapes and len(shapes) >= 10
    assert all(ms > 0 for _, ms in res["candidates"])
    best = min(ms for _, ms in res["candidates"])
    assert dict((tuple(s), ms) for s, ms in res["candidates"])[tuple(res["shape"])] == best
    assert H.get_shape("c128") == res["shape"]
    P1, _ = H.return_probability(c["state"], times)
    assert np.max(np.abs(P1 - P0)) <= 1e-12
    H.set_shape([0, 0, 0, 2, 0])
    P2, _ = H.return_probability(c["state"], times)
    assert np.array_equal(P2, P0)
    cache = str(tmp_path / "tune.json")
    r1 = H.autotune(c["state"], 1.0, dtype="c64", cache=cache)
    r2 = H.autotune(c["state"], 1.0, dtype="c64", cache=cache)
    assert r1["shape"] == r2["shape"]
    assert len(json.load(open(cache))) == 1


def test_autotune_batched(kry):
    L, N, K = 14, 7, 8
    h = [workloads.quasiperiodic_field(L, 1.0, p) for p in workloads.phases(11, K)]
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    times = workloads.log_times(10, 0.1, 20.0)
    P0, _ = H.return_probability(workloads.neel_state(L), times, dtype="c64", tol=1e-7)
    res = H.autotune(workloads.neel_state(L), 0.5, dtype="c64")
    P1, _ = H.return_probability(workloads.neel_state(L), times, dtype="c64", tol=1e-7)
    assert len(res["candidates"]) == 7   # the CTA count, then the chunk of realisations
    assert res["shape"][1:4] == [0, 0, 2] and res["shape"][4] in (0, 8, 16)
    assert np.max(np.abs(P1 - P0)) <= 1e-6


@pytest.mark.parametrize("K", [8, 64, 37])
def test_batched_chunks_give_the_same_bits(kry, K):
    """The batched H.v in chunks of 8 or 16 realisations (shape part 4) against all K at once:
    P bitwise equal, and each realisation against its own oracle evolution."""
    L, N = 12, 6
    h = [workloads.quasiperiodic_field(L, 1.2, p) for p in workloads.phases(13, K)]
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, 1.0, 1.0, h)
    times = workloads.log_times(8, 0.1, 10.0)
    st = workloads.neel_state(L)
    out = {}
    for dtype in ("c128", "c64"):
        for ch in (0, 8, 16):
            H.set_shape([0, 0, 0, 2, ch], dtype)
            out[(dtype, ch)], _ = H.return_probability(st, times, tol=1e-10 if dtype == "c128" else 1e-7, dtype=dtype)
        assert np.array_equal(out[(dtype, 0)], out[(dtype, 8)]) and np.array_equal(out[(dtype, 0)], out[(dtype, 16)])
    for k in (0, K - 1):
        Hc = ob.CSR(L, N, 1.0, 1.0, h[k], True)
        Po, _ = krylov.return_probability(Hc, ob.lookup(Hc.basis, st), times, m=30, tol=1e-12)
        assert np.max(np.abs(out[("c128", 16)][:, k] - Po)) <= 1e-10
        assert np.max(np.abs(out[("c64", 8)][:, k] - Po)) <= 1e-5


def test_bad_shapes_are_rejected(kry):
    B = kry.Basis(8, 4)
    H = kry.Hamiltonian(B, 1.0, 1.0, [0.0] * 8)
    with pytest.raises(kry.KryError):
        H.set_grid(-1)
    for bad in ([0, 4, 0, 2, 0], [0, 0, 3, 2, 0], [0, 0, 0, 3, 0], [-1, 0, 0, 2, 0], [0, 0, 0, 2, 4]):
        with pytest.raises(kry.KryError):
            H.set_shape(bad)
    assert H.get_shape() == [0, 0, 0, 2, 0]
