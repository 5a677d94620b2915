"""Launch-shape autotuner: picks a measured CTA count, keeps results within rounding of the
default shape, restores the default exactly, and round-trips through its cache file."""
import json

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def test_autotune_single(kry, tmp_path):
    c = workloads.config("L16_fp64")
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, 1.0, 1.0, c["h"][0])
    times = c["times"][:25]
    P0, _ = H.return_probability(c["state"], times)
    res = H.autotune(c["state"], 1.0, dtype="c128", reps=2)
    assert res["grid"] in res["candidates"]
    assert all(v > 0 for v in res["candidates"].values())
    assert res["candidates"][res["grid"]] == min(res["candidates"].values())
    P1, _ = H.return_probability(c["state"], times)
    assert np.max(np.abs(P1 - P0)) <= 1e-12
    H.set_grid(0)
    P2, _ = H.return_probability(c["state"], times)
    assert np.array_equal(P2, P0)
    cache = str(tmp_path / "tune.json")
    r1 = H.autotune(c["state"], 1.0, dtype="c64", cache=cache)
    r2 = H.autotune(c["state"], 1.0, dtype="c64", cache=cache)
    assert r1["grid"] == r2["grid"]
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
    assert res["grid"] in res["candidates"]
    assert np.max(np.abs(P1 - P0)) <= 1e-6


def test_set_grid_rejects_negative(kry):
    B = kry.Basis(8, 4)
    H = kry.Hamiltonian(B, 1.0, 1.0, [0.0] * 8)
    with pytest.raises(kry.KryError):
        H.set_grid(-1)
