"""Full-size parity: the five workloads at their configured sizes, and the largest split-table
sector (L = 32), against stored oracle values.

The oracle needs minutes to hours per evolution at these sizes, so its values are computed
once on the host by tests/golden/make_golden.py (which calls only oracle/ and the seeded
inputs of workloads/) and stored under tests/golden/.  Bars: complex128 |P_gpu - P_oracle|
<= 1e-10 at every stored time (the oracle ran at tol 1e-12); complex64 <= 1e-5; gradients
against the oracle's central differences <= 1e-6 (step 1e-5: truncation and rounding near
1e-7).  The measured error is printed for every case.
"""
import numpy as np
import pytest
import torch

from conftest import read_rows
import workloads

pytestmark = pytest.mark.gpu

BAR = {"c128": 1e-10, "c64": 1e-5, "c128e": 1e-10}
TOL = {"c128": 1e-10, "c64": 1e-7, "c128e": 1e-10}


def _report(name, err):
    print(f"[parity] {name}: max|dP| = {err:.3e}")


def _golden_P(name, cols="t P"):
    """{k: (times, P)} from a golden file whose rows are `cols`: 't P', 'k t P' or 't P bound'
    (the realisation k is 0 when absent)."""
    names = cols.split()
    out = {}
    for row in read_rows(name):
        r = dict(zip(names, row))
        k = int(r.get("k", 0))
        out.setdefault(k, ([], []))
        out[k][0].append(float(r["t"]))
        out[k][1].append(float(r["P"]))
    return {k: (np.array(v[0]), np.array(v[1])) for k, v in out.items()}


@pytest.mark.parametrize("dtype", ["c128", "c64", "c128e"])
def test_L24_all_output_times_vs_oracle(kry, dtype):
    """The L = 24 workload (D = 2,704,156) at all 40 output times, t = 0.1 .. 100: 143 and
    more Krylov steps, so step boundaries, dense output and the step-size control are all
    exercised at full size."""
    c = workloads.config("L24_mixed")
    times, Po = _golden_P("P_L24_mixed.txt")[0]
    assert np.allclose(times, c["times"], rtol=0, atol=0)
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
    P, st = H.return_probability(c["state"], c["times"], m=c["m"], tol=TOL[dtype], dtype=dtype)
    err = float(np.max(np.abs(P - Po)))
    _report(f"L24 {dtype}, 40 times to t=100 ({st['n_krylov_steps']} Krylov steps)", err)
    assert err <= BAR[dtype]


@pytest.mark.parametrize("hval", ["1.5", "0.5", "3"])
@pytest.mark.parametrize("dtype", ["c64", "c128", "c128e"])
def test_L22_batched_vs_oracle(kry, hval, dtype):
    """The K = 64 phase ensembles of L = 22 (D = 705,432) in one batched evolution each,
    every stored realisation against its own oracle evolution (all 64 at h = 1.5 to t = 10,
    realisations 0 and 63 to t = 100; every fourth at h = 0.5 and 3 to t = 10)."""
    c = workloads.config(f"L22_batched_h{hval}")
    gold = _golden_P(f"P_L22_batched_h{hval}.txt", "k t P")
    n_t = max(len(v[0]) for v in gold.values())
    if dtype != "c64":
        n_t = min(n_t, 27)   # t <= 10: the complex128 batched evolution to t = 100 is long
    times = c["times"][:n_t]
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, c["J"], c["Delta"], np.array(c["h"]), pbc=c["pbc"])
    P, st = H.return_probability(c["state"], times, m=c["m"], tol=TOL[dtype], dtype=dtype)
    assert P.shape == (n_t, 64)
    worst = 0.0
    for k, (tk, Pk) in gold.items():
        n = min(len(tk), n_t)
        assert np.allclose(tk[:n], times[:n], rtol=0, atol=0)
        worst = max(worst, float(np.max(np.abs(P[:n, k] - Pk[:n]))))
    _report(f"L22 K=64 h={hval} {dtype}, {len(gold)} realisations, t <= {times[-1]:.3g}", worst)
    assert worst <= BAR[dtype]
    # the disorder average of the stored realisations
    if hval == "1.5" and len(gold) == 64:
        n10 = min(len(v[0]) for v in gold.values())
        avg_o = np.mean([gold[k][1][:n10] for k in range(64)], axis=0)
        assert np.max(np.abs(np.mean(P[:n10], axis=1) - avg_o)) <= BAR[dtype]


def test_L20_gradient_vs_oracle_differences(kry):
    """dP(t=10)/dh_i for all 20 sites and dP/dDelta of the L = 20 workload (checkpoints every
    8 Krylov steps) against central differences of the oracle's P."""
    c = workloads.config("L20_grad")
    gold = {r[0]: float(r[1]) for r in read_rows("grad_L20.txt")}
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
    P, gh, gd, _ = H.grad(c["state"], c["times"][0], m=c["m"], tol=c["tol"], ckpt_every=c["ckpt_every"])
    want_h = np.array([gold[f"dP/dh_{i + 1}"] for i in range(c["L"])])
    err_h = float(np.max(np.abs(gh - want_h)))
    err_d = abs(gd - gold["dP/dDelta"])
    print(f"[parity] grad L20 vs oracle central differences: |dP| = {abs(P - gold['P']):.2e}, "
          f"max|d dP/dh| = {err_h:.3e}, |d dP/dDelta| = {err_d:.3e}")
    assert abs(P - gold["P"]) <= 1e-10
    assert err_h <= 1e-6 and err_d <= 1e-6


@pytest.mark.parametrize("name", ["L30_clean", "L30_qp"])
def test_L30_early_times_vs_moment_series(kry, name):
    """The L = 30 workloads (D = 155,117,520) at the output times the oracle's moment series
    reaches with a rigorous error bound <= 1e-12, in complex128 (84 GB of Krylov workspace),
    complex64, and complex128 with float-float arithmetic."""
    c = workloads.config(name)
    times, Po = _golden_P(f"P_{name}_early.txt", "t P bound")[0]
    assert len(times) >= 3 and np.allclose(times, c["times"][:len(times)], rtol=0, atol=0)
    B = kry.Basis(c["L"], c["n_up"])
    for dtype in ("c128", "c64", "c128e"):
        H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
        P, st = H.return_probability(c["state"], list(times), m=c["m"], tol=TOL[dtype], dtype=dtype)
        H.close()
        torch.cuda.empty_cache()
        err = float(np.max(np.abs(P - Po)))
        _report(f"{name} {dtype}, t <= {times[-1]:.3f}", err)
        assert err <= BAR[dtype]


def test_L32_largest_split_sector_vs_moment_series(kry):
    """The largest sector of the split rank tables: L = 32, N_up = 16 (D = 601,080,390; the
    lower-bit rank table has 2^16 entries and is read through L1), the quasiperiodic field,
    against the moment series at the output times its rigorous bound (<= 1e-12) covers, in
    every precision with a Krylov dimension of 12 (13 vectors of 9.6 GB in complex128)."""
    L, N = 32, 16
    times, Po = _golden_P("P_L32_qp_early.txt", "t P bound")[0]
    assert len(times) >= 3
    h = workloads.quasiperiodic_field(L, 1.5, workloads.phases(5)[0])
    B = kry.Basis(L, N)
    assert B.dim == 601080390
    for dtype in ("c64", "c128e", "c128"):
        H = kry.Hamiltonian(B, 1.0, 1.0, h, pbc=True)
        P, st = H.return_probability(workloads.neel_state(L), list(times), m=12, tol=TOL[dtype], dtype=dtype)
        H.close()
        torch.cuda.empty_cache()
        err = float(np.max(np.abs(P - Po)))
        _report(f"L32 {dtype}, t <= {times[-1]:.3f} ({st['n_krylov_steps']} Krylov steps)", err)
        assert err <= BAR[dtype]
