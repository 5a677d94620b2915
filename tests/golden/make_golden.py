"""Writes the stored oracle values that the full-size GPU parity tests compare against.

Every value here comes from the CPU oracle (`oracle/`) on the seeded inputs of `workloads/`;
nothing is read from the CUDA library.  The oracle at these sizes takes minutes to hours on
the host, far beyond a GPU test's budget, so its results are stored as small text files:

  P_L24_mixed.txt            P(t) of the L = 24 workload (D = 2,704,156) at its 40 output
                             times, t up to 100: krylov.return_probability, m = 30, tol 1e-12
  P_L22_batched_h<h>.txt     P(t) of realisations k of the K = 64 phase ensembles at L = 22
                             (D = 705,432), one oracle evolution per realisation
  grad_L20.txt               P(t = 10), dP/dh_i (i = 1..20) and dP/dDelta of the L = 20
                             workload by central differences (step 1e-5) of the oracle's P
  P_L30_<name>_early.txt     P at the first output times of the L = 30 workloads from the
                             moment series of oracle.moments, with its rigorous error bound
  P_L32_qp_early.txt         the same for the largest sector of the split rank tables, L = 32,
                             N_up = 16 (D = 601,080,390), h = 1.5 (phi: workloads.phases(5))

Each file's header states the workload, the oracle call, its tolerance and its run time.

    python tests/golden/make_golden.py L24|L22|L20grad|L30|L32 [--jobs N]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ORACLE_TOL = 1e-12
FD_STEP = 1e-5


def _oracle_P(L, N, J, Delta, h, pbc, state, times):
    """P at `times` from the oracle's CSR Hamiltonian and Krylov evolution (one process)."""
    from oracle import basis as ob
    from oracle import krylov
    t0 = time.perf_counter()
    H = ob.CSR(L, N, J, Delta, h, pbc)
    P, st = krylov.return_probability(H, ob.lookup(H.basis, state), times, m=30, tol=ORACLE_TOL)
    return [float(p) for p in P], st, time.perf_counter() - t0


def _job(args):
    key, L, N, J, Delta, h, pbc, state, times = args
    P, st, sec = _oracle_P(L, N, J, Delta, h, pbc, state, times)
    return key, P, st, sec


def _pool(jobs: int):
    # one BLAS thread per worker; spawn, so that no worker inherits a forked runtime
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(jobs)


def _header(f, lines):
    for ln in lines:
        f.write(f"# {ln}\n")


def make_L24(jobs: int):
    import workloads
    c = workloads.config("L24_mixed")
    P, st, sec = _oracle_P(c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"],
                           c["times"])
    with open(os.path.join(HERE, "P_L24_mixed.txt"), "w") as f:
        _header(f, [f"workload L24_mixed: L=24 N_up=12 PBC J=1 Delta=1 h=1.5 (phi: workloads.phases(2)), "
                    "Neel initial state",
                    f"oracle: krylov.return_probability on the CSR Hamiltonian, m=30, tol={ORACLE_TOL:g}",
                    f"oracle run: {st['steps']} Krylov steps, {st['hv']} H.v, {sec:.0f} s on the host",
                    "written by tests/golden/make_golden.py L24",
                    "columns: t P"])
        for t, p in zip(c["times"], P):
            f.write(f"{t!r} {p!r}\n")


def make_L22(jobs: int, hs=("1.5", "0.5", "3")):
    """K = 64 phase ensembles: every realisation of h = 1.5 to t = 10 (27 output times) and
    realisations 0 and 63 to t = 100; every fourth realisation of h = 0.5 and h = 3 to t = 10."""
    import workloads
    todo = []
    for hv in hs:
        c = workloads.config(f"L22_batched_h{hv}")
        n10 = sum(1 for t in c["times"] if t <= 10.0 + 1e-12)
        ks = range(64) if hv == "1.5" else range(0, 64, 4)
        for k in ks:
            full = hv == "1.5" and k in (0, 63)
            times = c["times"] if full else c["times"][:n10]
            todo.append(((hv, k), c["L"], c["n_up"], c["J"], c["Delta"], c["h"][k], c["pbc"], c["state"], times))
    # the long (t to 100) evolutions first, so that they overlap the short ones
    todo.sort(key=lambda a: -len(a[-1]))
    res = {hv: {} for hv in hs}
    t_start = time.time()
    with _pool(jobs) as pool:
        for key, P, st, sec in pool.imap_unordered(_job, todo):
            hv, k = key
            res[hv][k] = (P, st, sec)
            print(f"L22 h={hv} k={k}: {st['steps']} steps, {sec:.0f} s", flush=True)
    for hv in hs:
        c = workloads.config(f"L22_batched_h{hv}")
        tot = sum(v[2] for v in res[hv].values())
        with open(os.path.join(HERE, f"P_L22_batched_h{hv}.txt"), "w") as f:
            _header(f, [f"workload L22_batched_h{hv}: L=22 N_up=11 PBC J=1 Delta=1 h={hv}, K=64 phases "
                        "(workloads.phases(3, 64)), Neel initial state",
                        "realisation k evolved alone by the oracle: krylov.return_probability on the CSR "
                        f"Hamiltonian of row k, m=30, tol={ORACLE_TOL:g}",
                        f"{len(res[hv])} realisations, {tot:.0f} s of host time "
                        f"({time.time() - t_start:.0f} s wall on {jobs} processes)",
                        f"written by tests/golden/make_golden.py L22",
                        "columns: k t P"])
            for k in sorted(res[hv]):
                for t, p in zip(c["times"], res[hv][k][0]):
                    f.write(f"{k} {t!r} {p!r}\n")


def make_L20grad(jobs: int):
    import numpy as np
    import workloads
    c = workloads.config("L20_grad")
    L, N, t = c["L"], c["n_up"], c["times"][0]
    h = np.array(c["h"][0])
    todo = [("P", L, N, c["J"], c["Delta"], list(h), c["pbc"], c["state"], [t])]
    for i in range(L):
        for sgn in (1, -1):
            hh = h.copy()
            hh[i] += sgn * FD_STEP
            todo.append(((i, sgn), L, N, c["J"], c["Delta"], list(hh), c["pbc"], c["state"], [t]))
    for sgn in (1, -1):
        todo.append((("D", sgn), L, N, c["J"], c["Delta"] + sgn * FD_STEP, list(h), c["pbc"], c["state"], [t]))
    res = {}
    t0 = time.time()
    with _pool(jobs) as pool:
        for key, P, st, sec in pool.imap_unordered(_job, todo):
            res[key] = P[0]
    with open(os.path.join(HERE, "grad_L20.txt"), "w") as f:
        _header(f, ["workload L20_grad: L=20 N_up=10 PBC J=1 Delta=1 h=1.0 (phi: workloads.phases(4)), "
                    "Neel initial state, t=10",
                    f"oracle: krylov.return_probability, m=30, tol={ORACLE_TOL:g}; derivatives by central "
                    f"differences with step {FD_STEP:g} (oracle.gradient.central_fd's formula)",
                    f"{len(todo)} oracle evolutions, {time.time() - t0:.0f} s wall on {jobs} processes",
                    "written by tests/golden/make_golden.py L20grad",
                    "columns: name value"])
        f.write(f"P {res['P']!r}\n")
        for i in range(L):
            f.write(f"dP/dh_{i + 1} {(res[(i, 1)] - res[(i, -1)]) / (2 * FD_STEP)!r}\n")
        f.write(f"dP/dDelta {(res[('D', 1)] - res[('D', -1)]) / (2 * FD_STEP)!r}\n")


def make_L30(jobs: int, hops: int = 12):
    from oracle import moments
    import workloads
    for name in ("L30_clean", "L30_qp"):
        c = workloads.config(name)
        t0 = time.time()
        mu, nball = moments.moments(c["L"], c["J"], c["Delta"], c["h"][0], c["pbc"], c["state"], hops)
        sec = time.time() - t0
        rows = []
        for t in c["times"]:
            P, bound = moments.return_probability(mu, t)
            if bound > 1e-12:
                break
            rows.append((t, float(P), float(bound)))
        with open(os.path.join(HERE, f"P_{name}_early.txt"), "w") as f:
            _header(f, [f"workload {name}: L=30 N_up=15 PBC J=1 Delta=1 "
                        f"h={'0 (clean)' if name == 'L30_clean' else '1.5 (phi: workloads.phases(5))'}, "
                        "Neel initial state",
                        f"oracle: moments.moments over the {nball} states within {hops} hops of psi0 "
                        f"(moments mu_0..mu_{2 * hops}), moments.return_probability; {sec:.0f} s",
                        "the output times whose rigorous bound on |P_series - P| is <= 1e-12",
                        "written by tests/golden/make_golden.py L30",
                        "columns: t P bound"])
            for t, P, b in rows:
                f.write(f"{t!r} {P!r} {b!r}\n")


def make_L32(hops: int = 12):
    """The largest split-table sector: L = 32, N_up = 16, the quasiperiodic field of the L = 30
    workload's seed, Neel state; the output times where the series bound is <= 1e-12."""
    from oracle import moments
    import workloads
    L, N = 32, 16
    h = workloads.quasiperiodic_field(L, 1.5, workloads.phases(5)[0])
    state = workloads.neel_state(L)
    t0 = time.time()
    mu, nball = moments.moments(L, 1.0, 1.0, h, True, state, hops)
    sec = time.time() - t0
    with open(os.path.join(HERE, "P_L32_qp_early.txt"), "w") as f:
        _header(f, ["workload L32_qp: L=32 N_up=16 PBC J=1 Delta=1 h=1.5 (phi: workloads.phases(5)), "
                    "Neel initial state",
                    f"oracle: moments.moments over the {nball} states within {hops} hops of psi0 "
                    f"(moments mu_0..mu_{2 * hops}), moments.return_probability; {sec:.0f} s",
                    "the output times whose rigorous bound on |P_series - P| is <= 1e-12",
                    "written by tests/golden/make_golden.py L32",
                    "columns: t P bound"])
        for t in workloads.log_times():
            P, bound = moments.return_probability(mu, t)
            if bound > 1e-12:
                break
            f.write(f"{t!r} {float(P)!r} {float(bound)!r}\n")


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("target", choices=["L24", "L22", "L20grad", "L30", "L32"])
    ap.add_argument("--jobs", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    ap.add_argument("--h", nargs="*", default=None, help="L22: the field amplitudes to run")
    a = ap.parse_args()
    if a.target == "L24":
        make_L24(a.jobs)
    elif a.target == "L22":
        make_L22(a.jobs, tuple(a.h) if a.h else ("1.5", "0.5", "3"))
    elif a.target == "L20grad":
        make_L20grad(a.jobs)
    elif a.target == "L32":
        make_L32()
    else:
        make_L30(a.jobs)
