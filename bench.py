#!/usr/bin/env python
"""Krylov return-probability benchmark on one GB300 (replicas on N GPUs).

Workload: the L = 24, N_up = 12 sector (D = 2,704,156) of the quasiperiodic XXZ chain
(J = 1, Delta = 1, h = 1.5, phi from seed 2), Neel initial state, Krylov m = 30,
P(t) at 40 log-spaced times in [0.1, 100], tol = 1e-10.  One step = one full evolution
to t = 100 through kry_return_probability.  Metric: H.v state-updates per second
(D x number of H.v applications / time), FP64 (complex128) form; the mixed-precision
(complex64 vectors, FP64 coefficients) form is timed beside it with its error.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Krylov H.v state-updates/s (+ % HBM roofline), FP64 vs FP32/batched at set error"
WORKLOAD = "L24_mixed"
HBM_PEAK_FALLBACK = 6800.0
# profiled kernel kinds: pass A's H.v (k_hv) and dots (k_dots<.,0>), pass B's update
# (k_lincomb<.,0>), pass C (the second Gram-Schmidt pass), the small exponential, the combine
KIND_NAMES = ("hv", "dots", "update", "passC", "smallexp", "combine")
KERNEL_OF = {"hv": "k_hv", "dots": "k_dots<.,0>", "update": "k_lincomb<.,0>",
             "passC": "k_dots<.,1> + k_lincomb<.,1>", "smallexp": "k_smallexp", "combine": "k_lincomb<.,2>"}
# vector passes (reads + writes of D-element vectors) per launch at Lanczos index j
PASSES = {"hv": lambda j: 2, "dots": lambda j: j + 2, "update": lambda j: j + 3}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-l30", action="store_true", help="skip the L = 30 complex64 line")
    ap.add_argument("--l30", action="store_true",
                    help="only the L = 30 configuration in full: both fields, complex128 and complex64, e2e")
    ap.add_argument("--l32", action="store_true",
                    help="only the L = 32 sector (D = 601,080,390), complex64, to t = 100")
    ap.add_argument("--no-widened", action="store_true",
                    help="skip the temporal autocorrelation, random-state ensemble and L = 55 ring lines")
    ap.add_argument("--form", default="c128", choices=["c128", "c64", "c64b"],
                    help="precision of the timed region in --kernels-only mode")
    ap.add_argument("--kernels-only", action="store_true",
                    help="FP64 timed region only (no mixed, e2e or CPU legs)")
    ap.add_argument("--ncu-case", choices=["c128", "c64", "c64b", "c64l", "c128e"],
                    help="one Krylov step (m = 30, one output time) of the workload, nothing else: "
                         "a short, fixed launch sequence for ncu captures")
    ap.add_argument("--ncu-L", type=int, default=0,
                    help="ncu case: chain length L (N_up = L/2, h = 1.5, phi from seed 5; default: the workload)")
    ap.add_argument("--ncu-m", type=int, default=0, help="ncu case: Krylov dimension (default 30)")
    ap.add_argument("--ncu-shape", default=None, help="ncu case: launch shape, five comma-separated ints")
    a = ap.parse_args()
    if a.kernels_only:
        a.no_mixed = a.no_cpu_baseline = a.no_batched = a.no_widened = a.no_l30 = True
    return a


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return None


# ---------------------------------------------------------------- clocks during the run

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.rows, self.proc, self.thr = index, [], None, None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return self

        def reader():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])
        self.thr = threading.Thread(target=reader, daemon=True)
        self.thr.start()
        return self

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thr:
            self.thr.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 7 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 7 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 7
                          for i in range(4) if r[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


# ---------------------------------------------------------------- distributed helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def aggregate(units: float, seconds: float, world: int):
    """Whole-job throughput of independent replicas: sum of units / max of times."""
    if world == 1:
        return units, seconds
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- traffic from ncu

def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kry_hv.cu", "kry_batched.cu", "kry_device.cuh", "kry_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1704_02770_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind, algo_bytes_per_launch):
    """DRAM bytes per (average) launch of `kind`: the committed ncu capture of one launch,
    scaled by algorithmic bytes to the average launch; None if the kernel sources no
    longer hash to the value recorded with the capture."""
    path = os.path.join(ROOT, "profiles", "traffic_vector_kernels.txt")
    try:
        rows = dict(line.strip().split("=", 1) for line in open(path)
                    if "=" in line and not line.startswith("#"))
    except OSError:
        return None
    if rows.get("source_hash") != kernel_source_hash():
        return None
    dram, algo = rows.get(f"{kind}_captured_dram_bytes"), rows.get(f"{kind}_captured_algo_bytes")
    if not dram or not algo:
        return None
    return float(dram) / float(algo) * algo_bytes_per_launch


def fp64_flops(kind, D, m, krylov_steps, L, N, pbc):
    """Algorithmic FP64 flops of all launches of `kind` over `krylov_steps` full steps.

    Per element: a complex multiply-add is 8 flops, |w|^2 is 4.  At Lanczos index j the H.v
    row costs 2 flops per gathered neighbour and 10 for the diagonal term and the J/2 scale;
    the dots j+1 complex multiply-adds and ||u||^2; the update j+1 complex multiply-adds and
    ||w||^2 (the second Gram-Schmidt pass runs only when flagged and is counted under pass C).
    The average number of neighbours is 2N(L-N)/(L-1) on a ring, 2N(L-N)/L open."""
    nb = 2.0 * N * (L - N) / ((L - 1) if pbc else L)
    if kind == "hv":
        per = m * (10 + 2 * nb)
    elif kind in ("dots", "update"):
        per = sum(8 * (j + 1) + 4 for j in range(m))
    else:
        return 0.0
    return per * D * krylov_steps


def fp64_pipe_ops(kind, D, m, krylov_steps, L, N, pbc):
    """FP64 pipe instructions (per thread-element) of all launches of `kind`: a fused
    multiply-add, a multiply and an add each occupy the pipe once, so the adds of the H.v
    (two per gathered neighbour) cost as much pipe time as multiply-adds.  At index j: the
    H.v 2 per neighbour and 7 for the diagonal term and the scales; the dots 4 per vector
    (j+1) and 2 for ||u||^2; the update 4 per vector (j+1) and 2 for ||w||^2."""
    nb = 2.0 * N * (L - N) / ((L - 1) if pbc else L)
    if kind == "hv":
        per = m * (7 + 2 * nb)
    elif kind in ("dots", "update"):
        per = sum(4 * (j + 1) + 2 for j in range(m))
    else:
        return 0.0
    return per * D * krylov_steps


MEASURED_FP64 = {}   # filled by run_ours from kry_measure_peaks on this GPU


def roofline(prof, form, D, c, L, N, clocks, traffic_key=None):
    """Roofline of the dominant kernel kind over a profiled timed region.

    complex128: every element costs FP64 arithmetic, and GB300's FP64 pipe saturates before
    HBM, so the bound is the ALU, against the FP64 multiply-add rate measured on this GPU in
    the same run (kry_measure_peaks); the HBM view is given beside it.  complex64: the bound is
    HBM."""
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks and "hbm_gbs" in peaks else HBM_PEAK_FALLBACK
    dom = max(("hv", "dots", "update"), key=lambda k: prof[k]["ms"])   # the dominant kernel
    per = {k: {"ms": round(prof[k]["ms"], 3),
               "GBps": (prof[k]["bytes"] / (prof[k]["ms"] * 1e6)) if prof[k]["ms"] else None,
               "launches": prof[k]["launches"]} for k in KIND_NAMES}
    ach = prof[dom]["bytes"] / (prof[dom]["ms"] * 1e6)
    nl = max(prof[dom]["launches"], 1)
    hbm = {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
           "peak_source": "measured" if peaks else "fallback"}
    if traffic_key is None:
        traffic_key = "" if form == "c128" else "c64_"
    tr = ncu_traffic(traffic_key + dom, prof[dom]["bytes"] / nl)
    share = {k: prof[k]["ms"] / sum(prof[q]["ms"] for q in KIND_NAMES) for k in KIND_NAMES}
    if form == "c128":
        # Krylov steps that did work (replays after the last output time are no-ops):
        # recovered from the kernel's algorithmic bytes, PASSES[dom](j) vectors at index j
        per_step = sum(PASSES[dom](j) for j in range(c["m"])) * D * 16
        steps = prof[dom]["bytes"] / per_step
        fl = fp64_flops(dom, D, c["m"], steps, L, N, c["pbc"])
        mhz = clocks["sm_mhz"] or 2070.0
        if MEASURED_FP64.get("tflops"):
            fp64_peak = MEASURED_FP64["tflops"]
            src = ("measured in this run (kry_measure_peaks: FP64 multiply-add chains on every SM, "
                   f"{MEASURED_FP64['tflops']:.3f} TFLOP/s; nominal 152 SMs x 4 flop/clk x {mhz:.0f} MHz = "
                   f"{152 * 4 * mhz * 1e6 / 1e12:.3f})")
        else:
            fp64_peak = 152 * 4 * mhz * 1e6 / 1e12
            src = "nominal: 152 SMs x 4 flop/clk x median SM clock (no measurement)"
        ach_fl = fl / (prof[dom]["ms"] * 1e-3) / 1e12
        ops = fp64_pipe_ops(dom, D, c["m"], steps, L, N, c["pbc"])
        ach_ops = ops / (prof[dom]["ms"] * 1e-3) / 1e12
        ops_peak = fp64_peak / 2.0
        pipe = {"achieved": ach_ops, "peak": ops_peak, "unit": "T FP64 instr/s", "frac": ach_ops / ops_peak,
                "peak_source": "the measured multiply-add rate, one instruction each",
                "note": "adds occupy the pipe like multiply-adds; the H.v is add-heavy"}
        return {"bound": "alu", "kernel": KERNEL_OF[dom], "kind": dom, "achieved": ach_fl, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": ach_fl / fp64_peak,
                "peak_source": src,
                "traffic": tr, "algo_bytes_per_launch": prof[dom]["bytes"] / nl,
                "fp64_pipe_view": pipe,
                "hbm_view": hbm, "per_kind": per, "kernel_time_share": share,
                "profiled_region_s": prof.get("_sec"), "timing": TIMING_NOTE}
    return dict(bound="hbm", kernel=KERNEL_OF[dom], kind=dom, traffic=tr, algo_bytes_per_launch=prof[dom]["bytes"] / nl,
                per_kind=per, kernel_time_share=share, profiled_region_s=prof.get("_sec"),
                timing=TIMING_NOTE, **hbm)


TIMING_NOTE = ("per-kind CUDA-event times from a second timed region of the same evolutions with "
               "event nodes captured between the kernels of the step graph; value comes from the "
               "uninstrumented region")


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch

    import paper_1704_02770_gb300 as kry
    import workloads

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    kry.load()
    f64, f32 = kry.measure_peaks()
    MEASURED_FP64.update(tflops=f64, fp32_tflops=f32)
    c = workloads.config(args.workload)
    L, N, times = c["L"], c["n_up"], c["times"]
    B = kry.Basis(L, N)
    H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
    D = B.dim
    stream = torch.cuda.current_stream()

    def timed(dtype, tol, profile, Hx=None, cx=None, warmup=None, steps=None):
        """Time n_steps evolutions (the value: no instrumentation in the graph); with
        `profile`, time them once more with CUDA event nodes captured between the kernels
        of the step graph, for the per-kernel times of the roofline."""
        Hx = H if Hx is None else Hx
        cx = c if cx is None else cx
        n_warm = args.warmup if warmup is None else warmup
        n_steps = args.steps if steps is None else steps
        # launch shape chosen by the autotuner on a short probe of this workload
        tune[f"{dtype}_K{Hx.K}"] = Hx.autotune(cx["state"], 1.0, dtype=dtype)

        def evolve(dt, tl):
            return Hx.return_probability(cx["state"], cx["times"], m=cx["m"], tol=tl, dtype=dt)

        def region():
            barrier(world)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            hv = launches = 0
            P = st = None
            e0.record(stream)
            for _ in range(n_steps):
                P, st = evolve(dtype, tol)
                hv += st["n_hv"]
                launches += st["n_launches"]
            e1.record(stream)
            torch.cuda.synchronize()
            barrier(world)
            return e0.elapsed_time(e1) / 1e3, hv, launches, P, st

        for _ in range(n_warm):
            evolve(dtype, tol)
        sec, hv, launches, P, st = region()
        prof = None
        if profile:
            Hx.profile(True)
            evolve(dtype, tol)          # captures the instrumented graph
            Hx.profile(True)            # and drops its counts
            sec_p, _, _, _, _ = region()
            prof = Hx.profile_read()
            prof["_sec"] = sec_p
            Hx.profile(False)
        return sec, hv, launches, P, st, prof

    tune = {}
    if args.kernels_only and args.form == "c64b":
        # batched K = 64 ensemble alone (for kernel captures)
        cb = workloads.config("L22_batched_h1.5")
        Bb = kry.Basis(cb["L"], cb["n_up"])
        Hb = kry.Hamiltonian(Bb, cb["J"], cb["Delta"], cb["h"], pbc=cb["pbc"])
        clk = ClockSampler(local).start()
        secb, hvb, lb, Pb, stb, profb = timed("c64", 1e-7, profile=True, Hx=Hb, cx=cb)
        clocks = clk.stop()
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": Bb.dim * Hb.K * hvb / secb, "unit": "state-updates/s",
                              "ms_per_step": 1e3 * secb / args.steps, "workload": "L22_batched_h1.5 K=64 c64",
                              "roofline": roofline(profb, "c64", Bb.dim * Hb.K, cb, cb["L"], cb["n_up"], clocks,
                                                   traffic_key="b64_"),
                              "clocks": clocks}))
        return
    form = args.form if args.kernels_only else "c128"
    clk = ClockSampler(local).start()
    sec, hv, launches, P128, st128, prof = timed(form, c["tol"] if form == "c128" else 1e-7,
                                                 profile=True)
    clocks = clk.stop()
    units, sec_all = aggregate(D * hv, sec, world)
    value = units / sec_all
    out = {"metric": METRIC, "value": value, "unit": "state-updates/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * sec_all / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "c128 (fp64)" if form == "c128" else "c64 vectors, fp64 coefficients",
           "data": "synthetic (seeded quasiperiodic field, Neel state)"}
    cfg = {"workload": f"{args.workload}: L={L} N_up={N} D={D} PBC J=1 Delta=1 h=1.5 "
                       f"m={c['m']} tol={c['tol']:g} 40 log times in [0.1,100]",
           "krylov_steps_per_step": st128["n_krylov_steps"], "hv_per_step": st128["n_hv"],
           "second_passes_per_step": st128["n_second_pass"],
           "parallelism": f"replicas x{world}",
           "l2": "no flush: each step sweeps a 1.4 GB Krylov basis (31 vectors x 43 MB) > 129 MB L2"}
    # roofline of the dominant kernel kind, from CUDA events inside the timed region
    out["roofline"] = roofline(prof, form, D, c, L, N, clocks)
    out["gpu_launches"] = launches
    out["clocks"] = clocks
    # mixed precision at the same stated accuracy target
    if not args.no_mixed:
        sec64, hv64, l64, P64, st64, prof64 = timed("c64", 1e-7, profile=True)
        u64, s64 = aggregate(D * hv64, sec64, world)
        out["mixed"] = {"dtype": "c64 vectors, fp64 coefficients", "value": u64 / s64,
                        "unit": "state-updates/s", "ms_per_step": 1e3 * s64 / args.steps,
                        "speedup_vs_fp64": (u64 / s64) / value,
                        "max_abs_dP_vs_fp64": float(np.max(np.abs(P64 - P128))),
                        "tol": 1e-7, "roofline": roofline(prof64, "c64", D, c, L, N, clocks)}
        out["gpu_launches"] += l64
        # the FP64 form at the same stated accuracy (tol 1e-7): time to solution of both forms
        sec7, hv7, l7, P7, st7, _ = timed("c128", 1e-7, profile=False)
        u7, s7 = aggregate(D * hv7, sec7, world)
        out["gpu_launches"] += l7
        out["fp64_same_tol"] = {"tol": 1e-7, "value": u7 / s7, "unit": "state-updates/s",
                                "ms_per_step": 1e3 * s7 / args.steps, "krylov_steps_per_step": st7["n_krylov_steps"],
                                "max_abs_dP_vs_fp64_tol_1e-10": float(np.max(np.abs(P7 - P128)))}
        out["mixed"]["time_to_solution_speedup_vs_fp64_same_tol"] = s7 / s64
        out["mixed"]["krylov_steps_per_step"] = st64["n_krylov_steps"]
        # complex128 vectors with float-float arithmetic on the FP32 pipe, at the FP64 tol
        sece, hve, le, Pe, ste, profe = timed("c128e", c["tol"], profile=True)
        ue, se_ = aggregate(D * hve, sece, world)
        out["gpu_launches"] += le
        out["fp64_emulated"] = {
            "dtype": "complex128 in and out; float-float vectors and arithmetic on the FP32 pipe (about 48 bits)",
            "value": ue / se_, "unit": "state-updates/s", "ms_per_step": 1e3 * se_ / args.steps,
            "tol": c["tol"], "speedup_vs_fp64": (ue / se_) / value,
            "krylov_steps_per_step": ste["n_krylov_steps"],
            "max_abs_dP_vs_fp64": float(np.max(np.abs(Pe - P128))),
            "roofline": roofline(profe, "c128e", D, c, L, N, clocks, traffic_key="e_")}
    # batched realisations: the K = 64 phase ensemble of L = 22 in one interleaved launch
    if not args.no_batched:
        cb = workloads.config("L22_batched_h1.5")
        Bb = kry.Basis(cb["L"], cb["n_up"])
        Hb = kry.Hamiltonian(Bb, cb["J"], cb["Delta"], cb["h"], pbc=cb["pbc"])
        Kb = Hb.K
        # one warm-up and one timed evolution: a full 64-phase evolution runs for tens of seconds
        secb, hvb, lb, Pb, stb, profb = timed("c64", 1e-7, profile=True, Hx=Hb, cx=cb, warmup=1, steps=1)
        ub, sb = aggregate(Bb.dim * Kb * hvb, secb, world)
        out["batched"] = {
            "workload": f"L22_batched_h1.5: L=22 N_up=11 D={Bb.dim} K={Kb} phases, h=1.5, "
                        "40 log times in [0.1,100], tol 1e-7",
            "dtype": "c64 vectors [D][K] interleaved, fp64 coefficients",
            "value": ub / sb, "unit": "state-updates/s (D x K x H.v / s)",
            "ms_per_step": 1e3 * sb, "warmup": 1, "steps": 1,
            "krylov_steps_per_step": stb["n_krylov_steps"],
            "speedup_vs_fp64": (ub / sb) / value,
            "disorder_avg_P_last": float(np.mean(Pb[-1])),
            "roofline": roofline(profb, "c64", Bb.dim * Kb, cb, cb["L"], cb["n_up"], clocks, traffic_key="b64_")}
        out["gpu_launches"] += lb
        # time to solution against the FP64 form at the same tol: realisations 0 and 1 evolved
        # one by one in complex128, scaled to the 64 of the ensemble
        t64 = 0.0
        for k in (0, 1):
            Hk = kry.Hamiltonian(Bb, cb["J"], cb["Delta"], cb["h"][k], pbc=cb["pbc"])
            Hk.return_probability(cb["state"], [0.1], dtype="c128", tol=1e-7)   # capture
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, stk = Hk.return_probability(cb["state"], cb["times"], dtype="c128", tol=1e-7)
            e1.record(stream)
            torch.cuda.synchronize()
            t64 += e0.elapsed_time(e1) / 1e3
            out["gpu_launches"] += stk["n_launches"]
            del Hk
        out["batched"]["time_to_solution_speedup_vs_fp64_same_tol"] = (t64 * Kb / 2.0) / sb
        out["batched"]["fp64_same_tol_note"] = ("64 single complex128 evolutions at tol 1e-7, extrapolated from "
                                                f"realisations 0 and 1 ({t64 / 2:.2f} s each)")
        # the same ensemble at the FP64 bar (tol 1e-10) with float-float vectors, to t = 10,
        # against single complex128 evolutions at the same tol
        cb10 = dict(cb, times=cb["times"][:27])
        sece, hve, le, Pe, ste, _ = timed("c128e", 1e-10, profile=False, Hx=Hb, cx=cb10, warmup=1, steps=1)
        ue, se_ = aggregate(Bb.dim * Kb * hve, sece, world)
        out["gpu_launches"] += le
        t128 = 0.0
        for k in (0, 1):
            Hk = kry.Hamiltonian(Bb, cb["J"], cb["Delta"], cb["h"][k], pbc=cb["pbc"])
            Hk.return_probability(cb["state"], [0.1], dtype="c128", tol=1e-10)   # capture
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, stk = Hk.return_probability(cb["state"], cb10["times"], dtype="c128", tol=1e-10)
            e1.record(stream)
            torch.cuda.synchronize()
            t128 += e0.elapsed_time(e1) / 1e3
            out["gpu_launches"] += stk["n_launches"]
            del Hk
        out["batched_fp64_emulated"] = {
            "workload": f"L22_batched_h1.5 to t = 10 (27 output times), K={Kb}, tol 1e-10",
            "dtype": "complex128 in and out; float-float vectors [D][K] and arithmetic on the FP32 pipe",
            "value": ue / se_, "unit": "state-updates/s (D x K x H.v / s)", "ms_per_step": 1e3 * se_,
            "krylov_steps_per_step": ste["n_krylov_steps"], "second_passes": ste["n_second_pass"],
            "time_to_solution_speedup_vs_fp64_same_tol": (t128 * Kb / 2.0) / se_,
            "fp64_same_tol_note": ("64 single complex128 evolutions at tol 1e-10 to t = 10, extrapolated from "
                                   f"realisations 0 and 1 ({t128 / 2:.3f} s each)")}
    if not args.no_widened:
        try:
            out["widened"] = widened(args, kry, workloads, H, c, D, out, world)
            out["gpu_launches"] += out["widened"].pop("_launches")
        except Exception as e:   # the widened rows must not cost the headline line
            out["widened"] = {"error": f"{type(e).__name__}: {e}"}
    if not args.no_batched:
        del Hb, Bb
    if not args.no_l30:
        try:
            out["l30"] = l30_leg(kry, workloads, world, tune, clocks, full=False)
            out["gpu_launches"] += out["l30"].pop("_launches")
        except Exception as e:   # the L = 30 line must not cost the headline line
            out["l30"] = {"error": f"{type(e).__name__}: {e}"}
    cfg["autotune"] = {k: {"shape": v["shape"], "probe_ms": v["candidates"],
                           "default_shape_ms": next((ms for s_, ms in v["candidates"] if s_ == [0, 0, 0, 2, 0]), None)}
                       for k, v in tune.items()}
    cfg["measured_peaks"] = {"fp64_tflops": MEASURED_FP64.get("tflops"), "fp32_tflops": MEASURED_FP64.get("fp32_tflops"),
                             "how": "kry_measure_peaks: independent multiply-add chains on every SM, CUDA events"}
    out["config"] = cfg
    if args.kernels_only:
        if rank == 0:
            print(json.dumps(out))
        return
    # end to end through the public API with host buffers: psi0 from pinned memory every step
    psi_host = torch.zeros(D, dtype=torch.complex128).pin_memory()
    r0 = B.rank(torch.tensor([c["state"]], dtype=torch.int64, device="cuda")).item()
    psi_host[r0] = 1.0
    x = torch.empty(D, dtype=torch.complex128, device="cuda")
    for _ in range(max(1, args.warmup // 2)):
        x.copy_(psi_host, non_blocking=True)
        H.evolve(x, times, m=c["m"], tol=c["tol"])
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hv_e = 0
    e0.record(stream)
    for _ in range(args.steps):
        x.copy_(psi_host, non_blocking=True)
        Pe, ste = H.evolve(x, times, m=c["m"], tol=c["tol"])
        hv_e += ste["n_hv"]
        out["gpu_launches"] += ste["n_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    ue, se = aggregate(D * hv_e, e0.elapsed_time(e1) / 1e3, world)
    out["e2e"] = {"value": ue / se, "unit": "state-updates/s",
                  "h2d_bytes_per_step": D * 16, "d2h_bytes_per_step": len(times) * 8,
                  "api": "Hamiltonian.evolve (kry_evolve) on a psi0 copied from pinned host memory",
                  "max_abs_dP_vs_basis_state_call": float(np.max(np.abs(Pe - P128)))}
    out["config"] = cfg
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, cores=1)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def l32_config(workloads):
    """The largest sector of the split rank tables: L = 32, N_up = 16 (D = 601,080,390), the
    quasiperiodic field of the L = 30 workload's seed (h = 1.5), Neel state, m = 30, the 40
    log times."""
    c = dict(workloads.config("L30_qp"))
    c.update(name="L32_qp", L=32, n_up=16, state=workloads.neel_state(32),
             h=[workloads.quasiperiodic_field(32, 1.5, workloads.phases(5)[0])])
    return c


def l30_leg(kry, workloads, world, tune, clocks, full=False, l32=False):
    """The largest single-GPU configuration: L = 30, N_up = 15 (D = 155,117,520), Neel state,
    m = 30, 40 log times to t = 100.  Default: the quasiperiodic field (h = 1.5) in complex64
    (42 GB of Krylov workspace), one evolution after a short capture run.  full: both fields,
    complex128 (84 GB), complex64 and complex128 with float-float vectors (84 GB), and the
    end-to-end call with psi0 copied from pinned host memory.  One evolution per case, with CUDA event nodes between the kernels for the
    per-kind times (at this size their overhead is far below a kernel's duration)."""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    res = {"workload": "L=30 N_up=15 D=155117520 PBC J=1 Delta=1, Neel psi0, m=30, 40 log times in [0.1,100]",
           "timing": "one evolution per case after a capture run to t=0.1; per-kind times from event "
                     "nodes in the same run"}
    launches = 0
    Ps = {}
    cases = ([("L30_qp", "c64")] if not full else
             [(n, d) for n in ("L30_clean", "L30_qp") for d in ("c64", "c128", "c128e")])
    if l32:   # complex64 only: 31 vectors of 4.8 GB (complex128 would need 298 GB)
        cases = [("L32_qp", "c64")]
        res["workload"] = ("L=32 N_up=16 D=601080390 PBC J=1 Delta=1 h=1.5 (phi: phases(5)), Neel psi0, m=30, "
                           "40 log times in [0.1,100]")
    B = None
    for name, dt in cases:
        c = l32_config(workloads) if name == "L32_qp" else workloads.config(name)
        if B is None:
            B = kry.Basis(c["L"], c["n_up"])
        D = B.dim
        H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
        # launch shape tuned on this sector (one Krylov step per probe)
        t_ = H.autotune(c["state"], 0.02, dtype=dt, reps=1)
        res.setdefault("autotune", {})[f"{name}_{dt}"] = t_
        tol = 1e-7 if dt == "c64" else c["tol"]
        H.return_probability(c["state"], [0.1], m=c["m"], tol=tol, dtype=dt)
        H.profile(True)
        H.return_probability(c["state"], [0.1], m=c["m"], tol=tol, dtype=dt)   # instrumented capture
        H.profile(True)
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        P, st = H.return_probability(c["state"], c["times"], m=c["m"], tol=tol, dtype=dt)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        prof = H.profile_read()
        prof["_sec"] = sec
        H.profile(False)
        u, s = aggregate(D * st["n_hv"], sec, world)
        launches += st["n_launches"]
        Ps[(name, dt)] = np.asarray(P, dtype=np.float64)
        line = {"dtype": dt, "tol": tol, "value": u / s, "unit": "state-updates/s", "ms_per_step": 1e3 * s,
                "krylov_steps": st["n_krylov_steps"], "hv": st["n_hv"], "second_passes": st["n_second_pass"],
                "P_first": float(P[0]), "P_last": float(P[-1]),
                "roofline": roofline(prof, dt, D, c, c["L"], c["n_up"], clocks, traffic_key="l30_")}
        res[f"{name}_{dt}"] = line
        if full and name == "L30_qp" and dt == "c64":
            # end to end: psi0 from pinned host memory through kry_evolve, P back to the host
            psi_h = torch.zeros(D, dtype=torch.complex64).pin_memory()
            r0 = B.rank(torch.tensor([c["state"]], dtype=torch.int64, device="cuda")).item()
            psi_h[r0] = 1.0
            x = torch.empty(D, dtype=torch.complex64, device="cuda")
            torch.cuda.synchronize()
            e0.record(stream)
            x.copy_(psi_h, non_blocking=True)
            Pe, ste = H.evolve(x, c["times"], m=c["m"], tol=tol)
            e1.record(stream)
            torch.cuda.synchronize()
            ue, se = aggregate(D * ste["n_hv"], e0.elapsed_time(e1) / 1e3, world)
            launches += ste["n_launches"]
            line["e2e"] = {"value": ue / se, "unit": "state-updates/s", "h2d_bytes_per_step": D * 8,
                           "d2h_bytes_per_step": len(c["times"]) * 8,
                           "max_abs_dP_vs_basis_state_call": float(np.max(np.abs(Pe - P)))}
            del x, psi_h
        H.close()
        del H
        torch.cuda.empty_cache()
    if full:
        for name in ("L30_clean", "L30_qp"):
            a = res.get(f"{name}_c128")
            for dt in ("c64", "c128e"):
                b = res.get(f"{name}_{dt}")
                if a and b:
                    b["speedup_vs_fp64"] = b["value"] / a["value"]
                    b["time_to_solution_speedup_vs_fp64"] = a["ms_per_step"] / b["ms_per_step"]
                    b["max_abs_dP_vs_fp64_40_times"] = float(np.max(np.abs(Ps[(name, dt)] - Ps[(name, "c128")])))
    res["_launches"] = launches
    return res


def widened(args, kry, workloads, H, c, D, out, world):
    """Throughput of the rows widened past the hot path, each from CUDA events around whole
    calls of its public entry point (inputs resident, one warm-up call first):
      autocorrelation   kry_autocorrelation (P and C(t)) on the L = 24 workload, complex64
      ensemble          kry_return_probability_states: L = 22, K = 64 random basis states
                        with their own phases, complex64, 40 log times in [0.1, 10]
      list_basis        the L = 55 Fibonacci ring at N = 5 (D = 3,478,761, sorted-list basis,
                        Aubry-Andre field at lambda = 2), complex128 and complex64"""
    import numpy as np
    import torch
    stream = torch.cuda.current_stream()
    launches = 0

    def clock(fn, n_warm, n_steps):
        nonlocal launches
        for _ in range(n_warm):
            fn()
        barrier(world)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hv = 0
        res = None
        e0.record(stream)
        for _ in range(n_steps):
            res = fn()
            hv += res[-1]["n_hv"]
            launches += res[-1]["n_launches"]
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        return e0.elapsed_time(e1) / 1e3, hv, res

    w = {}
    # temporal autocorrelation on the L = 24 workload (complex64)
    sec, hv, (C, P, st) = clock(lambda: H.autocorrelation(c["state"], c["times"], m=c["m"], tol=1e-7,
                                                          dtype="c64"), 1, args.steps)
    u, s = aggregate(D * hv, sec, world)
    ref = out.get("mixed", {}).get("value")
    w["autocorrelation"] = {
        "workload": "L24_mixed, complex64, P and C(t) at the 40 log times (tol 1e-7)",
        "value": u / s, "unit": "state-updates/s", "ms_per_step": 1e3 * s / args.steps,
        "time_vs_P_only": (ref / (u / s)) if ref else None,
        "C_last": float(C[-1]), "gamma_fit_t10_100": kry.decay_exponent(c["times"], C, 10.0, 100.0)[0]}
    # random-initial-state ensemble: L = 22, K = 64
    cb = workloads.config("L22_batched_h1.5")
    Kb = len(cb["h"])
    Bb = kry.Basis(cb["L"], cb["n_up"])
    Hb = kry.Hamiltonian(Bb, cb["J"], cb["Delta"], cb["h"], pbc=cb["pbc"])
    states = workloads.random_basis_states(cb["L"], cb["n_up"], 6, Kb)
    tb = workloads.log_times(40, 0.1, 10.0)
    sec, hv, (Pb, Cb, st) = clock(lambda: Hb.return_probability_states(states, tb, m=cb["m"], tol=1e-7,
                                                                        dtype="c64", autocorrelation=True), 1, 1)
    u, s = aggregate(Bb.dim * Kb * hv, sec, world)
    w["ensemble"] = {
        "workload": f"L=22 N_up=11 D={Bb.dim} K={Kb}: random basis states (seed 6), phases of "
                    "L22_batched_h1.5, 40 log times in [0.1,10], P and C, tol 1e-7",
        "dtype": "c64 vectors [D][K], fp64 coefficients", "value": u / s,
        "unit": "state-updates/s (D x K x H.v / s)", "ms_per_step": 1e3 * s, "steps": 1,
        "ensemble_avg_C_last": float(np.mean(Cb[-1]))}
    del Hb, Bb
    # the L = 55 Fibonacci ring, N = 5, on the sorted-list basis
    L5, N5 = 55, 5
    h5 = workloads.aubry_andre_field(L5, 2.0, 1.0, workloads.phases(7)[0])
    st5 = sum(1 << (11 * i) for i in range(N5))
    B5 = kry.Basis(L5, N5)
    H5 = kry.Hamiltonian(B5, 1.0, 1.0, h5)
    lb = {"workload": f"L=55 ring, beta=34/55, N_up=5, D={B5.dim}, Aubry-Andre lambda=2 (phi seed 7), "
                      "Delta=1, psi0 = sites 1,12,23,34,45, m=30, 40 log times in [0.1,100]",
          "basis": "sorted list (Alg. 2), combinadic ranks"}
    for dt, tl in (("c128", 1e-10), ("c64", 1e-7)):
        H5.autotune(st5, 1.0, dtype=dt)
        sec, hv, (P5, st) = clock(lambda: H5.return_probability(st5, c["times"], m=30, tol=tl, dtype=dt), 1, 1)
        u, s = aggregate(B5.dim * hv, sec, world)
        H5.profile(True)
        H5.return_probability(st5, c["times"], m=30, tol=tl, dtype=dt)
        pr = H5.profile_read()
        H5.profile(False)
        lb[dt] = {"value": u / s, "unit": "state-updates/s", "ms_per_step": 1e3 * s,
                  "krylov_steps": st["n_krylov_steps"],
                  "GBps_by_kind": {k: (v["bytes"] / (v["ms"] * 1e6) if v["ms"] else None) for k, v in pr.items()}}
    w["list_basis"] = lb
    del H5, B5
    w["_launches"] = launches
    return w


# ---------------------------------------------------------------- CPU oracle

def oracle_sample(workload: str):
    """One Krylov step (m = 30 Arnoldi with CGS2 and one Pade exponential) of the workload
    with the CPU oracle, as it stands.  Returns (state-updates, seconds, D)."""
    import numpy as np

    from oracle import basis as ob
    from oracle import krylov, pade
    import workloads

    c = workloads.config(workload)
    H = ob.CSR(c["L"], c["n_up"], c["J"], c["Delta"], c["h"][0], c["pbc"])
    psi = krylov.basis_vector(H.D, ob.lookup(H.basis, c["state"]))
    t0 = time.perf_counter()
    V, Hb, me = krylov.arnoldi_cgs2(H.matvec, psi, c["m"], H.norm_inf())
    A = np.zeros((me + 1, me + 1), complex)
    A[:me, :me] = -1j * 0.5 * Hb[:me, :me]
    A[me, me - 1] = -1j * 0.5 * Hb[me, me - 1]
    E = pade.expm(A)
    _ = E[:me, 0] @ V[:me]
    sec = time.perf_counter() - t0
    return H.D * me, sec, H.D


def cpu_baseline(workload: str, cores: int = 1):
    env = dict(os.environ, OMP_NUM_THREADS=str(cores), OPENBLAS_NUM_THREADS=str(cores),
               MKL_NUM_THREADS=str(cores))
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "u,s,D=bench.oracle_sample(%r); print(json.dumps([u,s,D]))" % (ROOT, workload))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    u, s, D = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": u / s, "unit": "state-updates/s", "cores": cores, "kind": "oracle",
            "sample": f"one Krylov step (m=30 Arnoldi+CGS2, Pade exp) of {workload}, D={D}, "
                      f"{s:.1f} s on {cores} host thread(s)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"   # before numpy loads: the oracle runs on one host thread
    samples = []
    for i in range(args.warmup + args.steps):
        u, s, D = oracle_sample(args.workload)
        if i >= args.warmup:
            samples.append((u, s))
    units = sum(u for u, _ in samples)
    sec = sum(s for _, s in samples)
    v = units / sec
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "state-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec / max(len(samples), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128)",
        "data": "synthetic (seeded quasiperiodic field, Neel state)",
        "config": {"workload": args.workload,
                   "step": "one Krylov step (m=30) of the CPU oracle, a bounded sample"},
        "cpu_baseline": {"value": v, "unit": "state-updates/s", "kind": "oracle",
                         "cores": 1,
                         "sample": "one Krylov step (m=30 Arnoldi+CGS2, Pade exp) per step"},
        "e2e": {"value": v, "unit": "state-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def run_ncu_case(args):
    """One Krylov step of the workload in the given precision, with no autotuning and no
    warm-up, so that a kernel's launch index is known: per Lanczos index j the launches
    are k_hv, k_dots (pass A), k_lincomb (pass B), k_dots, k_lincomb (pass C, no-ops unless
    flagged), then the small exponential and the combine.  c64b: the batched K = 64
    ensemble of L = 22 in complex64.  c64l: the L = 55, N = 5 ring (sorted-list basis)."""
    import numpy as np
    import torch

    import paper_1704_02770_gb300 as kry
    import workloads

    kry.load()
    torch.cuda.set_device(0)
    if args.ncu_case == "c64l":   # the L = 55, N = 5 ring on the sorted-list basis
        B = kry.Basis(55, 5)
        H = kry.Hamiltonian(B, 1.0, 1.0, workloads.aubry_andre_field(55, 2.0, 1.0, workloads.phases(7)[0]))
        H.profile(2)
        P, st = H.return_probability(sum(1 << (11 * i) for i in range(5)), [0.5], m=30, tol=1e-7, dtype="c64")
        torch.cuda.synchronize()
        print(json.dumps({"ncu_case": "c64l", "workload": "L55 N5 ring", "krylov_steps": st["n_krylov_steps"],
                          "hv": st["n_hv"], "P": float(np.asarray(P).ravel()[0])}))
        return
    batched = args.ncu_case == "c64b"   # the K = 64 phase ensemble of L = 22
    c = workloads.config("L22_batched_h1.5" if batched else args.workload)
    if args.ncu_L and not batched:
        L = args.ncu_L
        c = dict(c, name=f"L{L} qp", L=L, n_up=L // 2, state=workloads.neel_state(L),
                 h=[workloads.quasiperiodic_field(L, 1.5, workloads.phases(5)[0])])
    m = args.ncu_m or c["m"]
    B = kry.Basis(c["L"], c["n_up"])
    H = kry.Hamiltonian(B, c["J"], c["Delta"], c["h"] if batched else c["h"][0], pbc=c["pbc"])
    dt = "c64" if batched else args.ncu_case
    H.profile(2)   # no conditional nodes: ncu cannot see kernels in graphs that have them
    if args.ncu_shape:
        H.set_shape([int(x) for x in args.ncu_shape.split(",")], dt)
    P, st = H.return_probability(c["state"], [0.5], m=m, tol=1e-7, dtype=dt)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "workload": c["name"], "krylov_steps": st["n_krylov_steps"],
                      "hv": st["n_hv"], "P": float(np.asarray(P).ravel()[0])}))


def run_l30(args):
    """python bench.py --l30: the L = 30 configuration in full (one JSON line); --l32: the
    L = 32 sector in complex64."""
    import torch

    import paper_1704_02770_gb300 as kry
    import workloads

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    kry.load()
    f64, f32 = kry.measure_peaks()
    MEASURED_FP64.update(tflops=f64, fp32_tflops=f32)
    # launch shapes from short probes of the L = 24 workload
    c = workloads.config("L24_mixed")
    H24 = kry.Hamiltonian(kry.Basis(c["L"], c["n_up"]), c["J"], c["Delta"], c["h"][0], pbc=c["pbc"])
    tune = {f"{dt}_K1": H24.autotune(c["state"], 1.0, dtype=dt) for dt in ("c128", "c64")}
    H24.close()
    clk = ClockSampler(local).start()
    res = l30_leg(kry, workloads, world, tune, {"sm_mhz": None}, full=True, l32=args.l32)
    clocks = clk.stop()
    res.pop("_launches")
    if rank == 0:
        print(json.dumps({"metric": METRIC, ("l32" if args.l32 else "l30"): res, "clocks": clocks,
                          "shapes": {k: v["shape"] for k, v in tune.items()},
                          "measured_peaks": {"fp64_tflops": f64, "fp32_tflops": f32}}))


if __name__ == "__main__":
    a = parse()
    if a.l30 or a.l32:
        run_l30(a)
    elif a.ncu_case:
        run_ncu_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
