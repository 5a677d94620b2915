"""Host logic of bench.py: the algorithmic byte and flop counts behind the roofline, the
selection of the dominant kernel, and the DRAM-traffic lookup.  No GPU."""
import pytest

import bench


def test_vector_passes_of_a_krylov_step():
    """At m = 30: the H.v moves 2 vectors per Lanczos index, the dots j + 2, the update
    j + 3, and the combine 31: 1111 vector passes per Krylov step."""
    m = 30
    hv = sum(bench.PASSES["hv"](j) for j in range(m))
    dots = sum(bench.PASSES["dots"](j) for j in range(m))
    upd = sum(bench.PASSES["update"](j) for j in range(m))
    assert (hv, dots, upd) == (60, 495, 525)
    assert hv + dots + upd + (m + 1) == 1111


def test_fp64_flop_counts():
    """A complex multiply-add is 8 flops and |w|^2 4: the update at index j costs
    8 (j + 1) + 4 per element, like the dots; the H.v 2 per gathered neighbour plus 10."""
    D, m, steps, L, N = 1000, 30, 3, 24, 12
    per = sum(8 * (j + 1) + 4 for j in range(m))
    assert bench.fp64_flops("update", D, m, steps, L, N, True) == per * D * steps
    assert bench.fp64_flops("dots", D, m, steps, L, N, True) == per * D * steps
    nb = 2.0 * N * (L - N) / (L - 1)          # average antiparallel bonds on a ring
    assert bench.fp64_flops("hv", D, m, steps, L, N, True) == pytest.approx(m * (10 + 2 * nb) * D * steps)
    assert bench.fp64_flops("passC", D, m, steps, L, N, True) == 0.0
    # FP64 pipe instructions: a multiply-add is one instruction, 4 per complex element
    assert bench.fp64_pipe_ops("update", D, m, steps, L, N, True) == sum(4 * (j + 1) + 2 for j in range(m)) * D * steps


def _prof(ms, mult=1.0):
    """A profile as Hamiltonian.profile_read returns it, for `steps` full Krylov steps."""
    D, m, steps = 2704156, 30, 10
    out = {}
    for k in bench.KIND_NAMES:
        passes = sum(bench.PASSES[k](j) for j in range(m)) if k in bench.PASSES else 0
        out[k] = {"ms": ms.get(k, 0.0), "bytes": passes * D * 8 * steps * mult, "launches": m * steps}
    return out, D, m, steps


def test_roofline_picks_the_slowest_vector_kernel(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6000.0})
    monkeypatch.setattr(bench, "ncu_traffic", lambda kind, b: None)
    prof, D, m, steps = _prof({"hv": 50.0, "dots": 200.0, "update": 150.0, "passC": 300.0, "smallexp": 5.0})
    c = {"m": m, "pbc": True}
    r = bench.roofline(prof, "c64", D, c, 24, 12, {"sm_mhz": 2070.0})
    # pass C is not a candidate (no-ops unless flagged); the dots are the slowest of the three
    assert r["kind"] == "dots" and r["kernel"] == "k_dots<.,0>" and r["bound"] == "hbm"
    want = prof["dots"]["bytes"] / (200.0 * 1e6)
    assert r["achieved"] == pytest.approx(want) and r["frac"] == pytest.approx(want / 6000.0)
    assert sum(r["kernel_time_share"].values()) == pytest.approx(1.0)


def test_roofline_of_complex128_counts_flops(monkeypatch):
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 6000.0})
    monkeypatch.setattr(bench, "ncu_traffic", lambda kind, b: None)
    monkeypatch.setattr(bench, "MEASURED_FP64", {"tflops": 1.0})
    prof, D, m, steps = _prof({"hv": 50.0, "dots": 100.0, "update": 200.0}, mult=2.0)   # 16-byte elements
    c = {"m": m, "pbc": True}
    r = bench.roofline(prof, "c128", D, c, 24, 12, {"sm_mhz": 2070.0})
    assert r["bound"] == "alu" and r["kind"] == "update" and r["peak"] == 1.0
    flops = bench.fp64_flops("update", D, m, steps, 24, 12, True)
    assert r["achieved"] == pytest.approx(flops / 0.2 / 1e12)
    assert r["hbm_view"]["achieved"] == pytest.approx(prof["update"]["bytes"] / (200.0 * 1e6))


def test_traffic_is_null_once_the_kernels_change(monkeypatch, tmp_path):
    """The committed DRAM traffic scales to the average launch by algorithmic bytes, and is
    withheld once the kernel sources no longer hash to the recorded value."""
    f = tmp_path / "profiles"
    f.mkdir()
    (f / "traffic_vector_kernels.txt").write_text(
        "# test\nsource_hash=abc\nc64_dots_captured_algo_bytes=100\nc64_dots_captured_dram_bytes=110\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    assert bench.ncu_traffic("c64_dots", 1000.0) == pytest.approx(1100.0)
    assert bench.ncu_traffic("c64_update", 1000.0) is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "def")
    assert bench.ncu_traffic("c64_dots", 1000.0) is None


def test_committed_traffic_file_matches_the_sources():
    """The committed capture was taken on the current kernel sources."""
    assert bench.ncu_traffic("update", 1.0) is not None
    assert bench.ncu_traffic("c64_dots", 1.0) == pytest.approx(1.0, rel=0.1)
