"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the Krylov method: it only draws random numbers and
lays out the model parameters of Eq. 1 (the on-site quasiperiodic field, the Neel initial
state of Sec. 4, the output-time grid).  Both sides consume the arrays it returns.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), implemented here from its published definition, so the
phases phi are reproducible on every machine without numpy's generator state.
"""
from __future__ import annotations

import math

_MASK64 = (1 << 64) - 1
GOLDEN_Q = (math.sqrt(5.0) - 1.0) / 2.0   # inverse golden ratio, Eq. 1 (beta)


def splitmix64_stream(seed: int, n: int) -> list[int]:
    """First n outputs of the SplitMix64 sequence started at state `seed`."""
    out = []
    state = seed & _MASK64
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out.append(z ^ (z >> 31))
    return out


def uniform53(seed: int, n: int) -> list[float]:
    """n doubles uniform on [0, 1): the top 53 bits of each SplitMix64 output."""
    return [(z >> 11) * (1.0 / (1 << 53)) for z in splitmix64_stream(seed, n)]


def phases(seed: int, k: int = 1) -> list[float]:
    """k phases phi ~ U[0, 2 pi): the k-th realisation uses the k-th draw of the stream."""
    return [2.0 * math.pi * u for u in uniform53(seed, k)]


def quasiperiodic_field(L: int, h: float, phi: float, q: float = GOLDEN_Q) -> list[float]:
    """On-site field of Eq. 1: h_i = h cos(2 pi q i + phi) for sites i = 1..L.

    Element i-1 of the returned list belongs to site i (bit i-1 of a state).
    """
    return [h * math.cos(2.0 * math.pi * q * i + phi) for i in range(1, L + 1)]


def random_basis_states(L: int, N: int, seed: int, k: int) -> list[int]:
    """k random product states of the (L, N) sector, each uniform over the C(L, N) site sets:
    N sites drawn without replacement by a partial Fisher-Yates shuffle of 1..L, with
    SplitMix64 draws (N per realisation) mapped to indices by floor(u * remaining)."""
    u = uniform53(seed, k * N)
    out = []
    for r in range(k):
        sites = list(range(L))
        s = 0
        for i in range(N):
            j = i + min(int(u[r * N + i] * (L - i)), L - i - 1)
            sites[i], sites[j] = sites[j], sites[i]
            s |= 1 << sites[i]
        out.append(s)
    return out


def fibonacci_beta(L: int) -> float:
    """beta = F_{n-1} / F_n for a ring of L = F_n sites (Sec. 2: a rational approximant of the
    inverse golden ratio that closes the quasiperiodic cycle on the ring, e.g. 34/55)."""
    a, b = 1, 1
    while b < L:
        a, b = b, a + b
    if b != L:
        raise ValueError(f"L = {L} is not a Fibonacci number")
    return a / b


def aubry_andre_field(L: int, lam: float, J: float, phi: float, beta: float | None = None) -> list[float]:
    """On-site field of the Aubry-Andre chain (Sec. 4) at lambda = h / t, with the hopping
    t = J / 2 of Eq. 1's XXZ form: h_i = (lambda J / 2) cos(2 pi beta i + phi); beta defaults
    to the Fibonacci ratio of L."""
    q = fibonacci_beta(L) if beta is None else beta
    return quasiperiodic_field(L, 0.5 * lam * J, phi, q)


def neel_state(L: int) -> int:
    """Neel product state (...010101) of Sec. 4: sites 1, 3, 5, ... occupied (bits 0, 2, 4, ...)."""
    s = 0
    for b in range(0, L, 2):
        s |= 1 << b
    return s


def log_times(n: int = 40, t0: float = 0.1, t1: float = 100.0) -> list[float]:
    """n log-spaced output times from t0 to t1, both ends included."""
    if n == 1:
        return [t0]
    a, b = math.log10(t0), math.log10(t1)
    return [10.0 ** (a + (b - a) * k / (n - 1)) for k in range(n)]


def config(name: str) -> dict:
    """The five seeded workloads: each entry gives L, n_up, J, Delta, the field rows h[K][L],
    the boundary, the initial state, Krylov size m, tolerance and output times."""
    if name == "L16_fp64":
        L, hh, seed = 16, 2.0, 1
        return dict(name=name, L=L, n_up=8, J=1.0, Delta=1.0,
                    h=[quasiperiodic_field(L, hh, phases(seed)[0])], pbc=True,
                    state=neel_state(L), m=30, tol=1e-10, times=log_times())
    if name == "L24_mixed":
        L, hh, seed = 24, 1.5, 2
        return dict(name=name, L=L, n_up=12, J=1.0, Delta=1.0,
                    h=[quasiperiodic_field(L, hh, phases(seed)[0])], pbc=True,
                    state=neel_state(L), m=30, tol=1e-10, times=log_times())
    if name.startswith("L22_batched"):
        # L22_batched_h{0.5,1.5,3}: K = 64 phases drawn from one seeded stream
        L, seed, K = 22, 3, 64
        hh = float(name.split("_h")[1]) if "_h" in name else 1.5
        return dict(name=name, L=L, n_up=11, J=1.0, Delta=1.0,
                    h=[quasiperiodic_field(L, hh, p) for p in phases(seed, K)], pbc=True,
                    state=neel_state(L), m=30, tol=1e-6, times=log_times())
    if name == "L20_grad":
        L, hh, seed = 20, 1.0, 4
        return dict(name=name, L=L, n_up=10, J=1.0, Delta=1.0,
                    h=[quasiperiodic_field(L, hh, phases(seed)[0])], pbc=True,
                    state=neel_state(L), m=30, tol=1e-10, times=[10.0], ckpt_every=8)
    if name in ("L30_clean", "L30_qp"):
        L, seed = 30, 5
        hh = 0.0 if name == "L30_clean" else 1.5
        return dict(name=name, L=L, n_up=15, J=1.0, Delta=1.0,
                    h=[quasiperiodic_field(L, hh, phases(seed)[0])], pbc=True,
                    state=neel_state(L), m=30, tol=1e-10, times=log_times())
    raise KeyError(name)


CONFIG_NAMES = ["L16_fp64", "L24_mixed", "L22_batched_h0.5", "L22_batched_h1.5",
                "L22_batched_h3", "L20_grad", "L30_clean", "L30_qp"]
