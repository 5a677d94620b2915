"""The seeded input generators (no arithmetic of the method): determinism, ranges and the
distributions they promise."""
import collections
import math

import pytest

import workloads


def test_splitmix64_published_first_outputs():
    # SplitMix64 from state 0: the first outputs of the published generator
    assert workloads.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_fibonacci_ratio_and_aubry_andre_field():
    assert workloads.fibonacci_beta(55) == 34 / 55
    assert workloads.fibonacci_beta(21) == 13 / 21
    with pytest.raises(ValueError):
        workloads.fibonacci_beta(54)
    h = workloads.aubry_andre_field(55, 2.0, 1.0, 0.0)
    assert len(h) == 55 and max(abs(x) for x in h) <= 1.0 + 1e-15   # amplitude lambda J / 2
    assert abs(sum(h)) < 1e-12                                      # a full period on the ring
    assert h[0] == pytest.approx(math.cos(2 * math.pi * 34 / 55))


def test_random_basis_states_are_sector_states_and_seeded():
    s1 = workloads.random_basis_states(22, 11, 5, 64)
    s2 = workloads.random_basis_states(22, 11, 5, 64)
    s3 = workloads.random_basis_states(22, 11, 6, 64)
    assert s1 == s2 and s1 != s3
    assert all(bin(s).count("1") == 11 and s >> 22 == 0 for s in s1)
    assert all(bin(s).count("1") == 3 and s >> 55 == 0 for s in workloads.random_basis_states(55, 3, 1, 50))


def test_random_basis_states_uniform_over_the_sector():
    """Chi-square test of uniformity over the C(6, 3) = 20 site sets (99.9% quantile of
    chi-square with 19 degrees of freedom: 43.8)."""
    n = 40000
    c = collections.Counter(workloads.random_basis_states(6, 3, 9, n))
    assert len(c) == 20
    e = n / 20
    chi2 = sum((v - e) ** 2 / e for v in c.values())
    assert chi2 < 43.8


def test_neel_and_log_times():
    assert workloads.neel_state(6) == 0b010101
    t = workloads.log_times(40, 0.1, 100.0)
    assert len(t) == 40 and t[0] == pytest.approx(0.1) and t[-1] == pytest.approx(100.0)
    assert all(b > a for a, b in zip(t, t[1:]))
