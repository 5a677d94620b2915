"""kry_tridiag_expv_noalloc: the small exponential for callers that must not allocate.

Some callers give all device memory to their own capped pool, or cannot afford the
device-wide synchronisation of cudaFree; this entry point keeps its device scratch in a
fixed array instead.  The test calls it through the C ABI several times in a row (large m,
then smaller m, then m = 1, where beta is not copied at all) with the host outputs filled
with NaN before every call, and compares each result with the allocating kry_tridiag_expv
at the tolerance of the small-exponential tests: a value left in the scratch by an earlier
call, or an output the call did not write, would show.  It runs last in the suite and also
passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_dp = ctypes.POINTER(ctypes.c_double)


def _call(lib, name, a, b, h, tau):
    m = a.size
    y = np.full(2 * m, np.nan)     # NaN sentinels: every element must be written by the call
    err = np.full(1, np.nan)
    bb = b if b.size else np.zeros(1)
    rc = getattr(lib, name)(a.ctypes.data_as(_dp), bb.ctypes.data_as(_dp), m, h, tau,
                            y.ctypes.data_as(_dp), err.ctypes.data_as(_dp), None)
    return rc, y[0::2] + 1j * y[1::2], float(err[0])


def test_noalloc_matches_the_allocating_call(kry):
    lib = kry.load()
    for call, (m, tau) in enumerate([(30, 0.8), (7, 2.5), (1, 1.7), (32, 0.3), (2, 4.0)]):
        rng = np.random.default_rng(100 + call)
        a = rng.normal(size=m) * 3.0
        b = np.abs(rng.normal(size=m - 1)) + 0.2
        h = 1.3
        rc1, y1, e1 = _call(lib, "kry_tridiag_expv", a, b, h, tau)
        rc2, y2, e2 = _call(lib, "kry_tridiag_expv_noalloc", a, b, h, tau)
        assert rc1 == kry.KRY_OK and rc2 == kry.KRY_OK
        assert np.all(np.isfinite(y2)) and np.isfinite(e2)
        assert np.max(np.abs(y1 - y2)) < 1e-13
        assert abs(e1 - e2) <= 1e-11 * e1 + 1e-20
        assert abs(np.linalg.norm(y2) - 1.0) < 1e-12
        if m == 1:   # exp(-i tau alpha) e_1, exactly
            assert abs(y2[0] - np.exp(-1j * tau * a[0])) < 1e-14


def test_noalloc_rejects_sizes_beyond_its_scratch(kry):
    lib = kry.load()
    a, b = np.zeros(33), np.zeros(32)
    rc, _, _ = _call(lib, "kry_tridiag_expv_noalloc", a, b, 1.0, 1.0)
    assert rc == kry.KRY_EINVAL
    assert b"maximum 32" in lib.kry_last_error()
