"""kry_tridiag_expv_noalloc: the small exponential for callers that must not allocate.

Some callers give all device memory to their own capped pool, or cannot afford the
device-wide synchronisation of cudaFree; this entry point keeps its device scratch in a
fixed array instead.  The test calls it through the C ABI twice in a row (the second call
smaller than the first, so stale scratch would show) and compares each result with the
allocating kry_tridiag_expv, at the tolerance of the small-exponential tests.  It runs
last in the suite and also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_dp = ctypes.POINTER(ctypes.c_double)


def _call(lib, name, a, b, h, tau):
    m = a.size
    y = np.zeros(2 * m)
    err = np.zeros(1)
    bb = b if b.size else np.zeros(1)
    rc = getattr(lib, name)(a.ctypes.data_as(_dp), bb.ctypes.data_as(_dp), m, h, tau,
                            y.ctypes.data_as(_dp), err.ctypes.data_as(_dp), None)
    return rc, y[0::2] + 1j * y[1::2], float(err[0])


def test_noalloc_matches_the_allocating_call(kry):
    lib = kry.load()
    for call, (m, tau) in enumerate([(30, 0.8), (7, 2.5)]):
        rng = np.random.default_rng(100 + call)
        a = rng.normal(size=m) * 3.0
        b = np.abs(rng.normal(size=m - 1)) + 0.2
        h = 1.3
        rc1, y1, e1 = _call(lib, "kry_tridiag_expv", a, b, h, tau)
        rc2, y2, e2 = _call(lib, "kry_tridiag_expv_noalloc", a, b, h, tau)
        assert rc1 == kry.KRY_OK and rc2 == kry.KRY_OK
        assert np.max(np.abs(y1 - y2)) < 1e-13
        assert abs(e1 - e2) <= 1e-11 * e1 + 1e-20
        assert abs(np.linalg.norm(y2) - 1.0) < 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch(kry):
    lib = kry.load()
    a, b = np.zeros(33), np.zeros(32)
    rc, _, _ = _call(lib, "kry_tridiag_expv_noalloc", a, b, 1.0, 1.0)
    assert rc == kry.KRY_EINVAL
    assert b"maximum 32" in lib.kry_last_error()
