"""The float-float accumulation of the dot kernels, emulated on the CPU in IEEE float32.

Each GPU thread sums its products with an error-free product (p = a*b, e = fma(a, b, -p)),
Knuth's TwoSum of the leading parts into s, and the rounding errors gathered in a plain float
c.  Left alone, c grows with the terms and its own rounding -- of order |c| 2^-24 per term --
makes the error grow like n 2^-48 of the sum.  Folding c back into s by a TwoSum after every
tile (4 rows per thread in the float-float dots) keeps c at a few units in the last place of
s, and the error grows like a random walk, sqrt(n) 2^-48.  The emulation (numpy float32
arithmetic, fused multiply-adds rounded once from the exact float64 product, one lane per
thread) runs at the terms per thread of the L = 24, 28 and 30 dots (278, 4K and 16K) against
the exact sum in float64: the reason the kernels renormalise once per tile.
"""
import numpy as np

F = np.float32
U = 2.0 ** -48          # unit roundoff of a float-float pair
RT = 4                  # rows per thread and tile of the float-float dots


def _fma(a, b, c):
    """fma in float32: the product of two floats is exact in float64, then one rounding."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def _two_sum(a, b):
    """Knuth's TwoSum: s + e == a + b exactly."""
    s = (a + b).astype(F)
    z = (s - a).astype(F)
    e = ((a - (s - z)).astype(F) + (b - z).astype(F)).astype(F)
    return s, e


def _dot2(a, b, renorm_every):
    """sum_k a[k] b[k] per column (one lane per column) in float-float, as the kernels do."""
    n, lanes = a.shape
    s = np.zeros(lanes, F)
    c = np.zeros(lanes, F)
    for k in range(n):
        p = (a[k] * b[k]).astype(F)
        e = _fma(a[k], b[k], -p)
        s, err = _two_sum(s, p)
        c = (c + (err + e).astype(F)).astype(F)
        if renorm_every and (k + 1) % renorm_every == 0:
            s, c = _two_sum(s, c)
    return s.astype(np.float64) + c.astype(np.float64)


def _case(n, lanes=64, seed=0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, lanes)).astype(F)
    b = (a + 0.01 * rng.standard_normal((n, lanes))).astype(F)   # norm-like: a large sum
    exact = np.sum(a.astype(np.float64) * b.astype(np.float64), axis=0)
    scale = np.sum(np.abs(a.astype(np.float64) * b.astype(np.float64)), axis=0)
    return a, b, exact, scale


def test_the_emulated_primitives_are_error_free():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(1000).astype(F)
    b = (rng.standard_normal(1000) * 1e-3).astype(F)
    s, e = _two_sum(a, b)
    assert np.all(s.astype(np.float64) + e.astype(np.float64) == a.astype(np.float64) + b.astype(np.float64))
    p = (a * b).astype(F)
    assert np.all(p.astype(np.float64) + _fma(a, b, -p).astype(np.float64) == a.astype(np.float64) * b.astype(np.float64))


def test_renormalised_error_grows_like_a_random_walk_and_the_plain_one_like_n():
    errs_no, errs_rn = [], []
    for n in (256, 4096, 16384):
        a, b, exact, scale = _case(n, seed=n)
        e_no = np.max(np.abs(_dot2(a, b, 0) - exact) / scale)
        e_rn = np.max(np.abs(_dot2(a, b, RT) - exact) / scale)
        assert e_rn < 2.0 * np.sqrt(n) * U
        assert e_no > 0.05 * n * U
        errs_no.append(e_no)
        errs_rn.append(e_rn)
    assert errs_no[2] > 20 * errs_no[0]          # 64 times the terms
    assert errs_no[2] > 20 * errs_rn[2]          # at the L = 30 terms per thread
