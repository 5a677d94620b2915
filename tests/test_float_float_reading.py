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
RT_C64 = 8              # rows per thread and tile of the complex64 dots


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


def _fast_two_sum(a, b):
    """Dekker's FastTwoSum: s + e == a + b exactly when |a| >= |b|."""
    s = (a + b).astype(F)
    return s, (b - (s - a).astype(F)).astype(F)


def _dot2_offset(a, b, rt, amax_bound):
    """The same sum with Dekker's FastTwoSum (3 operations) in place of TwoSum (6): every tile
    adds a power of two sigma > 2 (rt max|a| max|b| + 2 max(|s|, |c|)) to s, so that the
    running sum dominates every product of the tile, and takes it off exactly (Sterbenz) at
    the tile's end.  With amax_bound False, max|a| is replaced by 1, the bound that the unit
    norm of a Krylov vector gives without a pass over its rows."""
    n, lanes = a.shape
    s = np.zeros(lanes, F)
    c = np.zeros(lanes, F)
    for t0 in range(0, n, rt):
        at, bt = a[t0:t0 + rt], b[t0:t0 + rt]
        amax = np.max(np.abs(at), axis=0) if amax_bound else F(1)
        m = ((F(rt) * np.max(np.abs(bt), axis=0)).astype(F) * amax + F(2) * np.maximum(np.abs(s), np.abs(c))).astype(F)
        m = np.maximum(m, F(2.0 ** -100))
        sig = ((m.view(np.uint32) & np.uint32(0x7f800000)) + np.uint32(2 << 23)).view(F)
        t1, e1 = _fast_two_sum(sig, s)
        S, c = _fast_two_sum(t1, (c + e1).astype(F))
        for k in range(at.shape[0]):
            p = (at[k] * bt[k]).astype(F)
            assert np.all(np.abs(S) >= np.abs(p))
            e = _fma(at[k], bt[k], -p)
            S, err = _fast_two_sum(S, p)
            c = (c + (err + e).astype(F)).astype(F)
        s = (S - sig).astype(F)
        assert np.all(s.astype(np.float64) == S.astype(np.float64) - sig.astype(np.float64))
    s, c = _two_sum(s, c)
    return s.astype(np.float64) + c.astype(np.float64)


def test_a_fast_two_sum_against_a_per_tile_offset_loses_bits():
    """The cheaper accumulation weighed for the complex64 dots (7 instead of 10 operations per
    product) keeps every sum error-free but lets the rounding of c act on units of the offset
    instead of the running sum: on vectors normalised over an L = 24 and an L = 30 sector it is
    2.5 to 4.5 bits less accurate than TwoSum (2^-38 to 2^-44 of the sum of |terms|, against
    2^-42 to 2^-47), and 6 to 12 bits less with the unit-norm bound on |a|, which is why the
    dots keep TwoSum."""
    for n, D in ((278, 2.7e6), (16384, 1.55e8)):
        rng = np.random.default_rng(n)
        a = (rng.standard_normal((n, 64)) / np.sqrt(D)).astype(F)
        for b in ((a * 7 + 0.01 * rng.standard_normal((n, 64)) / np.sqrt(D)).astype(F),   # norm-like
                  (3 * rng.standard_normal((n, 64)) / np.sqrt(D)).astype(F)):           # orthogonal
            exact = np.sum(a.astype(np.float64) * b.astype(np.float64), axis=0)
            scale = np.sum(np.abs(a.astype(np.float64) * b.astype(np.float64)), axis=0)
            bits = lambda x: -np.log2(np.max(np.abs(x - exact) / scale))
            b_ts, b_off, b_unit = bits(_dot2(a, b, RT_C64)), bits(_dot2_offset(a, b, RT_C64, True)), bits(_dot2_offset(a, b, RT_C64, False))
            assert b_ts > 41 and b_off > 37
            assert 2 < b_ts - b_off < 6
            assert b_ts - b_unit > 6 and b_unit < 36
