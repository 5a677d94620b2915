// Device helpers of the GB300 Krylov library: rank lookups, the matrix-free H.v row,
// complex arithmetic and dot-product accumulators.
#pragma once

#include "kry_internal.cuh"

namespace kry {

// ---------------------------------------------------------------- element types

template <class V> struct VT;
template <> struct VT<double2> {
    using R = double;
    __device__ __forceinline__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ __forceinline__ static double ehlo(const DevHam &h, uint32_t p) { return __ldg(h.ehlo_d + p); }
    __device__ __forceinline__ static double ehhi(const DevHam &h, uint32_t p) { return __ldg(h.ehhi_d + p); }
    __device__ __forceinline__ static double eh8(const DevHam &h, size_t p) { return __ldg(h.eh8_d + p); }
    __device__ __forceinline__ static double2 from(double2 c) { return c; }
};
template <> struct VT<float2> {
    using R = float;
    __device__ __forceinline__ static float2 zero() { return make_float2(0.f, 0.f); }
    __device__ __forceinline__ static float ehlo(const DevHam &h, uint32_t p) { return __ldg(h.ehlo_f + p); }
    __device__ __forceinline__ static float ehhi(const DevHam &h, uint32_t p) { return __ldg(h.ehhi_f + p); }
    __device__ __forceinline__ static float eh8(const DevHam &h, size_t p) { return __ldg(h.eh8_f + p); }
    __device__ __forceinline__ static float2 from(double2 c) { return make_float2((float)c.x, (float)c.y); }
};

// ---------------------------------------------------------------- float-float vectors
// GB300 runs FP64 arithmetic, and conversions between FP64 and FP32, at 1/64 of its FP32
// rate, so the complex128 passes are bound by the FP64 pipe at about a third of the HBM rate.
// dtype KRY_C128E keeps the Krylov vectors as float-float pairs (ffc, kry_internal.cuh: 16
// bytes per element like complex128, about 48 significant bits) and does all vector
// arithmetic on the FP32 pipe: products are formed exactly for the leading parts (the fused
// multiply-add error term) with the cross terms in float, and sums are float-float (Knuth's
// TwoSum).  A dot product is accurate to about 2^-47 of the sum of |terms| (FP64: 2^-53).
// Complex128 inputs and coefficients are converted at the boundary: a double is split by
// integer operations on its bits into its leading 24 significant bits and the next 23.

__device__ __forceinline__ void ff_combine(float &s, float &c, float s2, float c2);

// hi + lo floats of x (|x| in [2^-80, 2^128); smaller magnitudes give 0, which for vectors of
// norm of order one changes a dot product by less than 2^-80 D^(1/2))
__device__ __forceinline__ float2 dsplit(double x)
{
    const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
    const unsigned ex = (hw >> 20) & 0x7ffu;
    const bool ok = ex >= 943u && ex <= 1150u;
    const unsigned sg = hw & 0x80000000u;
    const float hi = __uint_as_float(ok ? (sg | ((ex - 896u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29)) : 0u);
    const float lm = __fsub_rn(__uint_as_float(0x4b000000u | ((lw >> 6) & 0x7fffffu)), 8388608.0f);   // exact
    const float sc = __uint_as_float(ok ? (sg | ((ex - 942u) << 23)) : 0u);                            // +-2^(e-46)
    return make_float2(hi, __fmul_rn(lm, sc));
}
// a float as a double, exactly, by integer operations (zero and subnormal floats give 0)
__device__ __forceinline__ double f2d(float f)
{
    const unsigned b = __float_as_uint(f), e = (b >> 23) & 0xffu;
    const unsigned hi = e ? ((b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)) : 0u;
    const unsigned lo = e ? ((b & 7u) << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
// float-float s + c rounded to FP64 (one FP64 add)
__device__ __forceinline__ double ff2d(float s, float c) { return f2d(s) + f2d(c); }
// (s, c) += (ah + al)(bh + bl): the leading product split exactly (TwoSum into s), the error
// term and the cross terms into c
__device__ __forceinline__ void ff_mac(float ah, float al, float bh, float bl, float &s, float &c)
{
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}
// (s, c) renormalised so that |c| is at most half an ulp of s (TwoSum: exact for any order of
// magnitudes, so also after a cancellation has left |c| > |s|)
__device__ __forceinline__ void ff_renorm(float &s, float &c)
{
    const float t = __fadd_rn(s, c);
    const float z = __fsub_rn(t, s);
    c = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(c, z));
    s = t;
}

template <> struct VT<ffc> {
    using R = double;
    __device__ __forceinline__ static ffc zero() { return ffc{0.f, 0.f, 0.f, 0.f}; }
    __device__ __forceinline__ static double ehlo(const DevHam &h, uint32_t p) { return __ldg(h.ehlo_d + p); }
    __device__ __forceinline__ static double ehhi(const DevHam &h, uint32_t p) { return __ldg(h.ehhi_d + p); }
    __device__ __forceinline__ static double eh8(const DevHam &h, size_t p) { return __ldg(h.eh8_d + p); }
    __device__ __forceinline__ static ffc from(double2 c)
    {
        const float2 a = dsplit(c.x), b = dsplit(c.y);
        return ffc{a.x, a.y, b.x, b.y};
    }
};
__device__ __forceinline__ ffc ldg(const ffc *p)
{
    const float4 v = __ldg((const float4 *)p);
    return ffc{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ float2 ldg(const float2 *p) { return __ldg(p); }
__device__ __forceinline__ double2 ldg(const double2 *p) { return __ldg(p); }

// Per element type: the accumulator of a neighbour sum (HvSum), of a linear combination (Lin),
// a coefficient as kept in shared memory (Coef), a right-hand vector element prepared for
// several dot products (Pre).  For complex64 and complex128 these are the element itself.
struct FF4 {   // two float-float numbers (real, imaginary)
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
};
template <class V> struct Arith {
    using HvSum = V;
    using Lin = V;
    using Coef = V;
    using Pre = V;
};
template <> struct Arith<ffc> {
    using HvSum = FF4;
    using Lin = FF4;
    using Coef = float4;   // (re hi, re lo, im hi, im lo)
    using Pre = ffc;
};

__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// w - c v (complex)
__device__ __forceinline__ double2 cfms(double2 c, double2 v, double2 w)
{
    return make_double2(fma(-c.x, v.x, fma(c.y, v.y, w.x)), fma(-c.x, v.y, fma(-c.y, v.x, w.y)));
}
__device__ __forceinline__ float2 cfms(float2 c, float2 v, float2 w)
{
    return make_float2(fmaf(-c.x, v.x, fmaf(c.y, v.y, w.x)), fmaf(-c.x, v.y, fmaf(-c.y, v.x, w.y)));
}

// d x + s acc  (real d, s)
__device__ __forceinline__ double2 axpby(double d, double2 x, double s, double2 a)
{
    return make_double2(fma(d, x.x, s * a.x), fma(d, x.y, s * a.y));
}
__device__ __forceinline__ float2 axpby(float d, float2 x, float s, float2 a)
{
    return make_float2(fmaf(d, x.x, s * a.x), fmaf(d, x.y, s * a.y));
}
// neighbour sums of the H.v row: acc += v, then y = sd x + shj acc
template <class V> __device__ __forceinline__ void hv_add(V &acc, V v) { acc = acc + v; }
__device__ __forceinline__ void hv_add(FF4 &acc, ffc v)
{
    ff_combine(acc.sr, acc.cr, v.xh, v.xl);
    ff_combine(acc.si, acc.ci, v.yh, v.yl);
}
__device__ __forceinline__ double2 axpby(double d, double2 x, double s, double2 a);
__device__ __forceinline__ float2 axpby(float d, float2 x, float s, float2 a);
template <class V, class R> __device__ __forceinline__ V hv_finish(R sd, V x, R shj, V acc) { return axpby(sd, x, shj, acc); }
__device__ __forceinline__ ffc hv_finish(double sd, ffc x, double shj, const FF4 &acc)
{
    const float2 d = dsplit(sd), h = dsplit(shj);
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    ff_mac(d.x, d.y, x.xh, x.xl, sr, cr);
    ff_mac(h.x, h.y, acc.sr, acc.cr, sr, cr);
    ff_mac(d.x, d.y, x.yh, x.yl, si, ci);
    ff_mac(h.x, h.y, acc.si, acc.ci, si, ci);
    ff_renorm(sr, cr);
    ff_renorm(si, ci);
    return ffc{sr, cr, si, ci};
}
// linear combinations: w = src - sum_i c_i x_i
template <class V> __device__ __forceinline__ V lin_init(V src) { return src; }
template <class V> __device__ __forceinline__ V lin_out(V w) { return w; }
template <class V> __device__ __forceinline__ typename Arith<V>::Coef coef_from(double2 c) { return VT<V>::from(c); }
__device__ __forceinline__ FF4 lin_init(ffc src)
{
    FF4 w;
    w.sr = src.xh; w.cr = src.xl; w.si = src.yh; w.ci = src.yl;
    return w;
}
__device__ __forceinline__ ffc lin_out(FF4 w)
{
    ff_renorm(w.sr, w.cr);
    ff_renorm(w.si, w.ci);
    return ffc{w.sr, w.cr, w.si, w.ci};
}
template <> __device__ __forceinline__ float4 coef_from<ffc>(double2 c)
{
    const float2 a = dsplit(c.x), b = dsplit(c.y);
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ double2 cfms(double2 c, double2 v, double2 w);
__device__ __forceinline__ float2 cfms(float2 c, float2 v, float2 w);
template <class V> __device__ __forceinline__ void lin_fms(V &w, V c, V x) { w = cfms(c, x, w); }
__device__ __forceinline__ void lin_fms(FF4 &w, float4 c, ffc x)
{
    // w -= c x: re -= cr xr - ci xi, im -= cr xi + ci xr
    ff_mac(-c.x, -c.y, x.xh, x.xl, w.sr, w.cr);
    ff_mac(c.z, c.w, x.yh, x.yl, w.sr, w.cr);
    ff_mac(-c.x, -c.y, x.yh, x.yl, w.si, w.ci);
    ff_mac(-c.z, -c.w, x.xh, x.xl, w.si, w.ci);
}
// a right-hand vector element prepared for several dot products
template <class V> __device__ __forceinline__ V pre(V u) { return u; }

__device__ __forceinline__ double2 scale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// s a for a float-float element: the product of the split scale with each component
__device__ __forceinline__ ffc scale(ffc a, double s)
{
    const float2 f = dsplit(s);
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    ff_mac(f.x, f.y, a.xh, a.xl, sr, cr);
    ff_mac(f.x, f.y, a.yh, a.yl, si, ci);
    ff_renorm(sr, cr);
    ff_renorm(si, ci);
    return ffc{sr, cr, si, ci};
}
__device__ __forceinline__ float2 scale(float2 a, double s) { return make_float2(a.x * (float)s, a.y * (float)s); }
__device__ __forceinline__ float2 scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ---------------------------------------------------------------- launch ordering

// First statement of every kernel of the replayed step: wait until the kernel before it
// has completed and its writes are visible (griddepcontrol.wait; it returns at once for a
// kernel launched without programmatic dependence), then let the next kernel begin its
// launch, so that launches overlap the tails of the kernels before them.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- dot accumulators
// sum conj(a) b.  complex128: FP64 fused multiply-adds.  complex64 and float-float: every
// product is split exactly (p = a*b rounded, e = fma(a, b, -p)) and summed with Knuth's
// TwoSum into a float pair (s, c): the rounding errors of s are kept exactly, and c gathers
// them in plain float.  c is folded back into s (renorm, a TwoSum) after every few terms --
// the callers do it once per tile -- so that its own rounding stays at 2^-48 of |s|: left to
// grow over the N terms of a thread, c's rounding errors add up to about N 2^-48 of the sum
// (5e-11 relative at N = 16K, the rows per thread of an L = 30 sector).

__device__ __forceinline__ double2 warp_sum(double2 v);

struct DotAccD {
    double re = 0.0, im = 0.0;
    __device__ __forceinline__ void add(double2 a, double2 b)
    {
        re = fma(a.x, b.x, re); re = fma(a.y, b.y, re);
        im = fma(a.x, b.y, im); im = fma(-a.y, b.x, im);
    }
    __device__ __forceinline__ void add_norm(double2 a) { re = fma(a.x, a.x, re); re = fma(a.y, a.y, re); }
    __device__ __forceinline__ void renorm() {}
    __device__ __forceinline__ double2 value() const { return make_double2(re, im); }
    // the sum over the warp (valid in every lane)
    __device__ __forceinline__ double2 warp_value() const { return warp_sum(value()); }
};

// Float-float sum (s, c) += (s2, c2): TwoSum of the leading parts, the trailing parts and the
// rounding error added, then renormalised.  Symmetric in its two operands.
__device__ __forceinline__ void ff_combine(float &s, float &c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
    const float cc = __fadd_rn(__fadd_rn(c, c2), e);
    s = __fadd_rn(t, cc);
    c = __fsub_rn(cc, __fsub_rn(s, t));
}
// Sum of a float-float value over the warp, in FP32 arithmetic (GB300 runs FP64, and the
// conversions to it, at 1/64 of the FP32 rate, so per-thread FP64 epilogues of the streaming
// kernels cost as much as their streams at small j): every lane ends with the total.
__device__ __forceinline__ void ff_warp_sum(float &s, float &c)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
        ff_combine(s, c, s2, c2);
    }
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
__device__ __forceinline__ void exact_fma(float a, float b, float &s, float &c)
{
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    float t, err;
    two_sum(s, p, t, err);
    s = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}
struct DotAccF {
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    __device__ __forceinline__ void add(float2 a, float2 b)
    {
        exact_fma(a.x, b.x, sr, cr); exact_fma(a.y, b.y, sr, cr);
        exact_fma(a.x, b.y, si, ci); exact_fma(-a.y, b.x, si, ci);
    }
    // |a|^2 (the imaginary part of conj(a) a is zero and is not accumulated)
    __device__ __forceinline__ void add_norm(float2 a) { exact_fma(a.x, a.x, sr, cr); exact_fma(a.y, a.y, sr, cr); }
    __device__ __forceinline__ void renorm()
    {
        ff_renorm(sr, cr);
        ff_renorm(si, ci);
    }
    __device__ __forceinline__ double2 value() const
    {
        return make_double2((double)sr + (double)cr, (double)si + (double)ci);
    }
    __device__ __forceinline__ double2 warp_value() const
    {
        float a = sr, b = cr, c = si, d = ci;
        ff_warp_sum(a, b);
        ff_warp_sum(c, d);
        return make_double2((double)a + (double)b, (double)c + (double)d);
    }
};
// complex64 dots with packed FP32x2 arithmetic (sm_100 and later): the same error-free
// products and TwoSum as DotAccF, two components per instruction.  With b_x2 = (bx, bx)
// and b_y2 = (by, by), the pair products a*b_x2 = (ax bx, ay bx) and a*b_y2 = (ax by, ay by)
// are summed into two float-float pairs; conj(a) b = (ax bx + ay by, ax by - ay bx) is formed
// in FP64 at the end.
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ void ff_pair_add(float2 &s, float2 &c, float2 a, float2 b)
{
    const float2 p = __fmul2_rn(a, b);
    const float2 e = __ffma2_rn(a, b, make_float2(-p.x, -p.y));   // a*b - p, exact
    const float2 t = __fadd2_rn(s, p);
    const float2 z = fsub2(t, s);
    const float2 err = __fadd2_rn(fsub2(s, fsub2(t, z)), fsub2(p, z));
    s = t;
    c = __fadd2_rn(c, __fadd2_rn(err, e));
}
// (s, c) renormalised by TwoSum, two float-float lanes per instruction
__device__ __forceinline__ void ff_renorm2(float2 &s, float2 &c)
{
    const float2 t = __fadd2_rn(s, c);
    const float2 z = fsub2(t, s);
    c = __fadd2_rn(fsub2(s, fsub2(t, z)), fsub2(c, z));
    s = t;
}
struct DotAccF2 {
    float2 s1 = make_float2(0.f, 0.f), c1 = make_float2(0.f, 0.f);
    float2 s2 = make_float2(0.f, 0.f), c2 = make_float2(0.f, 0.f);
    // b4 = (bx, bx, by, by)
    __device__ __forceinline__ void add(float2 a, float4 b4)
    {
        ff_pair_add(s1, c1, a, make_float2(b4.x, b4.y));
        ff_pair_add(s2, c2, a, make_float2(b4.z, b4.w));
    }
    __device__ __forceinline__ void add2(float2 a0, float4 b0, float2 a1, float4 b1)
    {
        add(a0, b0);
        add(a1, b1);
    }
    // b = (bx, by), broadcast per use
    __device__ __forceinline__ void add(float2 a, float2 b)
    {
        ff_pair_add(s1, c1, a, make_float2(b.x, b.x));
        ff_pair_add(s2, c2, a, make_float2(b.y, b.y));
    }
    __device__ __forceinline__ void add2(float2 a0, float2 b0, float2 a1, float2 b1)
    {
        add(a0, b0);
        add(a1, b1);
    }
    __device__ __forceinline__ void renorm()
    {
        ff_renorm2(s1, c1);
        ff_renorm2(s2, c2);
    }
    __device__ __forceinline__ double2 value() const
    {
        const double axbx = (double)s1.x + (double)c1.x, aybx = (double)s1.y + (double)c1.y;
        const double axby = (double)s2.x + (double)c2.x, ayby = (double)s2.y + (double)c2.y;
        return make_double2(axbx + ayby, axby - aybx);
    }
    // the sum over the warp, reduced in FP32 float-float arithmetic; converted to FP64 once
    __device__ __forceinline__ double2 warp_value() const
    {
        float a = s1.x, b = c1.x, c = s1.y, d = c1.y, e = s2.x, f = c2.x, g = s2.y, h = c2.y;
        ff_warp_sum(a, b);
        ff_warp_sum(c, d);
        ff_warp_sum(e, f);
        ff_warp_sum(g, h);
        const double axbx = (double)a + (double)b, aybx = (double)c + (double)d;
        const double axby = (double)e + (double)f, ayby = (double)g + (double)h;
        return make_double2(axbx + ayby, axby - aybx);
    }
};

// sum conj(a) b for float-float vectors (ffc)
struct DotAccFF {
    float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
    __device__ __forceinline__ void add(ffc a, ffc b)
    {
        ff_mac(a.xh, a.xl, b.xh, b.xl, sr, cr);
        ff_mac(a.yh, a.yl, b.yh, b.yl, sr, cr);
        ff_mac(a.xh, a.xl, b.yh, b.yl, si, ci);
        ff_mac(-a.yh, -a.yl, b.xh, b.xl, si, ci);
    }
    __device__ __forceinline__ void add_norm(ffc a)
    {
        ff_mac(a.xh, a.xl, a.xh, a.xl, sr, cr);
        ff_mac(a.yh, a.yl, a.yh, a.yl, sr, cr);
    }
    __device__ __forceinline__ void renorm()
    {
        ff_renorm(sr, cr);
        ff_renorm(si, ci);
    }
    __device__ __forceinline__ double2 value() const { return make_double2(ff2d(sr, cr), ff2d(si, ci)); }
    __device__ __forceinline__ double2 warp_value() const
    {
        float a = sr, b = cr, c = si, d = ci;
        ff_warp_sum(a, b);
        ff_warp_sum(c, d);
        return make_double2(ff2d(a, b), ff2d(c, d));
    }
};

template <class V> struct DotAcc;
template <> struct DotAcc<double2> : DotAccD {};
template <> struct DotAcc<float2> : DotAccF {};
template <> struct DotAcc<ffc> : DotAccFF {};

__device__ __forceinline__ double2 warp_sum(double2 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ---------------------------------------------------------------- rank tables

// Locate rank r0 + t (< D) as (block hi, offset in block, particles in the lower part):
// start from the block of the enclosing tile's first rank and step over whole blocks.
__device__ __forceinline__ void tile_unrank(const DevBasis &b, const uint32_t *bsz_s, uint32_t r0,
                                            uint32_t t, uint32_t &hi, uint32_t &off, int &klo)
{
    const uint32_t nhi = 1u << b.Lhi;
    uint32_t h = __ldg(b.tstart + r0 / (uint32_t)TILE);
    uint32_t o = r0 - __ldg(b.blk + h) + t;
    int k = b.N - __popc(h);
    while (o >= bsz_s[k]) {
        o -= bsz_s[k];
        do { ++h; k = b.N - __popc(h); } while ((k < 0 || k > b.Llo) && h + 1 < nhi);
        if (k < 0 || k > b.Llo) { k = 0; o = 0; break; }   // unreachable when r0 + t < D
    }
    hi = h; off = o; klo = k;
}

// Stage the small tables (and optionally ranklo, 2^Llo 16-bit entries) in shared memory.
__device__ __forceinline__ void stage_tables(const DevBasis &b, uint32_t *koff_s, uint32_t *bsz_s,
                                             uint16_t *rl_s, int rl_smem)
{
    for (int i = threadIdx.x; i < b.Llo + 2; i += blockDim.x) koff_s[i] = __ldg(b.koff + i);
    for (int i = threadIdx.x; i < b.Llo + 1; i += blockDim.x) bsz_s[i] = __ldg(b.bsz + i);
    if (rl_smem) {
        const uint32_t n2 = (1u << b.Llo) >> 1;   // Llo >= 1, so the count is even
        const uint32_t *src = (const uint32_t *)b.ranklo;
        uint32_t *dst = (uint32_t *)rl_s;
        for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) dst[i] = __ldg(src + i);
    }
}

// ---------------------------------------------------------------- matrix-free H.v
// Row r of H x for the state s = (hi << Llo) | lo (Eq. 1, XXZ form):
//   (H x)[r] = d(s) x[r] + (J/2) sum_{antiparallel bonds b} x[rank(s ^ bondmask_b)],
//   d(s) = (J Delta / 4)(nbonds - 2 n_anti(s)) + sum_i h_i (n_i - 1/2).
// Pull form (one writer per row, no atomics).  The re-rank of a hopped state takes two
// table lookups; a hop inside the upper part keeps the lower bits, so its target is
// blk[hi'] + off and the lanes of one block read consecutive elements.
template <class V>
__device__ __forceinline__ V hv_row(const DevBasis &b, const DevHam &hm, const V *__restrict__ x,
                                    uint32_t hi, uint32_t off, int klo, const uint32_t *koff_s,
                                    const uint16_t *rl)
{
    using R = typename VT<V>::R;
    const int Llo = b.Llo, L = b.L;
    const uint32_t pos = koff_s[klo] + off;
    const uint32_t lo = __ldg(b.lolist + pos);
    const uint32_t s = (hi << Llo) | lo;
    const uint32_t base = __ldg(b.blk + hi);
    const uint32_t lomask = (1u << Llo) - 1u;
    const uint32_t obc = (L >= 2) ? ((1u << (L - 1)) - 1u) : 0u;
    const uint32_t anti = (s ^ (s >> 1)) & obc;
    const uint32_t wrap = hm.pbc ? ((s ^ (s >> (L - 1))) & 1u) : 0u;
    const int nanti = __popc(anti) + (int)wrap;
    const R d = (R)hm.cz * (R)(hm.nbonds - 2 * nanti) + VT<V>::ehlo(hm, pos) + VT<V>::ehhi(hm, hi);
    V acc = VT<V>::zero();
    uint32_t a = anti & ((1u << (Llo - 1)) - 1u);          // bonds inside the lower part
    while (a) {
        const int p = __ffs(a) - 1;
        a &= a - 1u;
        acc = acc + __ldg(x + base + rl[lo ^ (3u << p)]);
    }
    if (b.Lhi > 0 && ((anti >> (Llo - 1)) & 1u)) {         // bond joining the two parts
        const uint32_t s2 = s ^ (3u << (Llo - 1));
        acc = acc + __ldg(x + __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask]);
    }
    uint32_t ah = anti >> Llo;                              // bonds inside the upper part
    while (ah) {
        const int q = __ffs(ah) - 1;
        ah &= ah - 1u;
        acc = acc + __ldg(x + __ldg(b.blk + (hi ^ (3u << q))) + off);
    }
    if (wrap) {                                             // ring bond (L-1, 0)
        const uint32_t s2 = s ^ ((1u << (L - 1)) | 1u);
        acc = acc + __ldg(x + __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask]);
    }
    return axpby(d, __ldg(x + base + off), (R)hm.halfJ, acc);
}

// sigma (H x)[r] for the row of hv_row, with the bond energy read from a table
// dz[n] = (J Delta / 4)(nbonds - 2 n) and sigma folded into the two factors:
//   sigma (d x_r + (J/2) acc) = (sigma d) x_r + (sigma J/2) acc.
template <class V>
__device__ __forceinline__ V hv_row_scaled(const DevBasis &b, const DevHam &hm, const V *__restrict__ x,
                                           uint32_t hi, uint32_t off, int klo, const uint32_t *koff_s,
                                           const uint16_t *rl, const typename VT<V>::R *dz,
                                           typename VT<V>::R sigma, typename VT<V>::R sigma_halfJ)
{
    using R = typename VT<V>::R;
    const int Llo = b.Llo, L = b.L;
    const uint32_t pos = koff_s[klo] + off;
    const uint32_t lo = __ldg(b.lolist + pos);
    const uint32_t s = (hi << Llo) | lo;
    const uint32_t base = __ldg(b.blk + hi);
    const uint32_t lomask = (1u << Llo) - 1u;
    const uint32_t obc = (L >= 2) ? ((1u << (L - 1)) - 1u) : 0u;
    const uint32_t anti = (s ^ (s >> 1)) & obc;
    const uint32_t wrap = hm.pbc ? ((s ^ (s >> (L - 1))) & 1u) : 0u;
    const R d = dz[__popc(anti) + (int)wrap] + VT<V>::ehlo(hm, pos) + VT<V>::ehhi(hm, hi);
    typename Arith<V>::HvSum acc{};
    uint32_t a = anti & ((1u << (Llo - 1)) - 1u);          // bonds inside the lower part
    while (a) {
        const int p = __ffs(a) - 1;
        a &= a - 1u;
        hv_add(acc, ldg(x + base + rl[lo ^ (3u << p)]));
    }
    if (b.Lhi > 0 && ((anti >> (Llo - 1)) & 1u)) {         // bond joining the two parts
        const uint32_t s2 = s ^ (3u << (Llo - 1));
        hv_add(acc, ldg(x + __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask]));
    }
    uint32_t ah = anti >> Llo;                              // bonds inside the upper part
    while (ah) {
        const int q = __ffs(ah) - 1;
        ah &= ah - 1u;
        hv_add(acc, ldg(x + __ldg(b.blk + (hi ^ (3u << q))) + off));
    }
    if (wrap) {                                             // ring bond (L-1, 0)
        const uint32_t s2 = s ^ ((1u << (L - 1)) | 1u);
        hv_add(acc, ldg(x + __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask]));
    }
    return hv_finish(sigma * d, ldg(x + base + off), sigma_halfJ, acc);
}

// The same row as hv_row_scaled with the gathers issued in rounds: the targets of up to
// RND hops are computed first (taking the antiparallel bonds in ascending order) and
// their loads issued together, so a thread has up to RND gathers in flight instead of one
// (a warp issues in order, and the loop of hv_row_scaled waits for each gathered value
// before it computes the next target).  The terms are added in the same order as in
// hv_row_scaled, so the result is bitwise the same.
template <class V, int RND = 4>
__device__ __forceinline__ V hv_row_chunked(const DevBasis &b, const DevHam &hm, const V *__restrict__ x,
                                            uint32_t hi, uint32_t off, int klo, const uint32_t *koff_s,
                                            const uint16_t *rl, const typename VT<V>::R *dz,
                                            typename VT<V>::R sigma, typename VT<V>::R sigma_halfJ)
{
    using R = typename VT<V>::R;
    const int Llo = b.Llo, L = b.L;
    const uint32_t pos = koff_s[klo] + off;
    const uint32_t lo = __ldg(b.lolist + pos);
    const uint32_t s = (hi << Llo) | lo;
    const uint32_t base = __ldg(b.blk + hi);
    const uint32_t lomask = (1u << Llo) - 1u;
    const uint32_t obc = (L >= 2) ? ((1u << (L - 1)) - 1u) : 0u;
    const uint32_t anti = (s ^ (s >> 1)) & obc;
    const uint32_t wrap = hm.pbc ? ((s ^ (s >> (L - 1))) & 1u) : 0u;
    const R d = dz[__popc(anti) + (int)wrap] + VT<V>::ehlo(hm, pos) + VT<V>::ehhi(hm, hi);
    const V xr = ldg(x + base + off);
    typename Arith<V>::HvSum acc{};
    uint32_t a = anti & ((1u << (Llo - 1)) - 1u);          // bonds inside the lower part
    while (a) {
        uint32_t t[RND];
        int n = 0;
#pragma unroll
        for (int u = 0; u < RND; ++u) {
            if (a) {
                const int p = __ffs(a) - 1;
                a &= a - 1u;
                t[u] = base + rl[lo ^ (3u << p)];
                n = u + 1;
            }
        }
        V v[RND];
#pragma unroll
        for (int u = 0; u < RND; ++u)
            if (u < n) v[u] = ldg(x + t[u]);
#pragma unroll
        for (int u = 0; u < RND; ++u)
            if (u < n) hv_add(acc, v[u]);
    }
    const bool cross = b.Lhi > 0 && ((anti >> (Llo - 1)) & 1u);   // bond joining the two parts
    V vc = VT<V>::zero(), vr = VT<V>::zero();
    if (cross) {
        const uint32_t s2 = s ^ (3u << (Llo - 1));
        vc = ldg(x + __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask]);
    }
    if (wrap) {                                                    // ring bond (L-1, 0)
        const uint32_t s2 = s ^ ((1u << (L - 1)) | 1u);
        vr = ldg(x + __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask]);
    }
    if (cross) hv_add(acc, vc);
    uint32_t ah = anti >> Llo;                                     // bonds inside the upper part
    while (ah) {
        uint32_t t[RND];
        int n = 0;
#pragma unroll
        for (int u = 0; u < RND; ++u) {
            if (ah) {
                const int q = __ffs(ah) - 1;
                ah &= ah - 1u;
                t[u] = __ldg(b.blk + (hi ^ (3u << q)));
                n = u + 1;
            }
        }
        V v[RND];
#pragma unroll
        for (int u = 0; u < RND; ++u)
            if (u < n) v[u] = ldg(x + t[u] + off);
#pragma unroll
        for (int u = 0; u < RND; ++u)
            if (u < n) hv_add(acc, v[u]);
    }
    if (wrap) hv_add(acc, vr);
    return hv_finish(sigma * d, xr, sigma_halfJ, acc);
}

}  // namespace kry
