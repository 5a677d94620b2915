// Small exponential, error estimate and step control of one Krylov step (Sec. 2:
// psi(t + tau) ~ beta V_m exp(-i tau T_m) e_1 with time stepping and error estimation),
// run by one warp in FP64 without a host round trip.
//
// T (m_eff x m_eff, symmetric tridiagonal from Lanczos) is shifted and scaled into
// [-1, 1]: T~ = (T - c)/r with c, r the centre and half-width of its Gershgorin interval.
// Then (Jacobi-Anger expansion)
//     exp(-i tau T) e_1 = exp(-i tau c) sum_k w_k J_k(tau r) T_k(T~) e_1,
//     w_0 = 1, w_k = 2 (-i)^k,
// with Bessel functions J_k from Miller's backward recurrence normalised by
// J_0 + 2 sum J_2k = 1.  The leading term of the Krylov error (Saad 1992; the estimate
// of Sidje's Expokit that the paper relies on) is
//     err(tau) = beta h |e_m^T tau phi_1(-i tau (T - c)) e_1|
//              = (beta h / r) |sum_k w_k I_k(tau r) [T_k(T~) e_1]_m|,
// where I_k(x) = int_0^x J_k = 2 sum_n J_{k+2n+1}(x) (Abramowitz & Stegun 11.1.2) and h is
// the coupling of v_m to the next Krylov vector.  A ladder of 32 candidate steps (one per
// lane) is scanned and the largest tau with err(tau) <= 0.05 tol tau / t_end is taken;
// the Krylov basis is reused, so a rejected candidate costs no H.v.  Every output time in
// [t, t + tau] is read from the same expansion (dense output):
//     <psi0|psi(t + tau')> = beta exp(-i tau' c) sum_k w_k J_k(tau' r) sum_j g_j [T_k(T~) e_1]_j,
// g_j = <psi0|v_j>.
#include <cuda_runtime.h>

#include "kry_device.cuh"

namespace kry {

constexpr double STEP_SAFETY = 0.1;   // fraction of the local error budget a step may use
constexpr double LADDER = 0.85;       // ratio of consecutive candidate steps

struct ExpSmem {
    double al[MMAX], be[MMAX];
    double2 g[MMAX];
    double tch[(KMAX + 1) * 32];      // T_k(T~) e_1, component j at [k * 32 + j]
    double jb[32 * (KMAX + 2)];       // per-lane Bessel sequences
    double2 gk[KMAX + 1];             // sum_j g_j [T_k(T~) e_1]_j
};

__device__ __forceinline__ int cheb_degree(double x)
{
    const int K = (int)ceil(x + 8.0 * cbrt(x) + 24.0);
    return K < KMAX ? K : KMAX;
}

// J_k(x) for k = 0..K into out[0..K] (x >= 0).
__device__ void bessel_seq(double x, int K, double *out)
{
    if (x < 1e-6) {
        for (int k = 0; k <= K; ++k) out[k] = 0.0;
        out[0] = 1.0 - 0.25 * x * x;
        if (K >= 1) out[1] = 0.5 * x - x * x * x / 16.0;
        if (K >= 2) out[2] = x * x / 8.0;
        if (K >= 3) out[3] = x * x * x / 48.0;
        return;
    }
    int ns = (K > (int)x ? K : (int)x) + 40;
    ns += ns & 1;
    const double inv = 2.0 / x;
    double jp1 = 0.0, jk = 1e-280, sum = 0.0;
    for (int k = ns; k >= 1; --k) {
        const double jm1 = (double)k * inv * jk - jp1;
        jp1 = jk;
        jk = jm1;
        const int idx = k - 1;
        if (idx <= K) out[idx] = jm1;
        if (idx >= 2 && !(idx & 1)) sum += jm1;
        if (fabs(jk) > 1e250) {
            jk *= 1e-250;
            jp1 *= 1e-250;
            sum *= 1e-250;
            for (int t = idx; t <= K; ++t) out[t] *= 1e-250;
        }
    }
    const double invS = 1.0 / (out[0] + 2.0 * sum);
    for (int k = 0; k <= K; ++k) out[k] *= invS;
}

// sum_k w_k c_k v_k as a complex number, for real c_k, v_k
__device__ __forceinline__ double2 jacobi_anger_sum(const double *c, const double *v, int vstride, int K)
{
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= K; ++k) {
        const double t = c[k] * v[k * vstride] * (k == 0 ? 1.0 : 2.0);
        switch (k & 3) {
        case 0: re += t; break;
        case 1: im -= t; break;
        case 2: re -= t; break;
        default: im += t; break;
        }
    }
    return make_double2(re, im);
}

// Error-estimate sum: sum_k w_k I_k v_k with I_k = int_0^x J_k from the J sequence.
__device__ __forceinline__ double2 integral_sum(const double *J, const double *v, int vstride, int K)
{
    double re = 0.0, im = 0.0, ip1 = 0.0, ip2 = 0.0;   // I_{k+1}, I_{k+2}
    for (int k = K; k >= 0; --k) {
        const double Ik = (k + 1 <= K ? 2.0 * J[k + 1] : 0.0) + ip2;
        ip2 = ip1;
        ip1 = Ik;
        const double t = Ik * v[k * vstride] * (k == 0 ? 1.0 : 2.0);
        switch (k & 3) {
        case 0: re += t; break;
        case 1: im -= t; break;
        case 2: re -= t; break;
        default: im += t; break;
        }
    }
    return make_double2(re, im);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Gershgorin centre c and half-width r of T (lanes own rows), then the Chebyshev vectors
// T_k(T~) e_1 for k = 0..K into sm.tch.  Returns (c, r) in every lane.
__device__ double2 chebyshev_basis(ExpSmem &sm, int me, int K)
{
    const int j = threadIdx.x;
    const double a = (j < me) ? sm.al[j] : 0.0;
    const double bl = (j >= 1 && j < me) ? fabs(sm.be[j - 1]) : 0.0;
    const double br = (j + 1 < me) ? fabs(sm.be[j]) : 0.0;
    double lo = (j < me) ? a - bl - br : 1e300, hi = (j < me) ? a + bl + br : -1e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double c = 0.5 * (lo + hi);
    double r = 0.5 * (hi - lo);
    const double rmin = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
    if (!(r > rmin)) r = rmin;
    const double ir = 1.0 / r;
    const double dj = (j < me) ? (a - c) * ir : 0.0;
    const double ol = (j >= 1 && j < me) ? sm.be[j - 1] * ir : 0.0;
    const double orr = (j + 1 < me) ? sm.be[j] * ir : 0.0;
    double v0 = (j == 0) ? 1.0 : 0.0;
    sm.tch[j] = v0;
    double up = __shfl_up_sync(0xffffffffu, v0, 1), dn = __shfl_down_sync(0xffffffffu, v0, 1);
    double v1 = dj * v0 + ol * up + orr * dn;
    if (K >= 1) sm.tch[32 + j] = v1;
    for (int k = 2; k <= K; ++k) {
        up = __shfl_up_sync(0xffffffffu, v1, 1);
        dn = __shfl_down_sync(0xffffffffu, v1, 1);
        const double v2 = 2.0 * (dj * v1 + ol * up + orr * dn) - v0;
        sm.tch[k * 32 + j] = v2;
        v0 = v1;
        v1 = v2;
    }
    __syncwarp();
    return make_double2(c, r);
}

// <psi0|psi(t_now + tp)> from the expansion of the step (one Bessel sequence into J).
__device__ double2 step_readout(const ExpSmem &sm, double tp, double c, double r, int K, double beta0,
                                double *J)
{
    bessel_seq(tp * r, K, J);
    double re = 0.0, im = 0.0;
    for (int k = 0; k <= K; ++k) {
        const double t = J[k] * (k == 0 ? 1.0 : 2.0);
        const double2 G = sm.gk[k];
        // w_k G_k with w_k = (-i)^k
        switch (k & 3) {
        case 0: re += t * G.x; im += t * G.y; break;
        case 1: re += t * G.y; im -= t * G.x; break;
        case 2: re -= t * G.x; im -= t * G.y; break;
        default: re -= t * G.y; im += t * G.x; break;
        }
    }
    double sn, cs;
    sincos(tp * c, &sn, &cs);
    return cmul(make_double2(cs, -sn), make_double2(re * beta0, im * beta0));
}

// int_{t_now}^{t_now + s} P(t') dt' by NGL-point Gauss-Legendre on the step's expansion
// (warp-collective: every lane passes the same s and gets the sum).  P is an entire
// function of t' whose frequencies are bounded by the half-width r, and s r <= XMAX = 50,
// so 64 nodes integrate it to rounding.
__device__ double step_integral(const ExpSmem &sm, const double *glx, const double *glw, double s, double c,
                                double r, int K, double beta0, double *J)
{
    double acc = 0.0;
    for (int q = threadIdx.x; q < NGL; q += 32) {
        const double2 A = step_readout(sm, 0.5 * s * (1.0 + glx[q]), c, r, K, beta0, J);
        acc += glw[q] * (A.x * A.x + A.y * A.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return 0.5 * s * acc;
}

__global__ void __launch_bounds__(32) k_smallexp(ExpArgs ea)
{
    pdl_begin();
    KryCtl *ctl = ea.ctl;
    if (ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ExpSmem &sm = *(ExpSmem *)smem_raw;
    const int lane = threadIdx.x;
    const int me = ctl->m_eff;
    if (lane < me) {
        sm.al[lane] = ctl->alpha[lane];
        sm.be[lane] = ctl->beta[lane];
        double2 g;
        if (ctl->r0 >= 0) {
            const size_t idx = (size_t)lane * ea.ldW + (size_t)ctl->r0;
            double2 w;
            if (ea.c64) { float2 f = ((const float2 *)ea.W)[idx]; w = make_double2(f.x, f.y); }
            else if (ea.ff) { float4 f = ((const float4 *)ea.W)[idx]; w = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w); }
            else w = ((const double2 *)ea.W)[idx];
            // <psi0|v_j> with psi0 = e_{r0}: the (real-valued psi0) conjugate is trivial
            const double s = ctl->sigma[lane];
            g = make_double2(w.x * s, w.y * s);
        } else {
            g = ctl->g[lane];
        }
        sm.g[lane] = g;
    }
    __syncwarp();
    const double beta0 = ctl->beta0, h = sm.be[me - 1];
    const double t_now = ctl->t_now, t_end = ctl->t_end, tol = ctl->tol;
    const double remaining = t_end - t_now;
    // provisional radius for the step cap (recomputed exactly by chebyshev_basis)
    double2 cr;
    {
        const int j = lane;
        const double a = (j < me) ? sm.al[j] : 0.0;
        const double bl = (j >= 1 && j < me) ? fabs(sm.be[j - 1]) : 0.0;
        const double br = (j + 1 < me) ? fabs(sm.be[j]) : 0.0;
        double lo = (j < me) ? a - bl - br : 1e300, hi = (j < me) ? a + bl + br : -1e300;
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        double r = 0.5 * (hi - lo);
        const double rmin = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
        cr = make_double2(0.5 * (lo + hi), r > rmin ? r : rmin);
    }
    const double tau_hi = fmin(remaining, XMAX / cr.y);
    const int K = cheb_degree(tau_hi * cr.y);
    cr = chebyshev_basis(sm, me, K);
    // T holds the coefficients of H - s I: the phase centre of exp(-i tau T) gets s back
    const double c = cr.x + ctl->shift, r = cr.y;
    double *myJ = sm.jb + lane * (KMAX + 2);

    // ---- step-size ladder
    double tau_top = tau_hi, tau = 0.0, err = 0.0;
    int pick = -1;
    for (int round = 0; round < 4 && pick < 0; ++round) {
        const double tq = tau_top * pow(LADDER, (double)lane);
        bessel_seq(tq * r, K, myJ);
        double eq = 0.0;
        if (h != 0.0) {
            const double2 s = integral_sum(myJ, sm.tch + (me - 1), 32, K);
            eq = beta0 * fabs(h) / r * sqrt(s.x * s.x + s.y * s.y);
        }
        // a step's error budget must stay above the FP64 rounding unit of psi, otherwise
        // the tolerance is unreachable (KRY_ETOL) rather than met by ever smaller steps
        const double budget = STEP_SAFETY * 0.5 * tol * tq / t_end;
        const bool ok = tq > 0.0 && budget >= 2.3e-16 * beta0 && eq <= budget;
        const unsigned mask = __ballot_sync(0xffffffffu, ok || (remaining <= 0.0));
        if (mask) {
            pick = __ffs(mask) - 1;
            tau = __shfl_sync(0xffffffffu, tq, pick);
            err = __shfl_sync(0xffffffffu, eq, pick);
        } else {
            tau_top *= pow(LADDER, 32.0);
        }
    }
    __syncwarp();
    if (pick < 0) {
        if (lane == 0) { ctl->err = KRY_ETOL; ctl->done = 1; }
        return;
    }
    const bool last = (tau >= remaining);
    // ---- y(tau) -> combine coefficients
    const double *Jp = sm.jb + pick * (KMAX + 2);
    if (lane < me) {
        const double2 s = jacobi_anger_sum(Jp, sm.tch + lane, 32, K);
        double sn, cs;
        sincos(tau * c, &sn, &cs);
        const double2 y = cmul(make_double2(cs, -sn), s);
        const double f = -beta0 * ctl->sigma[lane];
        ctl->coefY[lane] = make_double2(f * y.x, f * y.y);
    }
    // ---- G_k = sum_j g_j [T_k e_1]_j
    for (int k = lane; k <= K; k += 32) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < me; ++j) {
            const double t = sm.tch[k * 32 + j];
            re += sm.g[j].x * t;
            im += sm.g[j].y * t;
        }
        sm.gk[k] = make_double2(re, im);
    }
    __syncwarp();
    // ---- dense output at every output time inside [t_now, t_now + tau]
    int next = ctl->next_out;
    const int n_times = ctl->n_times;
    while (next < n_times) {
        const int o = next + lane;
        double tp = 0.0;
        bool in = false;
        if (o < n_times) {
            tp = ea.times[o] - t_now;
            in = last ? true : (tp <= tau * (1.0 + 1e-12));
            if (tp < 0.0) tp = 0.0;
        }
        const unsigned mk = __ballot_sync(0xffffffffu, in);
        const int cnt = __popc(mk & ~(mk + 1u));   // leading run of lanes (times are sorted)
        if (lane < cnt) {
            const double2 A = step_readout(sm, tp, c, r, K, beta0, myJ);
            ea.P[o] = A.x * A.x + A.y * A.y;
        }
        if (ea.Yout) {
            // whole-vector dense output: psi(t_o) = sum_j Yout[o][j] W_j with
            // Yout[o][j] = beta sigma_j [exp(-i tau' T) e_1]_j, from the same Bessel rows
            __syncwarp();
            for (int bq = 0; bq < cnt; ++bq) {
                const double tpb = __shfl_sync(0xffffffffu, tp, bq);
                if (lane < me) {
                    const double2 s = jacobi_anger_sum(sm.jb + bq * (KMAX + 2), sm.tch + lane, 32, K);
                    double sn, cs;
                    sincos(tpb * c, &sn, &cs);
                    const double2 y = cmul(make_double2(cs, -sn), s);
                    const double f = beta0 * ctl->sigma[lane];
                    ea.Yout[(size_t)(next + bq) * MMAX + lane] = make_double2(f * y.x, f * y.y);
                }
            }
            __syncwarp();
        }
        next += cnt;
        if (cnt < 32) break;
    }
    if (ea.C) {
        // temporal autocorrelation (Sec. 4): C(t_o) = (int_0^{t_o} P) / t_o for the output
        // times of this step, and the running integral over the whole step
        __syncwarp();
        const double pint = ctl->pint;
        for (int o = ctl->next_out; o < next; ++o) {
            const double to = ea.times[o];
            const double s = fmax(to - t_now, 0.0);
            const double I = step_integral(sm, ea.glx, ea.glw, s, c, r, K, beta0, myJ);
            if (lane == 0) ea.C[o] = to > 0.0 ? (pint + I) / to : 1.0;
        }
        if (!last) {
            const double I = step_integral(sm, ea.glx, ea.glw, tau, c, r, K, beta0, myJ);
            if (lane == 0) ctl->pint = pint + I;
        }
        __syncwarp();
    }
    if (lane == 0) {
        ctl->out_begin = ctl->next_out;
        ctl->out_end = next;
        ctl->next_out = next;
        ctl->t_now = last ? t_end : t_now + tau;
        ctl->tau_prev = tau;
        ctl->n_steps += 1;
        ctl->err_sum += err;
        if (next >= n_times) ctl->finishing = 1;
    }
}

// Test hook: y = exp(-i tau T) e_1 and err(tau) for given T, h (beta = 1).
__global__ void __launch_bounds__(32) k_expv_test(const double *alpha, const double *beta, int me,
                                                  double h, double tau, double *y, double *err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ExpSmem &sm = *(ExpSmem *)smem_raw;
    const int lane = threadIdx.x;
    if (lane < me) {
        sm.al[lane] = alpha[lane];
        sm.be[lane] = (lane + 1 < me) ? beta[lane] : h;
    }
    __syncwarp();
    // radius first (with K = 0), then the full basis for the needed degree
    double2 cr = chebyshev_basis(sm, me, 0);
    const int K = cheb_degree(tau * cr.y);
    cr = chebyshev_basis(sm, me, K);
    double *myJ = sm.jb + lane * (KMAX + 2);
    bessel_seq(tau * cr.y, K, myJ);
    __syncwarp();
    const double *J0 = sm.jb;   // lane 0's sequence (all lanes computed the same)
    if (lane < me) {
        const double2 s = jacobi_anger_sum(J0, sm.tch + lane, 32, K);
        double sn, cs;
        sincos(tau * cr.x, &sn, &cs);
        const double2 yy = cmul(make_double2(cs, -sn), s);
        y[2 * lane] = yy.x;
        y[2 * lane + 1] = yy.y;
    }
    if (lane == 0) {
        const double2 s = integral_sum(J0, sm.tch + (me - 1), 32, K);
        *err = fabs(h) / cr.y * sqrt(s.x * s.x + s.y * s.y);
    }
}

// ---------------------------------------------------------------- batched realisations
// Every realisation k has its own T_k, coupling h_k and norm beta_k.  k_exp_scan_b finds,
// per realisation, the largest ladder step that meets the error budget; k_exp_apply_b takes
// the smallest of those (the leading error term grows with the step, so every realisation
// stays within its budget), builds exp(-i tau T_k) e_1 for the combine and reads P_k at
// every output time inside the step.

__device__ void load_tridiag_b(ExpSmem &sm, const KryCtlB *ctl, int k, int me, const ExpArgsB &ea)
{
    const int lane = threadIdx.x;
    if (lane < me) {
        sm.al[lane] = ctl->alpha[lane][k];
        sm.be[lane] = ctl->beta[lane][k];
        double2 g;
        if (ctl->hd.r0 >= 0) {
            const size_t idx = (size_t)lane * ea.ldW + (size_t)ctl->r0k[k] * ea.K + k;
            double2 w;
            if (ea.c64) { float2 f = ((const float2 *)ea.W)[idx]; w = make_double2(f.x, f.y); }
            else if (ea.ff) { float4 f = ((const float4 *)ea.W)[idx]; w = make_double2((double)f.x + (double)f.y, (double)f.z + (double)f.w); }
            else w = ((const double2 *)ea.W)[idx];
            const double s = ctl->sigma[lane][k];
            g = make_double2(w.x * s, w.y * s);
        } else {
            g = ctl->g[lane][k];
        }
        sm.g[lane] = g;
    }
    __syncwarp();
}

__device__ double2 gershgorin(const ExpSmem &sm, int me)
{
    const int j = threadIdx.x;
    const double a = (j < me) ? sm.al[j] : 0.0;
    const double bl = (j >= 1 && j < me) ? fabs(sm.be[j - 1]) : 0.0;
    const double br = (j + 1 < me) ? fabs(sm.be[j]) : 0.0;
    double lo = (j < me) ? a - bl - br : 1e300, hi = (j < me) ? a + bl + br : -1e300;
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const double r = 0.5 * (hi - lo);
    const double rmin = 1e-12 * fmax(1.0, fmax(fabs(lo), fabs(hi)));
    return make_double2(0.5 * (lo + hi), r > rmin ? r : rmin);
}

__global__ void __launch_bounds__(32) k_exp_scan_b(ExpArgsB ea)
{
    KryCtlB *ctl = ea.ctl;
    const KryHdrB &H = ctl->hd;
    if (H.done) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ExpSmem &sm = *(ExpSmem *)smem_raw;
    const int k = blockIdx.x, lane = threadIdx.x;
    const int me = ctl->m_eff[k];
    load_tridiag_b(sm, ctl, k, me, ea);
    const double beta0 = ctl->beta0[k], h = sm.be[me - 1];
    const double remaining = H.t_end - H.t_now;
    double2 cr = gershgorin(sm, me);
    const double tau_hi = fmin(remaining, XMAX / cr.y);
    const int Kc = cheb_degree(tau_hi * cr.y);
    cr = chebyshev_basis(sm, me, Kc);
    const double r = cr.y;
    double *myJ = sm.jb + lane * (KMAX + 2);
    double tau_top = tau_hi, tau = 0.0;
    int pick = -1;
    for (int round = 0; round < 4 && pick < 0; ++round) {
        const double tq = tau_top * pow(LADDER, (double)lane);
        bessel_seq(tq * r, Kc, myJ);
        double eq = 0.0;
        if (h != 0.0) {
            const double2 s = integral_sum(myJ, sm.tch + (me - 1), 32, Kc);
            eq = beta0 * fabs(h) / r * sqrt(s.x * s.x + s.y * s.y);
        }
        const double budget = STEP_SAFETY * 0.5 * H.tol * tq / H.t_end;
        const bool ok = tq > 0.0 && budget >= 2.3e-16 * beta0 && eq <= budget;
        const unsigned mask = __ballot_sync(0xffffffffu, ok || (remaining <= 0.0));
        if (mask) {
            pick = __ffs(mask) - 1;
            tau = __shfl_sync(0xffffffffu, tq, pick);
        } else {
            tau_top *= pow(LADDER, 32.0);
        }
    }
    if (lane == 0) {
        ctl->tau_ok[k] = (pick < 0) ? -1.0 : tau;
        if (pick < 0) ctl->hd.err = KRY_ETOL;
    }
}

__global__ void __launch_bounds__(32) k_exp_apply_b(ExpArgsB ea)
{
    KryCtlB *ctl = ea.ctl;
    KryHdrB &H = ctl->hd;
    if (H.done) return;
    const int k = blockIdx.x, lane = threadIdx.x;
    if (H.err) {
        if (k == 0 && lane == 0) H.done = 1;
        return;
    }
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ExpSmem &sm = *(ExpSmem *)smem_raw;
    double tau = 1e300;
    for (int kk = lane; kk < ea.K; kk += 32) tau = fmin(tau, ctl->tau_ok[kk]);
    for (int o = 16; o > 0; o >>= 1) tau = fmin(tau, __shfl_xor_sync(0xffffffffu, tau, o));
    const int me = ctl->m_eff[k];
    load_tridiag_b(sm, ctl, k, me, ea);
    const double beta0 = ctl->beta0[k], h = sm.be[me - 1];
    const double t_now = H.t_now, t_end = H.t_end, remaining = t_end - t_now;
    const bool last = (tau >= remaining);
    double2 cr = gershgorin(sm, me);
    const int Kc = cheb_degree(tau * cr.y);
    cr = chebyshev_basis(sm, me, Kc);
    const double c = cr.x + ctl->shift[k], r = cr.y;   // T holds H_k - s_k I
    double *myJ = sm.jb + lane * (KMAX + 2);
    bessel_seq(tau * r, Kc, myJ);
    if (lane < me) {
        const double2 s = jacobi_anger_sum(myJ, sm.tch + lane, 32, Kc);
        double sn, cs;
        sincos(tau * c, &sn, &cs);
        const double2 y = cmul(make_double2(cs, -sn), s);
        const double f = -beta0 * ctl->sigma[lane][k];
        ctl->coefY[lane][k] = make_double2(f * y.x, f * y.y);
    } else if (lane < MMAX) {
        ctl->coefY[lane][k] = make_double2(0.0, 0.0);
    }
    if (lane == 0) {
        double e = 0.0;
        if (h != 0.0) {
            const double2 s = integral_sum(myJ, sm.tch + (me - 1), 32, Kc);
            e = beta0 * fabs(h) / r * sqrt(s.x * s.x + s.y * s.y);
        }
        ctl->err_k[k] = e;
    }
    for (int kk = lane; kk <= Kc; kk += 32) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < me; ++j) {
            const double t = sm.tch[kk * 32 + j];
            re += sm.g[j].x * t;
            im += sm.g[j].y * t;
        }
        sm.gk[kk] = make_double2(re, im);
    }
    __syncwarp();
    int next = H.next_out;
    const int n_times = H.n_times;
    while (next < n_times) {
        const int o = next + lane;
        double tp = 0.0;
        bool in = false;
        if (o < n_times) {
            tp = ea.times[o] - t_now;
            in = last ? true : (tp <= tau * (1.0 + 1e-12));
            if (tp < 0.0) tp = 0.0;
        }
        const unsigned mk = __ballot_sync(0xffffffffu, in);
        const int cnt = __popc(mk & ~(mk + 1u));
        if (lane < cnt) {
            const double2 A = step_readout(sm, tp, c, r, Kc, beta0, myJ);
            ea.P[(size_t)o * ea.K + k] = A.x * A.x + A.y * A.y;
        }
        next += cnt;
        if (cnt < 32) break;
    }
    if (ea.C) {
        // temporal autocorrelation of realisation k (Sec. 4), as in the single path
        __syncwarp();
        const double pint = ctl->pint[k];
        for (int o = H.next_out; o < next; ++o) {
            const double to = ea.times[o];
            const double s = fmax(to - t_now, 0.0);
            const double I = step_integral(sm, ea.glx, ea.glw, s, c, r, Kc, beta0, myJ);
            if (lane == 0) ea.C[(size_t)o * ea.K + k] = to > 0.0 ? (pint + I) / to : 1.0;
        }
        if (!last) {
            const double I = step_integral(sm, ea.glx, ea.glw, tau, c, r, Kc, beta0, myJ);
            if (lane == 0) ctl->pint[k] = pint + I;
        }
        __syncwarp();
    }
    if (k == 0 && lane == 0) {
        H.next_out_new = next;
        H.t_next = last ? t_end : t_now + tau;
        H.finishing = (next >= n_times) ? 1 : 0;
    }
}

int launch_exp_b(const ExpArgsB &a, cudaStream_t s)
{
    KRY_CU(cudaFuncSetAttribute(k_exp_scan_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ExpSmem)));
    KRY_CU(cudaFuncSetAttribute(k_exp_apply_b, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ExpSmem)));
    k_exp_scan_b<<<a.K, 32, sizeof(ExpSmem), s>>>(a);
    KRY_CU(cudaGetLastError());
    k_exp_apply_b<<<a.K, 32, sizeof(ExpSmem), s>>>(a);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_smallexp(const ExpArgs &a, cudaStream_t s, int pdl)
{
    KRY_CU(cudaFuncSetAttribute(k_smallexp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(ExpSmem)));
    KRY_CU(launch_ex(pdl, k_smallexp, 1, 32, sizeof(ExpSmem), s, a));
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

}  // namespace kry

using namespace kry;

extern "C" int kry_tridiag_expv(const double *alpha, const double *beta, int m, double h, double tau,
                                double *y_out, double *err_out, void *stream)
{
    if (!alpha || (m > 1 && !beta) || !y_out || !err_out || m < 1 || m > MMAX || !(tau >= 0.0) ||
        !(tau * 1.0 < 1e300)) {
        set_error("kry_tridiag_expv: bad arguments");
        return KRY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double *d = nullptr;
    KRY_CU(cudaMalloc(&d, sizeof(double) * (4 * MMAX + 2)));
    double *da = d, *db = d + MMAX, *dy = d + 2 * MMAX, *de = d + 4 * MMAX;
    cudaError_t e = cudaMemcpyAsync(da, alpha, sizeof(double) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && m > 1)
        e = cudaMemcpyAsync(db, beta, sizeof(double) * (m - 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_expv_test, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ExpSmem));
    if (e == cudaSuccess) {
        k_expv_test<<<1, 32, sizeof(ExpSmem), s>>>(da, db, m, h, tau, dy, de);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_out, dy, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err_out, de, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "kry_tridiag_expv");
    return KRY_OK;
}

// ---------------------------------------------------------------- allocation-free variant
//
// kry_tridiag_expv_noalloc runs the same kernel as kry_tridiag_expv, but its device-side
// copies of alpha, beta and the results live in the fixed array below instead of memory
// from cudaMalloc.  It serves callers that hand all device memory to their own pool with a
// hard cap, and callers that cannot accept the device-wide synchronisation that cudaFree
// performs while their other streams are busy.
//
// The array holds alpha[32], beta[32], y[64] and err (about 1 KB).  Every GPU that loads
// this library keeps it for the life of the process.  Host code cannot pass the array's
// name to a kernel (in host code it is a stand-in, not a device address), so the call looks
// up the real address with cudaGetSymbolAddress while the caller's device is current, once
// per device and CUDA context: the address is kept together with the id of the context it
// was looked up in, and looked up again when the current context differs (after a
// cudaDeviceReset the module is loaded anew and the array may move).  When the driver
// cannot report a context id the address is looked up on every call.

#include <mutex>

static __device__ __align__(256) double g_expv_scratch[4 * kry::MMAX + 8];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_expv_mu;
struct ScratchAddr {
    unsigned long long ctx_id;   // 0 = not looked up
    double *ptr;
};
ScratchAddr g_expv_addr[kMaxDevices] = {};

// Id of the calling thread's current CUDA context (unique over the process's lifetime), or 0
// if there is none or the driver cannot say.  The two driver calls are fetched through the
// runtime, so the library does not link the driver library itself.
unsigned long long current_context_id()
{
    typedef int (*get_current_t)(void **);
    typedef int (*get_id_t)(void *, unsigned long long *);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (get_current_t)p;
        p = nullptr;
        q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (get_id_t)p;
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return 0;
    unsigned long long id = 0;
    if (get_id(ctx, &id) != 0) return 0;
    return id;
}

int expv_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("kry_tridiag_expv_noalloc: device ordinal %d is above %d", dev, kMaxDevices - 1);
        return KRY_EINVAL;
    }
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_expv_mu);
    ScratchAddr &a = g_expv_addr[dev];
    if (id == 0 || a.ctx_id != id || !a.ptr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_expv_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_expv_scratch)");
        a.ptr = (double *)p;
        a.ctx_id = current_context_id();   // the lookup made the runtime's context current
    }
    *out = a.ptr;
    return KRY_OK;
}
}  // namespace

extern "C" int kry_tridiag_expv_noalloc(const double *alpha, const double *beta, int m, double h,
                                        double tau, double *y_out, double *err_out, void *stream)
{
    if (m > MMAX) {
        set_error("kry_tridiag_expv_noalloc: m = %d exceeds the maximum %d that its fixed "
                  "device scratch holds", m, MMAX);
        return KRY_EINVAL;
    }
    if (!alpha || (m > 1 && !beta) || !y_out || !err_out || m < 1 || !(tau >= 0.0) ||
        !(tau < 1e300)) {
        set_error("kry_tridiag_expv_noalloc: bad arguments");
        return KRY_EINVAL;
    }
    double *d = nullptr;
    if (int rc = expv_scratch(&d)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    double *da = d, *db = d + MMAX, *dy = d + 2 * MMAX, *de = d + 4 * MMAX;
    // Every element the kernel reads is copied in below and every element read back is
    // written by the kernel, so nothing left over from an earlier call is used.
    cudaError_t e = cudaMemcpyAsync(da, alpha, sizeof(double) * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && m > 1)
        e = cudaMemcpyAsync(db, beta, sizeof(double) * (m - 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_expv_test, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(ExpSmem));
    if (e == cudaSuccess) {
        k_expv_test<<<1, 32, sizeof(ExpSmem), s>>>(da, db, m, h, tau, dy, de);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_out, dy, sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(err_out, de, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "kry_tridiag_expv_noalloc");
    return KRY_OK;
}
