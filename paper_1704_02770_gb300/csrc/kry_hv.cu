// Vector kernels of the Krylov step (Sec. 2, "Krylov subspace methods"):
//   k_apply     y = H x (matrix-free, Eq. 1)
//   k_hv        u = sigma_j H v_j with alpha_j = <v_j, u> and ||u||^2 (pass A, part 1)
//   k_dots      <v_i, y> for the Krylov vectors, a tall-skinny GEMV with plain loads
//               (pass A part 2 with y = u; pass C1 with y = w)
//   k_lincomb   w = src - sum_i c_i W_i (MODE 0: Lanczos update, pass B; 1: the second
//               Gram-Schmidt subtraction, pass C2; 2: combine psi = beta V y; 3: load the
//               initial vector)
// Every reduction ends in the last CTA to finish (ticket counter), which sums the
// per-CTA partials in CTA order: results are bitwise reproducible for a fixed grid.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kry_device.cuh"

namespace kry {

struct SmemHead {
    uint32_t koff[20];
    uint32_t bsz[20];
};

// ---------------------------------------------------------------- y = H x

template <class V>
__global__ void __launch_bounds__(NTHR) k_apply(DevBasis b, DevHam hm, const V *__restrict__ x,
                                                V *__restrict__ y, int rl_smem)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemHead *hd = (SmemHead *)smem;
    uint16_t *rl_s = (uint16_t *)(smem + sizeof(SmemHead));
    stage_tables(b, hd->koff, hd->bsz, rl_s, rl_smem);
    __syncthreads();
    const uint16_t *rl = rl_smem ? rl_s : b.ranklo;
    const uint32_t ntiles = (b.D + TILE - 1) / TILE;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TILE, t = threadIdx.x;
        if (r0 + t < b.D) {
            uint32_t hi, off;
            int klo;
            tile_unrank(b, hd->bsz, r0, t, hi, off, klo);
            y[r0 + t] = hv_row<V>(b, hm, x, hi, off, klo, hd->koff, rl);
        }
    }
}

// ---------------------------------------------------------------- reductions

// Write this CTA's partials, then let the last CTA to finish sum all partials into
// fin[0..PSTRIDE).  Returns true in the last CTA (all its threads).  Only the slots [0, nlead)
// and, with tail set, SLOT_NRM and SLOT_G are summed (the others of fin are zero), and all
// NTHR threads share the work: each of the ns needed slots gets TPS = NTHR / ns threads
// (rounded down to a power of two), thread t of a slot adds the partials of CTAs t, t + TPS,
// ..., and the TPS sums are added by a pairwise tree.  With few slots (the updates need two)
// this keeps the serial tail of the last CTA to a few loads per thread.  The summation order
// depends only on the grid and the slot count, so results are bitwise reproducible.
__device__ __forceinline__ bool finish_partials(const double2 *red, double2 *part, KryCtl *ctl,
                                                double2 *fin, int *flag, unsigned *counter = nullptr,
                                                int nlead = PSTRIDE, bool tail = true)
{
    __shared__ double2 tsum[NTHR];
    __shared__ int slots[PSTRIDE];
    const int tid = threadIdx.x;
    if (!counter) counter = &ctl->counter;
    if (tid < PSTRIDE) part[(size_t)blockIdx.x * PSTRIDE + tid] = red[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) *flag = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
    __syncthreads();
    if (!*flag) return false;
    __threadfence();
    int ns = 0;
    for (int sl = 0; sl < PSTRIDE; ++sl)
        if (sl < nlead || (tail && (sl == SLOT_NRM || sl == SLOT_G))) {
            if (tid == 0) slots[ns] = sl;
            ++ns;
        }
    int tps = 1;
    while (tps * 2 * ns <= NTHR && tps < 128) tps *= 2;
    if (tid < PSTRIDE) fin[tid] = make_double2(0.0, 0.0);
    __syncthreads();
    const int si = tid / tps, t = tid - si * tps;
    if (si < ns) {
        const int slot = slots[si];
        double2 sum = make_double2(0.0, 0.0);
#pragma unroll 4
        for (unsigned c = t; c < gridDim.x; c += tps) {
            const double2 v = __ldcg(part + (size_t)c * PSTRIDE + slot);
            sum.x += v.x;
            sum.y += v.y;
        }
        tsum[tid] = sum;
    }
    __syncthreads();
    for (int w = tps / 2; w > 0; w >>= 1) {
        if (si < ns && t < w) {
            tsum[tid].x += tsum[tid + w].x;
            tsum[tid].y += tsum[tid + w].y;
        }
        __syncthreads();
    }
    if (si < ns && t == 0) fin[slots[si]] = tsum[tid];
    __syncthreads();
    return true;
}

// Sum per-thread values over the CTA (warp shuffles, then warps in order) into red[slot].
__device__ __forceinline__ void cta_sum_into(double2 v, double2 *red, int slot, double2 *wtmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) wtmp[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < NTHR / 32; ++w) { s.x += wtmp[w].x; s.y += wtmp[w].y; }
        red[slot] = s;
    }
    __syncthreads();
}

// The same for per-thread dot accumulators (float-float warp sums for complex64).
template <class Acc>
__device__ __forceinline__ void cta_sum_into(const Acc &acc, double2 *red, int slot, double2 *wtmp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double2 v = acc.warp_value();
    if (lane == 0) wtmp[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < NTHR / 32; ++w) { s.x += wtmp[w].x; s.y += wtmp[w].y; }
        red[slot] = s;
    }
    __syncthreads();
}

// beta_j = ||w|| and the scale of the next vector, or the end of the Krylov space
__device__ __forceinline__ void finalize_beta(KryCtl *ctl, int jj, double nw2, double2 gdot)
{
    const double bt = sqrt(nw2);
    ctl->beta[jj] = bt;
    if (!(bt > ctl->eta_bd * sqrt(ctl->normu2))) {   // invariant subspace (or zero vector)
        ctl->m_eff = jj + 1;
        ctl->n_bd += 1;
    } else {
        const double s = 1.0 / bt;
        ctl->sigma[jj + 1] = s;
        ctl->g[jj + 1] = make_double2(gdot.x * s, gdot.y * s);
    }
}

// ---------------------------------------------------------------- pass A

// u = sigma_j H W_j, written to U (pass A, part 1).  One thread per row at full occupancy
// and nothing else: the gathers of the hops are latency-bound, so as many rows as possible
// are kept in flight.  alpha_j, ||u||^2 and the dots with the earlier vectors are taken by
// the streaming pass that follows (k_dots, mode 0).  FORM 0 gathers the hops one by one
// (hv_row_scaled), FORM 1 in rounds of four loads in flight (hv_row_chunked); both give the
// same bits, the launch shape picks the faster (kry_autotune).
template <class V, int FORM>
__global__ void __launch_bounds__(NTHR) k_hv(EvArgs<V> a, int jj)
{
    pdl_begin();
    KryCtl *ctl = a.ctl;
    if (ctl->done || jj >= ctl->m_eff) return;
    using R = typename VT<V>::R;
    extern __shared__ __align__(16) unsigned char smem[];
    SmemHead *hd = (SmemHead *)smem;
    uint16_t *rl_s = (uint16_t *)(smem + sizeof(SmemHead));
    __shared__ R dz[64];
    if (threadIdx.x <= (unsigned)a.b.L) dz[threadIdx.x] = (R)(a.h.cz * (double)(a.h.nbonds - 2 * (int)threadIdx.x));
    stage_tables(a.b, hd->koff, hd->bsz, rl_s, a.rl_smem);
    __syncthreads();
    const uint16_t *rl = a.rl_smem ? rl_s : a.b.ranklo;
    const double s = ctl->sigma[jj];
    const R sj = (R)s, shj = (R)(s * a.h.halfJ);
    const V *x = a.W + (size_t)jj * a.ldW;
    const uint32_t D = a.b.D, ntiles = (D + TILE - 1) / TILE;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TILE, r = r0 + threadIdx.x;
        if (r < D) {
            uint32_t hi, off;
            int klo;
            tile_unrank(a.b, hd->bsz, r0, threadIdx.x, hi, off, klo);
            a.U[r] = FORM == 1 ? hv_row_chunked<V>(a.b, a.h, x, hi, off, klo, hd->koff, rl, dz, sj, shj)
                               : hv_row_scaled<V>(a.b, a.h, x, hi, off, klo, hd->koff, rl, dz, sj, shj);
        }
    }
}

// Dots <W_i, y>, i <= j, of a right-hand vector y with the Krylov vectors: a tall-skinny
// GEMV with plain loads.  The vectors are read as KC interleaved columns of rows (thread k
// takes rows r0 + k + KC e, so a warp loads 32 consecutive rows), and thread (k, g) takes
// the vectors i = g, g + NG, ... with one accumulator per vector, so the accumulations of
// different vectors overlap.  The rows of the next vector are loaded before the current
// vector's products are accumulated (software prefetch), so the loads of one vector are in
// flight during the arithmetic of the one before: the complex64 accumulation is error-free
// float-float arithmetic, about as much FP32 work per byte as the HBM stream supplies, and
// without the overlap the kernel alternates between waiting on loads and on the FP32 pipe.
// complex64: KC = 32 (a warp per group of vectors), two CTAs per SM (the prefetch buffer
// needs the registers); complex128 (FP64-bound, no prefetch): KC = 64, two.  The sums over
// the columns are taken in a fixed order at the end.  PFT = 0 turns the prefetch off (a
// launch-shape choice of kry_autotune; the bits are the same).
//   MODE 0 (pass A): y = U = sigma_j H W_j; fills coefA[0..j], alpha_j and ||u||^2.
//   MODE 1 (pass C1, when pass B flagged it): y = W_{j+1}; measures the loss of
//          orthogonality and sets up the subtraction of pass C2 when it exceeds eta_corr.
template <class V, int MODE, int PFT>
__global__ void __launch_bounds__(NTHR, 2) k_dots(EvArgs<V> a, int jj)
{
    pdl_begin();
    KryCtl *ctl = a.ctl;
    if (ctl->done || jj >= ctl->m_eff) return;
    if (MODE == 1 && !ctl->corr) return;
    constexpr bool DD = std::is_same<V, ffc>::value;   // float-float vectors
    constexpr bool F32 = std::is_same<V, float2>::value;
    constexpr int KC = (F32 || DD) ? 32 : 64;          // columns (rows in flight per vector)
    constexpr int RT = DD ? 4 : 8;                      // rows per column and tile
    constexpr int NG = NTHR / KC, QD = (MMAX + NG - 1) / NG, TR = KC * RT;
    constexpr bool PF = PFT && (F32 || DD);   // prefetch (complex128 is FP64-bound: no gain)
    using Acc = typename std::conditional<F32, DotAccF2, DotAcc<V>>::type;
    __shared__ double2 red[PSTRIDE];
    __shared__ double2 wred[NTHR / 32][QD + 1];
    __shared__ int flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = tid % KC, g = tid / KC;
    if (tid < PSTRIDE) red[tid] = make_double2(0.0, 0.0);
    const V *y = (MODE == 0) ? a.U : a.W + (size_t)(jj + 1) * a.ldW;
    const int nv = jj + 1;   // vectors W_0 .. W_j
    const uint32_t D = a.b.D, ntiles = (D + TR - 1) / TR;
    // Work split: with nv = NG A + B, every group takes A whole vectors (g, g + NG, ...) over
    // all the CTA's tiles, and the B remaining vectors are shared by all groups: RX = NG / B
    // groups per remaining vector (group g: vector NG A + g mod B, every RX-th tile of the
    // CTA from g / B), so every warp streams about the same number of rows at every j; the
    // partial sums of the groups that share a vector are added at the end.
    const int A = nv / NG, Bn = nv % NG;
    const int RX = Bn > 0 ? NG / Bn : 1;
    const bool hasx = Bn > 0 && g < Bn * RX;
    const int xv = NG * A + (Bn > 0 ? g % Bn : 0), xs = Bn > 0 ? g / Bn : 0;
    const int nslot = A + (hasx ? 1 : 0);   // accumulators this group uses
    Acc acc[QD];
    DotAcc<V> nrm;
    // the norm of y: group 0 over all tiles when A > 0, else the groups of vector 0
    const bool own_norm = MODE == 0 && (A > 0 ? g == 0 : (hasx && xv == 0));
    uint32_t tl = 0;   // local index of the tile within this CTA
    for (uint32_t tile = blockIdx.x; nslot > 0 && tile < ntiles; tile += gridDim.x, ++tl) {
        const bool xt = hasx && (int)(tl % (uint32_t)RX) == xs;
        const int nq = A + (xt ? 1 : 0);   // vectors of this tile: A whole ones, then the shared one
        if (nq == 0) continue;
        const uint32_t r0 = tile * TR + k;
        const bool full = tile * TR + TR <= D;
        // rows r0 + KC e of vector p (zero past D; one test per tile when the tile is full)
        auto load = [&](const V *p, V *dst) {
            if (full) {
#pragma unroll
                for (int e = 0; e < RT; ++e) dst[e] = ldg(p + r0 + KC * e);
            } else {
#pragma unroll
                for (int e = 0; e < RT; ++e) dst[e] = (r0 + KC * e < D) ? ldg(p + r0 + KC * e) : VT<V>::zero();
            }
        };
        auto vec = [&](int q) { return a.W + (size_t)(q < A ? g + NG * q : xv) * a.ldW; };
        V uu[RT], cur[RT];
        load(y, uu);
        if (own_norm && (A > 0 || xt)) {
#pragma unroll
            for (int e = 0; e < RT; ++e) nrm.add_norm(uu[e]);
        }
        typename Arith<V>::Pre up[RT];   // y's rows prepared once for every vector of the tile
#pragma unroll
        for (int e = 0; e < RT; ++e) up[e] = pre(uu[e]);
        if (PF) {
            V nxt[RT];
            load(vec(0), cur);
#pragma unroll
            for (int q = 0; q < QD; ++q) {
                if (q < nq) {
                    if (q + 1 < nq) load(vec(q + 1), nxt);
#pragma unroll
                    for (int e = 0; e < RT; ++e) acc[q].add(cur[e], up[e]);
#pragma unroll
                    for (int e = 0; e < RT; ++e) cur[e] = nxt[e];
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < QD; ++q) {
                if (q < nq) {
                    load(vec(q), cur);
#pragma unroll
                    for (int e = 0; e < RT; ++e) acc[q].add(cur[e], up[e]);
                }
            }
        }
        // fold the float-float compensations back once per tile
#pragma unroll
        for (int q = 0; q < QD; ++q)
            if (q < nq) acc[q].renorm();
        nrm.renorm();
    }
    // per warp: the sum over its 32 columns; then the warps of a vector's groups, in order
#pragma unroll
    for (int q = 0; q < QD; ++q) {
        if (q < nslot) {   // (warp-uniform)
            const double2 v = acc[q].warp_value();
            if (lane == 0) wred[warp][q] = v;
        } else if (lane == 0) {
            wred[warp][q] = make_double2(0.0, 0.0);
        }
    }
    if (MODE == 0) {
        const double2 v = nrm.warp_value();
        if (lane == 0) wred[warp][QD] = v;
    }
    __syncthreads();
    constexpr int WG = KC / 32;   // warps per group
    if (tid < nv) {
        // vector tid: group tid mod NG at slot tid / NG, or the RX groups sharing it at slot A
        double2 t = make_double2(0.0, 0.0);
        const bool whole = tid < NG * A;
        for (int sv = 0; sv < (whole ? 1 : RX); ++sv) {
            const int gg = whole ? tid % NG : (tid - NG * A) + Bn * sv, q = whole ? tid / NG : A;
#pragma unroll
            for (int w = 0; w < WG; ++w) {
                t.x += wred[WG * gg + w][q].x;
                t.y += wred[WG * gg + w][q].y;
            }
        }
        red[tid] = t;
    }
    if (MODE == 0 && tid == 0) {
        double t = 0.0;
        for (int sv = 0; sv < (A > 0 ? 1 : RX); ++sv) {
            const int gg = A > 0 ? 0 : Bn * sv;
#pragma unroll
            for (int w = 0; w < WG; ++w) t += wred[WG * gg + w][QD].x;
        }
        red[SLOT_NRM] = make_double2(t, 0.0);
    }
    __syncthreads();
    double2 *fin = red;
    if (!finish_partials(red, a.part, ctl, fin, &flag, nullptr, nv, MODE == 0)) return;
    if (tid != 0) return;
    if (MODE == 0) {
        for (int i = 0; i <= jj; ++i) {
            const double s = ctl->sigma[i];
            const double2 c = make_double2(fin[i].x * s, fin[i].y * s);   // <v_i, u>
            ctl->coefA[i] = make_double2(c.x * s, c.y * s);
            if (i == jj) ctl->alpha[jj] = c.x;
        }
        ctl->normu2 = fin[SLOT_NRM].x;
        ctl->n_hv += 1;
        ctl->vec_passes += (double)(jj + 4);
        ctl->vp_kind[KIND_PASSA] += (double)(jj + 2);   // u and v_0 .. v_j
        ctl->vp_kind[KIND_HV] += 2.0;                  // the H.v: v_j read, u written
        ctl->counter = 0;
        return;
    }
    const double nw2 = ctl->wnorm2;
    double nd2 = 0.0;
    for (int i = 0; i <= jj; ++i) {
        const double s = ctl->sigma[i];
        nd2 += (fin[i].x * fin[i].x + fin[i].y * fin[i].y) * s * s;
    }
    if (nw2 > 0.0) ctl->max_orth = fmax(ctl->max_orth, sqrt(nd2 / nw2));
    ctl->n_c1 += 1;
    ctl->vec_passes += (double)(jj + 2);
    ctl->vp_kind[KIND_PASSC] += (double)(jj + 2);
    ctl->corr = 0;
    if (nw2 > 0.0 && sqrt(nd2) > ctl->eta_corr * sqrt(nw2)) {
        ctl->corr2 = 1;
        for (int i = 0; i <= jj; ++i) {
            const double s = ctl->sigma[i];
            ctl->coefC[i] = make_double2(fin[i].x * s * s, fin[i].y * s * s);
        }
        ctl->alpha[jj] += fin[jj].x * ctl->sigma[jj];
    } else {
        ctl->corr2 = 0;
        finalize_beta(ctl, jj, nw2, ctl->wg);
    }
    ctl->counter = 0;
}

// ---------------------------------------------------------------- linear combinations

// w = src - sum_i c_i W_i, the terms taken in index order; w is then dotted with psi0.
// Plain loads, RR rows per thread (r, r + TILE, ...) and eight vectors unrolled (8 RR loads
// in flight per thread), four CTAs per SM (two with RR = 4): a pure stream, which this form
// keeps near the HBM rate.  RR is a launch-shape choice (kry_autotune); it changes which
// rows a thread sums into its partial norms, so results agree to rounding.
template <class V, int MODE, int RR, int COND = 0>
__global__ void __launch_bounds__(NTHR, RR == 4 ? 2 : 4) k_lincomb(EvArgs<V> a, int jj)
{
    pdl_begin();
    KryCtl *ctl = a.ctl;
    if (ctl->done) return;
    if (MODE <= 1 && jj >= ctl->m_eff) return;
    if (MODE == 1 && !ctl->corr2) return;
    const int nvec = (MODE == 2) ? ctl->m_eff : ((MODE == 3) ? 0 : jj + 1);
    __shared__ typename Arith<V>::Coef coef[MMAX + 1];
    __shared__ double2 red[PSTRIDE];
    __shared__ double2 wtmp[NTHR / 32];
    __shared__ int flag;
    const int tid = threadIdx.x;
    if (tid < PSTRIDE) red[tid] = make_double2(0.0, 0.0);
    if (tid < nvec) {
        const double2 c = (MODE == 0) ? ctl->coefA[tid] : (MODE == 1) ? ctl->coefC[tid] : ctl->coefY[tid];
        coef[tid] = coef_from<V>(c);
    }
    __syncthreads();
    V *out = (MODE >= 2) ? a.W : a.W + (size_t)(jj + 1) * a.ldW;
    const V *src = (MODE == 0) ? a.U : (MODE == 1) ? out : (MODE == 3) ? a.G : nullptr;
    const uint32_t D = a.b.D;
    DotAcc<V> nrm, gacc;
    const uint32_t ntr = (D + RR * TILE - 1) / (RR * TILE);
    for (uint32_t tile = blockIdx.x; tile < ntr; tile += gridDim.x) {
        const uint32_t r = tile * RR * TILE + tid;
        if (r >= D) continue;
        uint32_t q[RR];
        bool in[RR];
#pragma unroll
        for (int k = 0; k < RR; ++k) {
            in[k] = r + k * TILE < D;
            q[k] = in[k] ? r + k * TILE : r;   // past D a row repeats the first, unstored
        }
        typename Arith<V>::Lin w[RR];
#pragma unroll
        for (int k = 0; k < RR; ++k) w[k] = lin_init(src ? src[q[k]] : VT<V>::zero());
        if (MODE == 2) {   // reads W_0 while overwriting it: plain loads
#pragma unroll 8
            for (int i = 0; i < nvec; ++i) {
                const V *wi = a.W + (size_t)i * a.ldW;
                V x[RR];
#pragma unroll
                for (int k = 0; k < RR; ++k) x[k] = wi[q[k]];
#pragma unroll
                for (int k = 0; k < RR; ++k) lin_fms(w[k], coef[i], x[k]);
            }
        } else {
#pragma unroll 8
            for (int i = 0; i < nvec; ++i) {
                const V *wi = a.W + (size_t)i * a.ldW;
                V x[RR];
#pragma unroll
                for (int k = 0; k < RR; ++k) x[k] = ldg(wi + q[k]);
#pragma unroll
                for (int k = 0; k < RR; ++k) lin_fms(w[k], coef[i], x[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < RR; ++k) {
            if (!in[k]) continue;
            const V wv = (MODE == 3) ? src[q[k]] : lin_out(w[k]);   // (the load is a plain copy)
            out[q[k]] = wv;
            nrm.add_norm(wv);
            if (a.G && MODE != 3) gacc.add(ldg(a.G + q[k]), wv);
        }
        nrm.renorm();
        gacc.renorm();
    }
    cta_sum_into(nrm, red, SLOT_NRM, wtmp);
    if (a.G) cta_sum_into(gacc, red, SLOT_G, wtmp);
    double2 *fin = red;
    if (!finish_partials(red, a.part, ctl, fin, &flag, nullptr, 0, true)) return;
    if (tid != 0) return;
    const double nw2 = fin[SLOT_NRM].x;
    const double2 gdot = fin[SLOT_G];
    if (MODE == 0) {
        ctl->vec_passes += (double)(jj + 3) + (a.G ? 1.0 : 0.0);
        ctl->vp_kind[KIND_PASSB] += (double)(jj + 3) + (a.G ? 1.0 : 0.0);
        // One classical Gram-Schmidt pass is enough unless the projection cancelled most of
        // u (||w|| < eta ||u||, the Daniel-Gragg-Kaufman-Stewart test), or the lengths show a
        // loss of orthogonality: with c = V^H u and G = V^H V = I + E, ||w||^2 = ||u||^2 -
        // ||c||^2 + c^H E c, so |||w||^2 - (||u||^2 - ||c||^2)| / (||c|| ||w||) estimates
        // ||E c|| / ||w|| = ||V^H w|| / ||w|| (Pythagoras test).  Either way the dots of w
        // with every previous vector are taken (pass C1) and subtracted if needed (C2).
        // With orth_check set the dots are taken after every update.
        double c2 = 0.0;
        for (int i = 0; i <= jj; ++i) {
            const double s = ctl->sigma[i];
            c2 += (ctl->coefA[i].x * ctl->coefA[i].x + ctl->coefA[i].y * ctl->coefA[i].y) / (s * s);
        }
        // (the second term is the noise floor of the lengths of vectors in storage precision)
        const double pyth = fabs(nw2 - (ctl->normu2 - c2));
        const bool lost = pyth > ctl->eta_corr * sqrt(c2 * nw2) + 0.1 * ctl->eta_bd * ctl->normu2;
        if (ctl->verify || nw2 < ctl->eta_cancel * ctl->eta_cancel * ctl->normu2 || lost) {
            ctl->corr = 1;
            ctl->wnorm2 = nw2;
            ctl->wg = gdot;
        } else {
            ctl->corr = 0;
            finalize_beta(ctl, jj, nw2, gdot);
        }
        // (COND = 0 leaves the device graph call out of the kernel: profilers skip kernels
        // that make it, and the plain step graph does not need it)
        if (COND && a.use_cond) cudaGraphSetConditional(a.cond, ctl->corr ? 1u : 0u);
    } else if (MODE == 1) {
        ctl->n_corr += 1;
        ctl->vec_passes += (double)(jj + 3) + (a.G ? 1.0 : 0.0);
        ctl->vp_kind[KIND_PASSC] += (double)(jj + 3) + (a.G ? 1.0 : 0.0);
        ctl->corr2 = 0;
        finalize_beta(ctl, jj, nw2, gdot);
    } else {
        const double b0 = sqrt(nw2);
        if (!(b0 > 0.0)) {
            ctl->err = KRY_EINVAL;
            ctl->done = 1;
        } else {
            ctl->beta0 = b0;
            ctl->sigma[0] = 1.0 / b0;
            ctl->g[0] = (MODE == 3) ? make_double2(b0, 0.0)
                                    : make_double2(gdot.x / b0, gdot.y / b0);
        }
        ctl->vec_passes += (double)(nvec + 1) + ((a.G && MODE == 2) ? 1.0 : 0.0);
        if (MODE == 2) ctl->vp_kind[KIND_COMBINE] += (double)(nvec + 1) + (a.G ? 1.0 : 0.0);
        ctl->m_eff = ctl->m;
        ctl->corr = 0;
        ctl->corr2 = 0;
        if (MODE == 2 && ctl->finishing) ctl->done = 1;
    }
    ctl->counter = 0;
}

template <class V>
__global__ void k_set_basis_state(V *W0, uint32_t r0)
{
    V one = VT<V>::zero();
    one.x = 1;
    W0[r0] = one;
}

__global__ void k_set_basis_state_ff(ffc *W0, uint32_t r0) { W0[r0] = ffc{1.f, 0.f, 0.f, 0.f}; }

// ---------------------------------------------------------------- dense vector output

// psi(t_o) = sum_j Yout[o][j] W_j for every output time o inside the current step (the
// small exponential fills Yout and [out_begin, out_end)); runs before the combine
// overwrites W_0.
template <class V>
__global__ void __launch_bounds__(NTHR) k_vecout(VecOutArgs<V> a)
{
    pdl_begin();
    KryCtl *ctl = a.ctl;
    if (ctl->done) return;
    const int ob = ctl->out_begin, oe = ctl->out_end, me = ctl->m_eff;
    if (ob >= oe) return;
    __shared__ V cf[MMAX];
    for (int o = ob; o < oe; ++o) {
        __syncthreads();
        if (threadIdx.x < me) cf[threadIdx.x] = VT<V>::from(a.Yout[(size_t)o * MMAX + threadIdx.x]);
        __syncthreads();
        V *out = a.out + (size_t)o * a.ldOut;
        for (size_t r = (size_t)blockIdx.x * NTHR + threadIdx.x; r < a.D; r += (size_t)gridDim.x * NTHR) {
            V w = VT<V>::zero();
            for (int j = 0; j < me; ++j) {
                const V v = a.W[(size_t)j * a.ldW + r];
                const V c = cf[j];
                w.x += c.x * v.x - c.y * v.y;
                w.y += c.x * v.y + c.y * v.x;
            }
            out[r] = w;
        }
    }
}

// Copy psi (= W_0 after the combine) into checkpoint slot n_steps/every - 1 after every
// `every`-th Krylov step, and record its time.
template <class V>
__global__ void __launch_bounds__(NTHR) k_ckpt(const V *__restrict__ W0, V *__restrict__ ck, size_t ldC,
                                               KryCtl *ctl, uint32_t D)
{
    pdl_begin();
    if (ctl->done || ctl->ckpt_every <= 0) return;
    const long long ns = ctl->n_steps;
    if (ns % ctl->ckpt_every != 0) return;
    const long long slot = ns / ctl->ckpt_every - 1;
    if (slot < 0 || slot >= ctl->ckpt_cap) return;
    V *dst = ck + (size_t)slot * ldC;
    for (size_t r = (size_t)blockIdx.x * NTHR + threadIdx.x; r < D; r += (size_t)gridDim.x * NTHR) dst[r] = W0[r];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->ckpt_t[slot] = ctl->t_now;
        ctl->n_ckpt = (int)slot + 1;
    }
}

// ---------------------------------------------------------------- gradient integrand

__global__ void __launch_bounds__(NTHR) k_grad_acc(DevBasis b, DevHam hm, double J, const double2 *__restrict__ psi,
                                                   const double2 *__restrict__ lam, size_t ld,
                                                   const double *__restrict__ w, int nq, double2 *part,
                                                   double2 *acc_out, unsigned *counter, int site0)
{
    __shared__ uint32_t koff_s[20], bsz_s[20];
    __shared__ double2 red[PSTRIDE];
    __shared__ double2 wtmp[NTHR / 32];
    __shared__ int flag;
    const int tid = threadIdx.x, L = b.L;
    if (!b.list) stage_tables(b, koff_s, bsz_s, nullptr, 0);
    if (tid < PSTRIDE) red[tid] = make_double2(0.0, 0.0);
    __syncthreads();
    double2 acc[MMAX + 1];
#pragma unroll
    for (int i = 0; i <= MMAX; ++i) acc[i] = make_double2(0.0, 0.0);
    const uint32_t D = b.D, ntiles = (D + TILE - 1) / TILE;
    const uint64_t obc = (L >= 2) ? ((1ull << (L - 1)) - 1ull) : 0ull;
    const double czz = 0.25 * J;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r = tile * TILE + tid;
        if (r >= D) continue;
        uint64_t s;
        if (b.list) {
            s = __ldg(b.states + r);
        } else {
            uint32_t hi, off;
            int klo;
            tile_unrank(b, bsz_s, tile * TILE, tid, hi, off, klo);
            s = ((uint64_t)hi << b.Llo) | __ldg(b.lolist + koff_s[klo] + off);
        }
        double2 S = make_double2(0.0, 0.0);
        for (int q = 0; q < nq; ++q) {
            const double2 l = __ldg(lam + (size_t)(nq - 1 - q) * ld + r), p = __ldg(psi + (size_t)q * ld + r);
            const double wq = __ldg(w + q);
            S.x += wq * (l.x * p.x + l.y * p.y);
            S.y += wq * (l.x * p.y - l.y * p.x);
        }
#pragma unroll
        for (int i = 0; i < MMAX; ++i) {
            if (site0 + i < L) {
                const double z = ((s >> (site0 + i)) & 1ull) ? 0.5 : -0.5;
                acc[i].x += z * S.x;
                acc[i].y += z * S.y;
            }
        }
        if (site0 == 0) {
            const int nanti = __popcll((long long)((s ^ (s >> 1)) & obc)) +
                              (hm.pbc ? (int)((s ^ (s >> (L - 1))) & 1ull) : 0);
            const double zz = czz * (double)(hm.nbonds - 2 * nanti);
            acc[MMAX].x += zz * S.x;
            acc[MMAX].y += zz * S.y;
        }
    }
#pragma unroll
    for (int i = 0; i <= MMAX; ++i) {
        if (site0 + i < L || i == MMAX) cta_sum_into(acc[i], red, i, wtmp);
    }
    double2 *fin = red;
    if (!finish_partials(red, part, nullptr, fin, &flag, counter)) return;
    if (tid < MMAX && site0 + tid < L) {
        acc_out[site0 + tid].x += fin[tid].x;
        acc_out[site0 + tid].y += fin[tid].y;
    } else if (tid == MMAX && site0 == 0) {
        acc_out[L].x += fin[MMAX].x;
        acc_out[L].y += fin[MMAX].y;
    }
    if (tid == 0) *counter = 0;
}

// ---------------------------------------------------------------- launchers

size_t apply_smem(const DevBasis &b, int rl_smem, int)
{
    return sizeof(SmemHead) + (rl_smem ? (sizeof(uint16_t) << b.Llo) : 0);
}


template <class K>
static int prep_smem(K kernel, size_t smem)
{
    if (smem > 48 * 1024) KRY_CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KRY_OK;
}

static int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

int launch_apply(const DevBasis &b, const DevHam &h, int c64, const void *x, void *y, int rl_smem,
                 cudaStream_t s)
{
    if (b.list) return launch_list_apply(b, h, c64, 1, x, y, s);
    const size_t smem = apply_smem(b, rl_smem, c64);
    const uint32_t ntiles = (b.D + TILE - 1) / TILE;
    int grid = (int)std::min<uint32_t>(ntiles, (uint32_t)sm_count() * 8u);
    if (c64) {
        if (int rc = prep_smem(k_apply<float2>, smem)) return rc;
        k_apply<float2><<<grid, NTHR, smem, s>>>(b, h, (const float2 *)x, (float2 *)y, rl_smem);
    } else {
        if (int rc = prep_smem(k_apply<double2>, smem)) return rc;
        k_apply<double2><<<grid, NTHR, smem, s>>>(b, h, (const double2 *)x, (double2 *)y, rl_smem);
    }
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

// CTAs of the vector kernels, whole SMs times their resident CTAs: the streaming dots
// (returned; also pass C1), the H.v of pass A (*gridH) and the updates, combine and
// outputs (*gridB).  Also sets the kernels' shared-memory limits.  hv_form is part 1 of the
// launch shape: bit 0 chunked gathers, bit 1 the lower-bit rank table read through L1
// instead of staged in shared memory (more CTAs per SM when that table is large).
template <class V>
int vector_grid(const DevBasis &b, int rl_smem, int hv_form, int *gridH, int *gridB)
{
    const uint32_t es = sizeof(V);
    const int rlH = rl_smem && !(hv_form & 2);
    const size_t smH = apply_smem(b, rlH, es == sizeof(float2));
    if (int rc = prep_smem(k_hv<V, 0>, smH)) return -rc;
    if (int rc = prep_smem(k_hv<V, 1>, smH)) return -rc;
    int occA = 0, occB = 0, occH = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occA, k_dots<V, 0, 1>, NTHR, 0);
    if (hv_form & 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occH, k_hv<V, 1>, NTHR, smH);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occH, k_hv<V, 0>, NTHR, smH);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occB, k_lincomb<V, 0, 2>, NTHR, 0);
    const uint32_t ntiles = (b.D + TILE - 1) / TILE;
    auto fit = [&](int occ) {
        return (int)std::max<uint32_t>(1u, std::min<uint32_t>(ntiles, (uint32_t)(sm_count() * std::max(1, occ))));
    };
    *gridH = fit(occH);
    if (b.list) {
        if (int rc = list_hv_grid<V>(b, gridH)) return -rc;
    }
    *gridB = fit(occB);
    return fit(occA);
}

template <class V>
int launch_hv(const EvArgs<V> &a, int jj, int grid, cudaStream_t s, int pdl)
{
    if (a.b.list) return launch_list_hv<V>(a, jj, grid, s, pdl);
    EvArgs<V> ah = a;
    ah.rl_smem = a.rl_smem && !(a.hv_form & 2);
    const size_t smem = apply_smem(a.b, ah.rl_smem, sizeof(V) == sizeof(float2));
    KRY_CU(launch_ex(pdl, (a.hv_form & 1) ? k_hv<V, 1> : k_hv<V, 0>, grid, NTHR, smem, s, ah, jj));
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template <class V, int MODE, int COND>
static cudaError_t launch_lincomb_rr(const EvArgs<V> &a, int jj, int grid, cudaStream_t s, int pdl)
{
    switch (a.upd_rows) {
    case 1: return launch_ex(pdl, k_lincomb<V, MODE, 1, COND>, grid, NTHR, 0, s, a, jj);
    case 4: return launch_ex(pdl, k_lincomb<V, MODE, 4, COND>, grid, NTHR, 0, s, a, jj);
    default: return launch_ex(pdl, k_lincomb<V, MODE, 2, COND>, grid, NTHR, 0, s, a, jj);
    }
}

template <class V>
int launch_lincomb(const EvArgs<V> &a, int mode, int jj, int grid, cudaStream_t s, int pdl)
{
    switch (mode) {
    case 0:
        if (a.use_cond) KRY_CU((launch_lincomb_rr<V, 0, 1>(a, jj, grid, s, pdl)));
        else KRY_CU((launch_lincomb_rr<V, 0, 0>(a, jj, grid, s, pdl)));
        break;
    case 1: KRY_CU((launch_lincomb_rr<V, 1, 0>(a, jj, grid, s, pdl))); break;
    case 2: KRY_CU(launch_ex(pdl, k_lincomb<V, 2, 2>, grid, NTHR, 0, s, a, jj)); break;
    default: KRY_CU(launch_ex(pdl, k_lincomb<V, 3, 2>, grid, NTHR, 0, s, a, jj)); break;
    }
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_set_basis_state(void *W0, int c64, uint32_t r0, cudaStream_t s, int ff)
{
    if (c64) k_set_basis_state<float2><<<1, 1, 0, s>>>((float2 *)W0, r0);
    else if (ff) k_set_basis_state_ff<<<1, 1, 0, s>>>((ffc *)W0, r0);
    else k_set_basis_state<double2><<<1, 1, 0, s>>>((double2 *)W0, r0);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

// complex128 <-> float-float vectors (dtype KRY_C128E): in at the initial vector, out at psi(t)
__global__ void __launch_bounds__(NTHR) k_c128_to_ffc(const double2 *__restrict__ src, ffc *__restrict__ dst, size_t n)
{
    for (size_t r = (size_t)blockIdx.x * NTHR + threadIdx.x; r < n; r += (size_t)gridDim.x * NTHR)
        dst[r] = VT<ffc>::from(__ldg(src + r));
}
__global__ void __launch_bounds__(NTHR) k_ffc_to_c128(const ffc *__restrict__ src, double2 *__restrict__ dst, size_t n)
{
    for (size_t r = (size_t)blockIdx.x * NTHR + threadIdx.x; r < n; r += (size_t)gridDim.x * NTHR) {
        const ffc v = ldg(src + r);
        dst[r] = make_double2(ff2d(v.xh, v.xl), ff2d(v.yh, v.yl));
    }
}
static unsigned convert_grid(size_t n)
{
    return (unsigned)std::max<size_t>(1, std::min<size_t>((n + NTHR - 1) / NTHR, (size_t)sm_count() * 8));
}
int launch_c128_to_ffc(const void *src, void *dst, size_t n, cudaStream_t s)
{
    if (n == 0) return KRY_OK;
    k_c128_to_ffc<<<convert_grid(n), NTHR, 0, s>>>((const double2 *)src, (ffc *)dst, n);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}
int launch_ffc_to_c128(const void *src, void *dst, size_t n, cudaStream_t s)
{
    if (n == 0) return KRY_OK;
    k_ffc_to_c128<<<convert_grid(n), NTHR, 0, s>>>((const ffc *)src, (double2 *)dst, n);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template <class V>
int launch_vecout(const VecOutArgs<V> &a, int grid, cudaStream_t s)
{
    KRY_CU(launch_pdl(k_vecout<V>, grid, NTHR, 0, s, a));
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template <class V>
int launch_ckpt(const V *W0, V *ckpt, size_t ldC, KryCtl *ctl, uint32_t D, int grid, cudaStream_t s)
{
    KRY_CU(launch_pdl(k_ckpt<V>, grid, NTHR, 0, s, W0, ckpt, ldC, ctl, D));
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_grad_acc(const DevBasis &b, const DevHam &h, double J, const double2 *psi, const double2 *lam,
                    size_t ld, const double *w, int nq, double2 *part, double2 *acc, unsigned *counter,
                    int grid, cudaStream_t s)
{
    for (int site0 = 0; site0 < b.L; site0 += MMAX) {   // 32 sites per launch (L > 32: two)
        k_grad_acc<<<grid, NTHR, 0, s>>>(b, h, J, psi, lam, ld, w, nq, part, acc, counter, site0);
        KRY_CU(cudaGetLastError());
    }
    return KRY_OK;
}

template int launch_vecout<double2>(const VecOutArgs<double2> &, int, cudaStream_t);
template int launch_vecout<float2>(const VecOutArgs<float2> &, int, cudaStream_t);
template int launch_ckpt<double2>(const double2 *, double2 *, size_t, KryCtl *, uint32_t, int, cudaStream_t);
template int launch_ckpt<float2>(const float2 *, float2 *, size_t, KryCtl *, uint32_t, int, cudaStream_t);
template <class V>
int launch_dots(const EvArgs<V> &a, int mode, int jj, int grid, cudaStream_t s, int pdl)
{
    const int pf = a.dots_form == 0;
    if (mode == 0) KRY_CU(launch_ex(pdl, pf ? k_dots<V, 0, 1> : k_dots<V, 0, 0>, grid, NTHR, 0, s, a, jj));
    else KRY_CU(launch_ex(pdl, pf ? k_dots<V, 1, 1> : k_dots<V, 1, 0>, grid, NTHR, 0, s, a, jj));
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template int launch_dots<double2>(const EvArgs<double2> &, int, int, int, cudaStream_t, int);
template int launch_dots<float2>(const EvArgs<float2> &, int, int, int, cudaStream_t, int);
template int launch_dots<ffc>(const EvArgs<ffc> &, int, int, int, cudaStream_t, int);
template int vector_grid<double2>(const DevBasis &, int, int, int *, int *);
template int vector_grid<float2>(const DevBasis &, int, int, int *, int *);
template int vector_grid<ffc>(const DevBasis &, int, int, int *, int *);
template int launch_hv<double2>(const EvArgs<double2> &, int, int, cudaStream_t, int);
template int launch_hv<float2>(const EvArgs<float2> &, int, int, cudaStream_t, int);
template int launch_hv<ffc>(const EvArgs<ffc> &, int, int, cudaStream_t, int);
template int launch_lincomb<double2>(const EvArgs<double2> &, int, int, int, cudaStream_t, int);
template int launch_lincomb<float2>(const EvArgs<float2> &, int, int, int, cudaStream_t, int);
template int launch_lincomb<ffc>(const EvArgs<ffc> &, int, int, int, cudaStream_t, int);

}  // namespace kry
