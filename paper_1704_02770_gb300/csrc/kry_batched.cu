// Batched realisations: K copies of Eq. 1 that differ only in the on-site field (K disorder
// phases, Sec. 3 "many layers of disorder"), evolved together.  Vectors are interleaved
// [state][K] complex, so one rank computation and one neighbour lookup serve K contiguous
// amplitudes (a 512-byte row at K = 64 complex64).  Each realisation keeps its own Lanczos
// recurrence (alpha_k, beta_k, reorthogonalisation coefficients) in FP64; all share the
// time grid, so the step size is the smallest step every realisation accepts.
//
//   k_apply_b      y = H x for all K (warp per state, lanes over k)
//   k_hv_b         u = H v_j for all K (pass A, part 1)
//   k_dots_b       all dots <v_i, u> and ||u||^2 per realisation (pass A, part 2)
//   k_lincomb_b    update / correction / combine / load with per-realisation coefficients,
//                  and the dots of the new vector with the earlier ones (pass C1)
//   k_reduce_b     per-realisation sum of the per-CTA partials (CTA order, deterministic)
//                  and the scalar epilogue of each pass
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kry_device.cuh"

namespace kry {

struct SmemHeadB {
    uint32_t koff[20];
    uint32_t bsz[20];
};

// Row r of H x for every realisation: the rank arithmetic is the same for all k, the
// lanes of the warp run over k = lane + 32 q (k0 = lane), or one realisation k0 per lane.
template <class V, int KQ>
__device__ __forceinline__ void hv_row_b(const DevBasis &b, const DevHam &hm, const V *__restrict__ x,
                                         int K, uint32_t hi, uint32_t off, int klo,
                                         const uint32_t *koff_s, const uint16_t *rl, V out[KQ], int k0)
{
    using R = typename VT<V>::R;
    const int lane = k0;
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
    const R dz = (R)hm.cz * (R)(hm.nbonds - 2 * nanti);
    typename Arith<V>::HvSum acc[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) acc[q] = typename Arith<V>::HvSum{};
    // Neighbour rows in chunks of 4 bond positions (bit 31 = ring bond): the ranks are the
    // same for all lanes; every lane issues its loads of the whole chunk before summing.
    const uint32_t hops = anti | (wrap << 31);
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 4) {
        if (!((hops >> c0) & 0xFu)) continue;
        V v[4][KQ];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = c0 + u;
#pragma unroll
            for (int q = 0; q < KQ; ++q) v[u][q] = VT<V>::zero();
            if ((hops >> p) & 1u) {
                uint32_t t2;
                if (p == 31) {
                    const uint32_t s2 = s ^ ((1u << (L - 1)) | 1u);
                    t2 = __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask];
                } else if (p < Llo - 1) {
                    t2 = base + rl[lo ^ (3u << p)];
                } else if (p == Llo - 1) {
                    const uint32_t s2 = s ^ (3u << p);
                    t2 = __ldg(b.blk + (s2 >> Llo)) + rl[s2 & lomask];
                } else {
                    t2 = __ldg(b.blk + (hi ^ (3u << (p - Llo)))) + off;
                }
                const V *xr = x + (size_t)t2 * K;
#pragma unroll
                for (int q = 0; q < KQ; ++q) {
                    const int k = lane + 32 * q;
                    if (k < K) v[u][q] = ldg(xr + k);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < KQ; ++q) hv_add(acc[q], v[u][q]);
    }
    const V *xr = x + (size_t)(base + off) * K;
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int k = lane + 32 * q;
        if (k < K) {
            const R d = dz + VT<V>::ehlo(hm, pos * K + k) + VT<V>::ehhi(hm, hi * K + k);
            out[q] = hv_finish(d, ldg(xr + k), (R)hm.halfJ, acc[q]);
        } else {
            out[q] = VT<V>::zero();
        }
    }
}

// ---------------------------------------------------------------- y = H x (batched)

template <class V, int KQ>
__global__ void __launch_bounds__(NTHR) k_apply_b(DevBasis b, DevHam hm, int K, const V *__restrict__ x,
                                                  V *__restrict__ y, int rl_smem)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SmemHeadB *hd = (SmemHeadB *)smem;
    uint16_t *rl_s = (uint16_t *)(smem + sizeof(SmemHeadB));
    stage_tables(b, hd->koff, hd->bsz, rl_s, rl_smem);
    __syncthreads();
    const uint16_t *rl = rl_smem ? rl_s : b.ranklo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ntiles = (b.D + TROWS - 1) / TROWS;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TROWS;
        for (int rr = warp; rr < TROWS; rr += NTHR / 32) {
            if (r0 + rr >= b.D) break;
            uint32_t hi, off;
            int klo;
            tile_unrank(b, hd->bsz, r0, rr, hi, off, klo);
            V u[KQ];
            hv_row_b<V, KQ>(b, hm, x, K, hi, off, klo, hd->koff, rl, u, lane);
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                const int k = lane + 32 * q;
                if (k < K) y[(size_t)(r0 + rr) * K + k] = u[q];
            }
        }
    }
}

// ---------------------------------------------------------------- pass A (batched)

// Part 1: U[:, k] = sigma_j[k] H_k W_j[:, k] for every realisation (warp per state, lanes over
// k), at full occupancy: nothing but the gathers.
template <class V, int KQ>
__global__ void __launch_bounds__(NTHR) k_hv_b(EvArgsB<V> a, int jj)
{
    using R = typename VT<V>::R;
    KryCtlB *ctl = a.ctl;
    if (ctl->hd.done || jj >= ctl->hd.m_run) return;
    extern __shared__ __align__(16) unsigned char smem[];
    SmemHeadB *hd = (SmemHeadB *)smem;
    uint16_t *rl_s = (uint16_t *)(smem + sizeof(SmemHeadB));
    stage_tables(a.b, hd->koff, hd->bsz, rl_s, a.rl_smem);
    __syncthreads();
    const uint16_t *rl = a.rl_smem ? rl_s : a.b.ranklo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, K = a.K;
    R sg[KQ];
#pragma unroll
    for (int q = 0; q < KQ; ++q) {
        const int k = lane + 32 * q;
        sg[q] = (k < K) ? (R)ctl->sigma[jj][k] : (R)0;
    }
    const V *x = a.W + (size_t)jj * a.ldW;
    const uint32_t D = a.b.D, ntiles = (D + TROWS - 1) / TROWS;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TROWS;
        for (int rr = warp; rr < TROWS; rr += NTHR / 32) {
            if (r0 + rr >= D) break;
            uint32_t hi, off;
            int klo;
            tile_unrank(a.b, hd->bsz, r0, rr, hi, off, klo);
            V u[KQ];
            hv_row_b<V, KQ>(a.b, a.h, x, K, hi, off, klo, hd->koff, rl, u, lane);
#pragma unroll
            for (int q = 0; q < KQ; ++q) {
                const int k = lane + 32 * q;
                if (k < K) a.U[(size_t)(r0 + rr) * K + k] = scale(u[q], sg[q]);
            }
        }
    }
}

// Part 1 in chunks of KCH realisations: the work items are (chunk, tile) pairs in chunk-major
// order and a warp holds 32 / KCH states, KCH lanes each.  The CTAs sweep all tiles of one
// chunk before the next, so the gathered part of W_j (D x KCH amplitudes, e.g. 90 MB for
// L = 22 and KCH = 16 in complex64) stays in L2 while its rows are gathered about eleven
// times each; without chunks the whole [D][K] block (361 MB at K = 64) exceeds L2 and
// gathered rows come from HBM several times.  The rank arithmetic is repeated per chunk.
// Same hop order per amplitude as k_hv_b: the same bits.
template <class V, int KCH>
__global__ void __launch_bounds__(NTHR) k_hv_bc(EvArgsB<V> a, int jj)
{
    using R = typename VT<V>::R;
    KryCtlB *ctl = a.ctl;
    if (ctl->hd.done || jj >= ctl->hd.m_run) return;
    extern __shared__ __align__(16) unsigned char smem[];
    SmemHeadB *hd = (SmemHeadB *)smem;
    uint16_t *rl_s = (uint16_t *)(smem + sizeof(SmemHeadB));
    stage_tables(a.b, hd->koff, hd->bsz, rl_s, a.rl_smem);
    __syncthreads();
    const uint16_t *rl = a.rl_smem ? rl_s : a.b.ranklo;
    constexpr int SPW = 32 / KCH;   // states per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, K = a.K;
    const int sub = lane / KCH, kk = lane % KCH;
    const V *x = a.W + (size_t)jj * a.ldW;
    const uint32_t D = a.b.D, ntiles = (D + TROWS - 1) / TROWS;
    const uint32_t nch = (uint32_t)((K + KCH - 1) / KCH);
    for (uint32_t item = blockIdx.x; item < nch * ntiles; item += gridDim.x) {
        const uint32_t ch = item / ntiles, tile = item - ch * ntiles;
        const int k = (int)ch * KCH + kk;
        const R sg = (k < K) ? (R)ctl->sigma[jj][k] : (R)0;
        const uint32_t r0 = tile * TROWS;
        for (int rr = warp * SPW + sub; rr < TROWS; rr += (NTHR / 32) * SPW) {
            if (r0 + rr >= D) break;
            uint32_t hi, off;
            int klo;
            tile_unrank(a.b, hd->bsz, r0, rr, hi, off, klo);
            V u[1];
            hv_row_b<V, 1>(a.b, a.h, x, K, hi, off, klo, hd->koff, rl, u, k);
            if (k < K) a.U[(size_t)(r0 + rr) * K + k] = scale(u[0], sg);
        }
    }
}

// Part 2: the dots <W_i[:, k], U[:, k]>, i <= j, and ||U[:, k]||^2 of every realisation.
// Thread (k, g) takes column k and the vectors i = g, g + NG, ...; the rows of U of a tile
// are loaded once and serve all of them.
template <class V, int KQ>
__global__ void __launch_bounds__(NTHR, 2) k_dots_b(EvArgsB<V> a, int jj)
{
    KryCtlB *ctl = a.ctl;
    if (ctl->hd.done || jj >= ctl->hd.m_run) return;
    // vectors i = g + NG q < MMAX (j <= MMAX - 1); complex64 accumulates with the packed
    // float-float pairs while they fit the registers (K <= 64), else with the scalar pairs;
    // complex128 in FP64
    constexpr int Kp = 32 * KQ, NG = NTHR / Kp, QD = (MMAX + NG - 1) / NG;
    using Acc = typename std::conditional<sizeof(V) == sizeof(float2) && KQ <= 2, DotAccF2, DotAcc<V>>::type;
    constexpr int RH = TROWS / 2;   // rows per half tile
    const int tid = threadIdx.x, K = a.K;
    const int k = tid % Kp, g = tid / Kp;
    const uint32_t D = a.b.D, ntiles = (D + TROWS - 1) / TROWS;
    Acc acc[QD];
    DotAcc<V> nrm;
    if (k < K) {
        for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const uint32_t r0 = tile * TROWS;
            // rows past D are skipped by one test per half tile, not per element
            // (a select of FP64 values occupies the FP64 pipe)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t rh = r0 + h * RH;
                const int nr = rh >= D ? 0 : (int)min((uint32_t)RH, D - rh);
                V uu[RH];
#pragma unroll
                for (int rr = 0; rr < RH; ++rr) uu[rr] = VT<V>::zero();
                if (nr == RH) {
#pragma unroll
                    for (int rr = 0; rr < RH; ++rr) uu[rr] = ldg(a.U + (size_t)(rh + rr) * K + k);
                } else {
#pragma unroll
                    for (int rr = 0; rr < RH; ++rr)
                        if (rr < nr) uu[rr] = ldg(a.U + (size_t)(rh + rr) * K + k);
                }
                if (g == 0) {
#pragma unroll
                    for (int rr = 0; rr < RH; ++rr) nrm.add_norm(uu[rr]);
                }
                // rows rh .. rh + RH of vector iv, column k (zero past D)
                auto load = [&](int iv, V *dst) {
                    const V *wi = a.W + (size_t)iv * a.ldW + (size_t)rh * K + k;
                    if (nr == RH) {
#pragma unroll
                        for (int rr = 0; rr < RH; ++rr) dst[rr] = ldg(wi + (size_t)rr * K);
                    } else {
#pragma unroll
                        for (int rr = 0; rr < RH; ++rr) dst[rr] = (rr < nr) ? ldg(wi + (size_t)rr * K) : VT<V>::zero();
                    }
                };
                // (a prefetch of the next vector's rows, as in the single-realisation dots,
                // needs more registers than the eight accumulators of K = 64 leave, and spills)
#pragma unroll
                for (int q = 0; q < QD; ++q) {
                    const int iv = g + NG * q;
                    if (iv <= jj) {
                        V vv[RH];
                        load(iv, vv);
#pragma unroll
                        for (int rr = 0; rr < RH; ++rr) acc[q].add(vv[rr], uu[rr]);
                    }
                }
            }
            // fold the float-float compensations back once per tile
#pragma unroll
            for (int q = 0; q < QD; ++q)
                if (g + NG * q <= jj) acc[q].renorm();
            nrm.renorm();
        }
    }
    double2 *pc = a.part + (size_t)blockIdx.x * PSB * Kp;
#pragma unroll
    for (int q = 0; q < QD; ++q) {
        const int iv = g + NG * q;
        if (iv <= jj) pc[(size_t)iv * Kp + k] = acc[q].value();
    }
    if (g == 0) pc[(size_t)SLOT_NRM * Kp + k] = make_double2(nrm.value().x, 0.0);
}


// ---------------------------------------------------------------- linear combinations (batched)

// MODE 0: w = U - sum_i c_i W_i (pure update); 1: the correction of pass C2; 2: combine;
// 3: load psi0; 4: the dots <W_i, W_{j+1}> of pass C1 (no update), for realisations that
// flagged them.
template <class V, int MODE, int KQ>
__global__ void __launch_bounds__(NTHR, 1) k_lincomb_b(EvArgsB<V> a, int jj)
{
    KryCtlB *ctl = a.ctl;
    if (ctl->hd.done) return;
    if ((MODE <= 1 || MODE == 4) && jj >= ctl->hd.m_run) return;
    if (MODE == 1 && !ctl->hd.corr_any) return;
    if (MODE == 4 && !ctl->hd.dots_any) return;
    constexpr int Kp = 32 * KQ, NG = NTHR / Kp, QD = (MMAX + NG) / NG;
    const int nvec = (MODE == 2) ? ctl->hd.m_run : ((MODE == 3 || MODE == 4) ? 0 : jj + 1);
    extern __shared__ __align__(16) unsigned char smem[];
    using Coef = typename Arith<V>::Coef;
    static_assert(sizeof(Coef) == sizeof(V), "coefficient slots have the element size");
    Coef *coef = (Coef *)smem;                    // [MMAX+1][Kp]
    V *wtile = (V *)(coef + (MMAX + 1) * Kp);     // [TROWS][Kp]
    double2 *nred = (double2 *)(wtile + TROWS * Kp);   // [NG][Kp] (norm), then [NG][Kp] (G)
    const int tid = threadIdx.x, K = a.K;
    for (int e = tid; e < nvec * Kp; e += NTHR) {
        const int i = e / Kp, k = e % Kp;
        double2 c = make_double2(0.0, 0.0);
        if (k < K) c = (MODE == 0) ? ctl->coefA[i][k] : (MODE == 1) ? ctl->coefC[i][k] : ctl->coefY[i][k];
        coef[i * Kp + k] = coef_from<V>(c);
    }
    __syncthreads();
    V *out = (MODE == 2 || MODE == 3) ? a.W : a.W + (size_t)(jj + 1) * a.ldW;
    const V *src = (MODE == 0) ? a.U : (MODE == 1 || MODE == 4) ? out : (MODE == 3) ? a.G : nullptr;
    const uint32_t D = a.b.D, ntiles = (D + TROWS - 1) / TROWS;
    const int k = tid % Kp, g = tid / Kp;
    DotAcc<V> acc[QD];
    DotAcc<V> nrm, gacc;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t r0 = tile * TROWS;
        for (int rr = g; rr < TROWS; rr += NG) {
            V w = VT<V>::zero();
            if (r0 + rr < D && k < K) {
                const size_t idx = (size_t)(r0 + rr) * K + k;
                if (src) w = src[idx];
                if (MODE != 4) {
                    typename Arith<V>::Lin wl = lin_init(w);
                    if (MODE == 2) {
#pragma unroll 8
                        for (int i = 0; i < nvec; ++i) lin_fms(wl, coef[i * Kp + k], a.W[(size_t)i * a.ldW + idx]);
                    } else {
#pragma unroll 8
                        for (int i = 0; i < nvec; ++i) lin_fms(wl, coef[i * Kp + k], ldg(a.W + (size_t)i * a.ldW + idx));
                    }
                    w = (MODE == 3) ? w : lin_out(wl);
                    out[idx] = w;
                    nrm.add_norm(w);
                    if (a.G && MODE != 3) gacc.add(ldg(a.G + idx), w);
                }
            }
            if (MODE == 4) wtile[rr * Kp + k] = w;
        }
        nrm.renorm();
        gacc.renorm();
        if (MODE == 4) {
            __syncthreads();
            if (k < K) {
#pragma unroll
                for (int q = 0; q < QD; ++q) {
                    const int iv = g + NG * q;
                    if (iv <= jj) {
                        const V *wi = a.W + (size_t)iv * a.ldW + (size_t)r0 * K + k;
                        V vv[TROWS];
#pragma unroll
                        for (int rr = 0; rr < TROWS; ++rr)
                            vv[rr] = (r0 + rr < D) ? ldg(wi + (size_t)rr * K) : VT<V>::zero();
#pragma unroll
                        for (int rr = 0; rr < TROWS; ++rr) acc[q].add(vv[rr], wtile[rr * Kp + k]);
                        acc[q].renorm();
                    }
                }
            }
            __syncthreads();
        }
    }
    double2 *pc = a.part + (size_t)blockIdx.x * PSB * Kp;
    if (MODE == 4) {
#pragma unroll
        for (int q = 0; q < QD; ++q) {
            const int iv = g + NG * q;
            if (iv <= jj) pc[(size_t)iv * Kp + k] = acc[q].value();
        }
        return;
    }
    nred[g * Kp + k] = nrm.value();
    nred[(NG + g) * Kp + k] = gacc.value();
    __syncthreads();
    for (int kk = tid; kk < Kp; kk += NTHR) {
        double2 s = make_double2(0.0, 0.0), t = make_double2(0.0, 0.0);
        for (int gg = 0; gg < NG; ++gg) {
            s.x += nred[gg * Kp + kk].x;
            t.x += nred[(NG + gg) * Kp + kk].x;
            t.y += nred[(NG + gg) * Kp + kk].y;
        }
        pc[(size_t)SLOT_NRM * Kp + kk] = s;
        pc[(size_t)SLOT_G * Kp + kk] = t;
    }
}

// ---------------------------------------------------------------- per-realisation reductions

// mode: 0 pass A, 1 pass B, 3 pass C1 (dots of w), 2 pass C2 (correction), 4 combine,
// 5 load of a general psi0.
__global__ void __launch_bounds__(128) k_reduce_b(KryCtlB *ctl, const double2 *__restrict__ part,
                                                  int grid, int Kp, int mode, int jj, int general)
{
    KryHdrB &H = ctl->hd;
    if (H.done) return;
    if (mode <= 3 && jj >= H.m_run) return;
    const int k = blockIdx.x, tid = threadIdx.x;
    if (mode == 2 && !H.corr_any) return;   // pass C2 did not run
    if (mode == 3 && !H.dots_any) return;   // pass C1 did not run
    __shared__ double2 red[128];
    __shared__ double2 fin[PSB];
    const int nd = (mode == 0 || mode == 3) ? jj + 1 : 0;
    auto reduce_slot = [&](int slot) {
        double2 s = make_double2(0.0, 0.0);
        for (int c = tid; c < grid; c += 128) {
            const double2 v = __ldg(part + ((size_t)c * PSB + slot) * Kp + k);
            s.x += v.x;
            s.y += v.y;
        }
        red[tid] = s;
        __syncthreads();
        for (int o = 64; o > 0; o >>= 1) {
            if (tid < o) { red[tid].x += red[tid + o].x; red[tid].y += red[tid + o].y; }
            __syncthreads();
        }
        if (tid == 0) fin[slot] = red[0];
        __syncthreads();
    };
    for (int i = 0; i < nd; ++i) reduce_slot(i);
    if (mode != 3) reduce_slot(SLOT_NRM);
    if (general && mode != 0 && mode != 3) reduce_slot(SLOT_G);
    if (tid != 0) return;
    const double nw2 = (mode == 3) ? ctl->wnorm2[k] : fin[SLOT_NRM].x;
    const double2 gdot = (mode == 3) ? ctl->wg[k]
                                     : ((general && mode != 0) ? fin[SLOT_G] : make_double2(0.0, 0.0));
    auto finalize = [&](double w2, double2 gd) {
        const double bt = sqrt(w2);
        ctl->beta[jj][k] = bt;
        if (!(bt > H.eta_bd * sqrt(ctl->normu2[k]))) {
            ctl->m_eff[k] = jj + 1;
            atomicAdd(&H.n_bd, 1ull);
            ctl->sigma[jj + 1][k] = 0.0;
        } else {
            const double s = 1.0 / bt;
            ctl->sigma[jj + 1][k] = s;
            ctl->g[jj + 1][k] = make_double2(gd.x * s, gd.y * s);
        }
    };
    if (mode == 0) {
        if (k == 0) {
            H.n_hv += 1;
            H.vec_passes += (double)(jj + 4);
            H.vp_kind[KIND_PASSA] += (double)(jj + 2);   // u and v_0 .. v_j
            H.vp_kind[KIND_HV] += 2.0;                  // the H.v: v_j read, u written
            H.corr_any = 0;
            H.dots_any = 0;
        }
        if (jj >= ctl->m_eff[k]) {
            // invariant subspace already reached: this realisation's next vectors stay zero
            for (int i = 0; i <= jj; ++i) ctl->coefA[i][k] = make_double2(0.0, 0.0);
            return;
        }
        for (int i = 0; i <= jj; ++i) {
            const double s = ctl->sigma[i][k];
            const double2 c = make_double2(fin[i].x * s, fin[i].y * s);
            ctl->coefA[i][k] = make_double2(c.x * s, c.y * s);
            if (i == jj) ctl->alpha[jj][k] = c.x;
        }
        ctl->normu2[k] = nw2;
    } else if (mode == 1) {
        if (k == 0) {
            H.vec_passes += (double)(jj + 3) + (general ? 1.0 : 0.0);
            H.vp_kind[KIND_PASSB] += (double)(jj + 3) + (general ? 1.0 : 0.0);
        }
        ctl->corr[k] = 0;
        ctl->dots[k] = 0;
        for (int i = 0; i <= jj; ++i) ctl->coefC[i][k] = make_double2(0.0, 0.0);
        if (jj >= ctl->m_eff[k]) return;
        // One classical Gram-Schmidt pass is enough unless the projection cancelled most of
        // u (||w|| < eta ||u||, the Daniel-Gragg-Kaufman-Stewart test); then this
        // realisation takes the dots of w with every previous vector (pass C1).
        if (H.verify || nw2 < H.eta_cancel * H.eta_cancel * ctl->normu2[k]) {
            ctl->dots[k] = 1;
            ctl->wnorm2[k] = nw2;
            ctl->wg[k] = gdot;
            H.dots_any = 1;
        } else {
            finalize(nw2, gdot);
        }
    } else if (mode == 3) {
        if (k == 0) {
            H.vec_passes += (double)(jj + 2);
            H.vp_kind[KIND_PASSC] += (double)(jj + 2);
        }
        if (!ctl->dots[k] || jj >= ctl->m_eff[k]) return;
        double nd2 = 0.0;
        for (int i = 0; i <= jj; ++i) {
            const double s = ctl->sigma[i][k];
            nd2 += (fin[i].x * fin[i].x + fin[i].y * fin[i].y) * s * s;
        }
        if (nw2 > 0.0) ctl->orth[k] = fmax(ctl->orth[k], sqrt(nd2 / nw2));
        if (nw2 > 0.0 && sqrt(nd2) > H.eta_corr * sqrt(nw2)) {
            ctl->corr[k] = 1;
            H.corr_any = 1;
            for (int i = 0; i <= jj; ++i) {
                const double s = ctl->sigma[i][k];
                ctl->coefC[i][k] = make_double2(fin[i].x * s * s, fin[i].y * s * s);
            }
            ctl->alpha[jj][k] += fin[jj].x * ctl->sigma[jj][k];
        } else {
            finalize(nw2, gdot);
        }
    } else if (mode == 2) {
        if (k == 0) {
            H.vec_passes += (double)(jj + 3) + (general ? 1.0 : 0.0);
            H.vp_kind[KIND_PASSC] += (double)(jj + 3) + (general ? 1.0 : 0.0);
        }
        if (jj < ctl->m_eff[k] && ctl->corr[k]) {
            atomicAdd(&H.n_corr, 1ull);
            finalize(nw2, gdot);
        }
    } else {   // 4 combine, 5 load of psi0
        const double b0 = sqrt(nw2);
        if (!(b0 > 0.0)) {
            H.err = KRY_EINVAL;
            H.done = 1;
            return;
        }
        ctl->beta0[k] = b0;
        ctl->sigma[0][k] = 1.0 / b0;
        ctl->g[0][k] = (mode == 5) ? make_double2(b0, 0.0) : make_double2(gdot.x / b0, gdot.y / b0);
        ctl->m_eff[k] = H.m;
        ctl->corr[k] = 0;
    }
}

// Shared bookkeeping after the combine (one thread): advance time, count the step.
__global__ void k_step_done_b(KryCtlB *ctl, int general)
{
    KryHdrB &H = ctl->hd;
    if (H.done) return;
    double e = 0.0;
    for (int k = 0; k < H.K; ++k) e = fmax(e, ctl->err_k[k]);
    H.err_sum += e;
    H.n_steps += 1;
    H.vec_passes += (double)(H.m_run + 1) + (general ? 1.0 : 0.0);
    H.vp_kind[KIND_COMBINE] += (double)(H.m_run + 1) + (general ? 1.0 : 0.0);
    H.t_now = H.t_next;
    H.next_out = H.next_out_new;
    H.m_run = H.m;
    H.corr_any = 0;
    if (H.finishing) H.done = 1;
}

// m_run refresh after pass C ran (all per-realisation epilogues of pass C are complete).
__global__ void k_mrun_b(KryCtlB *ctl)
{
    KryHdrB &H = ctl->hd;
    if (H.done) return;
    int mr = 0;
    for (int k = 0; k < H.K; ++k) mr = max(mr, ctl->m_eff[k]);
    H.m_run = mr;
}

// psi0_k = e_{r0_k}: each realisation starts from its own basis state
template <class V>
__global__ void k_set_basis_state_b(V *W0, int K, const KryCtlB *ctl)
{
    const int k = threadIdx.x;
    if (k < K) W0[(size_t)ctl->r0k[k] * K + k] = VT<V>::from(make_double2(1.0, 0.0));
}

// ---------------------------------------------------------------- launchers

static int sm_count_b()
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

static size_t hv_b_smem(const DevBasis &b, int rl_smem)
{
    return sizeof(SmemHeadB) + (rl_smem ? (sizeof(uint16_t) << b.Llo) : 0);
}

static size_t lincomb_b_smem(int Kp, size_t es)
{
    return es * (MMAX + 1) * Kp + es * TROWS * Kp + sizeof(double2) * 2 * NTHR;
}

template <class K_>
static int set_smem(K_ kernel, size_t smem)
{
    if (smem > 48 * 1024) KRY_CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KRY_OK;
}

#define KRY_KQ_SWITCH(Kp, ...)                                \
    switch (Kp) {                                             \
    case 32: { constexpr int KQ = 1; __VA_ARGS__; } break;    \
    case 64: { constexpr int KQ = 2; __VA_ARGS__; } break;    \
    default: { constexpr int KQ = 4; __VA_ARGS__; } break;    \
    }

// CTAs of the batched dots (returned) and of the updates (*gridB): whole SMs times the
// resident CTAs of each.
template <class V>
int batched_grid(const DevBasis &b, int Kp, int rl_smem, int *gridB)
{
    const size_t es = sizeof(V);
    int o1 = 1, o2 = 1;
    KRY_KQ_SWITCH(Kp, {
        if (int rc = set_smem(k_hv_b<V, KQ>, hv_b_smem(b, rl_smem))) return -rc;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_dots_b<V, KQ>, NTHR, 0);
        const size_t sL = lincomb_b_smem(Kp, es);
        if (int rc = set_smem(k_lincomb_b<V, 0, KQ>, sL)) return -rc;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_lincomb_b<V, 0, KQ>, NTHR, sL);
    });
    const uint32_t ntiles = (b.D + TROWS - 1) / TROWS;
    auto fit = [&](int occ) {
        return (int)std::max<uint32_t>(1u, std::min<uint32_t>(ntiles, (uint32_t)(sm_count_b() * std::max(1, occ))));
    };
    *gridB = fit(o2);
    return fit(o1);
}

// pass A: the H.v at full occupancy (its own grid), then the dots on the common grid
// (their partials feed k_reduce_b); part 1 launches the H.v alone, part 2 the dots alone
template <class V>
int launch_passA_b(const EvArgsB<V> &a, int jj, int grid, cudaStream_t s, int part)
{
    if (part == 2) {
        KRY_KQ_SWITCH(a.Kp, { k_dots_b<V, KQ><<<grid, NTHR, 0, s>>>(a, jj); });
        KRY_CU(cudaGetLastError());
        return KRY_OK;
    }
    if (a.b.list) {
        if (int rc = launch_list_hv_b<V>(a, jj, s)) return rc;
        if (part == 1) return KRY_OK;
        KRY_KQ_SWITCH(a.Kp, { k_dots_b<V, KQ><<<grid, NTHR, 0, s>>>(a, jj); });
        KRY_CU(cudaGetLastError());
        return KRY_OK;
    }
    const size_t sH = hv_b_smem(a.b, a.rl_smem);
    const uint32_t ntiles = (a.b.D + TROWS - 1) / TROWS;
    auto hv_grid = [&](auto kernel, uint32_t items) {
        int oh = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oh, kernel, NTHR, sH);
        return (int)std::max<uint32_t>(1u, std::min<uint32_t>(items, (uint32_t)(sm_count_b() * std::max(1, oh))));
    };
    if (a.kch == 8 || a.kch == 16) {   // chunks of realisations (launch shape part 4)
        const uint32_t items = ntiles * (uint32_t)((a.K + a.kch - 1) / a.kch);
        if (a.kch == 8) {
            if (int rc = set_smem(k_hv_bc<V, 8>, sH)) return rc;
            k_hv_bc<V, 8><<<hv_grid(k_hv_bc<V, 8>, items), NTHR, sH, s>>>(a, jj);
        } else {
            if (int rc = set_smem(k_hv_bc<V, 16>, sH)) return rc;
            k_hv_bc<V, 16><<<hv_grid(k_hv_bc<V, 16>, items), NTHR, sH, s>>>(a, jj);
        }
        KRY_CU(cudaGetLastError());
    } else {
        KRY_KQ_SWITCH(a.Kp, { k_hv_b<V, KQ><<<hv_grid(k_hv_b<V, KQ>, ntiles), NTHR, sH, s>>>(a, jj); });
        KRY_CU(cudaGetLastError());
    }
    if (part == 1) return KRY_OK;
    KRY_KQ_SWITCH(a.Kp, { k_dots_b<V, KQ><<<grid, NTHR, 0, s>>>(a, jj); });
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template <class V>
int launch_lincomb_b(const EvArgsB<V> &a, int mode, int jj, int grid, cudaStream_t s)
{
    const size_t sL = lincomb_b_smem(a.Kp, sizeof(V));
    KRY_KQ_SWITCH(a.Kp, {
        switch (mode) {
        case 0: if (int rc = set_smem(k_lincomb_b<V, 0, KQ>, sL)) return rc; k_lincomb_b<V, 0, KQ><<<grid, NTHR, sL, s>>>(a, jj); break;
        case 1: if (int rc = set_smem(k_lincomb_b<V, 1, KQ>, sL)) return rc; k_lincomb_b<V, 1, KQ><<<grid, NTHR, sL, s>>>(a, jj); break;
        case 2: if (int rc = set_smem(k_lincomb_b<V, 2, KQ>, sL)) return rc; k_lincomb_b<V, 2, KQ><<<grid, NTHR, sL, s>>>(a, jj); break;
        case 4: if (int rc = set_smem(k_lincomb_b<V, 4, KQ>, sL)) return rc; k_lincomb_b<V, 4, KQ><<<grid, NTHR, sL, s>>>(a, jj); break;
        default: if (int rc = set_smem(k_lincomb_b<V, 3, KQ>, sL)) return rc; k_lincomb_b<V, 3, KQ><<<grid, NTHR, sL, s>>>(a, jj); break;
        }
    });
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

// mode 0, 1 follow passes A, B; 3 and 2 passes C1 and C2; 4 the combine (then the shared
// step bookkeeping); 5 the load of a general psi0.
int launch_reduce_b(KryCtlB *ctl, const double2 *part, int grid, int K, int Kp, int mode, int jj,
                    int general, double, cudaStream_t s)
{
    k_reduce_b<<<K, 128, 0, s>>>(ctl, part, grid, Kp, mode, jj, general);
    KRY_CU(cudaGetLastError());
    if (mode == 2) {
        k_mrun_b<<<1, 1, 0, s>>>(ctl);
        KRY_CU(cudaGetLastError());
    }
    if (mode == 4) {
        k_step_done_b<<<1, 1, 0, s>>>(ctl, general);
        KRY_CU(cudaGetLastError());
    }
    return KRY_OK;
}

int launch_apply_b(const DevBasis &b, const DevHam &h, int c64, int K, const void *x, void *y,
                   int rl_smem, cudaStream_t s)
{
    if (b.list) return launch_list_apply(b, h, c64, K, x, y, s);
    int Kp = 32;
    while (Kp < K) Kp *= 2;
    const size_t smem = sizeof(SmemHeadB) + (rl_smem ? (sizeof(uint16_t) << b.Llo) : 0);
    const uint32_t ntiles = (b.D + TROWS - 1) / TROWS;
    const int grid = (int)std::min<uint32_t>(ntiles, (uint32_t)sm_count_b() * 8u);
    KRY_KQ_SWITCH(Kp, {
        if (c64) {
            if (int rc = set_smem(k_apply_b<float2, KQ>, smem)) return rc;
            k_apply_b<float2, KQ><<<grid, NTHR, smem, s>>>(b, h, K, (const float2 *)x, (float2 *)y, rl_smem);
        } else {
            if (int rc = set_smem(k_apply_b<double2, KQ>, smem)) return rc;
            k_apply_b<double2, KQ><<<grid, NTHR, smem, s>>>(b, h, K, (const double2 *)x, (double2 *)y, rl_smem);
        }
    });
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_set_basis_state_b(void *W0, int c64, int K, const KryCtlB *ctl, cudaStream_t s, int ff)
{
    if (c64) k_set_basis_state_b<float2><<<1, KBMAX, 0, s>>>((float2 *)W0, K, ctl);
    else if (ff) k_set_basis_state_b<ffc><<<1, KBMAX, 0, s>>>((ffc *)W0, K, ctl);
    else k_set_basis_state_b<double2><<<1, KBMAX, 0, s>>>((double2 *)W0, K, ctl);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template int batched_grid<ffc>(const DevBasis &, int, int, int *);
template int launch_passA_b<ffc>(const EvArgsB<ffc> &, int, int, cudaStream_t, int);
template int launch_lincomb_b<ffc>(const EvArgsB<ffc> &, int, int, int, cudaStream_t);
template int batched_grid<double2>(const DevBasis &, int, int, int *);
template int batched_grid<float2>(const DevBasis &, int, int, int *);
template int launch_passA_b<double2>(const EvArgsB<double2> &, int, int, cudaStream_t, int);
template int launch_passA_b<float2>(const EvArgsB<float2> &, int, int, cudaStream_t, int);
template int launch_lincomb_b<double2>(const EvArgsB<double2> &, int, int, int, cudaStream_t);
template int launch_lincomb_b<float2>(const EvArgsB<float2> &, int, int, int, cudaStream_t);

}  // namespace kry
