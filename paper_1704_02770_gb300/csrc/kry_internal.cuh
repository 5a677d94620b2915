// Internal declarations of the GB300 Krylov library (not installed; see include/kry.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <utility>
#include <vector>

#include "kry.h"

namespace kry {

// A complex number as two float-float numbers, x = xh + xl and y = yh + yl (about 48
// significant bits each, 16 bytes like complex128): the Krylov vectors of dtype KRY_C128E,
// on which the vector kernels do float-float arithmetic on the FP32 pipe (kry_device.cuh).
// Inputs and outputs of that dtype stay complex128; they are converted at the boundary.
struct __align__(16) ffc {
    float xh, xl, yh, yl;
};

// Index of a dtype's launch shape: KRY_C128, KRY_C64, KRY_C128E.
inline int dtype_slot(int dtype) { return dtype == KRY_C64 ? 1 : (dtype == KRY_C128E ? 2 : 0); }
inline bool dtype_ok(int dtype) { return dtype == KRY_C128 || dtype == KRY_C64 || dtype == KRY_C128E; }

constexpr int MMAX = 32;       // largest Krylov dimension m (one warp holds the small problem)
constexpr int TILE = 256;      // consecutive ranks per CTA tile
constexpr int NTHR = 256;      // threads per CTA of the vector kernels
constexpr int PSTRIDE = 40;    // partial-sum slots per CTA: MMAX+1 dots, then extras
constexpr int SLOT_NRM = 34;   // slot of a squared norm
constexpr int SLOT_G = 35;     // slot of the readout dot <psi0, w>
constexpr int KMAX = 128;      // largest Chebyshev degree of the small exponential
constexpr double XMAX = 50.0;  // largest tau * r (half-width) handled in one step

void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// Launch with programmatic dependent launch allowed: the kernel may begin while the
// kernel before it in the stream finishes, and waits for that kernel's completion
// (griddepcontrol.wait, see pdl_begin) before reading anything it wrote.
// With pdl = 0 the launch is an ordinary one (full dependence on the work before it), as
// needed after a node that is not a kernel (a conditional node of the step graph).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(int pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    return launch_ex(1, kernel, grid, block, smem, s, std::forward<Args>(args)...);
}

#define KRY_CU(call)                                                 \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::kry::cuda_fail(e_, #call);   \
    } while (0)

// Rank/unrank tables of one sector, resident on the device.
//   rank(s) = blk[s >> Llo] + ranklo[s & ((1 << Llo) - 1)]
// blk[hi] is the first rank of the block of states whose upper Lhi bits equal hi (the
// block holds C(Llo, N - popc(hi)) states, in the order of their lower bits); blk is
// non-decreasing (entries of empty blocks repeat the next start), so the block of a rank
// is found by binary search.  lolist lists the Llo-bit patterns grouped by popcount k,
// each group ascending and starting at koff[k]; ranklo[lo] is lo's index in its group.
// tstart[t] is the block holding rank t * TILE (one entry per tile of the vector kernels,
// so a tile finds its first state with one load instead of a search).
struct DevBasis {
    const uint32_t *blk;
    const uint32_t *tstart;   // [ceil(D / TILE)]
    const uint16_t *ranklo;
    const uint16_t *lolist;
    const uint32_t *koff;   // [Llo + 2]
    const uint32_t *bsz;    // [Llo + 1], C(Llo, k)
    int *err;               // device error flag of rank/unrank
    int L, N, Llo, Lhi;
    uint32_t D;
    // sorted-list basis (L > 32, or on request): the split tables above are unused
    int list;
    const uint64_t *states;   // [D] sorted states
    const uint32_t *cbin;     // C(p, k) at [p * (N + 1) + k], p < L, k <= N (saturated at 2^32 - 1)
};

// Hamiltonian parameters for the matrix-free H.v.  The field energy
// sum_i h_{k,i} (n_i - 1/2) of a state in realisation k is
// ehlo[pos * K + k] + ehhi[hi * K + k], pos = position of lo in lolist.
struct DevHam {
    const double *ehlo_d, *ehhi_d;
    const float *ehlo_f, *ehhi_f;
    double cz;      // J Delta / 4
    double halfJ;   // J / 2
    int nbonds;     // bonds of the chain (L-1 open, L on a ring with L >= 3)
    int pbc;        // ring bond (L-1, 0) present
    int K;          // realisations (field rows)
    // sorted-list basis: field energy by bytes of the state,
    //   sum_i h_{k,i} (n_i - 1/2) = sum_c eh8[(c * 256 + byte_c(s)) * K + k]
    const double *eh8_d;
    const float *eh8_f;
    int nchunk;     // bytes of a state, ceil(L / 8)
};

// ---------------------------------------------------------------- batched realisations
constexpr int KBMAX = 128;   // largest K of one batched evolution
constexpr int PSB = 36;      // partial-sum slots per (CTA, realisation): dots, then NRM, G
constexpr int TROWS = 16;    // rows (states) per CTA tile of the batched kernels

// kernel kinds of the profile: pass A's dots (with alpha_j and ||u||^2), pass B (the Lanczos
// update), pass C (the second Gram-Schmidt pass), the small exponential, the combine, and
// pass A's H.v
enum { KIND_PASSA = 0, KIND_PASSB = 1, KIND_PASSC = 2, KIND_EXP = 3, KIND_COMBINE = 4, KIND_HV = 5, NKIND = 6 };

// Control block of a batched evolution: one Lanczos recurrence per realisation k
// (structure of arrays, k fastest), one shared time grid and step size.
struct KryHdrB {   // shared scalars (copied to the host when polling)
    double t_now, t_end, tol, t_next;
    double eta_corr, eta_bd;
    double err_sum, max_orth, vec_passes;
    double vp_kind[NKIND];
    unsigned long long n_hv, n_steps, n_corr, n_bd;
    int K, m, m_run, corr_any, finishing, done, err;
    int n_times, next_out, next_out_new, r0;
    // second Gram-Schmidt pass: dots_any = some realisation takes the dots of w (pass C1)
    double eta_cancel;
    int verify, dots_any;
};
struct KryCtlB {
    KryHdrB hd;
    double alpha[MMAX + 1][KBMAX], beta[MMAX + 1][KBMAX], sigma[MMAX + 2][KBMAX];
    double2 coefA[MMAX + 1][KBMAX], coefC[MMAX + 1][KBMAX], coefY[MMAX + 1][KBMAX];
    double2 g[MMAX + 2][KBMAX];
    double normu2[KBMAX], beta0[KBMAX], tau_ok[KBMAX], err_k[KBMAX], orth[KBMAX];
    int m_eff[KBMAX], corr[KBMAX];
    double wnorm2[KBMAX];   // ||w||^2 of pass B, kept for pass C1
    double2 wg[KBMAX];      // <psi0, w> of pass B
    int dots[KBMAX];        // this realisation takes the dots of w (pass C1)
    int r0k[KBMAX];         // basis index of each realisation's initial state (hd.r0 >= 0)
    double pint[KBMAX];     // int_0^t_now P_k(t') dt' (temporal autocorrelation)
    double shift[KBMAX];    // s_k of the Lanczos operator H_k - s_k I
};

template <class V>
struct EvArgsB {
    DevBasis b;
    DevHam h;
    V *W;            // Krylov vectors, element (r, k) of W_i at i*ldW + r*K + k
    size_t ldW;
    V *U;
    const V *G;      // psi0 of a general initial state, or nullptr
    double2 *part;   // partials [grid][PSB][Kp]
    KryCtlB *ctl;
    int K, Kp;       // realisations; Kp = K rounded up to a power of two >= 32
    int rl_smem;
    int kch;         // H.v in chunks of kch realisations (8 or 16; 0 = all K at once)
};

struct ExpArgsB {
    KryCtlB *ctl;
    const double *times;
    double *P;       // [n_times][K]
    const void *W;
    size_t ldW;
    int c64, K;
    int ff;          // the vectors are float-float (ffc)
    double *C;       // nullable: temporal autocorrelation [n_times][K]
    const double *glx, *glw;   // Gauss-Legendre nodes and weights on [-1, 1] (with C)
};

// pass A of the batched path: part 0 = the H.v and the dots, 1 = the H.v only, 2 = the dots only
template <class V> int launch_passA_b(const EvArgsB<V> &a, int jj, int grid, cudaStream_t s, int part = 0);
template <class V> int launch_lincomb_b(const EvArgsB<V> &a, int mode, int jj, int grid, cudaStream_t s);
int launch_reduce_b(KryCtlB *ctl, const double2 *part, int grid, int K, int Kp, int mode, int jj,
                    int general, double es_bytes_per_vec, cudaStream_t s);
template <class V> int batched_grid(const DevBasis &b, int Kp, int rl_smem, int *gridB);
int launch_apply_b(const DevBasis &b, const DevHam &h, int c64, int K, const void *x, void *y,
                   int rl_smem, cudaStream_t s);
int launch_set_basis_state_b(void *W0, int c64, int K, const KryCtlB *ctl, cudaStream_t s, int ff = 0);
int launch_exp_b(const ExpArgsB &a, cudaStream_t s);

// Device control block of one evolution: Lanczos coefficients of the current Krylov
// step, time-stepping state and counters.  Written only by single-thread epilogues.
struct KryCtl {
    double alpha[MMAX + 1], beta[MMAX + 1], sigma[MMAX + 2];
    double2 coefA[MMAX + 1];   // update coefficients c_i sigma_i of pass B
    double2 coefC[MMAX + 1];   // correction coefficients of pass C
    double2 coefY[MMAX + 1];   // combine coefficients -beta0 y_i sigma_i
    double2 g[MMAX + 2];       // readout <psi0, v_i>
    double normu2;             // ||H v_j||^2 of the last pass A
    double beta0;              // ||psi|| at the start of the Krylov step
    double t_now, t_end, tol, tau_prev;
    double eta_corr, eta_bd;   // second-pass and breakdown thresholds (relative)
    double err_sum, max_orth, vec_passes;
    double vp_kind[NKIND];     // vector passes by kernel kind (KIND_*)
    long long n_hv, n_steps, n_corr, n_bd;
    int m, m_eff, corr, finishing, done, err;
    int n_times, next_out, r0;
    unsigned int counter;      // ticket of the last-CTA reductions
    // second Gram-Schmidt pass: corr = take the dots of w (pass C1), corr2 = subtract them (C2)
    int corr2, verify;
    double eta_cancel, wnorm2;
    double2 wg;
    // dense vector output (outputs [out_begin, out_end) of the current step) and checkpoints
    int out_begin, out_end;
    int ckpt_every, n_ckpt, ckpt_cap;
    double *ckpt_t;            // device [ckpt_cap]: time of every checkpoint
    double pint;               // int_0^t_now P(t') dt' (temporal autocorrelation)
    double shift;              // s of the Lanczos operator H - s I (T holds alpha - s)
    long long n_c1;            // second-pass dots taken (pass C1 runs)
};

// Dense output of whole vectors: psi(t_o) = sum_j Yout[o][j] W_j, written to out + o * ldOut.
template <class V>
struct VecOutArgs {
    const V *W;
    size_t ldW;
    const double2 *Yout;       // [n_times][MMAX]
    V *out;
    size_t ldOut;
    KryCtl *ctl;
    uint32_t D;
};
template <class V> int launch_vecout(const VecOutArgs<V> &a, int grid, cudaStream_t s);
template <class V> int launch_ckpt(const V *W0, V *ckpt, size_t ldC, KryCtl *ctl, uint32_t D, int grid,
                                   cudaStream_t s);
// Gradient integrand: acc[i] += sum_q w_q sum_r conj(lam_{nq-1-q}[r]) psi_q[r] dH_i[r] over the L
// single-site Sz_i (i < L) and the bond sum J/4 (nbonds - 2 n_anti) (i = L).
int launch_grad_acc(const DevBasis &b, const DevHam &h, double J, const double2 *psi, const double2 *lam,
                    size_t ld, const double *w, int nq, double2 *part, double2 *acc, unsigned *counter,
                    int grid, cudaStream_t s);

template <class V>
struct EvArgs {
    DevBasis b;
    DevHam h;
    V *W;            // Krylov vectors W_0..W_m, v_i = sigma_i W_i
    size_t ldW;      // elements between consecutive W_i
    V *U;            // H v_j
    const V *G;      // readout vector psi0 (general initial state) or nullptr
    double2 *part;   // per-CTA partial sums [grid][PSTRIDE]
    KryCtl *ctl;
    int rl_smem;     // stage ranklo in shared memory
    // pass B sets this conditional node of the step graph to whether the second
    // Gram-Schmidt pass (pass C) runs (use_cond = 0: no node, pass C kernels always launched)
    cudaGraphConditionalHandle cond;
    int use_cond;
    // launch shape (host side only): H.v gather form, dots form, update rows per thread
    int hv_form, dots_form, upd_rows;
};

struct ExpArgs {
    KryCtl *ctl;
    const double *times;
    double *P;
    const void *W;   // Krylov vectors (element type given by c64 and ff)
    size_t ldW;
    int c64;
    int ff;          // the vectors are float-float (ffc)
    double2 *Yout;   // nullable: combine coefficients of every output time [n_times][MMAX]
    double *C;       // nullable: temporal autocorrelation C(t_o) of every output time
    const double *glx, *glw;   // NGL-point Gauss-Legendre nodes and weights on [-1, 1] (with C)
};
constexpr int NGL = 64;   // Gauss-Legendre nodes of the per-step integral of P

size_t apply_smem(const DevBasis &b, int rl_smem, int c64);

// sorted-list basis (kry_list.cu)
int list_build(DevBasis &b, cudaStream_t s);
int launch_list_rank(const DevBasis &b, const uint64_t *st, uint32_t *rk, int64_t n, cudaStream_t s);
int launch_list_unrank(const DevBasis &b, const uint32_t *rk, uint64_t *st, int64_t n, cudaStream_t s);
int launch_list_apply(const DevBasis &b, const DevHam &h, int c64, int K, const void *x, void *y, cudaStream_t s);
template <class V> int launch_list_hv(const EvArgs<V> &a, int jj, int grid, cudaStream_t s, int pdl = 1);
template <class V> int launch_list_hv_b(const EvArgsB<V> &a, int jj, cudaStream_t s);
template <class V> int list_hv_grid(const DevBasis &b, int *grid);
size_t list_smem(const DevBasis &b);

// kernel launchers (kry_hv.cu)
int launch_apply(const DevBasis &b, const DevHam &h, int c64, const void *x, void *y,
                 int rl_smem, cudaStream_t s);
template <class V> int launch_hv(const EvArgs<V> &a, int jj, int grid, cudaStream_t s, int pdl = 1);
template <class V> int launch_lincomb(const EvArgs<V> &a, int mode, int jj, int grid,
                                      cudaStream_t s, int pdl = 1);
template <class V> int launch_dots(const EvArgs<V> &a, int mode, int jj, int grid, cudaStream_t s, int pdl = 1);
template <class V> int vector_grid(const DevBasis &b, int rl_smem, int hv_form, int *gridH, int *gridB);
int launch_set_basis_state(void *W0, int c64, uint32_t r0, cudaStream_t s, int ff = 0);
// complex128 <-> float-float vectors of n elements (the boundary of KRY_C128E)
int launch_c128_to_ffc(const void *src, void *dst, size_t n, cudaStream_t s);
int launch_ffc_to_c128(const void *src, void *dst, size_t n, cudaStream_t s);
// small exponential (kry_exp.cu)
int launch_smallexp(const ExpArgs &a, cudaStream_t s, int pdl = 1);


}  // namespace kry

struct kry_basis_s {
    int L, N, Llo, Lhi;
    int64_t D;
    void *d_tab;
    kry::DevBasis dev;
    int device;
};

struct kry_ham_s {
    kry_basis b;
    double J, Delta;
    int K, boundary;
    std::vector<double> h;
    void *d_eh;
    kry::DevHam dev;
    // the Lanczos pass works on H - s_k I (s_k = tr(H_k)/D): the same tables with s_k taken
    // off the field energy, so that the diagonal offset does not dominate ||H v||
    kry::DevHam dev_lz;
    std::vector<double> shift;
    // evolution workspace (grown on demand, freed by kry_hamiltonian_destroy)
    void *ws;
    size_t ws_bytes;
    int ws_user;                // ws belongs to the caller (kry_set_workspace): never freed here
    // cached CUDA graph of one Krylov step
    cudaGraphExec_t gexec;
    int g_dtype, g_m, g_general, g_grid, g_gridB, g_gridH, g_shape, g_plain;
    int plain_graph;            // forced plain step graph (kry_profile_enable(H, 2))
    int cond_pass_c;            // pass C as a conditional node (kry_set_second_pass_node)
    void *g_ws;
    const void *g_G;
    const void *g_vec, *g_ck;   // optional vector-output and checkpoint buffers baked in the graph
    int g_C;                    // the graph integrates P for C(t)
    size_t g_ldo, g_ldc;
    // per precision, the launch shape of the vector kernels (kry_set_shape, kry_autotune):
    // [0] CTAs of the streaming kernels (0 = occupancy rule), [1] H.v form (bit 0: chunks of
    // eight gathers; bit 1: rank table through L1), [2] dots form (0 prefetch, 1 none), [3]
    // update rows per thread,
    // [4] batched H.v in chunks of this many realisations (0 = all K)
    int shape[3][5];
    int orth_check;             // measure <v_i, w> after every Lanczos update
    cudaStream_t cap_stream;
    cudaStream_t cap_stream2;   // captures the bodies of the step graph's conditional nodes
    void *h_poll;   // pinned host mirror of the control block
    // profiling: CUDA events recorded between the kernels of the captured step
    int prof_on;
    std::vector<cudaEvent_t> prof_ev;
    double prof_ms[kry::NKIND], prof_bytes[kry::NKIND];
    int64_t prof_launches[kry::NKIND];
};

// Launch shape of a new Hamiltonian: the occupancy-rule grid, prefetching dots, two update
// rows per thread, all realisations at once, and the H.v one hop at a time with the
// lower-bit rank table in shared memory -- except for lower parts of 14 bits or more (L >=
// 28), whose table (32-64 KB) would cap the H.v at three or four CTAs per SM: there the
// gathers go in rounds and the table is read through L1 (form 3; 2.9x faster at L = 30).
inline void default_shape(kry_ham_s *H, int Llo)
{
    const int v[5] = {0, Llo >= 14 ? 3 : 0, 0, 2, 0};
    for (int d = 0; d < 3; ++d)
        for (int q = 0; q < 5; ++q) H->shape[d][q] = v[q];
}
