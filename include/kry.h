/*
 * kry.h -- C ABI of the GB300 Krylov return-probability library (libkry_gb300.so).
 *
 * The library evaluates |psi(t)> = exp(-iHt)|psi0> and the return probability
 * P(t) = |<psi0|psi(t)>|^2 (Eq. SP, Sec. 4 of Brenes, Varma, Scardicchio, Girotto,
 * "Massively parallel implementation and approaches to simulate quantum dynamics using
 * Krylov subspace techniques") for the chain of Eq. 1, restricted to a sector of fixed
 * particle number N (Sec. 2, "Basis representation"), with Krylov subspaces (Sec. 2,
 * "Krylov subspace methods").  Everything runs on one CUDA device.
 *
 * Conventions shared by every call:
 *  - A state is an integer: bit i-1 is the occupation (spin up) of site i (Sec. 2).  The
 *    sector basis is the ascending list of the L-bit integers with N set bits; the rank of
 *    a state is its index in that list.
 *  - Hamiltonian (Eq. 1 written in spin-1/2 form, hard-core bosons = XXZ chain):
 *        H = J sum_b [ (S+_i S-_j + S-_i S+_j)/2 + Delta Sz_i Sz_j ] + sum_i h_i Sz_i,
 *    Sz = n - 1/2.  Bonds b = (i, i+1), i = 1..L-1, plus (L, 1) when boundary == KRY_PBC
 *    and L >= 3.  Eq. 1's t and V are J/2 and J*Delta; its on-site term h n_i equals
 *    h_i Sz_i up to a constant, which does not change P.
 *  - Pointers named d_* are device pointers, others are host pointers.  All buffers are
 *    owned by the caller; the library never frees them.  Handles are owned by the library
 *    and released by the matching *_destroy call.
 *  - Complex vectors are interleaved (re, im): complex128 (KRY_C128) or complex64
 *    (KRY_C64).  Vectors of a Hamiltonian with K field rows are stored state-major,
 *    element (state r, realisation k) at index r*K + k.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls
 *    that return host results synchronise that stream before returning.
 *  - Every call returns a status code; on failure kry_last_error() gives a message.  No
 *    C++ exception crosses this interface.  A handle must not be used by two host threads
 *    at the same time.
 */
#ifndef KRY_H
#define KRY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kry_basis_s *kry_basis;
typedef struct kry_ham_s *kry_ham;

enum {
    KRY_OK = 0,
    KRY_EINVAL = 1,    /* bad argument (size, pointer, state outside the sector, ...) */
    KRY_ENOMEM = 2,    /* device allocation failed or exceeds the configured cap        */
    KRY_ETOL = 3,      /* no step size meets the tolerance                              */
    KRY_ETIMEOUT = 4,  /* the evolution did not finish within its step budget           */
    KRY_ECUDA = 5      /* a CUDA runtime call failed                                    */
};
enum { KRY_OBC = 0, KRY_PBC = 1 };
/* Element types of the state vectors.  KRY_C128: complex128 with FP64 arithmetic.  KRY_C64:
 * complex64 vectors and H.v, FP64 Lanczos coefficients and FP64-grade (float-float) dots.
 * KRY_C128E: complex128 in and out (the same arguments as KRY_C128), with the Krylov vectors
 * held as float-float pairs (16 bytes per element, about 48 significant bits) and the vector
 * arithmetic (H.v sums, dots, updates) done in float-float on the FP32 pipe, because GB300
 * runs FP64 at 1/64 of its FP32 rate; the Lanczos coefficients, the small exponential and the
 * step control stay FP64.  KRY_C128E serves every basis and both single and batched
 * (K > 1, [D][K]) evolutions, like the other dtypes; kry_apply takes KRY_C128 and KRY_C64
 * only, and kry_grad runs in complex128. */
enum { KRY_C128 = 0, KRY_C64 = 1, KRY_C128E = 2 };

/* Counters of one kry_evolve / kry_return_probability call. */
typedef struct kry_stats {
    int64_t n_hv;            /* H.v applications (each over all K realisations)            */
    int64_t n_krylov_steps;  /* accepted time steps                                         */
    int64_t n_second_pass;   /* reorthogonalisation corrections applied                     */
    int64_t n_breakdowns;    /* Krylov spaces that became invariant before m vectors        */
    double err_estimate;     /* sum of the accepted local error estimates (bound on ||dpsi||) */
    double max_orth_loss;    /* max |<v_i, v_j>| / ||v_j|| seen before the correction        */
    double time_ms;          /* device time of the call (CUDA events)                        */
    double algo_bytes;       /* algorithmic HBM bytes of the call, by formula                 */
    int64_t n_launches;      /* kernels the call launched (including no-op launches)          */
    int64_t n_second_dots;   /* second-pass dots taken (the test before a correction)         */
} kry_stats;

/* ---------------------------------------------------------------- basis (Sec. 2, Alg. 2)
 * Create the sector basis of L sites and n_up particles: 1 <= L <= 64, 0 <= n_up <= L.
 * For L <= 32 no basis list is stored; rank and unrank tables of about 2^(L/2+2) bytes live
 * on the current device.  For L > 32 the call returns the sorted-list form of
 * kry_basis_create_list.  Returns KRY_EINVAL for bad sizes, KRY_ENOMEM/KRY_ECUDA on device
 * failure. */
int kry_basis_create(int L, int n_up, kry_basis *out);
/* Sorted-list form of the basis (the sorted integer list of Alg. 2, built on the device;
 * 8 bytes per state) for 1 <= L <= 64 with D = C(L, n_up) <= 2^31 - 1 (KRY_EINVAL above).
 * Ranks are combinadic numbers, rank(s) = sum_j C(p_j, j) over the occupied sites
 * p_1 < ... < p_N, so lookups need no search.  Every call below accepts either form. */
int kry_basis_create_list(int L, int n_up, kry_basis *out);
int kry_basis_destroy(kry_basis b);
/* Sector dimension D = L!/(N!(L-N)!) (Sec. 2); -1 for a NULL handle. */
int64_t kry_basis_dim(kry_basis b);

/* Rank: d_ranks[i] = index of state d_states[i] in the sorted basis (Sec. 2 "binary
 * lookup"; computed here without a stored list).  n >= 0 states, device arrays.  Returns
 * KRY_EINVAL (after the stream is synchronised) if any state has bits at or above L or a
 * particle number other than n_up; its rank is then written as 0xFFFFFFFF. */
int kry_basis_rank(kry_basis b, const uint64_t *d_states, uint32_t *d_ranks, int64_t n,
                   void *stream);
/* Unrank: d_states[i] = the basis state of rank d_ranks[i] (the d_ranks[i]-th element of
 * the list that Algorithm 2 generates).  Ranks >= D give state 0 and KRY_EINVAL. */
int kry_basis_unrank(kry_basis b, const uint32_t *d_ranks, uint64_t *d_states, int64_t n,
                     void *stream);

/* ---------------------------------------------------------------- Hamiltonian (Eq. 1)
 * Bind couplings to a basis.  h: host array [K][L] of on-site fields (row k is
 * realisation k; K >= 1; the quasiperiodic field of Eq. 1 is h_i = h cos(2 pi beta i +
 * phi)).  boundary: KRY_OBC or KRY_PBC.  The matrix is never stored: H.v is evaluated
 * on the fly.  The basis must outlive the Hamiltonian. */
int kry_hamiltonian_set(kry_basis b, double J, double Delta, const double *h, int K,
                        int boundary, kry_ham *out);
int kry_hamiltonian_destroy(kry_ham H);

/* y = H x (the operation H|Psi> of Sec. 2), device vectors of D*K elements of type
 * dtype.  x and y must not overlap. */
int kry_apply(kry_ham H, int dtype, const void *d_x, void *d_y, void *stream);

/* Time evolution (Sec. 2, Krylov subspace methods; Eq. SP).  d_psi0: device [D][K]
 * vector of type dtype (normalised per realisation for P to be a probability).  times:
 * host array of n_times >= 1 non-decreasing, non-negative output times.  m: Krylov
 * dimension, 1 <= m <= 32.  tol: absolute error budget of P at every output time.
 * P_out: host [n_times][K], P_out[t*K+k] = |<psi0_k|psi_k(t)>|^2.  d_psi_out (nullable):
 * device [D][K] vector receiving psi(times[n_times-1]).  stats nullable.
 * KRY_C64 keeps vectors and H.v in complex64 and the Lanczos coefficients, dot products,
 * small exponential and step control in FP64. */
int kry_evolve(kry_ham H, int dtype, const void *d_psi0, const double *times, int n_times,
               int m, double tol, void *d_psi_out, double *P_out, kry_stats *stats,
               void *stream);

/* Same as kry_evolve with psi0 = the basis state psi0_state (e.g. the Neel state
 * ...010101 of Sec. 4) for every realisation; no input vector is needed. */
int kry_return_probability(kry_ham H, int dtype, uint64_t psi0_state, const double *times,
                           int n_times, int m, double tol, double *P_out,
                           kry_stats *stats, void *stream);

/* Temporal autocorrelation (Sec. 4): C(t) = (1/t) int_0^t P(t') dt' with P of Eq. SP, for
 * psi0 = the basis state psi0_state in every realisation.  The integral is accumulated over
 * the Krylov steps of the same evolution that gives P: each step's share is a 64-point
 * Gauss-Legendre quadrature of P on the step's small exponential, so C carries P's error
 * budget tol plus a quadrature error far below it for the step lengths the error control
 * accepts.  C_out: host [n_times][K], C_out[o*K+k] = C_k(times[o]), C(0) = 1 (required).
 * P_out: host [n_times][K] (required).  Other arguments as kry_return_probability. */
int kry_autocorrelation(kry_ham H, int dtype, uint64_t psi0_state, const double *times,
                        int n_times, int m, double tol, double *C_out, double *P_out,
                        kry_stats *stats, void *stream);

/* Power-law decay exponent (Sec. 4): the least-squares fit log C = log a - gamma log t over
 * the n points (t[i], C[i]) with t_min <= t[i] <= t_max (host arrays, e.g. the output of
 * kry_autocorrelation).  Host arithmetic only; no device is touched.  Returns KRY_EINVAL
 * when fewer than two distinct times lie in the window or C <= 0 there.  log_a nullable. */
int kry_decay_exponent(const double *t, const double *C, int n, double t_min, double t_max,
                       double *gamma, double *log_a);

/* Ensembles of initial states (Sec. 2 disorder layers, Sec. 4 random initial states):
 * realisation k starts from the basis state psi0_states[k] (host [K], each in the sector,
 * KRY_EINVAL otherwise) and evolves under its own fields h_k.  P_out: host [n_times][K]
 * (required); C_out: host [n_times][K] temporal autocorrelations, or NULL to skip them.
 * K > 1 runs the batched path (one step size for all realisations, each within tol). */
int kry_return_probability_states(kry_ham H, int dtype, const uint64_t *psi0_states,
                                  const double *times, int n_times, int m, double tol,
                                  double *P_out, double *C_out, kry_stats *stats, void *stream);

/* Gradient of the return probability of Eq. SP with respect to the on-site fields and to
 * Delta, for psi0 = the basis state psi0_state and one time t >= 0 (a single-realisation
 * Hamiltonian, K = 1; complex128).  With psi(s) = exp(-iHs) psi0 and the costate
 * lambda(s) = exp(+iH(t-s)) psi0:
 *   dA/dtheta = -i int_0^t <lambda(s)| dH/dtheta |psi(s)> ds,  dP/dtheta = 2 Re(conj(A) dA/dtheta),
 *   dH/dh_i = Sz_i,  dH/dDelta = J sum_b Sz Sz.
 * The costate is evolved backward with the same Krylov kernels (a forward evolution
 * under -H); psi is checkpointed after every ckpt_every-th Krylov step of the forward
 * sweep and recomputed interval by interval during the backward sweep; the integral uses
 * composite 16-point Gauss-Legendre rules.  Outputs (host): P = P(t), dP_dh[L],
 * dP_dDelta.  Allocates its own temporary device buffers: a few vectors of D complex128,
 * the vectors at the quadrature nodes of one checkpoint interval, and the checkpoints.  The
 * checkpoint buffer starts with room for 8; a forward sweep of more than 8 * ckpt_every
 * Krylov steps grows it to (steps / ckpt_every) vectors and repeats the sweep.  KRY_ENOMEM
 * (with the sizes in the message) when they do not fit: a larger ckpt_every needs fewer.
 * Synchronises `stream`.  m, tol: as kry_evolve. */
int kry_grad(kry_ham H, uint64_t psi0_state, double t, int m, double tol, int ckpt_every,
             double *P, double *dP_dh, double *dP_dDelta, kry_stats *stats, void *stream);

/* Small-exponential kernel exposed for testing (Sec. 2: psi ~ V_m exp(-itA_m) e_1).
 * Given the symmetric tridiagonal T (alpha[m] diagonal, beta[m-1] off-diagonal, host
 * arrays), its coupling h to the next Krylov vector, and tau >= 0, computes on the
 * device y = exp(-i tau T) e_1 (host y_out[2m], interleaved) and the local error
 * estimate err = h |e_m^T tau phi_1(-i tau (T - c)) e_1| used by the step control, with c
 * the centre of T's Gershgorin interval.  1 <= m <= 32.  Synchronises `stream`. */
int kry_tridiag_expv(const double *alpha, const double *beta, int m, double h, double tau,
                     double *y_out, double *err_out, void *stream);

/* The paper has no counterpart to this call: it is kry_tridiag_expv for callers that must
 * not allocate device memory.  Some callers give every byte of device memory to their own
 * pool with a hard limit, so an extra cudaMalloc can fail.  Others cannot let cudaFree
 * synchronise the whole device while their other streams are running.  kry_tridiag_expv
 * does a cudaMalloc and a cudaFree on every call; this variant calls neither, nor any
 * other routine that allocates.  Arguments and results are those of kry_tridiag_expv.
 * Its device scratch is one fixed array of about 1 KB, which every GPU that loads the
 * library keeps until the process exits.  That array caps m at 32; a larger m returns
 * KRY_EINVAL with a message naming the limit.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current) and keeps it for
 * the CUDA context it was found in; a call from another context (for instance after
 * cudaDeviceReset) looks it up again.  Make the first call on a device, and the first after a
 * reset, before any stream capture.  All calls share the one array: calls
 * whose GPU work overlaps (two host threads, or two streams) race on it and must be
 * serialised by the caller.  Each call copies in every value its kernel reads, so nothing
 * left in the array by an earlier call affects the result.  Synchronises `stream`. */
int kry_tridiag_expv_noalloc(const double *alpha, const double *beta, int m, double h,
                             double tau, double *y_out, double *err_out, void *stream);

/* Per-kernel profile (not part of the paper's method; a measurement aid).
 * kry_profile_enable(H, 1) makes later kry_evolve / kry_return_probability calls on H
 * record CUDA events between the kernels of every Krylov step (on the caller's stream,
 * inside the replayed graph) and synchronise after each step; 0 turns it off.  With 2 no
 * events are recorded, and the step graph launches the second Gram-Schmidt pass as two plain
 * kernels in every Lanczos index (returning at once unless needed) even where
 * kry_set_second_pass_node asked for a conditional node: external profilers such as Nsight
 * Compute cannot see the kernels of a graph that has conditional nodes.  KRY_EINVAL for
 * other values.
 * kry_profile_read fills, for the six kernel kinds
 *   0 = pass A's dots (<v_i, u> for i <= j, alpha_j and ||u||^2), 1 = pass B (the Lanczos
 *   update w = u - sum c_i v_i and ||w||^2), 2 = pass C (the second Gram-Schmidt pass, when
 *   flagged), 3 = small exponential and step control, 4 = combine psi = beta V y,
 *   5 = pass A's H.v (u = sigma_j (H - s) v_j),
 * the summed event time in ms, the algorithmic HBM bytes (vector reads and writes by
 * formula; gathers of H.v beyond one read of v_j are not counted) and the count of
 * profiled intervals, accumulated since the last kry_profile_enable(H, 1).  Arrays have 6
 * entries, host. */
int kry_profile_enable(kry_ham H, int on);
int kry_profile_read(kry_ham H, double *ms, double *bytes, int64_t *launches);

/* Launch shape of the vector kernels (not part of the paper's method), per Hamiltonian and
 * dtype, five ints:
 *   shape[0] CTAs of the streaming kernels: 0 = the occupancy rule (whole SMs times the
 *            resident CTAs of each kernel), else that many CTAs;
 *   shape[1] form of the H.v, two bits: bit 0 set = the targets of up to four hops computed
 *            first and their loads issued together (else one hop at a time); bit 1 set = the
 *            lower-bit rank table read through the L1 cache instead of staged in shared memory
 *            (at L = 29, 30 that table takes 64 KB of shared memory per CTA);
 *   shape[2] dots of pass A: 0 = the next vector's rows loaded before the current vector's
 *            products are accumulated (complex64), 1 = without that prefetch;
 *   shape[3] rows per thread of the update pass: 1, 2 or 4;
 *   shape[4] H.v of batched Hamiltonians (K > 1) in chunks of 8 or 16 realisations, so that
 *            the gathered part of the vector fits in L2 (0 = all K at once).
 * Parts 1, 2 and 4 change only the order of independent loads (the results are bitwise the
 * same); parts 0 and 3 change which rows a thread or CTA sums into its partial norms and dots
 * (the results agree to rounding).  Single-realisation evolutions use parts 0-3, batched ones
 * parts 0 and 4.  New Hamiltonians start at {0, 0, 0, 2, 0}, or {0, 3, 0, 2, 0} for L >= 28
 * (split-table bases), where the rank table of the lower bits is 32-64 KB.
 * kry_set_shape returns KRY_EINVAL for values outside those lists; kry_set_grid sets part 0. */
int kry_set_shape(kry_ham H, int dtype, const int *shape);
int kry_get_shape(kry_ham H, int dtype, int *shape);
int kry_set_grid(kry_ham H, int dtype, int grid);

/* Launch-shape autotuner (not part of the paper's method).  Times a probe evolution of the
 * basis state probe_state to t_probe (reps replays after one capture run, best kept) for
 * candidate shapes, one part after another with the other parts at their best so far: part 0
 * over {0, 1, 2, 3, 4 x the SM count}, then part 1 over {0..3}, part 2 over {0, 1}, part 3 over
 * {2, 1, 4} (K > 1: part 0, then part 4 over {0, 16, 8}).  Keeps the fastest for later calls on
 * H with this dtype and returns it in shape_out[5].  cand_out (host, [max_cand][5]) and ms_out
 * ([max_cand]) receive the shapes tried and their times, *n_cand how many were stored. */
int kry_autotune(kry_ham H, int dtype, int m, uint64_t probe_state, double t_probe, int reps,
                 int *shape_out, int *cand_out, double *ms_out, int max_cand, int *n_cand,
                 void *stream);

/* Reorthogonalisation check (a diagnostic; single-realisation evolutions).  Every new
 * Lanczos vector is orthogonalised against all previous ones by one classical Gram-Schmidt
 * pass (Sec. 2: Arnoldi orthogonalises each new vector against the whole basis); a second
 * pass is made only when that pass cancelled most of the vector (||w|| < 0.1 ||H v_j||).
 * With on = 1 the dots of every new vector with all previous ones are measured after each
 * pass (kry_stats.max_orth_loss) and subtracted when they exceed eta ||w||, with eta about
 * 1e4 units of roundoff of the vector storage: 1e-12 (KRY_C128), 3e-11 (KRY_C128E), 1e-5
 * (KRY_C64); with on = 2 they are subtracted after every update (classical Gram-Schmidt
 * applied twice to every vector, as in the oracle).  Besides the cancellation test, the
 * second pass is also taken when the lengths of u = H v_j, of its projections c = V^H u and
 * of w = u - V c disagree with Pythagoras, | ||w||^2 - (||u||^2 - ||c||^2) | > eta ||c|| ||w||
 * plus the storage-precision noise, a sign that V has lost orthogonality.  Returns
 * KRY_EINVAL for other values of on. */
int kry_set_orth_check(kry_ham H, int on);

/* Form of the second Gram-Schmidt pass in the captured Krylov step (single-realisation
 * evolutions; not part of the paper's method).  on = 0 (the default): its two kernels are
 * launched in every Lanczos index and return at once unless pass B flagged the pass.  on = 1:
 * they are the body of a conditional graph node (CUDA 12.4+ IF node) whose value pass B's
 * last CTA sets on the device, so nothing is launched where the pass is not needed.  Both
 * forms give bitwise the same results.  The kernel after a conditional node cannot start
 * before the node ends (no programmatic dependent launch across it); on GB300 the
 * conditional form measured 0.7-2.1% slower over whole L = 24 evolutions, hence the default.
 * KRY_EINVAL unless on is 0 or 1. */
int kry_set_second_pass_node(kry_ham H, int on);

/* Bytes of device workspace an evolution of H (single or batched by H's K) needs in dtype
 * with Krylov dimension m and n_times output times, at the current launch shape (an autotuned
 * grid can change it); -1 on bad input.  kry_workspace_size is the same for one output time. */
int64_t kry_workspace_bytes(kry_ham H, int dtype, int m, int n_times);
int64_t kry_workspace_size(kry_ham H, int dtype, int m);
/* Give H a caller-owned device workspace (e.g. a torch tensor's memory): d_ws 256-byte
 * aligned, `bytes` long, used by every later kry_evolve / kry_return_probability /
 * kry_autocorrelation / kry_return_probability_states / kry_autotune call on H, never freed
 * by the library.  A call that needs more than `bytes` (kry_workspace_bytes) returns
 * KRY_EINVAL instead of allocating.  d_ws = NULL returns to library-managed memory.  The
 * buffer must outlive its use; kry_grad keeps its own buffers. */
int kry_set_workspace(kry_ham H, void *d_ws, int64_t bytes);

/* Measured arithmetic peaks of the current device (a measurement aid, not part of the paper's
 * method): FP64 and FP32 fused multiply-add throughput in TFLOP/s (2 flops per multiply-add),
 * from independent chains of multiply-adds on every SM timed with CUDA events on `stream`
 * (best of three after a warm-up).  Allocates and frees 4 bytes of device memory; takes about
 * 0.3 s; synchronises `stream`.  The complex128 kernels are bound by the FP64 rate on GB300,
 * and this is the denominator of their roofline. */
int kry_measure_peaks(double *fp64_tflops, double *fp32_tflops, void *stream);

/* Message of the last failing call on this host thread ("" if none). */
const char *kry_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KRY_H */
