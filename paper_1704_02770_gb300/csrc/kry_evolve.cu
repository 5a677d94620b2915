// Host side of the time evolution (Sec. 2, "Krylov subspace methods"; Eq. SP): workspace,
// CUDA-graph capture of one Krylov step, the replay loop and the C ABI entry points
// kry_apply / kry_evolve / kry_return_probability.
//
// One Krylov step, captured once per (precision, m) and replayed:
//   for j = 0..m-1:  pass A (u = H v_j, then the dots <v_i, u>)  ->  pass B (update)
//                    ->  pass C (second Gram-Schmidt pass, runs only when flagged)
//   small exponential + step control + dense output of P  ->  combine psi = beta V y.
// Device flags end the Lanczos loop early on an invariant subspace and turn every kernel
// into a no-op once the last output time is reached; the host only polls that flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>

#include "kry_internal.cuh"

using namespace kry;

namespace {

uint64_t binom_host(int n, int k)
{
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

size_t elem_size(int dtype) { return dtype == KRY_C64 ? sizeof(float2) : sizeof(double2); }   // (sizeof(ffc) = 16)

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int rl_in_smem(const DevBasis &b) { return (!b.list && b.Llo <= 15) ? 1 : 0; }

void drop_graph(kry_ham_s *H);

// Timing events of one call, released on every return path.
struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
    ~EventPair()
    {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

// The evolution workspace: grown on demand by the library, or the caller's buffer
// (kry_set_workspace), which must already be large enough.
int ensure_workspace(kry_ham_s *H, size_t bytes)
{
    if (H->ws && H->ws_bytes >= bytes) return KRY_OK;
    if (H->ws_user) {
        set_error("kry_evolve: the workspace given to kry_set_workspace holds %zu bytes; this call needs %zu",
                  H->ws_bytes, bytes);
        return KRY_EINVAL;
    }
    drop_graph(H);
    if (H->ws) cudaFree(H->ws);
    H->ws = nullptr;
    H->ws_bytes = 0;
    cudaError_t e = cudaMalloc(&H->ws, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(workspace)");
    H->ws_bytes = bytes;
    return KRY_OK;
}

struct Layout {
    size_t ldW, oW, oU, oG, oPart, oCtl, oTimes, oP, oY, oC, oGL, bytes;
};

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);   // (adjoint section)

// Upload the NGL Gauss-Legendre nodes and weights of the per-step integral of P (temporal
// autocorrelation) to dst = [nodes | weights].
int upload_gl(char *dst, cudaStream_t s)
{
    static const std::vector<double> gl = [] {   // [nodes | weights], built once (thread-safe)
        std::vector<double> x, w;
        gauss_legendre(NGL, x, w);
        x.insert(x.end(), w.begin(), w.end());
        return x;
    }();
    KRY_CU(cudaMemcpyAsync(dst, gl.data(), sizeof(double) * 2 * NGL, cudaMemcpyHostToDevice, s));
    return KRY_OK;
}

Layout layout(const kry_ham_s *H, int dtype, int m, int grid, int n_times)
{
    Layout l{};
    const size_t es = elem_size(dtype);
    const size_t n = (size_t)H->b->D * (size_t)H->K;
    l.ldW = round_up(n, 64);
    l.oW = 0;
    l.oU = l.oW + (size_t)(m + 1) * l.ldW * es;
    l.oG = l.oU + l.ldW * es;
    l.oPart = l.oG + l.ldW * es;
    l.oCtl = round_up(l.oPart + (size_t)grid * PSTRIDE * sizeof(double2), 256);
    l.oTimes = round_up(l.oCtl + sizeof(KryCtl), 256);
    l.oP = round_up(l.oTimes + sizeof(double) * (size_t)n_times, 256);
    l.oY = round_up(l.oP + sizeof(double) * (size_t)n_times * H->K, 256);
    l.oC = round_up(l.oY + sizeof(double2) * MMAX * (size_t)n_times, 256);
    l.oGL = round_up(l.oC + sizeof(double) * (size_t)n_times, 256);
    l.bytes = round_up(l.oGL + sizeof(double) * 2 * NGL, 256);
    return l;
}

// Optional outputs of an evolution used by the gradient: whole vectors at every output
// time, and checkpoints of psi after every `ckpt_every`-th Krylov step.
struct EvOpts {
    void *vec_out = nullptr;   // [n_times][ldOut] elements
    size_t ldOut = 0;
    void *ckpt = nullptr;      // [ckpt_cap][ldC] elements
    double *d_ckpt_t = nullptr;   // device [ckpt_cap]: checkpoint times
    size_t ldC = 0;
    int ckpt_every = 0, ckpt_cap = 0;
    int n_ckpt = 0;            // out: checkpoints written (at most ckpt_cap)
    std::vector<double> ckpt_t;   // out: their times
    double *C_out = nullptr;   // host [n_times]: temporal autocorrelation C(t_o)
};

// CTAs of the streaming dots (returned), of the H.v (*gridH) and of the updates (*gridB);
// an autotuned override sets the two streaming grids.
int grid_for(const kry_ham_s *H, int dtype, int *gridH, int *gridB)
{
    const DevBasis &b = H->b->dev;
    const int rl = rl_in_smem(b);
    const int hvf = H->shape[dtype_slot(dtype)][1];
    const int g = dtype == KRY_C64    ? vector_grid<float2>(b, rl, hvf, gridH, gridB)
                  : dtype == KRY_C128E ? vector_grid<ffc>(b, rl, hvf, gridH, gridB)
                                       : vector_grid<double2>(b, rl, hvf, gridH, gridB);
    const int ov = H->shape[dtype_slot(dtype)][0];
    if (g > 0 && ov > 0) *gridB = ov;
    return (g > 0 && ov > 0) ? ov : g;   // vector_grid also sets the kernels' smem limits
}

void drop_graph(kry_ham_s *H)
{
    if (H->gexec) cudaGraphExecDestroy(H->gexec);
    H->gexec = nullptr;
    for (cudaEvent_t e : H->prof_ev) cudaEventDestroy(e);
    H->prof_ev.clear();
}

// pass C launched in every Lanczos index (true) or as a conditional node
bool plain_step_graph(const kry_ham_s *H) { return H->plain_graph || !H->cond_pass_c; }

// Profile intervals of the captured step: four per Lanczos index (the H.v, pass A's dots,
// pass B, pass C), then the small exponential and the combine; kind of the k-th interval.
int n_intervals(int m) { return 4 * m + 2; }
int kind_of(int k, int m)
{
    if (k < 4 * m) {
        const int q = k % 4;
        return q == 0 ? KIND_HV : q == 1 ? KIND_PASSA : q == 2 ? KIND_PASSB : KIND_PASSC;
    }
    return k == 4 * m ? KIND_EXP : KIND_COMBINE;
}

template <class V>
int capture_step(kry_ham_s *H, const EvArgs<V> &a, const ExpArgs &ea, int m, int grid, int gridH,
                 int gridB, const EvOpts *opt)
{
    cudaStream_t cs = H->cap_stream;
    cudaGraph_t g = nullptr;
    if (H->prof_on) {
        H->prof_ev.resize(n_intervals(m) + 1);
        for (auto &e : H->prof_ev) KRY_CU(cudaEventCreate(&e));
    }
    KRY_CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = KRY_OK, k = 0;
    auto mark = [&]() {
        if (H->prof_on && rc == KRY_OK) {
            cudaError_t er = cudaEventRecordWithFlags(H->prof_ev[k], cs, cudaEventRecordExternal);
            if (er != cudaSuccess) rc = cuda_fail(er, "cudaEventRecord(capture)");
        }
        ++k;
    };
    // The second Gram-Schmidt pass (pass C: its dots, then the subtraction) runs only where
    // pass B flagged it, in one of two forms.  Plain (the default): its two kernels are
    // launched in every Lanczos index and return at once unless flagged; with programmatic
    // dependent launch they cost about 3 us each.  Conditional (kry_set_second_pass_node):
    // they are the body of a conditional node after pass B, whose last CTA sets the node's
    // value; the kernel after the node is launched without programmatic dependence (that
    // only links two kernels), and on GB300 this form measured 0.7-2.1% slower over whole
    // evolutions at L = 24.  kry_profile_enable(H, 2) forces the plain form (external
    // profilers cannot see the kernels of a graph that has conditional nodes).
    const bool plain = plain_step_graph(H);
    cudaStream_t cs2 = H->cap_stream2;
    int after_cond = 0;
    for (int jj = 0; jj < m && rc == KRY_OK; ++jj) {
        mark();
        rc = launch_hv<V>(a, jj, gridH, cs, after_cond ? 0 : 1);
        mark();
        if (rc == KRY_OK) rc = launch_dots<V>(a, 0, jj, grid, cs);
        mark();
        if (plain) {
            if (rc == KRY_OK) rc = launch_lincomb<V>(a, 0, jj, gridB, cs);
            mark();
            if (rc == KRY_OK) rc = launch_dots<V>(a, 1, jj, grid, cs);
            if (rc == KRY_OK) rc = launch_lincomb<V>(a, 1, jj, gridB, cs);
            continue;
        }
        EvArgs<V> ab = a;
        cudaGraph_t cg = nullptr;
        if (rc == KRY_OK) {
            cudaStreamCaptureStatus cst;
            cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg);
            if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&ab.cond, cg, 0, cudaGraphCondAssignDefault);
            if (e != cudaSuccess) rc = cuda_fail(e, "conditional handle");
            ab.use_cond = 1;
        }
        if (rc == KRY_OK) rc = launch_lincomb<V>(ab, 0, jj, gridB, cs);
        mark();
        if (rc == KRY_OK) {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t *deps = nullptr;
            const cudaGraphEdgeData *edges = nullptr;
            size_t nd = 0;
            cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, &edges, &nd);
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = ab.cond;
            cp.conditional.type = cudaGraphCondTypeIf;
            cp.conditional.size = 1;
            cudaGraphNode_t node = nullptr;
            if (e == cudaSuccess) e = cudaGraphAddNode(&node, cg, deps, edges, nd, &cp);
            if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(cs2, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) rc = cuda_fail(e, "conditional node");
            if (rc == KRY_OK) {
                rc = launch_dots<V>(a, 1, jj, grid, cs2, 0);
                if (rc == KRY_OK) rc = launch_lincomb<V>(a, 1, jj, gridB, cs2, 0);
                cudaGraph_t body = nullptr;
                e = cudaStreamEndCapture(cs2, &body);
                if (rc == KRY_OK && e != cudaSuccess) rc = cuda_fail(e, "conditional body capture");
            }
            after_cond = 1;
        }
    }
    mark();
    if (rc == KRY_OK) rc = launch_smallexp(ea, cs, after_cond ? 0 : 1);
    if constexpr (!std::is_same<V, ffc>::value) {
    if (rc == KRY_OK && opt && opt->vec_out) {
        VecOutArgs<V> va{};
        va.W = a.W;
        va.ldW = a.ldW;
        va.Yout = ea.Yout;
        va.out = (V *)opt->vec_out;
        va.ldOut = opt->ldOut;
        va.ctl = a.ctl;
        va.D = a.b.D;
        rc = launch_vecout<V>(va, gridB, cs);
    }
    }   // (the vector outputs of the adjoint are complex128 or complex64 only)
    mark();
    if (rc == KRY_OK) rc = launch_lincomb<V>(a, 2, 0, gridB, cs);
    if constexpr (!std::is_same<V, ffc>::value) {
        if (rc == KRY_OK && opt && opt->ckpt)
            rc = launch_ckpt<V>(a.W, (V *)opt->ckpt, opt->ldC, a.ctl, a.b.D, gridB, cs);
    }
    mark();
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != KRY_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&H->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { H->gexec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return KRY_OK;
}

template <class V>
int evolve_t(kry_ham_s *H, int dtype, const void *d_psi0, uint64_t state, bool general,
             const double *times, int n_times, int m, double tol, void *d_psi_out, double *P_out,
             kry_stats *st, cudaStream_t s, EvOpts *opt = nullptr)
{
    const DevBasis &b = H->b->dev;
    int gridH = 0, gridB = 0;
    const int grid = grid_for(H, dtype, &gridH, &gridB);
    if (grid <= 0) { set_error("kry_evolve: kernel configuration failed"); return KRY_ECUDA; }
    const Layout l = layout(H, dtype, m, std::max(grid, std::max(gridH, gridB)), n_times);
    if (int rc = ensure_workspace(H, l.bytes)) return rc;
    if (!H->cap_stream) KRY_CU(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    if (!H->cap_stream2) KRY_CU(cudaStreamCreateWithFlags(&H->cap_stream2, cudaStreamNonBlocking));
    if (!H->h_poll) KRY_CU(cudaMallocHost(&H->h_poll, sizeof(KryCtl)));
    char *base = (char *)H->ws;
    EvArgs<V> a{};
    a.b = b;
    a.h = H->dev_lz;   // the Lanczos pass runs on H - s I
    a.W = (V *)(base + l.oW);
    a.ldW = l.ldW;
    a.U = (V *)(base + l.oU);
    a.G = general ? (const V *)(base + l.oG) : nullptr;
    a.part = (double2 *)(base + l.oPart);
    a.ctl = (KryCtl *)(base + l.oCtl);
    a.rl_smem = rl_in_smem(b);
    const int *shp = H->shape[dtype_slot(dtype)];
    a.hv_form = shp[1];
    a.dots_form = shp[2];
    a.upd_rows = shp[3];
    ExpArgs ea{};
    ea.ctl = a.ctl;
    ea.times = (const double *)(base + l.oTimes);
    ea.P = (double *)(base + l.oP);
    ea.W = a.W;
    ea.ldW = l.ldW;
    ea.c64 = dtype == KRY_C64;
    ea.ff = std::is_same<V, ffc>::value;
    ea.Yout = (opt && opt->vec_out) ? (double2 *)(base + l.oY) : nullptr;
    const int want_C = (opt && opt->C_out) ? 1 : 0;
    if (want_C) {
        if (int rc = upload_gl(base + l.oGL, s)) return rc;
        ea.C = (double *)(base + l.oC);
        ea.glx = (const double *)(base + l.oGL);
        ea.glw = ea.glx + NGL;
    }
    const void *vkey = opt ? opt->vec_out : nullptr, *ckey = opt ? opt->ckpt : nullptr;
    // graph of one Krylov step (reused while the workspace and the shape are unchanged)
    const int skey = shp[1] * 100 + shp[2] * 10 + shp[3];
    if (H->gexec && (H->g_dtype != dtype || H->g_m != m || H->g_general != (int)general || H->g_shape != skey ||
                     H->g_plain != (int)plain_step_graph(H) ||
                     H->g_grid != grid || H->g_gridB != gridB || H->g_gridH != gridH || H->g_ws != H->ws ||
                     H->g_G != (const void *)(base + l.oP) ||
                     H->ws_bytes < l.bytes || (int)H->prof_ev.empty() == H->prof_on ||
                     H->g_vec != vkey || H->g_ck != ckey || H->g_C != want_C ||
                     (opt && (H->g_ldo != opt->ldOut || H->g_ldc != opt->ldC))))
        drop_graph(H);
    if (!H->gexec) {
        if (int rc = capture_step<V>(H, a, ea, m, grid, gridH, gridB, opt)) return rc;
        H->g_dtype = dtype; H->g_m = m; H->g_general = general; H->g_grid = grid; H->g_gridB = gridB;
        H->g_gridH = gridH;
        H->g_shape = skey;
        H->g_plain = plain_step_graph(H);
        H->g_ws = H->ws; H->g_G = base + l.oP;
        H->g_vec = vkey; H->g_ck = ckey; H->g_C = want_C;
        H->g_ldo = opt ? opt->ldOut : 0;
        H->g_ldc = opt ? opt->ldC : 0;
    }
    EventPair evp;
    KRY_CU(cudaEventCreate(&evp.a));
    KRY_CU(cudaEventCreate(&evp.b));
    cudaEvent_t ev0 = evp.a, ev1 = evp.b;
    KRY_CU(cudaEventRecord(ev0, s));
    // control block
    KryCtl c;
    std::memset(&c, 0, sizeof c);
    c.m = m;
    c.m_eff = m;
    c.t_end = times[n_times - 1];
    c.tol = tol;
    c.n_times = n_times;
    // second-pass threshold on the loss of orthogonality, about 1e4 units of roundoff of the
    // vector storage: FP64 (2^-53) 1e-12, float-float (2^-48) 3e-11, complex64 (2^-24) 1e-5
    c.eta_corr = H->orth_check == 2 ? 0.0 : (dtype == KRY_C64 ? 1e-5 : dtype == KRY_C128E ? 3e-11 : 1e-12);
    c.eta_bd = dtype == KRY_C64 ? 1e-6 : 1e-12;
    c.eta_cancel = 0.1;
    c.verify = H->orth_check ? 1 : 0;
    c.shift = H->shift[0];
    if (opt && opt->ckpt) {
        c.ckpt_every = opt->ckpt_every;
        c.ckpt_cap = opt->ckpt_cap;
        c.ckpt_t = opt->d_ckpt_t;
    }
    const size_t es = sizeof(V), nvec = (size_t)b.D * (size_t)H->K;
    if (general) {
        c.r0 = -1;
    } else {
        uint64_t r = 0;
        int j = 0;
        for (int p = 0; p < b.L; ++p)
            if ((state >> p) & 1ull) r += binom_host(p, ++j);
        c.r0 = (int)r;
        c.beta0 = 1.0;
        c.sigma[0] = 1.0;
        c.g[0] = make_double2(1.0, 0.0);
    }
    KRY_CU(cudaMemcpyAsync(a.ctl, &c, sizeof c, cudaMemcpyHostToDevice, s));
    KRY_CU(cudaMemcpyAsync((void *)ea.times, times, sizeof(double) * n_times, cudaMemcpyHostToDevice, s));
    constexpr bool FF = std::is_same<V, ffc>::value;   // complex128 in and out, float-float inside
    if (general) {
        if (FF) {
            if (int rc = launch_c128_to_ffc(d_psi0, (void *)a.G, nvec, s)) return rc;
        } else {
            KRY_CU(cudaMemcpyAsync((void *)a.G, d_psi0, nvec * es, cudaMemcpyDeviceToDevice, s));
        }
        if (int rc = launch_lincomb<V>(a, 3, 0, gridB, s)) return rc;
    } else {
        KRY_CU(cudaMemsetAsync(a.W, 0, nvec * es, s));
        if (int rc = launch_set_basis_state(a.W, dtype == KRY_C64, (uint32_t)c.r0, s, FF)) return rc;
    }
    // replay until the device reports the last output time
    KryCtl *hp = (KryCtl *)H->h_poll;
    long long launched = 0;
    const long long max_launch = 500000;   // Krylov steps before KRY_ETIMEOUT
    int batch = 1;
    const int nk = 3 * m + 2;   // kernels of the step graph (pass C not counted)
    const double vp0[NKIND] = {0, 0, 0, 0, 0, 0};
    for (;;) {
        if (H->prof_on) batch = 1;   // events are read after every step
        for (int i = 0; i < batch; ++i) KRY_CU(cudaGraphLaunch(H->gexec, s));
        launched += batch;
        KRY_CU(cudaMemcpyAsync(hp, a.ctl, sizeof(KryCtl), cudaMemcpyDeviceToHost, s));
        KRY_CU(cudaStreamSynchronize(s));
        if (H->prof_on) {
            for (int k = 0; k < n_intervals(m); ++k) {
                float ms = 0.f;
                KRY_CU(cudaEventElapsedTime(&ms, H->prof_ev[k], H->prof_ev[k + 1]));
                H->prof_ms[kind_of(k, m)] += ms;
                H->prof_launches[kind_of(k, m)] += 1;
            }
        }
        if (hp->done || hp->err) break;
        if (launched >= max_launch) {
            set_error("kry_evolve: no convergence after %lld Krylov steps (t = %g of %g)", launched,
                      hp->t_now, hp->t_end);
            return KRY_ETIMEOUT;
        }
        const double rem = hp->t_end - hp->t_now;
        const double est = hp->tau_prev > 0.0 ? rem / hp->tau_prev : 1.0;
        batch = (int)std::min(64.0, std::max(1.0, std::ceil(est * 1.05)));
    }
    KRY_CU(cudaEventRecord(ev1, s));
    if (H->prof_on)
        for (int q = 0; q < NKIND; ++q)
            H->prof_bytes[q] += (hp->vp_kind[q] - vp0[q]) * (double)nvec * (double)es;
    if (hp->err) {
        if (hp->err == KRY_ETOL) set_error("kry_evolve: no step size meets tol=%g at t=%g", tol, hp->t_now);
        else set_error("kry_evolve: initial vector has zero norm");
        return hp->err;
    }
    KRY_CU(cudaMemcpyAsync(P_out, ea.P, sizeof(double) * n_times * H->K, cudaMemcpyDeviceToHost, s));
    if (want_C) KRY_CU(cudaMemcpyAsync(opt->C_out, ea.C, sizeof(double) * n_times, cudaMemcpyDeviceToHost, s));
    if (d_psi_out && FF) {
        if (int rc = launch_ffc_to_c128(a.W, d_psi_out, nvec, s)) return rc;
    } else if (d_psi_out) {
        KRY_CU(cudaMemcpyAsync(d_psi_out, a.W, nvec * es, cudaMemcpyDeviceToDevice, s));
    }
    KRY_CU(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    if (st) {
        st->n_hv = hp->n_hv;
        st->n_krylov_steps = hp->n_steps;
        st->n_second_pass = hp->n_corr;
        st->n_breakdowns = hp->n_bd;
        st->err_estimate = hp->err_sum;
        st->max_orth_loss = hp->max_orth;
        st->time_ms = ms;
        st->algo_bytes = hp->vec_passes * (double)nvec * (double)es;
        const bool plain = plain_step_graph(H);
        st->n_launches = launched * (nk + (plain ? 2 * m : 0) + (ea.Yout ? 1 : 0) + ((opt && opt->ckpt) ? 1 : 0)) +
                         (plain ? 0 : 2 * hp->n_c1) + 1 + (FF && general ? 1 : 0) + (FF && d_psi_out ? 1 : 0);
        st->n_second_dots = hp->n_c1;
    }
    if (opt && opt->ckpt) {
        opt->n_ckpt = std::min(hp->n_ckpt, opt->ckpt_cap);
        opt->ckpt_t.assign((size_t)opt->n_ckpt, 0.0);
        if (opt->n_ckpt > 0) {
            KRY_CU(cudaMemcpyAsync(opt->ckpt_t.data(), opt->d_ckpt_t, sizeof(double) * opt->n_ckpt,
                                   cudaMemcpyDeviceToHost, s));
            KRY_CU(cudaStreamSynchronize(s));
        }
    }
    return KRY_OK;
}

// ---------------------------------------------------------------- batched realisations

int padded_k(int K)
{
    int Kp = 32;
    while (Kp < K) Kp *= 2;
    return Kp;
}

Layout layout_b(const kry_ham_s *H, int dtype, int m, int grid, int n_times)
{
    Layout l{};
    const size_t es = elem_size(dtype);
    const size_t n = (size_t)H->b->D * (size_t)H->K;
    const int Kp = padded_k(H->K);
    l.ldW = round_up(n, 64);
    l.oW = 0;
    l.oU = l.oW + (size_t)(m + 1) * l.ldW * es;
    l.oG = l.oU + l.ldW * es;
    l.oPart = l.oG + l.ldW * es;
    l.oCtl = round_up(l.oPart + (size_t)grid * PSB * Kp * sizeof(double2), 256);
    l.oTimes = round_up(l.oCtl + sizeof(KryCtlB), 256);
    l.oP = round_up(l.oTimes + sizeof(double) * (size_t)n_times, 256);
    l.oC = round_up(l.oP + sizeof(double) * (size_t)n_times * H->K, 256);
    l.oGL = round_up(l.oC + sizeof(double) * (size_t)n_times * H->K, 256);
    l.bytes = round_up(l.oGL + sizeof(double) * 2 * NGL, 256);
    return l;
}

// CTAs of the batched dots of pass A (returned) and of the update, second pass and combine
// (*gridB), both by the occupancy rule; an autotuned override sets *gridB.
int grid_for_b(const kry_ham_s *H, int dtype, int *gridB)
{
    const DevBasis &b = H->b->dev;
    const int Kp = padded_k(H->K);
    const int g = dtype == KRY_C64     ? batched_grid<float2>(b, Kp, rl_in_smem(b), gridB)
                  : dtype == KRY_C128E ? batched_grid<ffc>(b, Kp, rl_in_smem(b), gridB)
                                       : batched_grid<double2>(b, Kp, rl_in_smem(b), gridB);
    const int ov = H->shape[dtype_slot(dtype)][0];
    if (g > 0 && ov > 0) *gridB = ov;
    return g;
}

// One Krylov step of the batched path, in groups whose boundaries carry the profile events:
// per Lanczos index {H.v}, {pass A's dots, reduce}, {pass B, reduce}, {pass C1, reduce,
// pass C2, reduce, m_run}; then {exp scan, exp apply} and {combine, reduce, step bookkeeping}.
template <class V>
int capture_step_b(kry_ham_s *H, const EvArgsB<V> &a, const ExpArgsB &ea, int m, int grid, int gridB,
                   int general)
{
    cudaStream_t cs = H->cap_stream;
    cudaGraph_t g = nullptr;
    if (H->prof_on) {
        H->prof_ev.resize(n_intervals(m) + 1);
        for (auto &e : H->prof_ev) KRY_CU(cudaEventCreate(&e));
    }
    KRY_CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = KRY_OK, k = 0;
    auto mark = [&]() {
        if (H->prof_on && rc == KRY_OK) {
            cudaError_t er = cudaEventRecordWithFlags(H->prof_ev[k], cs, cudaEventRecordExternal);
            if (er != cudaSuccess) rc = cuda_fail(er, "cudaEventRecord(capture)");
        }
        ++k;
    };
    const double2 *part = a.part;
    for (int jj = 0; jj < m && rc == KRY_OK; ++jj) {
        mark();
        rc = launch_passA_b<V>(a, jj, grid, cs, 1);
        mark();
        if (rc == KRY_OK) rc = launch_passA_b<V>(a, jj, grid, cs, 2);
        if (rc == KRY_OK) rc = launch_reduce_b(a.ctl, part, grid, a.K, a.Kp, 0, jj, general, 0, cs);
        mark();
        if (rc == KRY_OK) rc = launch_lincomb_b<V>(a, 0, jj, gridB, cs);
        if (rc == KRY_OK) rc = launch_reduce_b(a.ctl, part, gridB, a.K, a.Kp, 1, jj, general, 0, cs);
        mark();
        if (rc == KRY_OK) rc = launch_lincomb_b<V>(a, 4, jj, gridB, cs);
        if (rc == KRY_OK) rc = launch_reduce_b(a.ctl, part, gridB, a.K, a.Kp, 3, jj, general, 0, cs);
        if (rc == KRY_OK) rc = launch_lincomb_b<V>(a, 1, jj, gridB, cs);
        if (rc == KRY_OK) rc = launch_reduce_b(a.ctl, part, gridB, a.K, a.Kp, 2, jj, general, 0, cs);
    }
    mark();
    if (rc == KRY_OK) rc = launch_exp_b(ea, cs);
    mark();
    if (rc == KRY_OK) rc = launch_lincomb_b<V>(a, 2, 0, gridB, cs);
    if (rc == KRY_OK) rc = launch_reduce_b(a.ctl, part, gridB, a.K, a.Kp, 4, 0, general, 0, cs);
    mark();
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (rc != KRY_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&H->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { H->gexec = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return KRY_OK;
}

template <class V>
int evolve_bt(kry_ham_s *H, int dtype, const void *d_psi0, uint64_t state, bool general,
              const double *times, int n_times, int m, double tol, void *d_psi_out, double *P_out,
              kry_stats *st, cudaStream_t s, const uint64_t *states = nullptr, double *C_out = nullptr)
{
    const DevBasis &b = H->b->dev;
    const int K = H->K, Kp = padded_k(K);
    int gridB = 0;
    const int grid = grid_for_b(H, dtype, &gridB);
    if (grid <= 0) { set_error("kry_evolve: kernel configuration failed"); return KRY_ECUDA; }
    const Layout l = layout_b(H, dtype, m, std::max(grid, gridB), n_times);
    if (int rc = ensure_workspace(H, l.bytes)) return rc;
    if (!H->cap_stream) KRY_CU(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    if (!H->h_poll) KRY_CU(cudaMallocHost(&H->h_poll, sizeof(KryCtl) > sizeof(KryHdrB) ? sizeof(KryCtl) : sizeof(KryHdrB)));
    char *base = (char *)H->ws;
    EvArgsB<V> a{};
    a.b = b;
    a.h = H->dev_lz;   // the Lanczos pass runs on H - s I
    a.W = (V *)(base + l.oW);
    a.ldW = l.ldW;
    a.U = (V *)(base + l.oU);
    a.G = general ? (const V *)(base + l.oG) : nullptr;
    a.part = (double2 *)(base + l.oPart);
    a.ctl = (KryCtlB *)(base + l.oCtl);
    a.K = K;
    a.Kp = Kp;
    a.rl_smem = rl_in_smem(b);
    a.kch = H->shape[dtype_slot(dtype)][4];
    ExpArgsB ea{};
    ea.ctl = a.ctl;
    ea.times = (const double *)(base + l.oTimes);
    ea.P = (double *)(base + l.oP);
    ea.W = a.W;
    ea.ldW = l.ldW;
    ea.c64 = dtype == KRY_C64;
    ea.ff = std::is_same<V, ffc>::value;
    ea.K = K;
    const int want_C = C_out ? 1 : 0;
    if (want_C) {
        if (int rc = upload_gl(base + l.oGL, s)) return rc;
        ea.C = (double *)(base + l.oC);
        ea.glx = (const double *)(base + l.oGL);
        ea.glw = ea.glx + NGL;
    }
    const int gkey = 2 + (int)general;   // distinguishes batched graphs from single ones
    if (H->gexec && (H->g_dtype != dtype || H->g_m != m || H->g_general != gkey || H->g_shape != a.kch ||
                     H->g_grid != grid || H->g_gridB != gridB || H->g_ws != H->ws || H->g_C != want_C ||
                     H->g_G != (const void *)(base + l.oP) || (int)H->prof_ev.empty() == H->prof_on))
        drop_graph(H);
    if (!H->gexec) {
        if (int rc = capture_step_b<V>(H, a, ea, m, grid, gridB, (int)general)) return rc;
        H->g_dtype = dtype; H->g_m = m; H->g_general = gkey; H->g_grid = grid; H->g_gridB = gridB;
        H->g_shape = a.kch;
        H->g_ws = H->ws; H->g_G = base + l.oP; H->g_C = want_C;
    }
    EventPair evp;
    KRY_CU(cudaEventCreate(&evp.a));
    KRY_CU(cudaEventCreate(&evp.b));
    cudaEvent_t ev0 = evp.a, ev1 = evp.b;
    KRY_CU(cudaEventRecord(ev0, s));
    KryCtlB *c = new (std::nothrow) KryCtlB();
    if (!c) { set_error("kry_evolve: host allocation failed"); return KRY_ENOMEM; }
    std::memset(c, 0, sizeof(KryCtlB));
    KryHdrB &hd = c->hd;
    hd.K = K;
    hd.m = m;
    hd.m_run = m;
    hd.t_end = times[n_times - 1];
    hd.tol = tol;
    hd.n_times = n_times;
    hd.eta_corr = dtype == KRY_C64 ? 1e-5 : dtype == KRY_C128E ? 3e-11 : 1e-12;
    hd.eta_cancel = 0.1;
    hd.verify = H->orth_check;
    hd.eta_bd = dtype == KRY_C64 ? 1e-6 : 1e-12;
    for (int k = 0; k < K; ++k) {
        c->m_eff[k] = m;
        c->shift[k] = H->shift[k];
    }
    const size_t es = sizeof(V), nvec = (size_t)b.D * (size_t)K;
    if (general) {
        hd.r0 = -1;
    } else {
        // one basis state for every realisation, or one per realisation (states[k])
        for (int k = 0; k < K; ++k) {
            const uint64_t sk = states ? states[k] : state;
            uint64_t r = 0;
            int j = 0;
            for (int p = 0; p < b.L; ++p)
                if ((sk >> p) & 1ull) r += binom_host(p, ++j);
            c->r0k[k] = (int)r;
        }
        hd.r0 = c->r0k[0];
        for (int k = 0; k < K; ++k) {
            c->beta0[k] = 1.0;
            c->sigma[0][k] = 1.0;
            c->g[0][k] = make_double2(1.0, 0.0);
        }
    }
    cudaError_t ce = cudaMemcpyAsync(a.ctl, c, sizeof(KryCtlB), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);   // c is freed next
    delete c;
    if (ce != cudaSuccess) return cuda_fail(ce, "control block upload");
    KRY_CU(cudaMemcpyAsync((void *)ea.times, times, sizeof(double) * n_times, cudaMemcpyHostToDevice, s));
    constexpr bool FF = std::is_same<V, ffc>::value;   // complex128 in and out, float-float inside
    if (general) {
        if (FF) {
            if (int rc = launch_c128_to_ffc(d_psi0, (void *)a.G, nvec, s)) return rc;
        } else {
            KRY_CU(cudaMemcpyAsync((void *)a.G, d_psi0, nvec * es, cudaMemcpyDeviceToDevice, s));
        }
        if (int rc = launch_lincomb_b<V>(a, 3, 0, gridB, s)) return rc;
        if (int rc = launch_reduce_b(a.ctl, a.part, gridB, K, Kp, 5, 0, 1, 0, s)) return rc;
    } else {
        KRY_CU(cudaMemsetAsync(a.W, 0, nvec * es, s));
        if (int rc = launch_set_basis_state_b(a.W, dtype == KRY_C64, K, a.ctl, s, FF)) return rc;
    }
    KryHdrB *hp = (KryHdrB *)H->h_poll;
    long long launched = 0;
    const long long max_launch = 500000;   // Krylov steps before KRY_ETIMEOUT
    int batch = 1;
    for (;;) {
        if (H->prof_on) batch = 1;
        for (int i = 0; i < batch; ++i) KRY_CU(cudaGraphLaunch(H->gexec, s));
        launched += batch;
        KRY_CU(cudaMemcpyAsync(hp, &a.ctl->hd, sizeof(KryHdrB), cudaMemcpyDeviceToHost, s));
        KRY_CU(cudaStreamSynchronize(s));
        if (H->prof_on) {
            for (int k = 0; k < n_intervals(m); ++k) {
                float ms = 0.f;
                KRY_CU(cudaEventElapsedTime(&ms, H->prof_ev[k], H->prof_ev[k + 1]));
                H->prof_ms[kind_of(k, m)] += ms;
                H->prof_launches[kind_of(k, m)] += 1;
            }
        }
        if (hp->done || hp->err) break;
        if (launched >= max_launch) {
            set_error("kry_evolve: no convergence after %lld Krylov steps (t = %g of %g)", launched,
                      hp->t_now, hp->t_end);
            return KRY_ETIMEOUT;
        }
        const double rem = hp->t_end - hp->t_now;
        const double est = (hp->t_next > 0.0 && hp->n_steps > 0) ? rem / (hp->t_now / (double)hp->n_steps) : 1.0;
        batch = (int)std::min(64.0, std::max(1.0, std::ceil(est * 1.05)));
    }
    KRY_CU(cudaEventRecord(ev1, s));
    if (H->prof_on)
        for (int q = 0; q < NKIND; ++q) H->prof_bytes[q] += hp->vp_kind[q] * (double)nvec * (double)es;
    if (hp->err) {
        if (hp->err == KRY_ETOL) set_error("kry_evolve: no step size meets tol=%g at t=%g", tol, hp->t_now);
        else set_error("kry_evolve: an initial vector has zero norm");
        return hp->err;
    }
    KRY_CU(cudaMemcpyAsync(P_out, ea.P, sizeof(double) * n_times * K, cudaMemcpyDeviceToHost, s));
    if (want_C) KRY_CU(cudaMemcpyAsync(C_out, ea.C, sizeof(double) * n_times * K, cudaMemcpyDeviceToHost, s));
    if (d_psi_out && FF) {
        if (int rc = launch_ffc_to_c128(a.W, d_psi_out, nvec, s)) return rc;
    } else if (d_psi_out) {
        KRY_CU(cudaMemcpyAsync(d_psi_out, a.W, nvec * es, cudaMemcpyDeviceToDevice, s));
    }
    std::vector<double> orth(K);
    KRY_CU(cudaMemcpyAsync(orth.data(), a.ctl->orth, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
    KRY_CU(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    if (st) {
        st->n_hv = (int64_t)hp->n_hv;
        st->n_krylov_steps = (int64_t)hp->n_steps;
        st->n_second_pass = (int64_t)hp->n_corr;
        st->n_breakdowns = (int64_t)hp->n_bd;
        st->err_estimate = hp->err_sum;
        st->max_orth_loss = *std::max_element(orth.begin(), orth.end());
        st->time_ms = ms;
        st->algo_bytes = hp->vec_passes * (double)nvec * (double)es;
        st->n_launches = launched * (10 * m + 5) + (general ? 2 : 1) + (FF && general ? 1 : 0) + (FF && d_psi_out ? 1 : 0);
        st->n_second_dots = 0;
    }
    return KRY_OK;
}

int check_evolve_args(kry_ham H, int dtype, const double *times, int n_times, int m, double tol,
                      double *P_out)
{
    if (!H || !times || n_times < 1 || !P_out || m < 1 || m > MMAX || !(tol > 0.0) || !dtype_ok(dtype)) {
        set_error("kry_evolve: bad arguments (need H, times, n_times >= 1, P_out, 1 <= m <= %d, tol > 0)", MMAX);
        return KRY_EINVAL;
    }
    for (int i = 0; i < n_times; ++i) {
        if (!(times[i] >= 0.0) || !std::isfinite(times[i]) || (i > 0 && times[i] < times[i - 1])) {
            set_error("kry_evolve: times must be finite, non-negative and non-decreasing");
            return KRY_EINVAL;
        }
    }
    return KRY_OK;
}

}  // namespace

extern "C" int kry_hamiltonian_destroy(kry_ham H)
{
    if (!H) return KRY_OK;
    drop_graph(H);
    if (H->ws && !H->ws_user) cudaFree(H->ws);
    if (H->d_eh) cudaFree(H->d_eh);
    if (H->h_poll) cudaFreeHost(H->h_poll);
    if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
    if (H->cap_stream2) cudaStreamDestroy(H->cap_stream2);
    delete H;
    return KRY_OK;
}

extern "C" int kry_profile_enable(kry_ham H, int on)
{
    if (!H) { set_error("kry_profile_enable: H is NULL"); return KRY_EINVAL; }
    if (on < 0 || on > 2) { set_error("kry_profile_enable: on must be 0, 1 or 2"); return KRY_EINVAL; }
    H->prof_on = on == 1 ? 1 : 0;
    H->plain_graph = on == 2 ? 1 : 0;
    for (int q = 0; q < NKIND; ++q) { H->prof_ms[q] = 0.0; H->prof_bytes[q] = 0.0; H->prof_launches[q] = 0; }
    return KRY_OK;
}

extern "C" int kry_set_second_pass_node(kry_ham H, int on)
{
    if (!H || on < 0 || on > 1) { set_error("kry_set_second_pass_node: bad arguments (on = 0 or 1)"); return KRY_EINVAL; }
    H->cond_pass_c = on;
    return KRY_OK;
}

extern "C" int kry_profile_read(kry_ham H, double *ms, double *bytes, int64_t *launches)
{
    if (!H || !ms || !bytes || !launches) { set_error("kry_profile_read: bad arguments"); return KRY_EINVAL; }
    for (int q = 0; q < NKIND; ++q) { ms[q] = H->prof_ms[q]; bytes[q] = H->prof_bytes[q]; launches[q] = H->prof_launches[q]; }
    return KRY_OK;
}

extern "C" int64_t kry_workspace_bytes(kry_ham H, int dtype, int m, int n_times)
{
    if (!H || m < 1 || m > MMAX || n_times < 1 || !dtype_ok(dtype)) return -1;
    if (H->K > 1) {
        int gridB = 0;
        const int grid = grid_for_b(H, dtype, &gridB);
        if (grid <= 0) return -1;
        return (int64_t)layout_b(H, dtype, m, std::max(grid, gridB), n_times).bytes;
    }
    int gridH = 0, gridB = 0;
    const int grid = grid_for(H, dtype, &gridH, &gridB);
    if (grid <= 0) return -1;
    return (int64_t)layout(H, dtype, m, std::max(grid, std::max(gridH, gridB)), n_times).bytes;
}

extern "C" int64_t kry_workspace_size(kry_ham H, int dtype, int m)
{
    return kry_workspace_bytes(H, dtype, m, 1);
}

extern "C" int kry_set_workspace(kry_ham H, void *d_ws, int64_t bytes)
{
    if (!H || (d_ws && bytes <= 0) || ((uintptr_t)d_ws & 255u)) {
        set_error("kry_set_workspace: bad arguments (need H, and a 256-byte aligned buffer with bytes > 0)");
        return KRY_EINVAL;
    }
    drop_graph(H);
    if (H->ws && !H->ws_user) cudaFree(H->ws);
    H->ws = d_ws;
    H->ws_bytes = d_ws ? (size_t)bytes : 0;
    H->ws_user = d_ws ? 1 : 0;
    return KRY_OK;
}

extern "C" int kry_apply(kry_ham H, int dtype, const void *d_x, void *d_y, void *stream)
{
    if (!H || !d_x || !d_y || d_x == d_y || (dtype != KRY_C128 && dtype != KRY_C64)) {
        set_error("kry_apply: bad arguments");
        return KRY_EINVAL;
    }
    const DevBasis &b = H->b->dev;
    if (H->K > 1)
        return launch_apply_b(b, H->dev, dtype == KRY_C64, H->K, d_x, d_y, rl_in_smem(b), (cudaStream_t)stream);
    return launch_apply(b, H->dev, dtype == KRY_C64, d_x, d_y, rl_in_smem(b), (cudaStream_t)stream);
}

extern "C" int kry_evolve(kry_ham H, int dtype, const void *d_psi0, const double *times, int n_times,
                          int m, double tol, void *d_psi_out, double *P_out, kry_stats *stats,
                          void *stream)
{
    if (int rc = check_evolve_args(H, dtype, times, n_times, m, tol, P_out)) return rc;
    if (!d_psi0) { set_error("kry_evolve: d_psi0 is NULL"); return KRY_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == KRY_C128E)
        return H->K > 1
                   ? evolve_bt<ffc>(H, dtype, d_psi0, 0, true, times, n_times, m, tol, d_psi_out, P_out, stats, s)
                   : evolve_t<ffc>(H, dtype, d_psi0, 0, true, times, n_times, m, tol, d_psi_out, P_out, stats, s);
    if (dtype == KRY_C64)
        return H->K > 1
                   ? evolve_bt<float2>(H, dtype, d_psi0, 0, true, times, n_times, m, tol, d_psi_out, P_out, stats, s)
                   : evolve_t<float2>(H, dtype, d_psi0, 0, true, times, n_times, m, tol, d_psi_out, P_out, stats, s);
    return H->K > 1
               ? evolve_bt<double2>(H, dtype, d_psi0, 0, true, times, n_times, m, tol, d_psi_out, P_out, stats, s)
               : evolve_t<double2>(H, dtype, d_psi0, 0, true, times, n_times, m, tol, d_psi_out, P_out, stats, s);
}

extern "C" int kry_return_probability(kry_ham H, int dtype, uint64_t psi0_state, const double *times,
                                      int n_times, int m, double tol, double *P_out, kry_stats *stats,
                                      void *stream)
{
    if (int rc = check_evolve_args(H, dtype, times, n_times, m, tol, P_out)) return rc;
    const int L = H->b->L;
    if ((L < 64 && (psi0_state >> L) != 0ull) || __builtin_popcountll(psi0_state) != H->b->N) {
        set_error("kry_return_probability: state is not in the (L=%d, N=%d) sector", L, H->b->N);
        return KRY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == KRY_C128E)
        return H->K > 1
                   ? evolve_bt<ffc>(H, dtype, nullptr, psi0_state, false, times, n_times, m, tol, nullptr, P_out, stats, s)
                   : evolve_t<ffc>(H, dtype, nullptr, psi0_state, false, times, n_times, m, tol, nullptr, P_out, stats, s);
    if (dtype == KRY_C64)
        return H->K > 1
                   ? evolve_bt<float2>(H, dtype, nullptr, psi0_state, false, times, n_times, m, tol, nullptr, P_out, stats, s)
                   : evolve_t<float2>(H, dtype, nullptr, psi0_state, false, times, n_times, m, tol, nullptr, P_out, stats, s);
    return H->K > 1
               ? evolve_bt<double2>(H, dtype, nullptr, psi0_state, false, times, n_times, m, tol, nullptr, P_out, stats, s)
               : evolve_t<double2>(H, dtype, nullptr, psi0_state, false, times, n_times, m, tol, nullptr, P_out, stats, s);
}

// Temporal autocorrelation (Sec. 4): C(t) = (1/t) int_0^t P(t') dt' at the output times,
// from the same evolution as P (the small exponential integrates P over each step of the
// dense output by Gauss-Legendre quadrature).  Single realisation (K = 1).
namespace {

// Basis-state initial vectors with an optional temporal autocorrelation: states[k] (or the one
// state) for realisation k; the single path for K = 1, the batched path otherwise.
int evolve_states(kry_ham H, int dtype, const uint64_t *states, const double *times, int n_times, int m,
                  double tol, double *P_out, double *C_out, kry_stats *stats, void *stream, const char *who)
{
    if (int rc = check_evolve_args(H, dtype, times, n_times, m, tol, P_out)) return rc;
    if (!states) { set_error("%s: no initial states", who); return KRY_EINVAL; }
    const int L = H->b->L;
    for (int k = 0; k < H->K; ++k) {
        if ((L < 64 && (states[k] >> L) != 0ull) || __builtin_popcountll(states[k]) != H->b->N) {
            set_error("%s: state of realisation %d is not in the (L=%d, N=%d) sector", who, k, L, H->b->N);
            return KRY_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (H->K > 1)
        return dtype == KRY_C64
                   ? evolve_bt<float2>(H, dtype, nullptr, 0, false, times, n_times, m, tol, nullptr, P_out, stats, s,
                                       states, C_out)
               : dtype == KRY_C128E
                   ? evolve_bt<ffc>(H, dtype, nullptr, 0, false, times, n_times, m, tol, nullptr, P_out, stats, s,
                                    states, C_out)
                   : evolve_bt<double2>(H, dtype, nullptr, 0, false, times, n_times, m, tol, nullptr, P_out, stats, s,
                                        states, C_out);
    EvOpts opt;
    opt.C_out = C_out;
    if (dtype == KRY_C128E)
        return evolve_t<ffc>(H, dtype, nullptr, states[0], false, times, n_times, m, tol, nullptr, P_out, stats, s,
                             &opt);
    return dtype == KRY_C64
               ? evolve_t<float2>(H, dtype, nullptr, states[0], false, times, n_times, m, tol, nullptr, P_out, stats,
                                  s, &opt)
               : evolve_t<double2>(H, dtype, nullptr, states[0], false, times, n_times, m, tol, nullptr, P_out, stats,
                                   s, &opt);
}

}  // namespace

extern "C" int kry_autocorrelation(kry_ham H, int dtype, uint64_t psi0_state, const double *times, int n_times,
                                   int m, double tol, double *C_out, double *P_out, kry_stats *stats,
                                   void *stream)
{
    if (!C_out) { set_error("kry_autocorrelation: C_out is NULL"); return KRY_EINVAL; }
    if (!H) { set_error("kry_autocorrelation: H is NULL"); return KRY_EINVAL; }
    std::vector<uint64_t> st((size_t)std::max(H->K, 1), psi0_state);
    return evolve_states(H, dtype, st.data(), times, n_times, m, tol, P_out, C_out, stats, stream,
                         "kry_autocorrelation");
}

// Ensembles of basis-state initial vectors (Sec. 2 disorder layers; Sec. 4): realisation k
// starts from psi0_states[k]; P and, when C_out is given, C for every realisation.
extern "C" int kry_return_probability_states(kry_ham H, int dtype, const uint64_t *psi0_states,
                                             const double *times, int n_times, int m, double tol, double *P_out,
                                             double *C_out, kry_stats *stats, void *stream)
{
    return evolve_states(H, dtype, psi0_states, times, n_times, m, tol, P_out, C_out, stats, stream,
                         "kry_return_probability_states");
}


// ---------------------------------------------------------------- adjoint gradient
//
// A(t) = <psi0| exp(-iHt) |psi0>, P = |A|^2 (Eq. SP).  For a parameter theta of H,
//     dA/dtheta = -i int_0^t <lambda(s)| dH/dtheta |psi(s)> ds,
//     psi(s) = exp(-iHs) psi0,   lambda(s) = exp(+iH(t - s)) psi0   (the costate),
//     dP/dtheta = 2 Re(conj(A) dA/dtheta),
// with dH/dh_i = Sz_i and dH/dDelta = J sum_b Sz Sz (both diagonal).  The costate is
// evolved backward from lambda(t) = psi0 with the same Krylov kernels, as a forward
// evolution under -H in u = t - s.  psi is checkpointed after every `ckpt_every`-th Krylov
// step of the forward sweep; the backward sweep visits the checkpoint intervals from the
// last to the first, recomputes psi from the interval's checkpoint at the quadrature nodes
// inside it, advances the costate through the same interval, and accumulates the
// integrand.  The integral uses composite 16-point Gauss-Legendre rules on segments short
// enough that (spectral width bound) x (segment length) <= 20.

namespace {

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    // Newton iteration on the Legendre polynomial P_n from cosine initial guesses
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), p1 = 0.0, p0 = 0.0, dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            p0 = 1.0;
            p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

void add_stats(kry_stats &a, const kry_stats &b)
{
    a.n_hv += b.n_hv;
    a.n_krylov_steps += b.n_krylov_steps;
    a.n_second_pass += b.n_second_pass;
    a.n_breakdowns += b.n_breakdowns;
    a.err_estimate += b.err_estimate;
    a.max_orth_loss = std::max(a.max_orth_loss, b.max_orth_loss);
    a.time_ms += b.time_ms;
    a.algo_bytes += b.algo_bytes;
    a.n_launches += b.n_launches;
    a.n_second_dots += b.n_second_dots;
}

}  // namespace

extern "C" int kry_grad(kry_ham H, uint64_t psi0_state, double t, int m, double tol, int ckpt_every,
                        double *P, double *dP_dh, double *dP_dDelta, kry_stats *stats, void *stream)
{
    if (!H || !P || !dP_dh || !dP_dDelta || !(t >= 0.0) || !std::isfinite(t) || m < 1 || m > MMAX ||
        !(tol > 0.0) || ckpt_every < 1) {
        set_error("kry_grad: bad arguments (need H, outputs, t >= 0, 1 <= m <= %d, tol > 0, ckpt_every >= 1)", MMAX);
        return KRY_EINVAL;
    }
    if (H->K != 1) { set_error("kry_grad: one realisation (K = 1) only"); return KRY_EINVAL; }
    const int L = H->b->L;
    if ((L < 64 && (psi0_state >> L) != 0ull) || __builtin_popcountll(psi0_state) != H->b->N) {
        set_error("kry_grad: state is not in the (L=%d, N=%d) sector", L, H->b->N);
        return KRY_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const DevBasis &b = H->b->dev;
    const size_t D = b.D, ldv = round_up(D, 64), vb = ldv * sizeof(double2);
    uint64_t r0 = 0;
    {
        int j = 0;
        for (int p = 0; p < L; ++p)
            if ((psi0_state >> p) & 1ull) r0 += binom_host(p, ++j);
    }
    kry_stats tot{};
    if (t == 0.0) {
        *P = 1.0;
        for (int i = 0; i < L; ++i) dP_dh[i] = 0.0;
        *dP_dDelta = 0.0;
        if (stats) *stats = tot;
        return KRY_OK;
    }
    // quadrature nodes over [0, t]
    double hsum = 0.0;
    for (int i = 0; i < L; ++i) hsum += std::fabs(H->h[i]);
    const int nb = H->dev.nbonds;
    const double wbound = 2.0 * (0.5 * std::fabs(H->J) * nb + 0.25 * std::fabs(H->J * H->Delta) * nb + 0.5 * hsum);
    const int nseg = std::max(1, (int)std::ceil(wbound * t / 20.0));
    std::vector<double> gx, gw, sq, wq;
    gauss_legendre(16, gx, gw);
    for (int sgi = 0; sgi < nseg; ++sgi) {
        const double a0 = t * sgi / nseg, a1 = t * (sgi + 1) / nseg, hh = 0.5 * (a1 - a0);
        for (int i = 0; i < 16; ++i) {
            sq.push_back(a0 + hh * (gx[i] + 1.0));
            wq.push_back(hh * gw[i]);
        }
    }
    // device buffers
    DevBuf bpsi0, bpsit, bck, bckt, blamA, blamB, bw, bacc, bpart;
    KRY_CU(cudaMalloc(&bpsi0.p, vb));
    KRY_CU(cudaMalloc(&bpsit.p, vb));
    KRY_CU(cudaMalloc(&blamA.p, vb));
    KRY_CU(cudaMalloc(&blamB.p, vb));
    KRY_CU(cudaMalloc(&bw.p, sizeof(double) * wq.size()));
    constexpr int NACC = 66;   // L <= 64 sites and Delta
    KRY_CU(cudaMalloc(&bacc.p, sizeof(double2) * NACC + 64));
    const int ggrid = (int)std::min<size_t>((D + TILE - 1) / TILE, 152 * 2);
    KRY_CU(cudaMalloc(&bpart.p, sizeof(double2) * PSTRIDE * (size_t)ggrid));
    double2 *acc = (double2 *)bacc.p;
    unsigned *counter = (unsigned *)(acc + NACC);
    KRY_CU(cudaMemsetAsync(bacc.p, 0, sizeof(double2) * NACC + 64, s));
    KRY_CU(cudaMemcpyAsync(bw.p, wq.data(), sizeof(double) * wq.size(), cudaMemcpyHostToDevice, s));
    KRY_CU(cudaMemsetAsync(bpsi0.p, 0, vb, s));
    if (int rc = launch_set_basis_state(bpsi0.p, 0, (uint32_t)r0, s)) return rc;
    // 1. forward sweep with checkpoints.  The buffer starts with room for a few checkpoints;
    // if the sweep takes more Krylov steps than that covers, it is grown to the number the
    // sweep needs and the sweep is repeated (the step sequence does not depend on it).
    EvOpts fo;
    fo.ldC = ldv;
    fo.ckpt_every = ckpt_every;
    double Pt = 0.0;
    kry_stats st{};
    for (int cap = 8;;) {
        if (bck.p) { cudaFree(bck.p); bck.p = nullptr; }
        if (bckt.p) { cudaFree(bckt.p); bckt.p = nullptr; }
        cudaError_t e = cudaMalloc(&bck.p, (size_t)cap * vb);
        if (e != cudaSuccess) {
            bck.p = nullptr;
            cudaGetLastError();
            set_error("kry_grad: %d checkpoints of %zu bytes do not fit in device memory; use a larger "
                      "ckpt_every", cap, vb);
            return KRY_ENOMEM;
        }
        KRY_CU(cudaMalloc(&bckt.p, sizeof(double) * cap));
        fo.ckpt = bck.p;
        fo.d_ckpt_t = (double *)bckt.p;
        fo.ckpt_cap = cap;
        if (int rc = evolve_t<double2>(H, KRY_C128, nullptr, psi0_state, false, &t, 1, m, tol, bpsit.p, &Pt, &st, s,
                                       &fo))
            return rc;
        add_stats(tot, st);
        const long long need = st.n_krylov_steps / ckpt_every;
        if (need <= cap) break;
        cap = (int)std::min<long long>(need, 1 << 20);
    }
    double2 A;
    KRY_CU(cudaMemcpyAsync(&A, (double2 *)bpsit.p + r0, sizeof(double2), cudaMemcpyDeviceToHost, s));
    KRY_CU(cudaStreamSynchronize(s));
    *P = A.x * A.x + A.y * A.y;
    const int C = fo.n_ckpt;
    std::vector<double> T(C + 2);
    T[0] = 0.0;
    for (int c = 0; c < C; ++c) T[c + 1] = fo.ckpt_t[c];
    T[C + 1] = t;
    // node ranges per interval and the largest one
    std::vector<int> qa(C + 1), qb(C + 1);
    int nmax = 1;
    for (int c = 0; c <= C; ++c) {
        int a = 0;
        while (a < (int)sq.size() && sq[a] < T[c]) ++a;
        int e = a;
        while (e < (int)sq.size() && (sq[e] < T[c + 1] || (c == C && sq[e] <= t))) ++e;
        qa[c] = a;
        qb[c] = e;
        nmax = std::max(nmax, e - a + 1);
    }
    DevBuf bP, bL;
    KRY_CU(cudaMalloc(&bP.p, (size_t)nmax * vb));
    KRY_CU(cudaMalloc(&bL.p, (size_t)nmax * vb));
    // 2. costate Hamiltonian -H (J -> -J at fixed Delta flips both bond terms; h -> -h)
    std::vector<double> hneg(L);
    for (int i = 0; i < L; ++i) hneg[i] = -H->h[i];
    kry_ham Hn = nullptr;
    if (int rc = kry_hamiltonian_set(H->b, -H->J, H->Delta, hneg.data(), 1, H->boundary, &Hn)) return rc;
    struct HamGuard { kry_ham h; ~HamGuard() { kry_hamiltonian_destroy(h); } } guard{Hn};
    KRY_CU(cudaMemcpyAsync(blamA.p, bpsi0.p, vb, cudaMemcpyDeviceToDevice, s));
    std::vector<double> tim, Pd(nmax + 1);
    for (int c = C; c >= 0; --c) {
        const int n = qb[c] - qa[c];
        const double Ta = T[c], Tb = T[c + 1];
        const void *start = (c == 0) ? bpsi0.p : (const void *)((char *)bck.p + (size_t)(c - 1) * vb);
        if (n > 0) {
            // 3a. psi at the nodes of the interval, recomputed from its checkpoint
            tim.clear();
            for (int q = qa[c]; q < qb[c]; ++q) tim.push_back(std::max(0.0, sq[q] - Ta));
            EvOpts po;
            po.vec_out = bP.p;
            po.ldOut = ldv;
            if (int rc = evolve_t<double2>(H, KRY_C128, start, 0, true, tim.data(), n, m, tol, nullptr, Pd.data(), &st, s, &po))
                return rc;
            add_stats(tot, st);
        }
        // 3b. costate through the same interval: u from t - Tb to t - Ta, outputs at u = t - s_q
        tim.clear();
        for (int q = qb[c] - 1; q >= qa[c]; --q) tim.push_back(std::max(0.0, (t - sq[q]) - (t - Tb)));
        tim.push_back(Tb - Ta);
        EvOpts lo;
        lo.vec_out = bL.p;
        lo.ldOut = ldv;
        if (int rc = evolve_t<double2>(Hn, KRY_C128, blamA.p, 0, true, tim.data(), (int)tim.size(), m, tol, blamB.p, Pd.data(), &st, s, &lo))
            return rc;
        add_stats(tot, st);
        std::swap(blamA.p, blamB.p);
        // 3c. integrand at the interval's nodes
        if (n > 0) {
            if (int rc = launch_grad_acc(b, H->dev, H->J, (const double2 *)bP.p, (const double2 *)bL.p, ldv,
                                         (const double *)bw.p + qa[c], n, (double2 *)bpart.p, acc, counter, ggrid, s))
                return rc;
        }
    }
    std::vector<double2> hacc(L + 1);
    KRY_CU(cudaMemcpyAsync(hacc.data(), acc, sizeof(double2) * (L + 1), cudaMemcpyDeviceToHost, s));
    KRY_CU(cudaStreamSynchronize(s));
    // dA = -i acc; dP = 2 Re(conj(A) dA) = 2 (A.x acc.y - A.y acc.x)
    for (int i = 0; i <= L; ++i) {
        const double dA_re = hacc[i].y, dA_im = -hacc[i].x;
        const double dp = 2.0 * (A.x * dA_re + A.y * dA_im);
        if (i < L) dP_dh[i] = dp;
        else *dP_dDelta = dp;
    }
    if (stats) *stats = tot;
    return KRY_OK;
}
