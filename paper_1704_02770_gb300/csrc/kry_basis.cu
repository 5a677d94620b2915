// Sector basis without a stored list: combinadic rank/unrank tables (Sec. 2 "Basis
// representation"; Algorithm 2 defines the sorted order that the ranks reproduce), and
// the Hamiltonian handle (Eq. 1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kry_internal.cuh"

namespace kry {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

int cuda_fail(cudaError_t e, const char *what)
{
    set_error("CUDA error in %s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? KRY_ENOMEM : KRY_ECUDA;
}

static uint64_t binom64(int n, int k)
{
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
    return r;
}

// ---------------------------------------------------------------- rank / unrank kernels

__device__ __forceinline__ uint32_t find_block(const DevBasis &b, uint32_t r)
{
    // largest hi with blk[hi] <= r (upper bound - 1); blk is non-decreasing
    uint32_t lo = 0, cnt = 1u << b.Lhi;
    while (cnt > 0) {
        uint32_t step = cnt >> 1;
        if (__ldg(b.blk + lo + step) <= r) { lo += step + 1; cnt -= step + 1; }
        else cnt = step;
    }
    return lo - 1;
}

__global__ void k_rank(DevBasis b, const uint64_t *__restrict__ st, uint32_t *__restrict__ rk,
                       int64_t n)
{
    const uint64_t lomask = (1ull << b.Llo) - 1ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t s = st[i];
        if ((s >> b.L) != 0ull || __popcll(s) != b.N) {
            rk[i] = 0xFFFFFFFFu;
            atomicOr(b.err, 1);
            continue;
        }
        rk[i] = __ldg(b.blk + (uint32_t)(s >> b.Llo)) + __ldg(b.ranklo + (uint32_t)(s & lomask));
    }
}

__global__ void k_unrank(DevBasis b, const uint32_t *__restrict__ rk, uint64_t *__restrict__ st,
                         int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t r = rk[i];
        if (r >= b.D) {
            st[i] = 0ull;
            atomicOr(b.err, 2);
            continue;
        }
        uint32_t hi = find_block(b, r);
        int klo = b.N - __popc(hi);
        uint32_t off = r - __ldg(b.blk + hi);
        uint32_t lo = __ldg(b.lolist + __ldg(b.koff + klo) + off);
        st[i] = ((uint64_t)hi << b.Llo) | (uint64_t)lo;
    }
}

}  // namespace kry

using namespace kry;

extern "C" const char *kry_last_error(void) { return g_err.c_str(); }

// C(n, k) saturated at 2^63 (exact below it)
static uint64_t binom_sat(int n, int k)
{
    if (k < 0 || k > n) return 0;
    if (k > n - k) k = n - k;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i) {
        r = r * (unsigned)(n - k + i) / (unsigned)i;
        if (r >= ((unsigned __int128)1 << 63)) return 1ull << 63;
    }
    return (uint64_t)r;
}

// Sorted-list basis of Alg. 2 (states on the device, combinadic ranks): 1 <= L <= 64.
extern "C" int kry_basis_create_list(int L, int n_up, kry_basis *out)
{
    if (!out) { set_error("kry_basis_create_list: out is NULL"); return KRY_EINVAL; }
    *out = nullptr;
    if (L < 1 || L > 64 || n_up < 0 || n_up > L) {
        set_error("kry_basis_create_list: need 1 <= L <= 64 and 0 <= n_up <= L (got L=%d, n_up=%d)", L, n_up);
        return KRY_EINVAL;
    }
    const uint64_t D = binom_sat(L, n_up);
    if (D > 0x7FFFFFFFull) {
        set_error("kry_basis_create_list: sector dimension C(%d, %d) exceeds 2^31 - 1", L, n_up);
        return KRY_EINVAL;
    }
    const int N1 = n_up + 1;
    std::vector<uint32_t> cb((size_t)L * N1);
    for (int p = 0; p < L; ++p)
        for (int k = 0; k <= n_up; ++k) cb[(size_t)p * N1 + k] = (uint32_t)std::min<uint64_t>(binom_sat(p, k), 0xFFFFFFFFull);
    const size_t o_st = 0, o_cb = (8 * (size_t)D + 255) & ~(size_t)255;
    const size_t o_er = (o_cb + sizeof(uint32_t) * cb.size() + 15) & ~(size_t)15, bytes = o_er + 16;
    kry_basis b = new (std::nothrow) kry_basis_s();
    if (!b) { set_error("kry_basis_create_list: host allocation failed"); return KRY_ENOMEM; }
    b->L = L; b->N = n_up; b->Llo = 0; b->Lhi = 0; b->D = (int64_t)D;
    cudaGetDevice(&b->device);
    cudaError_t e = cudaMalloc(&b->d_tab, bytes);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaMalloc(basis list)"); }
    char *base = (char *)b->d_tab;
    DevBasis &d = b->dev;
    d = DevBasis{};
    d.list = 1;
    d.states = (const uint64_t *)(base + o_st);
    d.cbin = (const uint32_t *)(base + o_cb);
    d.err = (int *)(base + o_er);
    d.L = L; d.N = n_up; d.Llo = 0; d.Lhi = 0; d.D = (uint32_t)D;
    e = cudaMemcpy(base + o_cb, cb.data(), sizeof(uint32_t) * cb.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(base + o_er, 0, 16);
    int rc = (e == cudaSuccess) ? list_build(d, 0) : KRY_OK;
    if (e == cudaSuccess && rc == KRY_OK) e = cudaDeviceSynchronize();
    if (e != cudaSuccess || rc != KRY_OK) {
        cudaFree(b->d_tab);
        delete b;
        return e != cudaSuccess ? cuda_fail(e, "basis list build") : rc;
    }
    *out = b;
    return KRY_OK;
}

extern "C" int kry_basis_create(int L, int n_up, kry_basis *out)
{
    if (!out) { set_error("kry_basis_create: out is NULL"); return KRY_EINVAL; }
    *out = nullptr;
    if (L > 32 && L <= 64) return kry_basis_create_list(L, n_up, out);
    if (L < 1 || L > 64 || n_up < 0 || n_up > L) {
        set_error("kry_basis_create: need 1 <= L <= 64 and 0 <= n_up <= L (got L=%d, n_up=%d)",
                  L, n_up);
        return KRY_EINVAL;
    }
    const int Llo = (L + 1) / 2, Lhi = L - Llo;
    const uint64_t D = binom64(L, n_up);
    const uint32_t nlo = 1u << Llo, nhi = 1u << Lhi;
    // host tables
    std::vector<uint32_t> blk(nhi), koff(Llo + 2), bsz(Llo + 1);
    std::vector<uint16_t> ranklo(nlo), lolist(nlo);
    koff[0] = 0;
    for (int k = 0; k <= Llo; ++k) {
        bsz[k] = (uint32_t)binom64(Llo, k);
        koff[k + 1] = koff[k] + bsz[k];
    }
    {
        std::vector<uint32_t> fill(koff.begin(), koff.end() - 1);
        for (uint32_t lo = 0; lo < nlo; ++lo) {
            int k = __builtin_popcount(lo);
            uint32_t r = 0;
            int j = 0;
            for (int p = 0; p < Llo; ++p)
                if ((lo >> p) & 1u) r += (uint32_t)binom64(p, ++j);
            ranklo[lo] = (uint16_t)r;
            if (fill[k] - koff[k] != r) {
                set_error("kry_basis_create: internal table mismatch (lo=%u)", lo);
                return KRY_EINVAL;
            }
            lolist[fill[k]++] = (uint16_t)lo;
        }
    }
    // block starts: valid blocks in increasing hi are contiguous in rank order
    const uint32_t INV = 0xFFFFFFFFu;
    uint64_t expect = 0;
    for (uint32_t hi = 0; hi < nhi; ++hi) {
        int khi = __builtin_popcount(hi), klo = n_up - khi;
        if (klo < 0 || klo > Llo) { blk[hi] = INV; continue; }
        uint64_t v = 0;
        int j = 0;
        for (int q = 0; q < Lhi; ++q)
            if ((hi >> q) & 1u) { ++j; v += binom64(Llo + q, klo + j); }
        if (v != expect) {
            set_error("kry_basis_create: internal block order mismatch (hi=%u)", hi);
            return KRY_EINVAL;
        }
        blk[hi] = (uint32_t)v;
        expect = v + bsz[klo];
    }
    if (expect != D) {
        set_error("kry_basis_create: internal dimension mismatch");
        return KRY_EINVAL;
    }
    uint32_t next = (uint32_t)D;
    for (int64_t hi = (int64_t)nhi - 1; hi >= 0; --hi) {
        if (blk[hi] == INV) blk[hi] = next;
        else next = blk[hi];
    }
    // block of the first rank of every tile: the largest hi with blk[hi] <= t * TILE
    const uint64_t ntiles = (D + TILE - 1) / TILE;
    std::vector<uint32_t> tstart(ntiles > 0 ? ntiles : 1, 0);
    {
        uint32_t hi = 0;
        for (uint64_t t = 0; t < ntiles; ++t) {
            const uint64_t r = t * TILE;
            while (hi + 1 < nhi && blk[hi + 1] <= r) ++hi;
            tstart[t] = hi;
        }
    }
    // device upload: one allocation holding every table and the error flag
    size_t o_blk = 0, o_rl = o_blk + sizeof(uint32_t) * nhi;
    size_t o_ll = o_rl + sizeof(uint16_t) * nlo;
    size_t o_ko = (o_ll + sizeof(uint16_t) * nlo + 15) & ~(size_t)15;
    size_t o_bs = o_ko + sizeof(uint32_t) * (Llo + 2);
    size_t o_er = (o_bs + sizeof(uint32_t) * (Llo + 1) + 15) & ~(size_t)15;
    size_t o_ts = o_er + 16;
    size_t bytes = o_ts + sizeof(uint32_t) * tstart.size();
    kry_basis b = new (std::nothrow) kry_basis_s();
    if (!b) { set_error("kry_basis_create: host allocation failed"); return KRY_ENOMEM; }
    b->L = L; b->N = n_up; b->Llo = Llo; b->Lhi = Lhi; b->D = (int64_t)D;
    cudaGetDevice(&b->device);
    cudaError_t e = cudaMalloc(&b->d_tab, bytes);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaMalloc(tables)"); }
    char *base = (char *)b->d_tab;
    const struct { size_t off; const void *src; size_t n; } up[] = {
        {o_blk, blk.data(), sizeof(uint32_t) * nhi},
        {o_rl, ranklo.data(), sizeof(uint16_t) * nlo},
        {o_ll, lolist.data(), sizeof(uint16_t) * nlo},
        {o_ko, koff.data(), sizeof(uint32_t) * (Llo + 2)},
        {o_bs, bsz.data(), sizeof(uint32_t) * (Llo + 1)},
        {o_ts, tstart.data(), sizeof(uint32_t) * tstart.size()},
    };
    for (const auto &u : up)
        if (e == cudaSuccess) e = cudaMemcpy(base + u.off, u.src, u.n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(base + o_er, 0, 16);
    if (e != cudaSuccess) { cudaFree(b->d_tab); delete b; return cuda_fail(e, "table upload"); }
    DevBasis &d = b->dev;
    d.blk = (const uint32_t *)(base + o_blk);
    d.tstart = (const uint32_t *)(base + o_ts);
    d.ranklo = (const uint16_t *)(base + o_rl);
    d.lolist = (const uint16_t *)(base + o_ll);
    d.koff = (const uint32_t *)(base + o_ko);
    d.bsz = (const uint32_t *)(base + o_bs);
    d.err = (int *)(base + o_er);
    d.L = L; d.N = n_up; d.Llo = Llo; d.Lhi = Lhi; d.D = (uint32_t)D;
    *out = b;
    return KRY_OK;
}

extern "C" int kry_basis_destroy(kry_basis b)
{
    if (!b) return KRY_OK;
    cudaFree(b->d_tab);
    delete b;
    return KRY_OK;
}

extern "C" int64_t kry_basis_dim(kry_basis b) { return b ? b->D : -1; }

static int rank_common(kry_basis b, int64_t n, const void *in, void *out, void *stream,
                       bool unrank)
{
    if (!b || n < 0 || (n > 0 && (!in || !out))) {
        set_error("kry_basis_%s: bad arguments", unrank ? "unrank" : "rank");
        return KRY_EINVAL;
    }
    if (n == 0) return KRY_OK;
    cudaStream_t s = (cudaStream_t)stream;
    KRY_CU(cudaMemsetAsync(b->dev.err, 0, sizeof(int), s));
    int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    if (b->dev.list) {
        const int rc = unrank ? launch_list_unrank(b->dev, (const uint32_t *)in, (uint64_t *)out, n, s)
                              : launch_list_rank(b->dev, (const uint64_t *)in, (uint32_t *)out, n, s);
        if (rc) return rc;
    } else if (unrank) {
        k_unrank<<<grid, 256, 0, s>>>(b->dev, (const uint32_t *)in, (uint64_t *)out, n);
    } else {
        k_rank<<<grid, 256, 0, s>>>(b->dev, (const uint64_t *)in, (uint32_t *)out, n);
    }
    KRY_CU(cudaGetLastError());
    int flag = 0;
    KRY_CU(cudaMemcpyAsync(&flag, b->dev.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KRY_CU(cudaStreamSynchronize(s));
    if (flag) {
        set_error(unrank ? "kry_basis_unrank: rank >= D" :
                           "kry_basis_rank: state outside the sector (bits >= L or wrong N)");
        return KRY_EINVAL;
    }
    return KRY_OK;
}

extern "C" int kry_basis_rank(kry_basis b, const uint64_t *d_states, uint32_t *d_ranks,
                              int64_t n, void *stream)
{
    return rank_common(b, n, d_states, d_ranks, stream, false);
}

extern "C" int kry_basis_unrank(kry_basis b, const uint32_t *d_ranks, uint64_t *d_states,
                                int64_t n, void *stream)
{
    return rank_common(b, n, d_ranks, d_states, stream, true);
}

// ---------------------------------------------------------------- Hamiltonian handle

// s_k = tr(H_k) / D, the mean diagonal of the sector: every bond is antiparallel in a fraction
// 2N(L-N)/(L(L-1)) of the states and every site occupied in a fraction N/L.
static double mean_diagonal(int L, int N, double J, double Delta, const double *hk, int nbonds)
{
    const double panti = (L >= 2) ? 2.0 * N * (double)(L - N) / ((double)L * (L - 1)) : 0.0;
    double e = 0.25 * J * Delta * (nbonds - 2.0 * nbonds * panti);
    for (int i = 0; i < L; ++i) e += hk[i] * ((double)N / L - 0.5);
    return e;
}

// Sorted-list basis: field energy by bytes of the state, realisation fastest,
//   sum_i h_{k,i} (n_i - 1/2) = sum_c eh8[(c * 256 + byte_c) * K + k]   (-sum_i h_{k,i}/2 in c = 0).
static void fill_dev_ham(DevHam &d, double J, double Delta, int L, int K, int boundary)
{
    d.cz = 0.25 * J * Delta;
    d.halfJ = 0.5 * J;
    d.pbc = (boundary == KRY_PBC && L >= 3) ? 1 : 0;
    d.nbonds = d.pbc ? L : (L - 1);
    d.K = K;
}

static int ham_set_list(kry_basis b, double J, double Delta, const double *h, int K, int boundary, kry_ham *out)
{
    const int L = b->L, nc = (L + 7) / 8;
    const size_t n8 = (size_t)nc * 256 * K;
    std::vector<double> eh(n8);
    std::vector<float> ehf(n8);
    for (int k = 0; k < K; ++k) {
        const double *hk = h + (size_t)k * L;
        double hsum = 0.0;
        for (int i = 0; i < L; ++i) hsum += hk[i];
        for (int c = 0; c < nc; ++c)
            for (int v = 0; v < 256; ++v) {
                double e = (c == 0) ? -0.5 * hsum : 0.0;
                for (int q = 0; q < 8 && 8 * c + q < L; ++q) if ((v >> q) & 1) e += hk[8 * c + q];
                eh[((size_t)c * 256 + v) * K + k] = e;
            }
    }
    for (size_t i = 0; i < n8; ++i) ehf[i] = (float)eh[i];
    kry_ham H = new (std::nothrow) kry_ham_s();
    if (!H) { set_error("kry_hamiltonian_set: host allocation failed"); return KRY_ENOMEM; }
    default_shape(H, b->dev.list ? 0 : b->Llo);
    fill_dev_ham(H->dev, J, Delta, L, K, boundary);
    // shifted copy for the Lanczos pass: s_k taken off the byte-0 entries
    H->shift.resize(K);
    std::vector<double> ehs(eh);
    for (int k = 0; k < K; ++k) {
        H->shift[k] = mean_diagonal(L, b->N, J, Delta, h + (size_t)k * L, H->dev.nbonds);
        for (int v = 0; v < 256; ++v) ehs[(size_t)v * K + k] -= H->shift[k];
    }
    std::vector<float> ehsf(n8);
    for (size_t i = 0; i < n8; ++i) ehsf[i] = (float)ehs[i];
    cudaError_t e = cudaMalloc(&H->d_eh, 24 * n8);
    if (e != cudaSuccess) { delete H; return cuda_fail(e, "cudaMalloc(field tables)"); }
    char *base = (char *)H->d_eh;
    e = cudaMemcpy(base, eh.data(), 8 * n8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + 8 * n8, ehf.data(), 4 * n8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + 12 * n8, ehs.data(), 8 * n8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + 20 * n8, ehsf.data(), 4 * n8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(H->d_eh); delete H; return cuda_fail(e, "field upload"); }
    H->b = b; H->J = J; H->Delta = Delta; H->K = K; H->boundary = boundary;
    H->h.assign(h, h + (size_t)K * L);
    DevHam &d = H->dev;
    d.eh8_d = (const double *)base;
    d.eh8_f = (const float *)(base + 8 * n8);
    d.nchunk = nc;
    H->dev_lz = d;
    H->dev_lz.eh8_d = (const double *)(base + 12 * n8);
    H->dev_lz.eh8_f = (const float *)(base + 20 * n8);
    *out = H;
    return KRY_OK;
}

extern "C" int kry_hamiltonian_set(kry_basis b, double J, double Delta, const double *h, int K,
                                   int boundary, kry_ham *out)
{
    if (!out) { set_error("kry_hamiltonian_set: out is NULL"); return KRY_EINVAL; }
    *out = nullptr;
    if (!b || !h || K < 1 || (boundary != KRY_OBC && boundary != KRY_PBC) ||
        !std::isfinite(J) || !std::isfinite(Delta)) {
        set_error("kry_hamiltonian_set: bad arguments");
        return KRY_EINVAL;
    }
    const int L = b->L;
    for (int i = 0; i < K * L; ++i)
        if (!std::isfinite(h[i])) { set_error("kry_hamiltonian_set: non-finite field"); return KRY_EINVAL; }
    if (K > KBMAX) {
        set_error("kry_hamiltonian_set: K = %d realisations exceeds the maximum %d", K, KBMAX);
        return KRY_EINVAL;
    }
    if (b->dev.list) return ham_set_list(b, J, Delta, h, K, boundary, out);
    const int Llo = b->Llo, Lhi = b->Lhi;
    const uint32_t nlo = 1u << Llo, nhi = 1u << Lhi;
    // field energy tables, realisation fastest:
    //   sum_i h_{k,i} (n_i - 1/2) = ehlo[pos(lo) * K + k] + ehhi[hi * K + k]
    std::vector<uint16_t> lolist(nlo);
    {
        std::vector<uint32_t> koff(Llo + 2, 0);
        for (int k = 0; k <= Llo; ++k) koff[k + 1] = koff[k] + (uint32_t)binom64(Llo, k);
        for (uint32_t lo = 0; lo < nlo; ++lo) lolist[koff[__builtin_popcount(lo)]++] = (uint16_t)lo;
    }
    std::vector<double> ehlo((size_t)nlo * K), ehhi((size_t)nhi * K);
    for (int k = 0; k < K; ++k) {
        const double *hk = h + (size_t)k * L;
        double hsum = 0.0;
        for (int i = 0; i < L; ++i) hsum += hk[i];
        for (uint32_t p = 0; p < nlo; ++p) {
            uint32_t lo = lolist[p];
            double e = 0.0;
            for (int i = 0; i < Llo; ++i) if ((lo >> i) & 1u) e += hk[i];
            ehlo[(size_t)p * K + k] = e;
        }
        for (uint32_t hi = 0; hi < nhi; ++hi) {
            double e = -0.5 * hsum;
            for (int q = 0; q < Lhi; ++q) if ((hi >> q) & 1u) e += hk[Llo + q];
            ehhi[(size_t)hi * K + k] = e;
        }
    }
    kry_ham H = new (std::nothrow) kry_ham_s();
    if (!H) { set_error("kry_hamiltonian_set: host allocation failed"); return KRY_ENOMEM; }
    default_shape(H, b->dev.list ? 0 : b->Llo);
    fill_dev_ham(H->dev, J, Delta, L, K, boundary);
    // shifted copy of the upper-bit table for the Lanczos pass: s_k taken off every entry
    H->shift.resize(K);
    std::vector<double> ehhs(ehhi);
    for (int k = 0; k < K; ++k) {
        H->shift[k] = mean_diagonal(L, b->N, J, Delta, h + (size_t)k * L, H->dev.nbonds);
        for (uint32_t hi = 0; hi < nhi; ++hi) ehhs[(size_t)hi * K + k] -= H->shift[k];
    }
    std::vector<float> ehlo_f(ehlo.size()), ehhi_f(ehhi.size()), ehhs_f(ehhs.size());
    for (size_t p = 0; p < ehlo.size(); ++p) ehlo_f[p] = (float)ehlo[p];
    for (size_t p = 0; p < ehhi.size(); ++p) { ehhi_f[p] = (float)ehhi[p]; ehhs_f[p] = (float)ehhs[p]; }
    const size_t nl = (size_t)nlo * K, nh = (size_t)nhi * K;
    size_t o_ld = 0, o_hd = o_ld + 8 * nl, o_lf = o_hd + 8 * nh;
    size_t o_hf = o_lf + 4 * nl, o_sd = o_hf + 4 * nh, o_sf = o_sd + 8 * nh, bytes = o_sf + 4 * nh;
    cudaError_t e = cudaMalloc(&H->d_eh, bytes);
    if (e != cudaSuccess) { delete H; return cuda_fail(e, "cudaMalloc(field tables)"); }
    char *base = (char *)H->d_eh;
    e = cudaMemcpy(base + o_ld, ehlo.data(), 8 * nl, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_hd, ehhi.data(), 8 * nh, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_lf, ehlo_f.data(), 4 * nl, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_hf, ehhi_f.data(), 4 * nh, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_sd, ehhs.data(), 8 * nh, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + o_sf, ehhs_f.data(), 4 * nh, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(H->d_eh); delete H; return cuda_fail(e, "field upload"); }
    H->b = b; H->J = J; H->Delta = Delta; H->K = K; H->boundary = boundary;
    H->h.assign(h, h + (size_t)K * L);
    DevHam &d = H->dev;
    d.ehlo_d = (const double *)(base + o_ld);
    d.ehhi_d = (const double *)(base + o_hd);
    d.ehlo_f = (const float *)(base + o_lf);
    d.ehhi_f = (const float *)(base + o_hf);
    H->dev_lz = d;
    H->dev_lz.ehhi_d = (const double *)(base + o_sd);
    H->dev_lz.ehhi_f = (const float *)(base + o_sf);
    *out = H;
    return KRY_OK;
}
