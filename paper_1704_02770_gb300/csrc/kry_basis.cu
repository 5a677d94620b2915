// Sector basis without a stored list: combinadic rank/unrank tables (Sec. 2 "Basis
// representation"; Algorithm 2 defines the sorted order that the ranks reproduce), and
// the Hamiltonian handle (Eq. 1).
#include <cuda_runtime.h>

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

extern "C" int kry_basis_create(int L, int n_up, kry_basis *out)
{
    if (!out) { set_error("kry_basis_create: out is NULL"); return KRY_EINVAL; }
    *out = nullptr;
    if (L < 1 || L > 32 || n_up < 0 || n_up > L) {
        set_error("kry_basis_create: need 1 <= L <= 32 and 0 <= n_up <= L (got L=%d, n_up=%d)",
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
    cudaMemcpy(base + o_blk, blk.data(), sizeof(uint32_t) * nhi, cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_rl, ranklo.data(), sizeof(uint16_t) * nlo, cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_ll, lolist.data(), sizeof(uint16_t) * nlo, cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_ko, koff.data(), sizeof(uint32_t) * (Llo + 2), cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_bs, bsz.data(), sizeof(uint32_t) * (Llo + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_ts, tstart.data(), sizeof(uint32_t) * tstart.size(), cudaMemcpyHostToDevice);
    e = cudaMemset(base + o_er, 0, 16);
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
    if (unrank) k_unrank<<<grid, 256, 0, s>>>(b->dev, (const uint32_t *)in, (uint64_t *)out, n);
    else k_rank<<<grid, 256, 0, s>>>(b->dev, (const uint64_t *)in, (uint32_t *)out, n);
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
    std::vector<float> ehlo_f(ehlo.size()), ehhi_f(ehhi.size());
    for (size_t p = 0; p < ehlo.size(); ++p) ehlo_f[p] = (float)ehlo[p];
    for (size_t p = 0; p < ehhi.size(); ++p) ehhi_f[p] = (float)ehhi[p];
    const size_t nl = (size_t)nlo * K, nh = (size_t)nhi * K;
    size_t o_ld = 0, o_hd = o_ld + 8 * nl, o_lf = o_hd + 8 * nh;
    size_t o_hf = o_lf + 4 * nl, bytes = o_hf + 4 * nh;
    kry_ham H = new (std::nothrow) kry_ham_s();
    if (!H) { set_error("kry_hamiltonian_set: host allocation failed"); return KRY_ENOMEM; }
    cudaError_t e = cudaMalloc(&H->d_eh, bytes);
    if (e != cudaSuccess) { delete H; return cuda_fail(e, "cudaMalloc(field tables)"); }
    char *base = (char *)H->d_eh;
    cudaMemcpy(base + o_ld, ehlo.data(), 8 * nl, cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_hd, ehhi.data(), 8 * nh, cudaMemcpyHostToDevice);
    cudaMemcpy(base + o_lf, ehlo_f.data(), 4 * nl, cudaMemcpyHostToDevice);
    e = cudaMemcpy(base + o_hf, ehhi_f.data(), 4 * nh, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(H->d_eh); delete H; return cuda_fail(e, "field upload"); }
    H->b = b; H->J = J; H->Delta = Delta; H->K = K; H->boundary = boundary;
    H->h.assign(h, h + (size_t)K * L);
    DevHam &d = H->dev;
    d.ehlo_d = (const double *)(base + o_ld);
    d.ehhi_d = (const double *)(base + o_hd);
    d.ehlo_f = (const float *)(base + o_lf);
    d.ehhi_f = (const float *)(base + o_hf);
    d.cz = 0.25 * J * Delta;
    d.halfJ = 0.5 * J;
    d.pbc = (boundary == KRY_PBC && L >= 3) ? 1 : 0;
    d.nbonds = d.pbc ? L : (L - 1);
    d.K = K;
    *out = H;
    return KRY_OK;
}
