// Sorted-list basis: chains longer than the split rank tables reach (33 <= L <= 64), such as
// the L = 55 Fibonacci rings of Sec. 2 and Sec. 4, and any L on request.
//
// The basis is kept as the sorted integer list of Alg. 2, built on the device by combinadic
// unranking (row r holds the r-th smallest L-bit integer with N set bits).  The rank of a
// state is its combinadic number (the lookup of Sec. 3 replaced by arithmetic):
//     rank(s) = sum_{j=1..N} C(p_j, j),   p_1 < ... < p_N the occupied sites.
// A hop across bond (p, p+1) moves one particle, the i-th from the left, by one site and
// leaves the order of the particles unchanged, so the rank moves by C(p, i-1): up when the
// particle moves right, down when it moves left.  Only the ring bond (L-1, 0) reorders the
// particles; its neighbour is re-ranked in full.  The binomials C(p, k), p < L, k <= N, sit in
// shared memory; the list costs 8 bytes per row of every H.v.
//
//   k_list_build    states[r] for every rank r
//   k_list_rank     ranks of given states (validated)
//   k_list_unrank   states of given ranks (validated)
//   k_list_apply    y = H x for [D][K] vectors (K = 1 for one realisation)
//   k_list_hv       u = sigma_j H W_j (pass A, part 1, one realisation)
//   k_list_hv_b     u = sigma_j[k] H_k W_j[:, k] (pass A, part 1, K realisations)
#include <cuda_runtime.h>

#include <algorithm>

#include "kry_device.cuh"

namespace kry {

namespace {

int sm_count_l()
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

__device__ __forceinline__ void stage_cbin(const DevBasis &b, uint32_t *cb)
{
    const int n = b.L * (b.N + 1);
    for (int i = threadIdx.x; i < n; i += blockDim.x) cb[i] = __ldg(b.cbin + i);
}

// combinadic number of s (s must hold N set bits below bit L)
__device__ __forceinline__ uint32_t list_rank(uint64_t s, const uint32_t *cb, int N1)
{
    uint32_t r = 0;
    int j = 0;
    while (s) {
        const int p = __ffsll((long long)s) - 1;
        s &= s - 1ull;
        r += cb[p * N1 + (++j)];
    }
    return r;
}

// Row r (state s) of H x for realisation k of K interleaved ones: returns the sum of the
// neighbour amplitudes, and the diagonal d(s) in *d.
template <class V>
__device__ __forceinline__ typename Arith<V>::HvSum list_row(const DevBasis &b, const DevHam &hm,
                                                             const V *__restrict__ x, uint32_t r, uint64_t s,
                                                             int k, int K, const uint32_t *cb,
                                                             typename VT<V>::R *d)
{
    using R = typename VT<V>::R;
    const int L = b.L, N1 = b.N + 1;
    const uint64_t obc = (L >= 2) ? ((1ull << (L - 1)) - 1ull) : 0ull;
    const uint64_t anti = (s ^ (s >> 1)) & obc;
    const uint64_t wrap = hm.pbc ? ((s ^ (s >> (L - 1))) & 1ull) : 0ull;
    const int nanti = __popcll((long long)anti) + (int)wrap;
    R e = (R)hm.cz * (R)(hm.nbonds - 2 * nanti);
    for (int c = 0; c < hm.nchunk; ++c) {
        const uint32_t v = (uint32_t)(s >> (8 * c)) & 0xFFu;
        e += VT<V>::eh8(hm, ((size_t)c * 256 + v) * K + k);
    }
    *d = e;
    typename Arith<V>::HvSum acc{};
    uint64_t a = anti;
    while (a) {
        const int p = __ffsll((long long)a) - 1;
        a &= a - 1ull;
        const int cnt = __popcll((long long)(s & ((1ull << p) - 1ull)));
        const uint32_t step = cb[p * N1 + cnt];
        const uint32_t t = ((s >> p) & 1ull) ? r + step : r - step;
        hv_add(acc, ldg(x + (size_t)t * K + k));
    }
    if (wrap) {
        const uint64_t s2 = s ^ ((1ull << (L - 1)) | 1ull);
        hv_add(acc, ldg(x + (size_t)list_rank(s2, cb, N1) * K + k));
    }
    return acc;
}

__global__ void k_list_build(DevBasis b, uint64_t *states)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cb = (uint32_t *)smem;
    stage_cbin(b, cb);
    __syncthreads();
    const int N1 = b.N + 1;
    for (uint32_t r0 = blockIdx.x * blockDim.x + threadIdx.x; r0 < b.D; r0 += gridDim.x * blockDim.x) {
        // largest p with C(p, k) <= the remaining rank, for k = N down to 1 (p decreasing)
        uint32_t r = r0;
        uint64_t s = 0;
        int p = b.L;
        for (int k = b.N; k >= 1; --k) {
            do { --p; } while (p > 0 && cb[p * N1 + k] > r);
            r -= cb[p * N1 + k];
            s |= 1ull << p;
        }
        states[r0] = s;
    }
}

__global__ void k_list_rank(DevBasis b, const uint64_t *__restrict__ st, uint32_t *__restrict__ rk, int64_t n)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cb = (uint32_t *)smem;
    stage_cbin(b, cb);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t s = st[i];
        if ((b.L < 64 && (s >> b.L) != 0ull) || __popcll((long long)s) != b.N) {
            rk[i] = 0xFFFFFFFFu;
            atomicOr(b.err, 1);
            continue;
        }
        rk[i] = list_rank(s, cb, b.N + 1);
    }
}

__global__ void k_list_unrank(DevBasis b, const uint32_t *__restrict__ rk, uint64_t *__restrict__ st, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = rk[i];
        if (r >= b.D) {
            st[i] = 0ull;
            atomicOr(b.err, 2);
            continue;
        }
        st[i] = __ldg(b.states + r);
    }
}

// y = H x over the D*K elements, realisation fastest
template <class V>
__global__ void __launch_bounds__(NTHR) k_list_apply(DevBasis b, DevHam hm, int K, const V *__restrict__ x,
                                                     V *__restrict__ y)
{
    using R = typename VT<V>::R;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cb = (uint32_t *)smem;
    stage_cbin(b, cb);
    __syncthreads();
    const size_t n = (size_t)b.D * (size_t)K;
    for (size_t i = (size_t)blockIdx.x * NTHR + threadIdx.x; i < n; i += (size_t)gridDim.x * NTHR) {
        const uint32_t r = (uint32_t)(i / (size_t)K);
        const int k = (int)(i - (size_t)r * K);
        R d;
        const auto acc = list_row<V>(b, hm, x, r, __ldg(b.states + r), k, K, cb, &d);
        y[i] = hv_finish(d, ldg(x + i), (R)hm.halfJ, acc);
    }
}

// pass A, part 1, one realisation: U = sigma_j H W_j
template <class V>
__global__ void __launch_bounds__(NTHR) k_list_hv(EvArgs<V> a, int jj)
{
    pdl_begin();
    KryCtl *ctl = a.ctl;
    if (ctl->done || jj >= ctl->m_eff) return;
    using R = typename VT<V>::R;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cb = (uint32_t *)smem;
    stage_cbin(a.b, cb);
    __syncthreads();
    const double sd = ctl->sigma[jj];
    const R sj = (R)sd, shj = (R)(sd * a.h.halfJ);
    const V *x = a.W + (size_t)jj * a.ldW;
    for (uint32_t r = blockIdx.x * NTHR + threadIdx.x; r < a.b.D; r += gridDim.x * NTHR) {
        R d;
        const auto acc = list_row<V>(a.b, a.h, x, r, __ldg(a.b.states + r), 0, 1, cb, &d);
        a.U[r] = hv_finish(sj * d, ldg(x + r), shj, acc);
    }
}

// pass A, part 1, K realisations: U[:, k] = sigma_j[k] H_k W_j[:, k]
template <class V>
__global__ void __launch_bounds__(NTHR) k_list_hv_b(EvArgsB<V> a, int jj)
{
    KryCtlB *ctl = a.ctl;
    if (ctl->hd.done || jj >= ctl->hd.m_run) return;
    using R = typename VT<V>::R;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cb = (uint32_t *)smem;
    stage_cbin(a.b, cb);
    __syncthreads();
    const int K = a.K;
    const V *x = a.W + (size_t)jj * a.ldW;
    const size_t n = (size_t)a.b.D * (size_t)K;
    for (size_t i = (size_t)blockIdx.x * NTHR + threadIdx.x; i < n; i += (size_t)gridDim.x * NTHR) {
        const uint32_t r = (uint32_t)(i / (size_t)K);
        const int k = (int)(i - (size_t)r * K);
        R d;
        const auto acc = list_row<V>(a.b, a.h, x, r, __ldg(a.b.states + r), k, K, cb, &d);
        const double sd = ctl->sigma[jj][k];
        a.U[i] = hv_finish((R)sd * d, ldg(x + i), (R)(sd * a.h.halfJ), acc);
    }
}

template <class Kern>
int list_prep(Kern kernel, size_t smem)
{
    if (smem > 48 * 1024) KRY_CU(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KRY_OK;
}

template <class Kern>
int list_grid_of(Kern kernel, size_t smem, size_t work)
{
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NTHR, smem);
    const size_t blocks = (work + NTHR - 1) / NTHR;
    return (int)std::max<size_t>(1, std::min<size_t>(blocks, (size_t)sm_count_l() * (size_t)std::max(1, occ)));
}

}  // namespace

size_t list_smem(const DevBasis &b) { return sizeof(uint32_t) * (size_t)b.L * (size_t)(b.N + 1); }

int list_build(DevBasis &b, cudaStream_t s)
{
    const size_t sm = list_smem(b);
    if (int rc = list_prep(k_list_build, sm)) return rc;
    const int grid = list_grid_of(k_list_build, sm, b.D);
    k_list_build<<<grid, NTHR, sm, s>>>(b, (uint64_t *)b.states);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_list_rank(const DevBasis &b, const uint64_t *st, uint32_t *rk, int64_t n, cudaStream_t s)
{
    const size_t sm = list_smem(b);
    if (int rc = list_prep(k_list_rank, sm)) return rc;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_list_rank<<<grid, 256, sm, s>>>(b, st, rk, n);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_list_unrank(const DevBasis &b, const uint32_t *rk, uint64_t *st, int64_t n, cudaStream_t s)
{
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    k_list_unrank<<<grid, 256, 0, s>>>(b, rk, st, n);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

int launch_list_apply(const DevBasis &b, const DevHam &h, int c64, int K, const void *x, void *y, cudaStream_t s)
{
    const size_t sm = list_smem(b), work = (size_t)b.D * (size_t)K;
    if (c64) {
        if (int rc = list_prep(k_list_apply<float2>, sm)) return rc;
        k_list_apply<float2><<<list_grid_of(k_list_apply<float2>, sm, work), NTHR, sm, s>>>(
            b, h, K, (const float2 *)x, (float2 *)y);
    } else {
        if (int rc = list_prep(k_list_apply<double2>, sm)) return rc;
        k_list_apply<double2><<<list_grid_of(k_list_apply<double2>, sm, work), NTHR, sm, s>>>(
            b, h, K, (const double2 *)x, (double2 *)y);
    }
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template <class V>
int list_hv_grid(const DevBasis &b, int *grid)
{
    const size_t sm = list_smem(b);
    if (int rc = list_prep(k_list_hv<V>, sm)) return rc;
    *grid = list_grid_of(k_list_hv<V>, sm, b.D);
    return KRY_OK;
}

template <class V>
int launch_list_hv(const EvArgs<V> &a, int jj, int grid, cudaStream_t s, int pdl)
{
    KRY_CU(launch_ex(pdl, k_list_hv<V>, grid, NTHR, list_smem(a.b), s, a, jj));
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template <class V>
int launch_list_hv_b(const EvArgsB<V> &a, int jj, cudaStream_t s)
{
    const size_t sm = list_smem(a.b);
    if (int rc = list_prep(k_list_hv_b<V>, sm)) return rc;
    const int grid = list_grid_of(k_list_hv_b<V>, sm, (size_t)a.b.D * (size_t)a.K);
    k_list_hv_b<V><<<grid, NTHR, sm, s>>>(a, jj);
    KRY_CU(cudaGetLastError());
    return KRY_OK;
}

template int list_hv_grid<ffc>(const DevBasis &, int *);
template int launch_list_hv<ffc>(const EvArgs<ffc> &, int, int, cudaStream_t, int);
template int launch_list_hv_b<ffc>(const EvArgsB<ffc> &, int, cudaStream_t);
template int list_hv_grid<double2>(const DevBasis &, int *);
template int list_hv_grid<float2>(const DevBasis &, int *);
template int launch_list_hv<double2>(const EvArgs<double2> &, int, int, cudaStream_t, int);
template int launch_list_hv<float2>(const EvArgs<float2> &, int, int, cudaStream_t, int);
template int launch_list_hv_b<double2>(const EvArgsB<double2> &, int, cudaStream_t);
template int launch_list_hv_b<float2>(const EvArgsB<float2> &, int, cudaStream_t);

}  // namespace kry
