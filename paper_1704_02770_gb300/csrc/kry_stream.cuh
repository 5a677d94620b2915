// Streaming of Krylov-vector tiles through shared memory with the bulk-copy engine
// (cp.async.bulk global -> shared, completion counted in bytes on an mbarrier).
//
// A vector kernel walks its tiles of TILE consecutive rows; for every tile it needs the
// same rows of several vectors (the "chunks": a right-hand operand, then W_0..W_j).  Chunks
// are grouped in units (the operand alone, then up to GV vectors each) and the units of all
// tiles of a CTA form one sequence q = 0, 1, ... (tile-major).  Unit q lands in ring slot q % nr; one thread keeps nr units in flight,
// so the bytes in flight per CTA are set by the ring, not by registers or occupancy.
//
// Every wait is bounded by the global timer: a unit that has not landed after WAIT_NS
// makes the kernel record an error, wait (bounded again) for its own copies still in
// flight, and return.
#pragma once

#include <stdint.h>

#include "kry_internal.cuh"

namespace kry {

constexpr int GV = 8;                          // chunks per unit (one per warp in the dots)
constexpr unsigned long long WAIT_NS = 1000000000ull;   // 1 s
constexpr uint32_t RING_BUDGET = 108u * 1024u;  // dynamic smem per CTA (two CTAs per SM with static smem)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// bytes must be a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Test the phase; a thread whose phase is not complete is suspended (it issues nothing)
// until the phase completes or about SUSPEND_NS pass, so a waiting warp costs no issue slots.
constexpr uint32_t SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(SUSPEND_NS)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier, at most WAIT_NS.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > WAIT_NS) return false;
    return true;
}

// Ring of nr units in dynamic shared memory: nr barriers, then nr * GV chunk buffers.
struct Ring {
    uint64_t *bar;
    unsigned char *buf;
    int nr;
    uint32_t chunk;   // TILE * sizeof(element)
    __device__ __forceinline__ unsigned char *slot(int st, int c) const
    {
        return buf + ((size_t)st * GV + c) * chunk;
    }
};

// bytes of a ring of nr units (barriers padded to 128 bytes)
__host__ __device__ inline size_t ring_bytes(int nr, size_t es) { return 128 + (size_t)nr * GV * TILE * es; }

// ring depth that fits `fixed` other bytes into the per-CTA budget (2..8 units)
inline int ring_units(size_t fixed, size_t es, uint32_t budget = RING_BUDGET)
{
    const size_t unit = (size_t)GV * TILE * es;
    long long n = ((long long)budget - (long long)fixed - 128) / (long long)unit;
    if (n < 2) n = 2;
    if (n > 8) n = 8;
    return (int)n;
}

// Tiles of this CTA (tile = blockIdx.x + k * gridDim.x).
__device__ __forceinline__ uint32_t cta_tiles(uint32_t ntiles)
{
    return ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0u;
}

// Issue unit q (called by one thread), q = k * ng + g, for tile k of this CTA.  Unit 0 of a
// tile holds the `lead` chunks [0, lead) (the tile's right-hand operand), unit g >= 1 the
// chunks [lead + (g-1) GV, lead + g GV) clipped to nch.  ptr(c) is the first element of
// chunk c's vector.
template <class V, class PtrF>
__device__ __forceinline__ void ring_issue(const Ring &R, uint32_t q, int ng, int nch, int lead, uint32_t D,
                                           PtrF ptr)
{
    const uint32_t k = q / (uint32_t)ng;
    const int g = (int)(q - k * (uint32_t)ng);
    const uint32_t r0 = (blockIdx.x + k * gridDim.x) * (uint32_t)TILE;
    const uint32_t rows = min((uint32_t)TILE, D - r0);
    const uint32_t bytes = (rows * (uint32_t)sizeof(V) + 15u) & ~15u;
    const int c0 = g == 0 ? 0 : lead + (g - 1) * GV;
    const int c1 = g == 0 ? lead : min(nch, c0 + GV);
    const int st = (int)(q % (uint32_t)R.nr);
    mbar_arrive_expect_tx(R.bar + st, bytes * (uint32_t)(c1 - c0));
    for (int c = c0; c < c1; ++c) bulk_g2s(R.slot(st, c - c0), ptr(c) + r0, bytes, R.bar + st);
}

// Initialise the barriers and issue the first units (thread 0), then sync the CTA.
template <class V, class PtrF>
__device__ __forceinline__ void ring_start(const Ring &R, uint32_t nq, int ng, int nch, int lead, uint32_t D,
                                           PtrF ptr)
{
    if (threadIdx.x == 0) {
        for (int i = 0; i < R.nr; ++i) mbar_init(R.bar + i, 1);
        fence_barrier_init();
        for (uint32_t q = 0; q < (uint32_t)R.nr && q < nq; ++q) ring_issue<V>(R, q, ng, nch, lead, D, ptr);
    }
    __syncthreads();
}

// After a timed-out wait on unit q: wait (bounded) for units q .. q+nr-1, the ones that
// may still be in flight.
__device__ __forceinline__ void ring_drain(const Ring &R, uint32_t q, uint32_t nq)
{
    for (uint32_t p = q; p < nq && p < q + (uint32_t)R.nr; ++p)
        mbar_wait(R.bar + p % (uint32_t)R.nr, (p / (uint32_t)R.nr) & 1u);
}

}  // namespace kry
