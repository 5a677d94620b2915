// Measured arithmetic peaks of the current GPU (a measurement aid, not part of the paper's
// method): the rate of FP64 fused multiply-adds and of FP32 fused multiply-adds when every SM
// runs independent chains of them, timed with CUDA events.  GB300 executes FP64 at a small
// fraction of its FP32 rate, so the complex128 kernels of this library are bound by the FP64
// pipe rather than by HBM; this measurement is the denominator of their roofline.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "kry_internal.cuh"

using namespace kry;

namespace {

constexpr int kChains = 8;   // independent multiply-add chains per thread

// Each thread runs kChains chains of `iters` dependent multiply-adds in FP64 (F64 = 1) or FP32.
template <int F64>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, float seed, float *sink)
{
    using T = typename std::conditional<F64 != 0, double, float>::type;
    T x[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = (T)(seed + (float)(threadIdx.x + i));
    const T a = (T)0.999, b = (T)0.001;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += x[i];
    if (s == (T)-1.0) sink[0] = (float)s;   // never true; keeps the chains alive
}

template <int F64>
int time_rate(int grid, int iters, cudaStream_t s, float *sink, double *flops_per_s)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KRY_CU(cudaEventCreate(&e0));
    cudaError_t err = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && err == cudaSuccess; ++rep) {   // first run warms up
        err = cudaEventRecord(e0, s);
        if (err == cudaSuccess) {
            k_fma_rate<F64><<<grid, 256, 0, s>>>(iters, 1.0f, sink);
            err = cudaGetLastError();
        }
        if (err == cudaSuccess) err = cudaEventRecord(e1, s);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && rep > 0) best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "kry_measure_peaks");
    *flops_per_s = 2.0 * (double)grid * 256.0 * (double)iters * kChains / (best * 1e-3);
    return KRY_OK;
}

}  // namespace

extern "C" int kry_measure_peaks(double *fp64_tflops, double *fp32_tflops, void *stream)
{
    if (!fp64_tflops || !fp32_tflops) {
        set_error("kry_measure_peaks: bad arguments");
        return KRY_EINVAL;
    }
    int dev = 0, sms = 0;
    KRY_CU(cudaGetDevice(&dev));
    KRY_CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = (cudaStream_t)stream;
    float *sink = nullptr;
    KRY_CU(cudaMalloc(&sink, sizeof(float)));
    double f64 = 0.0, f32 = 0.0;
    const int grid = sms * 8;
    int rc = time_rate<1>(grid, 512, s, sink, &f64);
    if (rc == KRY_OK) rc = time_rate<0>(grid, 1024, s, sink, &f32);
    cudaFree(sink);
    if (rc != KRY_OK) return rc;
    *fp64_tflops = f64 / 1e12;
    *fp32_tflops = f32 / 1e12;
    return KRY_OK;
}
