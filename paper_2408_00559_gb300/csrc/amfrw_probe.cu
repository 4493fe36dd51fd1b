// Arithmetic peak probe: the FP64 and FP32 FMA throughput of the current
// device, measured with CUDA events.  The roofline of the solver kernels is
// set by these pipes (their grids live in shared memory and move almost no
// HBM traffic), and the FP64 rate of a part is not among the copy/GEMM peaks
// measured elsewhere, so the library measures it itself.  The paper has no
// counterpart.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/amfrw.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hide the pipe latency)
constexpr int kThreads = 256;
__device__ double g_probe_sink;  // keeps the chains observable

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(int iters, T b, T c)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // a value the chains never reach: the store is never taken, but the
    // compiler cannot prove it, so the chains are not removed
    if (s == (T)-1234.5) g_probe_sink = (double)s;
}

}  // namespace

extern "C" int amfrw_peak_probe(int32_t precision, int32_t iters, double* tflops_out, void* cuda_stream)
{
    if (!tflops_out || iters < 1) return AMFRW_EINVAL;
    if (precision != AMFRW_FP64 && precision != 2) return AMFRW_EINVAL;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return AMFRW_ECUDA;
    int per_sm = 0;
    const void* f = precision == AMFRW_FP64 ? (const void*)fma_probe_kernel<double>
                                            : (const void*)fma_probe_kernel<float>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, kThreads, 0) != cudaSuccess || per_sm < 1)
        return AMFRW_ECUDA;
    const int grid = sms * per_sm;
    auto launch = [&]() {
        if (precision == AMFRW_FP64)
            fma_probe_kernel<double><<<grid, kThreads, 0, st>>>(iters, 0.999999, 1e-6);
        else
            fma_probe_kernel<float><<<grid, kThreads, 0, st>>>(iters, 0.9999f, 1e-4f);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return AMFRW_ECUDA;
    }
    int rc = AMFRW_OK;
    float best = 0.f;
    launch();  // warm-up
    for (int r = 0; r < 5 && rc == AMFRW_OK; ++r) {
        float ms = 0.f;
        if (cudaEventRecord(e0, st) != cudaSuccess) rc = AMFRW_ECUDA;
        launch();
        if (rc == AMFRW_OK && (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, st) != cudaSuccess ||
                               cudaEventSynchronize(e1) != cudaSuccess ||
                               cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            rc = AMFRW_ECUDA;
        if (rc == AMFRW_OK && (best == 0.f || ms < best)) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != AMFRW_OK || !(best > 0.f)) return AMFRW_ECUDA;
    const double flops = 2.0 * kChains * (double)iters * (double)grid * (double)kThreads;
    *tflops_out = flops / (best * 1e-3) / 1e12;
    return AMFRW_OK;
}
