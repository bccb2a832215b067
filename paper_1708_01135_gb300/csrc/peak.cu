// ewald_fma_peak: the CUDA-core fused multiply-add rate of the current GPU, measured.
//
// The real-space pair kernels and the CUDA-core reciprocal products are bound by FP32 or
// FP64 arithmetic issue, so their roofline needs the rate the device actually sustains,
// not a figure from unit counts and a nominal clock.  This file measures it: every thread
// runs kChains independent FMA recurrences a <- a * b + c for a fixed number of iterations
// (enough independent work per warp to hide the FMA latency), on a grid of resident
// blocks on every SM, timed with CUDA events.  Each FMA counts two flops.  The recurrence
// values stay bounded (|b| < 1), and one value per thread is kept live through a store that
// the compiler cannot drop.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ewald_internal.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

__device__ double g_peak_sink;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_loop(int64_t iters, T b, T c, int sink_flag)
{
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = T(threadIdx.x + k) * T(1e-3);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    // sink_flag is never equal to the thread index at run time (the host passes -1), but the
    // compiler cannot know that, so every chain stays live
    if ((int)threadIdx.x == sink_flag) g_peak_sink = (double)s;
}

template <class T>
int measure(int sms, double *tflops)
{
    const dim3 grid((unsigned)(sms * kBlocksPerSm)), block(kThreads);
    const double threads = (double)grid.x * kThreads;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return EWALD_E_CUDA;
    }
    // a short run to warm up and to size the timed run at ~0.1 s (bounded: at most 2^22
    // iterations, ~0.5 s for FP32 on a full GB300)
    int64_t iters = 1024;
    float ms = 0.f;
    int rc = EWALD_OK;
    for (int pass = 0; pass < 3 && rc == EWALD_OK; ++pass) {
        cudaEventRecord(e0);
        k_fma_loop<T><<<grid, block>>>(iters, T(0.999), T(1e-4), -1);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
            rc = EWALD_E_CUDA;
            break;
        }
        cudaEventElapsedTime(&ms, e0, e1);
        if (pass < 2) {
            const double want = 100.0;   // ms
            int64_t next = (int64_t)((double)iters * want / (ms > 1e-3 ? ms : 1e-3));
            if (next < 1024) next = 1024;
            if (next > (1ll << 22)) next = 1ll << 22;
            iters = next;
        }
    }
    if (rc == EWALD_OK)
        *tflops = 2.0 * kChains * (double)iters * threads / (ms * 1e-3) / 1e12;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace

extern "C" int ewald_fma_peak(int precision, double *tflops)
{
    if (!tflops || (precision != EWALD_FP64 && precision != EWALD_FP32)) return EWALD_E_INVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EWALD_E_CUDA;
    return precision == EWALD_FP64 ? measure<double>(sms, tflops) : measure<float>(sms, tflops);
}
