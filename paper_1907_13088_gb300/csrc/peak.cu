// fmx_fma_peak: the device's measured fused multiply-add rate in FP32 or
// FP64, the denominator of the arithmetic roofline reported beside the HBM
// one.  A measurement utility with no counterpart in the paper.
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA
// latency at full occupancy) for a fixed number of iterations; the grid
// fills every SM several times over.  The rate is 2 flops per FMA over the
// CUDA-event time of the launch on the given stream, best of a few launches
// after a warm-up.
#include <cuda_runtime.h>

#include "fmx.h"
#include "fmx_internal.h"

namespace fmx {
void set_last_error(const char *msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

// where a chain's result would be written (see below); never read
__device__ float g_sink32;
__device__ double g_sink64;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_loop(int iters, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // never true for the arguments the host passes (the chains stay positive);
    // keeps them from being optimised away
    if (s == (T)-1.2345e30) {
        if (sizeof(T) == 4) g_sink32 = (float)s;
        else g_sink64 = (double)s;
    }
}

template <typename T>
fmx_status measure(cudaStream_t s, double *flops) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FMX_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_loop<T>, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int blocks = sms * per_sm * 4;
    // FP32 runs ~64x faster on this class of part: more iterations to time
    const int iters = sizeof(T) == 4 ? 1 << 16 : 1 << 11;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return FMX_ECUDA;
    }
    const T a = (T)0.999999, b = (T)1e-7;
    float best = 0.f;
    fmx_status st = FMX_OK;
    for (int rep = 0; rep < 4 && st == FMX_OK; ++rep) {
        cudaEventRecord(e0, s);
        k_fma_loop<T><<<blocks, kThreads, 0, s>>>(iters, a, b);
        cudaEventRecord(e1, s);
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = FMX_ECUDA;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // launch 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FMX_OK || best <= 0.f) return FMX_ECUDA;
    *flops = 2.0 * kChains * (double)iters * blocks * kThreads / (best * 1e-3);
    return FMX_OK;
}

}  // namespace

extern "C" fmx_status fmx_fma_peak(int precision, void *stream, double *flops_per_s) {
    if (!flops_per_s || (precision != FMX_F32 && precision != FMX_F64)) {
        fmx::set_last_error("fmx_fma_peak: bad precision or NULL output");
        return FMX_EINVAL;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    fmx_status st = precision == FMX_F64 ? measure<double>(s, flops_per_s) : measure<float>(s, flops_per_s);
    if (st != FMX_OK) fmx::set_last_error("fmx_fma_peak: a CUDA call failed");
    return st;
}
