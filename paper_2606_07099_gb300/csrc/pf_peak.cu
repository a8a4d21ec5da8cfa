// pf_peak.cu -- FMA throughput of this GPU, measured: the denominators of the ALU
// roofline that the solve kernels are reported against (not part of the paper's method).
//
// Every thread runs kChains independent fused multiply-add chains (so that the pipe, not
// the chain latency, bounds the loop), over a grid of several CTAs per SM.  The result
// is written out so that the compiler keeps the arithmetic.
#include <cuda_runtime.h>

#include "pf.h"

namespace {

constexpr int kChains = 8;

// where a result would be stored if the loop's sum ever came out negative (it cannot:
// every chain grows from a non-negative start by a positive step)
__device__ double g_sink;

template <typename T>
__global__ void __launch_bounds__(256) fma_loop(int iters) {
    T a[kChains];
    const T x = T(1) + T(1e-7) * T(threadIdx.x & 7), y = T(0.5) - T(1e-8) * T(blockIdx.x & 3);
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = T(c) * T(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s < T(0)) g_sink = double(s);  // never true; keeps the arithmetic
}

template <typename T>
pf_err measure(int blocks_per_sm, int iters, double* tflops, cudaStream_t st) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PF_ECUDA;
    const int threads = 256, grid = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return PF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return PF_ECUDA;
    }
    fma_loop<T><<<grid, threads, 0, st>>>(iters / 4);  // warm-up (clocks, instruction cache)
    cudaEventRecord(e0, st);
    fma_loop<T><<<grid, threads, 0, st>>>(iters);
    cudaEventRecord(e1, st);
    pf_err r = PF_OK;
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || !(ms > 0.f)) {
        r = PF_ECUDA;
    } else {
        const double flops = 2.0 * kChains * (double)iters * threads * (double)grid;
        *tflops = flops / (ms * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return r;
}

}  // namespace

extern "C" pf_err pf_measure_fma_peak(int fp64, int iters, double* tflops, void* stream) {
    if (!tflops || iters < 16) return PF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return fp64 ? measure<double>(8, iters, tflops, st) : measure<float>(8, iters, tflops, st);
}
