// Instrumentation, not part of the method: a measured arithmetic peak for the
// benchmark's rooflines.  Every thread runs 8 independent fused multiply-add
// chains in registers (no memory traffic), on 8 CTAs of 256 threads per SM.
#include "internal.h"

namespace {

template <class R>
__global__ void __launch_bounds__(256) k_fma_peak(R a, R b, int iters, R* sink) {
    R x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (R)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    R s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == (R)-1.2345e-30) sink[threadIdx.x] = s;  // keeps the chains alive; never true
}

template <class R>
double run(int iters) {
    int dev = 0, sms = 0;
    SIM_CUDA(cudaGetDevice(&dev));
    SIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    R* sink = nullptr;
    SIM_CUDA(cudaMalloc(&sink, 256 * sizeof(R)));
    cudaEvent_t e0, e1;
    SIM_CUDA(cudaEventCreate(&e0));
    SIM_CUDA(cudaEventCreate(&e1));
    const int blocks = 8 * sms;
    const R a = (R)0.9999999, b = (R)1e-7;
    k_fma_peak<R><<<blocks, 256>>>(a, b, iters / 10, sink);  // warm-up
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaEventRecord(e0));
    k_fma_peak<R><<<blocks, 256>>>(a, b, iters, sink);
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaEventRecord(e1));
    SIM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    SIM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    const double flops = 2.0 * 8.0 * (double)iters * blocks * 256.0;
    return flops / (ms * 1e-3) / 1e12;
}

}  // namespace

// which = 0: FP64 FMA throughput, 1: FP32; *tflops receives TFLOP/s.
extern "C" sim_status sim_measure_fma_peak(int32_t which, double* tflops) {
    if (!tflops || (which != 0 && which != 1)) return SIM_ERR_INVALID_ARG;
    try {
        *tflops = which == 0 ? run<double>(1 << 16) : run<float>(1 << 18);
    } catch (...) {
        return SIM_ERR_CUDA;
    }
    return SIM_OK;
}
