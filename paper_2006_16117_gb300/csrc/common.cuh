// Shared device helpers of the SIM-M library: complex arithmetic on
// double2/float2, warp reductions, launch checks.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace sim {

// ---- complex arithmetic (x = re, y = im) ----------------------------------
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename R> using cplx = typename cplx_t<R>::type;

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cconjmul(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc += a*b
template <typename C> __host__ __device__ __forceinline__ C cfma(C a, C b, C acc) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
template <typename C> __host__ __device__ __forceinline__ C cscale(C a, decltype(a.x) s) { return mk(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ decltype(C().x) cabs2(C a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double cabsd(double2 a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ float cabsd(float2 a) { return hypotf(a.x, a.y); }
// a / b with scaling to avoid overflow (Smith's method)
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        double r = b.x / b.y, d = b.y + b.x * r;
        return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__host__ __device__ __forceinline__ float2 cdiv(float2 a, float2 b) {
    if (fabsf(b.x) >= fabsf(b.y)) {
        float r = b.y / b.x, d = b.x + b.y * r;
        return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    } else {
        float r = b.x / b.y, d = b.y + b.x * r;
        return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
    }
}
__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float2 a) { return mk((double)a.x, (double)a.y); }
template <typename C> __device__ __forceinline__ C from_c128(double2 a);
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_c128<float2>(double2 a) { return mk((float)a.x, (float)a.y); }

// ---- warp / block reductions -----------------------------------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}
__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// ---- error handling ------------------------------------------------------
struct CudaError {
    cudaError_t code;
    std::string what;
};

#define SIM_CUDA(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::sim::CudaError{e_, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// every kernel launch of the library is followed by this check, which also
// counts launches (sim_kernel_stats reports the count)
int64_t& launch_counter();
#define SIM_LAUNCH_CHECK()                 \
    do {                                   \
        ++::sim::launch_counter();         \
        SIM_CUDA(cudaGetLastError());      \
    } while (0)

// Optional per-kernel timing with CUDA events on the launching stream (off by
// default; sim_options.kernel_timing turns it on).  kprof_end adds the
// algorithmic bytes and flops of the launch.
void kprof_begin(const char* name, cudaStream_t st);
void kprof_end(const char* name, cudaStream_t st, double bytes, double flops);
bool kprof_enabled();
void kprof_enable(bool on);
void kprof_reset();
bool kprof_query(const char* name, double* ms, double* bytes, double* flops, int64_t* launches);

inline int cdiv_up(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace sim
