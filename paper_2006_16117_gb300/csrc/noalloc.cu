// sim_apply_shifted_noalloc: the shifted sparse apply y = (A - σB) x of
// sim_apply_shifted, for callers that must not allocate device memory.
//
// Who cannot allocate: a process whose device memory is already owned by
// another allocator (for example a framework's caching pool that reserved the
// GPU up front), where a cudaMalloc fails or fragments that pool; and
// latency-critical loops, where cudaMalloc/cudaFree may synchronise the device.
// sim_apply_shifted stages x and y in per-handle job vectors that the library
// allocates on first use; this variant stages them in one file-scope device
// array instead and calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array holds at most SIM_NOALLOC_MAX_N complex128 entries per vector
// (about 8 MiB in all).  The CUDA runtime reserves it on a device when it
// loads this file's module there: at context creation with
// CUDA_MODULE_LOADING=EAGER, otherwise (lazy loading, the default) on the
// first call made on that device.  A caller whose pool will later reserve the
// GPU should make that first call, or set CUDA_MODULE_LOADING=EAGER, before
// the pool does; an out-of-memory result of that load is reported as
// SIM_ERR_OOM.  The device keeps the array until the process exits.  In host
// code the array's name is only a stand-in for it, so the device address is
// obtained with cudaGetSymbolAddress once per device, on the first call made
// while that device is current; make that first call before any stream
// capture.  All calls share the array and it keeps the last call's contents:
// each call overwrites both staging vectors completely before reading them,
// and calls that overlap on the GPU (different streams or handles at once)
// race on it.  The call is synchronous: it returns once y is written.
#include <cstring>
#include <string>

#include "internal.h"

#define SIM_NOALLOC_MAX_N 262144

namespace {

// [0, 16): two int32 job indices (active list, shift id); then x and y, each
// SIM_NOALLOC_MAX_N complex128, starting 256 bytes in.
constexpr int64_t kHeader = 16;  // double2 units = 256 bytes
static __device__ __align__(256) double2 g_noalloc_scratch[kHeader + 2 * (int64_t)SIM_NOALLOC_MAX_N];

constexpr int kMaxDevices = 64;
double2* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (set up on first use).
cudaError_t scratch_address(double2** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double2*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

// The handle internals this entry point needs (defined in api.cu).
namespace sim {
struct NoallocView {
    const Pencil* P;
    double2* d_sigma;   // per-handle shift table, allocated by sim_create
    int scratch_slot;   // index of the table's scratch shift
    cudaStream_t st;
};
bool noalloc_view(sim_handle h, NoallocView* v);
void noalloc_fail(sim_handle h, const std::string& msg);
}  // namespace sim

extern "C" sim_status sim_apply_shifted_noalloc(sim_handle h, double sig_re, double sig_im, const double* x,
                                                double* y) {
    using namespace sim;
    NoallocView v;
    if (!h || !noalloc_view(h, &v)) return SIM_ERR_INVALID_ARG;
    try {
        noalloc_fail(h, "");  // clear the previous call's message
        if (!x || !y) {
            noalloc_fail(h, "sim_apply_shifted_noalloc: NULL vector");
            return SIM_ERR_INVALID_ARG;
        }
        const int64_t n = v.P->n;
        if (n > SIM_NOALLOC_MAX_N) {
            noalloc_fail(h, "sim_apply_shifted_noalloc: n = " + std::to_string(n) +
                                " exceeds the static scratch limit of " + std::to_string(SIM_NOALLOC_MAX_N) +
                                "; use sim_apply_shifted");
            return SIM_ERR_LIMIT;
        }
        double2* base = nullptr;
        cudaError_t e = scratch_address(&base);
        if (e != cudaSuccess) {
            noalloc_fail(h, std::string("sim_apply_shifted_noalloc: cudaGetSymbolAddress (loads the static scratch "
                                        "array on first use): ") + cudaGetErrorString(e));
            return e == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
        }
        const double2 sg = make_double2(sig_re, sig_im);
        const int idx[2] = {0, v.scratch_slot};  // active job 0, its shift id
        SIM_CUDA(cudaMemcpyAsync(v.d_sigma + v.scratch_slot, &sg, sizeof(double2), cudaMemcpyHostToDevice, v.st));
        SIM_CUDA(cudaMemcpyAsync(base, idx, sizeof(idx), cudaMemcpyHostToDevice, v.st));
        JobSpace js;
        js.J = 1;
        js.n = n;
        js.vec = base + kHeader;
        js.vstride = 2 * n;
        js.d_active = reinterpret_cast<int*>(base);
        js.d_jobshift = reinterpret_cast<int*>(base) + 1;
        SIM_CUDA(cudaMemcpyAsync(js.vec, x, sizeof(double2) * n, cudaMemcpyDeviceToDevice, v.st));
        spmv_shifted_jobs(*v.P, js, 1, nullptr, 0, 1, v.d_sigma, v.st);
        SIM_CUDA(cudaMemcpyAsync(y, js.vec + n, sizeof(double2) * n, cudaMemcpyDeviceToDevice, v.st));
        SIM_CUDA(cudaStreamSynchronize(v.st));
    } catch (const CudaError& err) {
        noalloc_fail(h, "sim_apply_shifted_noalloc: " + err.what);
        return err.code == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA;
    } catch (const std::bad_alloc&) {
        return SIM_ERR_OOM;  // host memory for the message itself ran out
    } catch (...) {
        return SIM_ERR_CUDA;
    }
    return SIM_OK;
}
