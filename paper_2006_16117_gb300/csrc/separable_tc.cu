// Mode products of the separable preconditioner on the 5th-generation tensor
// cores (tcgen05), complex64 data.
//
// A mode product along an axis of length N is a real GEMM once the complex
// vector is viewed as floats: with m = 2 r + c (row r of the mode product, c the
// real or imaginary part),
//     Y[m][k] = Σ_j X[m][j] Q[k][j]      (Q symmetric, real),
// where element (m, j) of X sits at base(m) + j ks floats:
//     axis 0 (P = 1):  base(m) = (m >> 1) 2N + (m & 1),        ks = 2,
//     axis d > 0:      base(m) = (m mod 2P) + 2PN (m div 2P),  ks = 2P.
// A CTA computes a 128 × NT tile of Y (NT <= 256 outputs) in tensor memory
// with tcgen05.mma kind::tf32 (M = 128, N = NT, K = 8 per instruction): the
// operands are staged by the CTA's threads in shared memory as K-major
// no-swizzle core matrices (8 rows × 16 bytes; next core matrix along K at
// +128 B, next 8 rows at +1024 B), 32 reduction indices per stage.  A launch
// of at least one CTA per SM uses one stage per CTA and as many CTAs per SM as
// shared memory allows (2 to 6), so that one CTA's staging overlaps the others'
// MMAs; a smaller launch uses two stages per CTA (staging of the next 32
// indices while the current ones multiply).  FP32 accuracy from TF32 units:
// every value is split as x = hi + lo with hi its leading 11 significand bits
// (exact in TF32), and Y = X_hi Q_hi + X_hi Q_lo + X_lo Q_hi accumulated in
// FP32 (the dropped X_lo Q_lo term is below FP32 rounding); Q's halves are
// tables made once.
// One thread issues the MMAs and commits them to the stage's mbarrier; the
// epilogue reads the accumulator with tcgen05.ld (warp w: lanes 32 (w mod 4) ..,
// half the columns each) and stores Y.  Every wait has an iteration limit.
#include <cstdint>

#include "internal.h"
#include "separable.h"

namespace sim {

namespace {

constexpr int TC_M = 128;          // tile rows = tensor-memory lanes
constexpr int TC_KC = 32;          // reduction indices per stage
constexpr int TC_THREADS = 256;    // 8 warps: staging; all 8 read the accumulator
constexpr int TC_A_BYTES = TC_M * TC_KC * 4;  // one A tile (hi or lo): 16 KB
constexpr long long TC_WAIT = 1ll << 26;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle, LBO = 128 B (next core
// matrix along K), SBO = 1024 B (next 8 rows), descriptor version 1
__device__ __forceinline__ uint64_t kmajor_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// byte offset of element (row, k) of a K-major tile with 32 reduction indices
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
    return (uint32_t)((row & 7) * 16 + (k & 3) * 4 + (k >> 2) * 128 + (row >> 3) * 1024);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait; false (and the error flag) if the limit ran out
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (long long it = 0; it < TC_WAIT; ++it)
        if (bar_try(bar, parity)) return true;
    atomicExch(err, 5);
    return false;
}

__device__ __forceinline__ int64_t row_base(int64_t m, int N, int64_t P) {
    return P == 1 ? (m >> 1) * 2 * (int64_t)N + (m & 1) : (m % (2 * P)) + 2 * P * (int64_t)N * (m / (2 * P));
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS) k_sep_mode_tc(const float2* __restrict__ Xall, float2* __restrict__ Yall,
                                                               const float* __restrict__ Qhi,
                                                               const float* __restrict__ Qlo, int N, int64_t P,
                                                               int64_t rows, int64_t n, int NT, uint32_t tcols,
                                                               int nst, int* err) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    // nst stages, each [A_hi | A_lo | B_hi | B_lo]
    const uint32_t b_bytes = (uint32_t)NT * TC_KC * 4;
    const uint32_t stage_bytes = 2 * TC_A_BYTES + 2 * b_bytes;
    unsigned char* base = tc_raw + ((1024 - (smem_addr(tc_raw) & 1023)) & 1023);
    __shared__ uint64_t bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail, s_committed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* X = reinterpret_cast<const float*>(Xall + (size_t)blockIdx.z * n);
    float* Y = reinterpret_cast<float*>(Yall + (size_t)blockIdx.z * n);
    const int64_t Mtot = 2 * rows;
    const int64_t m0 = (int64_t)blockIdx.x * TC_M;
    const int n0 = blockIdx.y * NT;
    const int64_t ks = P == 1 ? 2 : 2 * P;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&s_tmem)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        s_committed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    // kind::tf32: D f32 (bits 4-5 = 1), A and B tf32 (bits 7-9, 10-12 = 2), both
    // K-major, N >> 3 at bit 17, M >> 4 at bit 24
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    const int nchunks = (N + TC_KC - 1) / TC_KC;
    const bool qvec = (N & 3) == 0;

    for (int c = 0; c < nchunks; ++c) {
        const int b = c % nst;
        unsigned char* st = base + (size_t)b * stage_bytes;
        float* Ahi = reinterpret_cast<float*>(st);
        float* Alo = reinterpret_cast<float*>(st + TC_A_BYTES);
        float* Bhi = reinterpret_cast<float*>(st + 2 * TC_A_BYTES);
        float* Blo = reinterpret_cast<float*>(st + 2 * TC_A_BYTES + b_bytes);
        // the MMAs of chunk c - nst read this stage: wait for their commit
        if (c >= nst && !bar_wait(&bar[b], (uint32_t)(((c - nst) / nst) & 1), err)) s_fail = 1;
        __syncthreads();
        if (s_fail) break;
        const int k0 = c * TC_KC;
        // A: item (row pair mp, 4 reduction indices k4), mp fastest; rows 2 mp and 2 mp + 1 are the
        // real and imaginary parts of one complex element
        for (int it = tid; it < (TC_M / 2) * (TC_KC / 4); it += TC_THREADS) {
            const int mp = it % (TC_M / 2), k4 = it / (TC_M / 2);
            const int64_t m = m0 + 2 * mp;
            float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
            if (m < Mtot) {
                const float* src = X + row_base(m, N, P);
                const int kb = k0 + 4 * k4;
                if (P == 1 && kb + 3 < N && ((reinterpret_cast<uintptr_t>(src + 2 * (int64_t)kb) & 15) == 0)) {
                    const float4 v0 = *reinterpret_cast<const float4*>(src + 2 * (int64_t)kb);
                    const float4 v1 = *reinterpret_cast<const float4*>(src + 2 * (int64_t)kb + 4);
                    re[0] = v0.x; im[0] = v0.y; re[1] = v0.z; im[1] = v0.w;
                    re[2] = v1.x; im[2] = v1.y; re[3] = v1.z; im[3] = v1.w;
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (kb + e < N) {
                            const float2 v = *reinterpret_cast<const float2*>(src + (int64_t)(kb + e) * ks);
                            re[e] = v.x;
                            im[e] = v.y;
                        }
                }
            }
            float4 h0, l0, h1, l1;
            h0.x = tf32_hi(re[0]); h0.y = tf32_hi(re[1]); h0.z = tf32_hi(re[2]); h0.w = tf32_hi(re[3]);
            h1.x = tf32_hi(im[0]); h1.y = tf32_hi(im[1]); h1.z = tf32_hi(im[2]); h1.w = tf32_hi(im[3]);
            l0 = make_float4(re[0] - h0.x, re[1] - h0.y, re[2] - h0.z, re[3] - h0.w);
            l1 = make_float4(im[0] - h1.x, im[1] - h1.y, im[2] - h1.z, im[3] - h1.w);
            const uint32_t o0 = tile_off(2 * mp, 4 * k4), o1 = tile_off(2 * mp + 1, 4 * k4);
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Ahi) + o0) = h0;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Alo) + o0) = l0;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Ahi) + o1) = h1;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Alo) + o1) = l1;
        }
        // B: item (output row nn, 4 reduction indices k4), nn fastest
        for (int it = tid; it < NT * (TC_KC / 4); it += TC_THREADS) {
            const int nn = it % NT, k4 = it / NT;
            const int kout = n0 + nn, kb = k0 + 4 * k4;
            float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
            if (kout < N) {
                const size_t q = (size_t)kout * N + kb;
                if (qvec && kb + 3 < N) {
                    h = *reinterpret_cast<const float4*>(Qhi + q);
                    l = *reinterpret_cast<const float4*>(Qlo + q);
                } else {
                    float hv[4] = {0.f, 0.f, 0.f, 0.f}, lv[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (kb + e < N) {
                            hv[e] = Qhi[q + e];
                            lv[e] = Qlo[q + e];
                        }
                    h = make_float4(hv[0], hv[1], hv[2], hv[3]);
                    l = make_float4(lv[0], lv[1], lv[2], lv[3]);
                }
            }
            const uint32_t o = tile_off(nn, 4 * k4);
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Bhi) + o) = h;
            *reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(Blo) + o) = l;
        }
        // the tensor cores read shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_addr(Ahi), al = smem_addr(Alo), bh = smem_addr(Bhi), bl = smem_addr(Blo);
#pragma unroll
            for (int kk = 0; kk < TC_KC / 8; ++kk) {
                const uint32_t o = (uint32_t)kk * 256;  // 8 reduction indices = 2 core matrices
                mma_tf32(tmem, kmajor_desc(ah + o), kmajor_desc(bh + o), idesc, (c > 0 || kk > 0) ? 1u : 0u);
                mma_tf32(tmem, kmajor_desc(ah + o), kmajor_desc(bl + o), idesc, 1u);
                mma_tf32(tmem, kmajor_desc(al + o), kmajor_desc(bh + o), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&bar[b]))
                         : "memory");
            s_committed = c + 1;
        }
    }
    // the last commit covers every MMA issued before it (also after a failed wait:
    // nothing leaves while its MMAs may still write the accumulator)
    __syncthreads();
    const int last = s_committed - 1;
    bool ok = !s_fail && last == nchunks - 1;
    if (last >= 0) ok = bar_wait(&bar[last % nst], (uint32_t)((last / nst) & 1), err) && ok;
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int quad = warp & 3, half = warp >> 2;
        const int64_t m = m0 + 32 * quad + lane;
        const int64_t rb = m < Mtot ? row_base(m, N, P) : 0;
        const int cb = half * (NT / 2), ce = cb + NT / 2;
        for (int c0 = cb; c0 < ce; c0 += 8) {
            uint32_t v[8];
            const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7])
                         : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < Mtot) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int kout = n0 + c0 + e;
                    if (kout < N) Y[rb + (int64_t)kout * ks] = __uint_as_float(v[e]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// Q = hi + lo with hi exact in TF32 (the leading 11 significand bits of the
// FP64 value rounded to FP32) and lo the FP32 remainder.
__global__ void k_sep_split(const double* Q64, int64_t NN, float* Qhi, float* Qlo) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= NN) return;
    const double q = Q64[t];
    const float h = tf32_hi((float)q);
    Qhi[t] = h;
    Qlo[t] = (float)(q - (double)h);
}

namespace {
int* g_tc_err = nullptr;
}

void sep_split_tables(const double* Q64, int N, float* Qhi, float* Qlo, cudaStream_t st) {
    const int64_t NN = (int64_t)N * N;
    k_sep_split<<<cdiv_up(NN, 256), 256, 0, st>>>(Q64, NN, Qhi, Qlo);
    SIM_LAUNCH_CHECK();
}

bool sep_mode_tc(const float2* cur, float2* nxt, const float* Qhi, const float* Qlo, int N, int64_t P, int64_t rows,
                 int64_t n, int na, cudaStream_t st) {
    if (N < 1 || na < 1 || rows < 1) return false;
    const int NT = N <= 256 ? ((N + 15) / 16) * 16 : 256;
    uint32_t tcols = 32;
    while ((int)tcols < NT) tcols <<= 1;
    const dim3 grid((unsigned)cdiv_up(2 * rows, TC_M), (unsigned)cdiv_up(N, NT), (unsigned)na);
    const int nst = (int64_t)grid.x * grid.y * grid.z >= 152 ? 1 : 2;
    const size_t smem = nst * (2 * (size_t)TC_A_BYTES + 2 * (size_t)NT * TC_KC * 4) + 1024;
    static size_t attr_set = 0;
    if (smem > attr_set) {
        SIM_CUDA(cudaFuncSetAttribute(k_sep_mode_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = smem;
    }
    if (!g_tc_err) {
        SIM_CUDA(cudaMalloc(&g_tc_err, sizeof(int)));
        SIM_CUDA(cudaMemset(g_tc_err, 0, sizeof(int)));
    }
    k_sep_mode_tc<<<grid, TC_THREADS, smem, st>>>(cur, nxt, Qhi, Qlo, N, P, rows, n, NT, tcols, nst, g_tc_err);
    SIM_LAUNCH_CHECK();
    return true;
}

}  // namespace sim
