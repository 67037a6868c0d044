// Block Thomas solve x = (A - σB)^{-1} r on a thread-block cluster.
//
// The factors of one shift are the dense T×T blocks Dinv_0..Dinv_{nb-1} and
// E_0..E_{nb-2} (krylov.cu).  The solve is a chain of 2nb-1 GEMVs,
//   forward   t_k = Dinv_k (r_k - L_k t_{k-1}),
//   backward  x_k = t_k - E_k x_{k+1},
// and only the vectors depend on the previous step — the matrices do not.  So
// each CTA of a cluster owns a slice of rows of every block, and a producer
// warp streams the slices, in chain order, through a ring of shared-memory
// stages (one 1-D bulk copy per row into a padded row, completing on the
// stage's "full" mbarrier) as far ahead as the ring allows; the consumers
// release a stage on its "empty" mbarrier.  Per step the eight consumer warps
// form the right-hand side, then for each chunk of rows run the GEMV with one
// row per lane (or a row per group of lanes) and a column range per warp, sum
// the warps' partials through shared memory, and send the new rows of the
// vector into every CTA's shared memory with st.async, which completes on the
// receiver's per-step mbarrier.  Up to R right-hand sides of the same shift
// share each pass over the matrices (the k random vectors of the
// multiplicity step).
//
// Every wait on an mbarrier has an iteration limit; a thread whose wait runs
// out records an error and the CTA stops computing and issuing copies, keeps
// taking part in its barriers (so no thread waits forever), and waits (again
// bounded) for its own copies in flight before it exits.
#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <vector>

#include "internal.h"
#include "solve_cluster.h"

namespace cg = cooperative_groups;

namespace sim {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// wait with cluster-scope acquire: the data arrived through st.async from other CTAs
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint32_t mapa_u32(const void* local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(local)), "r"(rank));
    return r;
}

// store one complex value into another CTA's shared memory; the bytes count
// against that CTA's mbarrier (addresses from mapa_u32)
__device__ __forceinline__ void st_async_c(uint32_t raddr, float2 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "f"(v.x), "f"(v.y), "r"(rbar)
                 : "memory");
}
__device__ __forceinline__ void st_async_c(uint32_t raddr, double2 v, uint32_t rbar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(raddr),
                 "d"(v.x), "d"(v.y), "r"(rbar)
                 : "memory");
}

constexpr long long WAIT_LIMIT = 1ll << 26;  // try_wait polls before a wait is declared failed

// Sum S values across the warp (S = 8 or 16): at each stage a lane keeps half
// of its values and trades the other half with its partner, so S-1 shuffles
// leave one partial per lane; the lanes below the value bits then finish with
// plain xor shuffles.  Afterwards lane L holds, in v[0], the warp sum of value
// (L >> (5 - log2 S)) & (S - 1).
template <class Rt, int S> __device__ __forceinline__ void butterfly(Rt (&v)[S], int lane) {
#pragma unroll
    for (int st = 0, width = S; width > 1; ++st, width >>= 1) {
        const int mask = 16 >> st;
        const bool upper = (lane & mask) != 0;
        const int half = width >> 1;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const Rt send = upper ? v[i] : v[i + half];
            const Rt keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
        }
    }
    constexpr int LOGS = S == 16 ? 4 : 3;
#pragma unroll
    for (int mask = (1 << (5 - LOGS)) >> 1; mask > 0; mask >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], mask);
}

template <class C> __device__ __forceinline__ C zero_c();
template <> __device__ __forceinline__ double2 zero_c<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zero_c<float2>() { return make_float2(0.f, 0.f); }


}  // namespace

// 16 bytes of complex values: two complex64 or one complex128
template <class C> struct Vec16;
template <> struct Vec16<float2> {
    using T = float4;
    static constexpr int N = 2;
    __device__ static __forceinline__ float2 get(const float4& v, int e) {
        return e == 0 ? make_float2(v.x, v.y) : make_float2(v.z, v.w);
    }
};
template <> struct Vec16<double2> {
    using T = double2;
    static constexpr int N = 1;
    __device__ static __forceinline__ double2 get(const double2& v, int) { return v; }
};

// two CTAs per SM for single right-hand sides in complex64 (see choose_shape)
constexpr bool kTwoPerSm = true;

constexpr int CL_WARPS = 8;                       // consumer warps: the GEMVs and the vector work
constexpr int CL_THREADS = (CL_WARPS + 1) * 32;   // + one producer warp that issues the copies

// barrier of the consumer warps only (the producer warp never joins it)
__device__ __forceinline__ void consumer_sync() {
    static_assert(CL_WARPS * 32 == 256, "named barrier thread count");
    asm volatile("bar.sync 1, 256;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool failed_flag(const int* f) { return *(const volatile int*)f != 0; }

// MINB: CTAs per SM the launch is built for (2 caps the registers at 112 so
// that two CTAs of at most ~112 KB of shared memory share an SM)
template <class C, int R, int MINB>
__global__ void __launch_bounds__(CL_THREADS, MINB) k_block_solve_cl(Pencil P, JobSpace js, int in_slot,
                                                                  int out_slot, void* const* fptrs,
                                                                  const int* grp_jobs, int SR, int NS, int TP,
                                                                  int* err) {
    cg::cluster_group cl = cg::this_cluster();
    const int Ccl = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int grp = blockIdx.x / Ccl;
    const int T = P.T, nb = P.nb;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    using VT = typename Vec16<C>::T;
    constexpr int VN = Vec16<C>::N;
    using Rt = decltype(zero_c<C>().x);

    // the group's job vectors (in shared memory: indexed by runtime job numbers)
    __shared__ const double2* s_in[R];
    __shared__ double2* s_out[R];
    __shared__ int s_fail;
    int nr = 0;
#pragma unroll
    for (int j = 0; j < R; ++j)
        if (grp_jobs[grp * R + j] >= 0) nr = j + 1;
    const int job0 = grp_jobs[grp * R];
    if (tid < R) {
        const int jb = grp_jobs[grp * R + tid];
        const int jj = jb >= 0 ? jb : job0;
        s_in[tid] = js.vec + (size_t)jj * js.vstride + (size_t)in_slot * js.n;
        s_out[tid] = js.vec + (size_t)jj * js.vstride + (size_t)out_slot * js.n;
    }
    const int s = js.d_jobshift[job0];
    const C* Dinv = reinterpret_cast<const C*>(fptrs[s]);
    const C* E = Dinv + (size_t)nb * T * T;
    const C* Lval = Dinv + factor_lval_offset(P);
    const C* L0val = Dinv + factor_l0_offset(P);

    const int Tc = (T + Ccl - 1) / Ccl;
    const int r0 = min(T, q * Tc), r1 = min(T, r0 + Tc);
    const int myrows = r1 - r0;
    const int nsub = (myrows + SR - 1) / SR;
    const int total = (2 * nb - 1) * nsub;

    extern __shared__ __align__(128) unsigned char raw[];
    C* stage = reinterpret_cast<C*>(raw);                  // [NS][SR][TP]: rows padded to TP
    C* vbuf = stage + (size_t)NS * SR * TP;                // [3][R][T]: the chain's vectors
    C* sbuf = vbuf + (size_t)3 * R * T;                    // [R][T]
    C* tbuf = sbuf + (size_t)R * T;                        // [R][T]: t_k rows of this CTA (backward)
    C* red = tbuf + (size_t)R * T;                         // [2][warps][R][SR]: per-warp partial sums
    uint64_t* full = reinterpret_cast<uint64_t*>(red + (size_t)2 * CL_WARPS * R * SR);  // [NS] stage filled
    uint64_t* empty = full + NS;                                                         // [NS] stage consumed
    uint64_t* vbar = empty + NS;                                                         // [3] vector received

    if (tid == 0) {
        s_fail = 0;
        for (int i = 0; i < NS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 3; ++i) mbar_init(&vbar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t vec_bytes = (uint32_t)((size_t)T * nr * sizeof(C));  // one step's vector, all rows
    if (tid == 0)
        for (int i = 0; i < 3 && i <= 2 * nb - 3; ++i) mbar_expect_tx(&vbar[i], vec_bytes);  // steps 0, 1, 2
    cl.sync();  // every CTA of the cluster is running, barriers initialised and armed, before any remote store

    if (warp == CL_WARPS) {
        // ---- producer: chunk c = up to SR rows of one block, one 1-D bulk copy
        // per row into its padded row of stage c % NS, once that stage is consumed
        int c = 0;
        for (; c < total; ++c) {
            const int slot = c % NS;
            int ok = 1;
            if (lane == 0) {
                if (c >= NS) {
                    const uint32_t par = (uint32_t)(((c / NS) - 1) & 1);
                    long long it = 0;
                    while (!mbar_try_wait(&empty[slot], par)) {
                        if (failed_flag(&s_fail)) {
                            ok = 0;
                            break;
                        }
                        if (++it > WAIT_LIMIT) {
                            s_fail = 1;
                            atomicExch(err, 4);
                            ok = 0;
                            break;
                        }
                    }
                }
                if (failed_flag(&s_fail)) ok = 0;
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            const int b = c / nsub, sub = c % nsub;
            const int rs = r0 + sub * SR;
            const int rows = min(SR, r1 - rs);
            const C* M = (b < nb ? Dinv + (size_t)b * T * T : E + (size_t)(2 * nb - 2 - b) * T * T) + (size_t)rs * T;
            C* dst = stage + (size_t)slot * SR * TP;
            if (lane == 0) mbar_expect_tx(&full[slot], (uint32_t)((size_t)rows * T * sizeof(C)));
            __syncwarp();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int i = lane; i < rows; i += 32)
                tma_load_1d(dst + (size_t)i * TP, M + (size_t)i * T, (uint32_t)(T * sizeof(C)), &full[slot]);
        }
        // stopped early (a failure): the last issued copies may still be in flight,
        // and this CTA's shared memory must outlive them
        if (lane == 0 && c < total) {
            for (int d = max(0, c - NS); d < c; ++d) {
                long long it = 0;
                while (!mbar_try_wait(&full[d % NS], (uint32_t)((d / NS) & 1)) && ++it < WAIT_LIMIT) {
                }
            }
        }
    } else {
        // ---- consumers
        // Prefetch of the next step's chain-independent inputs, one row per
        // thread, kept as loaded (no arithmetic on them until they are used):
        // r_k and the row's couplings (forward), t_k of this CTA's rows (backward).
        const bool pf_ok = T <= CL_WARPS * 32;
        double2 pf_v[R];
        int pf_lo = 0, pf_hi = 0, pf_c = 0;
        C pf_a = zero_c<C>();
        auto prefetch_fwd = [&](int kk) {
            const int64_t g = (int64_t)kk * T + tid;
            if (tid < T) {
                const bool in = g < P.n;
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (j < nr) pf_v[j] = in ? s_in[j][g] : make_double2(0.0, 0.0);
                if (in) {
                    pf_lo = P.Lptr[g];
                    pf_hi = P.Lptr[g + 1];
                    pf_c = P.L0col[g];
                    pf_a = L0val[g];
                } else {
                    pf_lo = pf_hi = 0;
                }
            }
        };
        auto prefetch_bwd = [&](int kk) {
            const int64_t g = (int64_t)kk * T + r0 + tid;
            if (tid < myrows) {
#pragma unroll
                for (int j = 0; j < R; ++j)
                    if (j < nr) pf_v[j] = g < P.n ? s_out[j][g] : make_double2(0.0, 0.0);
            }
        };
        if (pf_ok) prefetch_fwd(0);

        // this warp's 16-byte column units of every row
        const int U = T / VN;
        const int u0 = (warp * U) / CL_WARPS, u1 = ((warp + 1) * U) / CL_WARPS;

        int chunk = 0;
        for (int b = 0; b < 2 * nb - 1; ++b) {
            const bool fwd = b < nb;
            const int k = fwd ? b : 2 * nb - 2 - b;
            const int64_t g0 = (int64_t)k * T;
            const int cur = b % 3, prv = (b + 2) % 3;
            const C* vprev = vbuf + (size_t)prv * R * T;  // t_{k-1} (fwd) or x_{k+1} (bwd)
            const bool last = b == 2 * nb - 2;            // nobody reads the last vector: not sent
            if (b > 0 && !failed_flag(&s_fail)) {
                // the previous step's vector: every CTA's rows, delivered by st.async
                const uint32_t par = (uint32_t)(((b - 1) / 3) & 1);
                long long it = 0;
                while (!mbar_try_wait_cluster(&vbar[prv], par)) {
                    if (failed_flag(&s_fail)) break;
                    if (++it > WAIT_LIMIT) {
                        s_fail = 1;
                        atomicExch(err, 3);
                        break;
                    }
                }
            }
            consumer_sync();  // also: the previous step's reads of sbuf and tbuf are done
            // re-arm that barrier for step b+2 now: no CTA can send step b+2's rows
            // before it has ours of step b+1, so the expected bytes are always
            // registered before the first of them arrives
            if (tid == 0 && b > 0 && !failed_flag(&s_fail) && b + 2 <= 2 * nb - 3)
                mbar_expect_tx(&vbar[prv], vec_bytes);
            const bool failed = failed_flag(&s_fail);
            if (fwd) {
                // s_k = r_k - L_k t_{k-1}: every CTA forms the whole block
                if (failed) {
                } else if (pf_ok) {
                    if (tid < T) {
                        const int i = tid;
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (j >= nr) break;
                            C v = from_c128<C>(pf_v[j]);
                            if (pf_hi > pf_lo) {
                                const C tt = vprev[(size_t)j * T + pf_c];
                                v.x -= pf_a.x * tt.x - pf_a.y * tt.y;
                                v.y -= pf_a.x * tt.y + pf_a.y * tt.x;
                                for (int e = pf_lo + 1; e < pf_hi; ++e) {
                                    const C a = Lval[e];
                                    const C t2 = vprev[(size_t)j * T + P.Lcol[e]];
                                    v.x -= a.x * t2.x - a.y * t2.y;
                                    v.y -= a.x * t2.y + a.y * t2.x;
                                }
                            }
                            sbuf[(size_t)j * T + i] = v;
                        }
                    }
                    if (k + 1 < nb) prefetch_fwd(k + 1);
                    else prefetch_bwd(nb - 2 >= 0 ? nb - 2 : 0);
                } else {
                    for (int idx = tid; idx < T * nr; idx += CL_WARPS * 32) {
                        const int i = idx % T, j = idx / T;
                        const int64_t g = g0 + i;
                        C v = zero_c<C>();
                        if (g < P.n) {
                            v = from_c128<C>(s_in[j][g]);
                            const int e0 = P.Lptr[g], e1 = P.Lptr[g + 1];
                            for (int e = e0; e < e1; ++e) {
                                const C a = Lval[e];
                                const C t = vprev[(size_t)j * T + P.Lcol[e]];
                                v.x -= a.x * t.x - a.y * t.y;
                                v.y -= a.x * t.y + a.y * t.x;
                            }
                        }
                        sbuf[(size_t)j * T + i] = v;
                    }
                }
                consumer_sync();
            }
            const C* rhs = fwd ? sbuf : vprev;
            if (!fwd && !failed) {
                // t_k of this CTA's rows, for x_k = t_k - E_k x_{k+1} (read after the next barrier)
                if (pf_ok) {
                    if (tid < myrows) {
#pragma unroll
                        for (int j = 0; j < R; ++j)
                            if (j < nr) tbuf[(size_t)j * T + tid] = from_c128<C>(pf_v[j]);
                    }
                    if (k > 0) prefetch_bwd(k - 1);
                } else {
                    for (int idx = tid; idx < myrows * nr; idx += CL_WARPS * 32) {
                        const int i = idx % myrows, j = idx / myrows;
                        const int64_t g = g0 + r0 + i;
                        tbuf[(size_t)j * T + i] = g < P.n ? from_c128<C>(s_out[j][g]) : zero_c<C>();
                    }
                }
            }
            for (int sub = 0; sub < nsub; ++sub, ++chunk) {
                const int slot = chunk % NS;
                C* rbuf = red + (size_t)(chunk & 1) * CL_WARPS * R * SR;
                if (!failed_flag(&s_fail)) {
                    const uint32_t par = (uint32_t)((chunk / NS) & 1);
                    long long it = 0;
                    while (!mbar_try_wait(&full[slot], par)) {
                        if (failed_flag(&s_fail)) break;
                        if (++it > WAIT_LIMIT) {
                            s_fail = 1;
                            atomicExch(err, 2);
                            break;
                        }
                    }
                }
                const int rs = r0 + sub * SR;
                const int rows = min(SR, r1 - rs);
                // warp-uniform test: the GEMV's shuffles need every lane, and the
                // flag can change under a warp's feet (the producer sets it too)
                if (__all_sync(0xffffffffu, !failed_flag(&s_fail))) {
                    // lane = row r (of SRp, the power of two >= rows) + SRp * column phase cp
                    int lg = 0;
                    while ((1 << lg) < rows) ++lg;
                    const int SRp = 1 << lg;
                    const int CP = 32 >> lg;
                    const int r = lane & (SRp - 1), cp = lane >> lg;
                    Rt acc[2 * R];
#pragma unroll
                    for (int v = 0; v < 2 * R; ++v) acc[v] = Rt(0);
                    auto mac = [&](const VT& mv, const VT (&xv)[R]) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
#pragma unroll
                            for (int e = 0; e < VN; ++e) {
                                const C m = Vec16<C>::get(mv, e), x = Vec16<C>::get(xv[j], e);
                                acc[2 * j] = fma(m.x, x.x, acc[2 * j]);
                                acc[2 * j] = fma(-m.y, x.y, acc[2 * j]);
                                acc[2 * j + 1] = fma(m.x, x.y, acc[2 * j + 1]);
                                acc[2 * j + 1] = fma(m.y, x.x, acc[2 * j + 1]);
                            }
                        }
                    };
                    if (r < rows) {
                        const VT* Mrow = reinterpret_cast<const VT*>(stage + ((size_t)slot * SR + r) * TP);
                        const VT* X = reinterpret_cast<const VT*>(rhs);  // unit u of job j at X[j * U + u]
                        int u = u0 + cp;
                        if constexpr (sizeof(C) == 8) {
                            // complex64: the next unit's operands load while this one's FMAs run.
                            // Packed FP32 pairs: pa_j += (m.x, m.x) * (x.x, x.y) and
                            // pb_j += (m.y, m.y) * (x.x, x.y), so that m x = (pa.x - pb.y, pa.y + pb.x):
                            // two paired FMAs per complex product instead of four scalar ones
                            float2 pa[R], pb[R];
#pragma unroll
                            for (int j = 0; j < R; ++j) pa[j] = pb[j] = make_float2(0.f, 0.f);
                            auto mac2 = [&](const VT& mv, const VT (&xv)[R]) {
#pragma unroll
                                for (int e = 0; e < VN; ++e) {
                                    const C m = Vec16<C>::get(mv, e);
                                    const float2 mr = make_float2(m.x, m.x), mi = make_float2(m.y, m.y);
#pragma unroll
                                    for (int j = 0; j < R; ++j) {
                                        const C x = Vec16<C>::get(xv[j], e);
                                        const float2 xx = make_float2(x.x, x.y);
                                        pa[j] = __ffma2_rn(mr, xx, pa[j]);
                                        pb[j] = __ffma2_rn(mi, xx, pb[j]);
                                    }
                                }
                            };
                            if (u < u1) {
                                VT mv = Mrow[u];
                                VT xv[R];
#pragma unroll
                                for (int j = 0; j < R; ++j) xv[j] = X[(size_t)j * U + u];
                                while (true) {
                                    const int un = u + CP;
                                    const bool more = un < u1;
                                    VT mn = mv;
                                    VT xn[R];
#pragma unroll
                                    for (int j = 0; j < R; ++j) xn[j] = xv[j];
                                    if (more) {
                                        mn = Mrow[un];
#pragma unroll
                                        for (int j = 0; j < R; ++j) xn[j] = X[(size_t)j * U + un];
                                    }
                                    mac2(mv, xv);
                                    if (!more) break;
                                    mv = mn;
#pragma unroll
                                    for (int j = 0; j < R; ++j) xv[j] = xn[j];
                                    u = un;
                                }
                            }
#pragma unroll
                            for (int j = 0; j < R; ++j) {
                                acc[2 * j] = pa[j].x - pb[j].y;
                                acc[2 * j + 1] = pa[j].y + pb[j].x;
                            }
                        } else {
                            for (; u < u1; u += CP) {
                                const VT mv = Mrow[u];
                                VT xv[R];
#pragma unroll
                                for (int j = 0; j < R; ++j) xv[j] = X[(size_t)j * U + u];
                                mac(mv, xv);
                            }
                        }
                    }
                    // sum the column phases of each row
                    for (int mask = 16; mask >= SRp; mask >>= 1) {
#pragma unroll
                        for (int v = 0; v < 2 * R; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], mask);
                    }
                    if (cp == 0 && r < rows) {
#pragma unroll
                        for (int j = 0; j < R; ++j) {
                            if (j < nr) {
                                C v;
                                v.x = acc[2 * j];
                                v.y = acc[2 * j + 1];
                                rbuf[((size_t)warp * R + j) * SR + r] = v;
                            }
                        }
                    }
                }
                consumer_sync();  // partial sums written; the stage is consumed
                if (tid == 0) mbar_arrive(&empty[slot]);
                if (!failed_flag(&s_fail)) {
                    // one thread per (row, job): sum the warps' partials, store, broadcast
                    for (int t = tid; t < rows * nr; t += CL_WARPS * 32) {
                        const int r = t % rows, j = t / rows;
                        C v = rbuf[(size_t)j * SR + r];
#pragma unroll
                        for (int w = 1; w < CL_WARPS; ++w) {
                            const C p = rbuf[((size_t)w * R + j) * SR + r];
                            v.x += p.x;
                            v.y += p.y;
                        }
                        const int rr = rs + r;
                        const int64_t g = g0 + rr;
                        if (!fwd) v = csub(tbuf[(size_t)j * T + (rr - r0)], v);
                        // send first: the peers wait for these rows, nobody here waits for the store
                        if (!last) {
                            C* loc = vbuf + (size_t)cur * R * T + (size_t)j * T + rr;
                            for (int qq = 0; qq < Ccl; ++qq)
                                st_async_c(mapa_u32(loc, qq), v, mapa_u32(&vbar[cur], qq));
                        }
                        if (g < P.n) s_out[j][g] = to_c128(v);
                    }
                }
            }
        }
    }
    // the cluster barrier keeps every CTA's shared memory alive until all peers
    // have finished sending into it
    cl.sync();
}

// ---------------------------------------------------------------------------
namespace {

struct Plan {
    int R = 1, SR = 1, NS = 3, TP = 1;
    size_t smem = 0;
};

// Row stride (complex values) of a stage in shared memory: a whole number of
// 16-byte units, and an odd one, so that the 16-byte loads of 8 consecutive
// rows at the same column fall in distinct bank groups.
int padded_row(int T, size_t cs) {
    int TP = T;
    while ((TP * cs) % 16 != 0 || ((TP * cs / 16) & 1) == 0) ++TP;
    return TP;
}

size_t plan_smem(const Plan& p, int T, size_t cs) {
    return (size_t)p.NS * p.SR * p.TP * cs + (size_t)5 * p.R * T * cs + (size_t)2 * CL_WARPS * p.R * p.SR * cs +
           (2 * p.NS + 3) * sizeof(uint64_t) + 16;
}

// Largest R (right-hand sides per pass) and stage height SR that fit in
// `budget` bytes of shared memory.
bool make_plan(int T, size_t cs, int want_R, Plan& p, size_t budget = 220 * 1024) {
    const int TP = padded_row(T, cs);
    for (int R : {8, 4, 2, 1}) {
        if (R > want_R && R != 1) continue;
        const size_t vec = (size_t)5 * R * T * cs;
        if (vec + 96 >= budget) continue;
        const int NS = 3;
        const size_t per_row = (size_t)NS * TP * cs + (size_t)2 * CL_WARPS * R * cs;
        const int SR = (int)std::min<size_t>(32, (budget - vec - 96) / per_row);
        if (SR < 1) continue;
        p.R = R;
        p.SR = SR;
        p.NS = NS;
        p.TP = TP;
        p.smem = plan_smem(p, T, cs);
        return true;
    }
    return false;
}

// Stage height for a CTA of Tc rows: each chunk of `rows` rows occupies the
// lanes as rows x column phases with rows padded to a power of two, so the
// estimate charges the padded rows' multiply-adds (FP32: 4 warp-instructions a clock per SM,
// FP64: one per 16 clocks) plus a fixed cost per chunk (its waits, barrier and
// epilogue, about 2 us).
int choose_rows(int Tc, int SRmax, int T, size_t cs, int R) {
    const int VN = (int)(16 / cs);
    const int Uw = (T / VN + CL_WARPS - 1) / CL_WARPS;
    const double per_fma = cs == 16 ? 16.0 : 0.25;
    int best = SRmax;
    double best_c = 1e300;
    for (int SR = 1; SR <= SRmax; ++SR) {
        double c = 0.0;
        for (int a = 0; a < Tc; a += SR) {
            const int rows = std::min(SR, Tc - a);
            int SRp = 1;
            while (SRp < rows) SRp <<= 1;
            const int CP = 32 / SRp;
            c += (double)((Uw + CP - 1) / CP) * R * VN * 4 * CL_WARPS * per_fma + 4000.0;
        }
        if (c < best_c) {
            best_c = c;
            best = SR;
        }
    }
    return best;
}

template <class C, int R, int MINB> void set_smem_attr(size_t smem) {
    static size_t attr_set = 0;  // per instantiation
    static bool nonportable = false;
    if (!nonportable) {
        // clusters of up to 16 CTAs (beyond the portable 8) for launches of few groups
        // (where that is refused, the occupancy query reports no room for them)
        if (cudaFuncSetAttribute(k_block_solve_cl<C, R, MINB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
            (void)cudaGetLastError();
        nonportable = true;
    }
    if (smem > attr_set) {
        SIM_CUDA(cudaFuncSetAttribute(k_block_solve_cl<C, R, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        attr_set = smem;
    }
}

cudaLaunchConfig_t cluster_config(int ngroups, int Ccl, size_t smem, cudaStream_t st, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ngroups * Ccl);
    cfg.blockDim = dim3(CL_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Ccl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// How many clusters of Ccl CTAs with `smem` bytes each the GPU holds at once
// (the CUDA occupancy query: clusters are placed within a GPC, so this is not
// simply SMs / Ccl).  Cached per (instantiation, Ccl, smem).
template <class C, int R, int MINB> int max_active_clusters(int Ccl, size_t smem) {
    static std::map<std::pair<int, size_t>, int> cache;
    const auto key = std::make_pair(Ccl, smem);
    const auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    set_smem_attr<C, R, MINB>(smem);
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config(1, Ccl, smem, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_block_solve_cl<C, R, MINB>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        n = 0;
    }
    cache[key] = n;
    return n;
}

template <class C, int R, int MINB>
void launch_cl(const Pencil& P, const JobSpace& js, int in_slot, int out_slot, void* const* fptrs, const int* d_grp,
               int ngroups, int Ccl, const Plan& pl, int* d_err, cudaStream_t st) {
    set_smem_attr<C, R, MINB>(pl.smem);
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config(ngroups, Ccl, pl.smem, st, attr);
    SIM_CUDA(cudaLaunchKernelEx(&cfg, k_block_solve_cl<C, R, MINB>, P, js, in_slot, out_slot, fptrs, d_grp, pl.SR,
                                pl.NS, pl.TP, d_err));
    SIM_LAUNCH_CHECK();
}

// Launch shape: CTAs per group (cluster size), CTAs per SM, and the plan.
struct Shape {
    int Ccl = 1, minb = 1;
    Plan pl;
};

// The shape of a launch of ng groups: every group in one wave if the GPU holds
// that many clusters, and then the largest cluster (the most SMs, the fewest
// rows per CTA on the chain's critical path); cluster sizes need not be powers
// of two.  Two CTAs per SM are considered for single right-hand sides in
// complex64, whose plan then fits in half of an SM's shared memory.
template <class C, int R>
Shape choose_shape(const Pencil& P, size_t cs, const Plan& base, int ng) {
    Shape best;
    double best_cost = 1e300;
    const int cmax = std::min(16, P.T);
    for (int minb = 1; minb <= 2; ++minb) {
        if (minb == 2 && !(kTwoPerSm && R == 1 && sizeof(C) == 8)) continue;
        Plan pl = base;
        if (minb == 2 && !make_plan(P.T, cs, R, pl, 110 * 1024)) continue;
        for (int c = 1; c <= cmax; ++c) {
            Plan q = pl;
            q.SR = choose_rows((P.T + c - 1) / c, pl.SR, P.T, cs, pl.R);
            q.smem = plan_smem(q, P.T, cs);
            int maxc = 0;
            if constexpr (R == 1 && sizeof(C) == 8)
                maxc = minb == 1 ? max_active_clusters<C, R, 1>(c, q.smem) : max_active_clusters<C, R, 2>(c, q.smem);
            else
                maxc = max_active_clusters<C, R, 1>(c, q.smem);
            if (maxc <= 0) continue;
            const int waves = (ng + maxc - 1) / maxc;
            // waves first, then the fewest rows per CTA, then one CTA per SM
            const double cost = waves * 1e6 + (double)((P.T + c - 1) / c) * 10.0 + minb;
            if (cost < best_cost) {
                best_cost = cost;
                best.Ccl = c;
                best.minb = minb;
                best.pl = q;
            }
        }
    }
    if (best_cost == 1e300) {  // no occupancy answer: one CTA per group
        best.Ccl = 1;
        best.minb = 1;
        best.pl = base;
        best.pl.SR = choose_rows(P.T, base.SR, P.T, cs, base.R);
        best.pl.smem = plan_smem(best.pl, P.T, cs);
    }
    return best;
}

int* g_err = nullptr;
int* g_grp = nullptr;
int g_grp_cap = 0;
// pinned staging for the group table: a pageable upload would synchronise the stream
int* g_grp_h[2] = {nullptr, nullptr};
cudaEvent_t g_grp_ev[2] = {nullptr, nullptr};
int g_grp_h_cap = 0;
int g_grp_flip = 0;

}  // namespace

bool block_solve_cluster(const Pencil& P, int precision, const JobSpace& js, const std::vector<int>& active,
                         int in_slot, int out_slot, const double2* d_sigma, void* const* d_factor_ptrs,
                         cudaStream_t st) {
    if (active.empty()) return true;
    const size_t cs = precision == SIM_FP64 ? sizeof(double2) : sizeof(float2);
    if ((P.T * cs) % 16 != 0) return false;
    // group active jobs that share a shift (consecutive in the active list)
    std::vector<std::vector<int>> groups;
    int maxr = 1;
    for (size_t i = 0; i < active.size(); ++i) {
        const int j = active[i];
        if (!groups.empty() && js.h_jobshift[groups.back().back()] == js.h_jobshift[j] && groups.back().size() < 8)
            groups.back().push_back(j);
        else
            groups.push_back({j});
        maxr = std::max<int>(maxr, (int)groups.back().size());
    }
    Plan pl;
    if (!make_plan(P.T, cs, maxr, pl)) return false;
    // split groups larger than the plan's R
    std::vector<std::vector<int>> gs;
    for (auto& g : groups)
        for (size_t a = 0; a < g.size(); a += pl.R) gs.emplace_back(g.begin() + a, g.begin() + std::min(g.size(), a + pl.R));
    const int ng = (int)gs.size();
    std::vector<int> flat((size_t)ng * pl.R, -1);
    for (int g = 0; g < ng; ++g)
        for (size_t j = 0; j < gs[g].size(); ++j) flat[(size_t)g * pl.R + j] = gs[g][j];
    if (!g_err) {
        SIM_CUDA(cudaMalloc(&g_err, sizeof(int)));
        SIM_CUDA(cudaMemset(g_err, 0, sizeof(int)));
    }
    if ((int)flat.size() > g_grp_cap) {
        if (g_grp) {
            SIM_CUDA(cudaStreamSynchronize(st));
            cudaFree(g_grp);
        }
        g_grp_cap = (int)flat.size() * 2;
        SIM_CUDA(cudaMalloc(&g_grp, sizeof(int) * g_grp_cap * 2));
    }
    if ((int)flat.size() > g_grp_h_cap) {
        for (int b = 0; b < 2; ++b) {
            if (g_grp_ev[b]) SIM_CUDA(cudaEventSynchronize(g_grp_ev[b]));
            if (g_grp_h[b]) cudaFreeHost(g_grp_h[b]);
            SIM_CUDA(cudaMallocHost(&g_grp_h[b], sizeof(int) * flat.size() * 2));
            if (!g_grp_ev[b]) SIM_CUDA(cudaEventCreateWithFlags(&g_grp_ev[b], cudaEventDisableTiming));
        }
        g_grp_h_cap = (int)flat.size() * 2;
    }
    const int fb = g_grp_flip;
    g_grp_flip ^= 1;
    SIM_CUDA(cudaEventSynchronize(g_grp_ev[fb]));  // the copy that last used this buffer is done
    std::copy(flat.begin(), flat.end(), g_grp_h[fb]);
    int* d_grp = g_grp + (size_t)fb * g_grp_cap;
    SIM_CUDA(cudaMemcpyAsync(d_grp, g_grp_h[fb], sizeof(int) * flat.size(), cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaEventRecord(g_grp_ev[fb], st));
    Shape sh;
    if (precision == SIM_FP64) {
        if (pl.R == 8) sh = choose_shape<double2, 8>(P, cs, pl, ng);
        else if (pl.R == 4) sh = choose_shape<double2, 4>(P, cs, pl, ng);
        else if (pl.R == 2) sh = choose_shape<double2, 2>(P, cs, pl, ng);
        else sh = choose_shape<double2, 1>(P, cs, pl, ng);
    } else {
        if (pl.R == 8) sh = choose_shape<float2, 8>(P, cs, pl, ng);
        else if (pl.R == 4) sh = choose_shape<float2, 4>(P, cs, pl, ng);
        else if (pl.R == 2) sh = choose_shape<float2, 2>(P, cs, pl, ng);
        else sh = choose_shape<float2, 1>(P, cs, pl, ng);
    }
    const int Ccl = sh.Ccl;
    pl = sh.pl;
    const double TT = (double)P.T * P.T, blocks = 2.0 * P.nb - 1.0;
    // instrumentation also files each launch under its shape (right-hand sides
    // per pass, CTAs per group), e.g. "block_solve_r8_c2"
    char shape[40];
    snprintf(shape, sizeof shape, "block_solve_r%d_c%d%s", pl.R, Ccl, sh.minb == 2 ? "x2" : "");
    kprof_begin("block_solve", st);
    kprof_begin(shape, st);
#define SIM_LAUNCH_R(CT, RR, MB) \
    launch_cl<CT, RR, MB>(P, js, in_slot, out_slot, d_factor_ptrs, d_grp, ng, Ccl, pl, g_err, st)
    if (precision == SIM_FP64) {
        if (pl.R == 8) SIM_LAUNCH_R(double2, 8, 1);
        else if (pl.R == 4) SIM_LAUNCH_R(double2, 4, 1);
        else if (pl.R == 2) SIM_LAUNCH_R(double2, 2, 1);
        else SIM_LAUNCH_R(double2, 1, 1);
    } else {
        if (pl.R == 8) SIM_LAUNCH_R(float2, 8, 1);
        else if (pl.R == 4) SIM_LAUNCH_R(float2, 4, 1);
        else if (pl.R == 2) SIM_LAUNCH_R(float2, 2, 1);
        else if (sh.minb == 2) SIM_LAUNCH_R(float2, 1, 2);
        else SIM_LAUNCH_R(float2, 1, 1);
    }
#undef SIM_LAUNCH_R
    // algorithmic bytes: each group reads the factor once, and 4 vectors per job
    const double alg_bytes = ng * blocks * TT * cs + (double)active.size() * 4.0 * P.n * sizeof(double2);
    const double alg_flops = (double)active.size() * 8.0 * blocks * TT;
    kprof_end(shape, st, alg_bytes, alg_flops);
    kprof_end("block_solve", st, alg_bytes, alg_flops);
    return true;
}

int block_solve_error() {
    if (!g_err) return 0;
    int e = 0;
    cudaMemcpy(&e, g_err, sizeof(int), cudaMemcpyDeviceToHost);
    return e;
}

}  // namespace sim
