// Block Thomas solve x = (A - σB)^{-1} r on a thread-block cluster.
//
// The factors of one shift are the dense T×T blocks Dinv_0..Dinv_{nb-1} and
// E_0..E_{nb-2} (krylov.cu).  The solve is a chain of 2nb-1 GEMVs,
//   forward   t_k = Dinv_k (r_k - L_k t_{k-1}),
//   backward  x_k = t_k - E_k x_{k+1},
// and only the vectors depend on the previous step — the matrices do not.  So
// each CTA of a cluster owns a slice of rows of every block and streams its
// slices, in chain order, through a ring of shared-memory stages with 1-D TMA
// bulk copies (cp.async.bulk + mbarrier), as far ahead as the ring allows.  The
// per-step work is then a GEMV out of shared memory; the CTA broadcasts its
// rows of the new vector to every CTA of the cluster through distributed
// shared memory and one cluster barrier closes the step.  Up to R right-hand
// sides of the same shift share each pass over the matrices (the k random
// vectors of the multiplicity step).
//
// Every wait on an mbarrier has an iteration limit; a CTA whose wait runs out
// records an error, stops computing and issuing copies, keeps taking part in
// the cluster barriers (so no CTA waits forever), and waits (again bounded)
// for its own copies in flight before it exits.
#include <cooperative_groups.h>

#include <algorithm>
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

template <class C, int R>
__global__ void __launch_bounds__(256, 1) k_block_solve_cl(Pencil P, JobSpace js, int in_slot, int out_slot,
                                                        const double2* sigma, void* const* fptrs,
                                                        const int* grp_jobs, int SR, int NS, int* err) {
    cg::cluster_group cl = cg::this_cluster();
    const int Ccl = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int grp = blockIdx.x / Ccl;
    const int T = P.T, nb = P.nb;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

    int jb[R];
    int nr = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        jb[j] = grp_jobs[grp * R + j];
        if (jb[j] >= 0) nr = j + 1;
    }
    const int s = js.d_jobshift[jb[0]];
    const C* Dinv = reinterpret_cast<const C*>(fptrs[s]);
    const C* E = Dinv + (size_t)nb * T * T;
    const C* Lval = Dinv + factor_lval_offset(P);

    const int Tc = (T + Ccl - 1) / Ccl;
    const int r0 = min(T, q * Tc), r1 = min(T, r0 + Tc);
    const int myrows = r1 - r0;
    const int nsub = (myrows + SR - 1) / SR;
    const int total = (2 * nb - 1) * nsub;

    extern __shared__ __align__(128) unsigned char raw[];
    C* stage = reinterpret_cast<C*>(raw);                       // [NS][SR*T]
    C* vbuf = stage + (size_t)NS * SR * T;                      // [3][R][T]: the chain's vectors
    C* sbuf = vbuf + (size_t)3 * R * T;                         // [R][T]
    C* tbuf = sbuf + (size_t)R * T;                              // [R][T]: t_k rows of this CTA (backward)
    uint64_t* bars = reinterpret_cast<uint64_t*>(tbuf + (size_t)R * T);  // [NS] stage barriers
    uint64_t* vbar = bars + NS;                                           // [3] vector barriers
    __shared__ int s_fail;

    auto chunk_src = [&](int c, uint32_t& bytes) -> const C* {
        const int b = c / nsub, sub = c % nsub;
        const int rs = r0 + sub * SR;
        const int rows = min(SR, r1 - rs);
        bytes = (uint32_t)((size_t)rows * T * sizeof(C));
        const C* M = b < nb ? Dinv + (size_t)b * T * T : E + (size_t)(2 * nb - 2 - b) * T * T;
        return M + (size_t)rs * T;
    };

    if (tid == 0) {
        s_fail = 0;
        for (int i = 0; i < NS; ++i) mbar_init(&bars[i], 1);
        for (int i = 0; i < 3; ++i) mbar_init(&vbar[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0) {
        for (; issued < min(NS, total); ++issued) {
            uint32_t bytes;
            const C* src = chunk_src(issued, bytes);
            mbar_expect_tx(&bars[issued], bytes);
            tma_load_1d(stage + (size_t)issued * SR * T, src, bytes, &bars[issued]);
        }
    }
    const uint32_t vec_bytes = (uint32_t)((size_t)T * nr * sizeof(C));  // one step's vector, all rows
    if (tid == 0)
        for (int i = 0; i < 3 && i <= 2 * nb - 3; ++i) mbar_expect_tx(&vbar[i], vec_bytes);  // steps 0, 1, 2
    cl.sync();  // every CTA of the cluster is running, barriers initialised and armed, before any remote store

    const double2* in[R];
    double2* out[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const int jj = jb[j] >= 0 ? jb[j] : jb[0];
        in[j] = js.vec + (size_t)jj * js.vstride + (size_t)in_slot * js.n;
        out[j] = js.vec + (size_t)jj * js.vstride + (size_t)out_slot * js.n;
    }

    // Register prefetch of the next step's chain-independent inputs: r_k and
    // the first coupling of each row (forward), t_k of this CTA's rows (backward).
    constexpr int PFN = 8;
    const bool pf_ok = T * nr <= PFN * (int)blockDim.x;
    C pf_v[PFN], pf_a[PFN];
    int pf_c[PFN], pf_n[PFN];
    auto prefetch_fwd = [&](int kk) {
        const int64_t gg0 = (int64_t)kk * T;
#pragma unroll
        for (int t = 0; t < PFN; ++t) {
            const int idx = tid + t * (int)blockDim.x;
            pf_n[t] = -1;
            if (idx < T * nr) {
                const int i = idx % T, j = idx / T;
                const int64_t g = gg0 + i;
                if (g < P.n) {
                    pf_v[t] = from_c128<C>(in[j][g]);
                    const int e0 = P.Lptr[g], e1 = P.Lptr[g + 1];
                    pf_n[t] = e1 - e0;
                    if (e1 > e0) {
                        pf_c[t] = P.Lcol[e0];
                        pf_a[t] = Lval[e0];
                    }
                } else {
                    pf_n[t] = -2;
                }
            }
        }
    };
    auto prefetch_bwd = [&](int kk) {
        const int64_t gg0 = (int64_t)kk * T + r0;
#pragma unroll
        for (int t = 0; t < PFN; ++t) {
            const int idx = tid + t * (int)blockDim.x;
            pf_n[t] = -1;
            if (idx < myrows * nr) {
                const int i = idx % myrows, j = idx / myrows;
                const int64_t g = gg0 + i;
                pf_v[t] = g < P.n ? from_c128<C>(out[j][g]) : zero_c<C>();
                pf_n[t] = 0;
            }
        }
    };
    const bool pfb_ok = myrows * nr <= PFN * (int)blockDim.x;
    if (pf_ok) prefetch_fwd(0);

    int chunk = 0;
    for (int b = 0; b < 2 * nb - 1; ++b) {
        const bool fwd = b < nb;
        const int k = fwd ? b : 2 * nb - 2 - b;
        const int64_t g0 = (int64_t)k * T;
        const int cur = b % 3, prv = (b + 2) % 3;
        const C* vprev = vbuf + (size_t)prv * R * T;  // t_{k-1} (fwd) or x_{k+1} (bwd)
        const bool last = b == 2 * nb - 2;            // nobody reads the last vector: not sent
        if (b > 0 && !s_fail) {
            // the previous step's vector: every CTA's rows, delivered by st.async
            const uint32_t par = (uint32_t)(((b - 1) / 3) & 1);
            long long it = 0;
            while (!mbar_try_wait_cluster(&vbar[prv], par)) {
                if (++it > WAIT_LIMIT) {
                    s_fail = 1;
                    atomicExch(err, 3);
                    break;
                }
            }
        }
        __syncthreads();
        // re-arm that barrier for step b+2 now: no CTA can send step b+2's rows
        // before it has ours of step b+1, so the expected bytes are always
        // registered before the first of them arrives
        if (tid == 0 && b > 0 && !s_fail && b + 2 <= 2 * nb - 3) mbar_expect_tx(&vbar[prv], vec_bytes);
        const bool failed = s_fail != 0;
        if (fwd && !failed && pf_ok) {
            // s_k = r_k - L_k t_{k-1}: every CTA forms the whole block
#pragma unroll
            for (int t = 0; t < PFN; ++t) {
                const int idx = tid + t * (int)blockDim.x;
                if (idx >= T * nr) break;
                const int i = idx % T, j = idx / T;
                C v = zero_c<C>();
                if (pf_n[t] >= 0) {
                    v = pf_v[t];
                    if (pf_n[t] >= 1) {
                        const C a = pf_a[t];
                        const C tt = vprev[(size_t)j * T + pf_c[t]];
                        v.x -= a.x * tt.x - a.y * tt.y;
                        v.y -= a.x * tt.y + a.y * tt.x;
                    }
                    if (pf_n[t] > 1) {
                        const int64_t g = g0 + i;
                        for (int e = P.Lptr[g] + 1; e < P.Lptr[g + 1]; ++e) {
                            const C a = Lval[e];
                            const C tt = vprev[(size_t)j * T + P.Lcol[e]];
                            v.x -= a.x * tt.x - a.y * tt.y;
                            v.y -= a.x * tt.y + a.y * tt.x;
                        }
                    }
                }
                sbuf[(size_t)j * T + i] = v;
            }
            __syncthreads();
            if (k + 1 < nb) prefetch_fwd(k + 1);
            else if (pfb_ok) prefetch_bwd(nb - 2 >= 0 ? nb - 2 : 0);
        } else if (fwd && !failed) {
            for (int idx = tid; idx < T * nr; idx += blockDim.x) {
                const int i = idx % T, j = idx / T;
                const int64_t g = g0 + i;
                C v = zero_c<C>();
                if (g < P.n) {
                    v = from_c128<C>(in[j][g]);
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
            __syncthreads();
        }
        const C* rhs = fwd ? sbuf : vprev;
        if (!fwd && !failed) {
            // t_k of this CTA's rows, for x_k = t_k - E_k x_{k+1}
            if (pfb_ok) {
#pragma unroll
                for (int t = 0; t < PFN; ++t) {
                    const int idx = tid + t * (int)blockDim.x;
                    if (idx < myrows * nr) tbuf[(size_t)(idx / myrows) * T + idx % myrows] = pf_v[t];
                }
                if (k > 0) prefetch_bwd(k - 1);
            } else {
                for (int idx = tid; idx < myrows * nr; idx += blockDim.x) {
                    const int i = idx % myrows, j = idx / myrows;
                    const int64_t g = g0 + r0 + i;
                    tbuf[(size_t)j * T + i] = g < P.n ? from_c128<C>(out[j][g]) : zero_c<C>();
                }
            }
        }
        for (int sub = 0; sub < nsub; ++sub, ++chunk) {
            const int slot = chunk % NS;
            if (!s_fail) {
                const uint32_t par = (uint32_t)((chunk / NS) & 1);
                long long it = 0;
                while (!mbar_try_wait(&bars[slot], par)) {
                    if (++it > WAIT_LIMIT) {
                        s_fail = 1;
                        atomicExch(err, 2);
                        break;
                    }
                }
            }
            __syncthreads();
            if (!s_fail) {
                const C* M = stage + (size_t)slot * SR * T;
                const int rs = r0 + sub * SR;
                const int rows = min(SR, r1 - rs);
                constexpr int RP = R == 1 ? 4 : (R == 2 ? 2 : 1);  // rows per warp pass
                constexpr int NSC = 2 * RP * R;                      // real accumulators per lane
                constexpr int LOGS = NSC == 16 ? 4 : 3;
                constexpr int SH = 5 - LOGS;                         // lane bits below the value index
                using Rt = decltype(zero_c<C>().x);
                for (int rb = warp * RP; rb < rows; rb += nw * RP) {
                    Rt acc[NSC];
#pragma unroll
                    for (int u = 0; u < NSC; ++u) acc[u] = Rt(0);
                    for (int c = lane; c < T; c += 32) {
                        C xv[R];
#pragma unroll
                        for (int j = 0; j < R; ++j) xv[j] = rhs[(size_t)j * T + c];  // consecutive across lanes
#pragma unroll
                        for (int p = 0; p < RP; ++p) {
                            if (rb + p < rows) {
                                const C m = M[(size_t)(rb + p) * T + c];
#pragma unroll
                                for (int j = 0; j < R; ++j) {
                                    Rt& re = acc[(p * R + j) * 2];
                                    Rt& im = acc[(p * R + j) * 2 + 1];
                                    re = fma(m.x, xv[j].x, re);
                                    re = fma(-m.y, xv[j].y, re);
                                    im = fma(m.x, xv[j].y, im);
                                    im = fma(m.y, xv[j].x, im);
                                }
                            }
                        }
                    }
                    // butterfly: NSC sums over the warp with NSC shuffles in all;
                    // lane L ends with the sum of value (L >> SH) & (NSC - 1)
                    butterfly<Rt, NSC>(acc, lane);
                    const Rt mine = acc[0];
                    const Rt other = __shfl_xor_sync(0xffffffffu, mine, 1 << SH);
                    const int kv = (lane >> SH) & (NSC - 1);
                    if ((lane & ((1 << SH) - 1)) == 0 && (kv & 1) == 0) {
                        const int pair = kv >> 1;
                        const int p = pair / R, j = pair % R;
                        if (rb + p < rows && j < nr) {
                            const int r = rs + rb + p;
                            const int64_t g = g0 + r;
                            C val;
                            val.x = mine;
                            val.y = other;
                            if (!fwd) val = csub(tbuf[(size_t)j * T + (r - r0)], val);
                            if (g < P.n) out[j][g] = to_c128(val);
                            if (!last) {
                                C* loc = vbuf + (size_t)cur * R * T + (size_t)j * T + r;
                                for (int qq = 0; qq < Ccl; ++qq)
                                    st_async_c(mapa_u32(loc, qq), val, mapa_u32(&vbar[cur], qq));
                            }
                        }
                    }
                }
            }
            __syncthreads();  // the stage is consumed
            if (tid == 0 && !s_fail && issued < total) {
                uint32_t bytes;
                const C* src = chunk_src(issued, bytes);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bars[issued % NS], bytes);
                tma_load_1d(stage + (size_t)(issued % NS) * SR * T, src, bytes, &bars[issued % NS]);
                ++issued;
            }
        }
    }
    // a failed CTA still has copies in flight: wait for them (bounded) before exit;
    // the final cluster barrier keeps every CTA's shared memory alive until all
    // peers have finished
    if (tid == 0 && s_fail) {
        for (int c = chunk; c < issued; ++c) {
            long long it = 0;
            while (!mbar_try_wait(&bars[c % NS], (uint32_t)((c / NS) & 1)) && ++it < WAIT_LIMIT) {
            }
        }
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
namespace {

struct Plan {
    int R = 1, SR = 1, NS = 3;
    size_t smem = 0;
};

bool make_plan(int T, size_t cs, int want_R, Plan& p) {
    const size_t budget = 220 * 1024;
    for (int R : {8, 4, 2, 1}) {
        if (R > want_R && R != 1) continue;
        const size_t vec = (size_t)5 * R * T * cs;
        if (vec + 64 >= budget) continue;
        const int NS = 3;
        const size_t per_row = (size_t)NS * T * cs;
        int SR = (int)std::min<size_t>(32, (budget - vec - 64) / per_row);
        if (SR < 1) continue;
        p.R = R;
        p.SR = SR;
        p.NS = NS;
        p.smem = (size_t)NS * SR * T * cs + vec + (NS + 3) * sizeof(uint64_t) + 16;
        return true;
    }
    return false;
}

template <class C, int R>
void launch_cl(const Pencil& P, const JobSpace& js, int in_slot, int out_slot, const double2* d_sigma,
               void* const* fptrs, const int* d_grp, int ngroups, int Ccl, const Plan& pl, int* d_err,
               cudaStream_t st) {
    auto kern = k_block_solve_cl<C, R>;
    static size_t attr_set = 0;  // per instantiation
    if (pl.smem > attr_set) {
        SIM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
        attr_set = pl.smem;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ngroups * Ccl);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Ccl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SIM_CUDA(cudaLaunchKernelEx(&cfg, kern, P, js, in_slot, out_slot, d_sigma, fptrs, d_grp, pl.SR, pl.NS, d_err));
    SIM_LAUNCH_CHECK();
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
    // cluster size: as many CTAs per group as the 152 SMs allow, up to 8
    int Ccl = 8;
    while (Ccl > 1 && (int64_t)Ccl * ng > 152) Ccl >>= 1;
    Ccl = std::min(Ccl, P.T);
    {
        // equal chunks: a CTA's rows in as few stages-worth pieces as the ring allows
        const int Tc = (P.T + Ccl - 1) / Ccl;
        const int nsub = (Tc + pl.SR - 1) / pl.SR;
        pl.SR = (Tc + nsub - 1) / nsub;
    }
    const double TT = (double)P.T * P.T, blocks = 2.0 * P.nb - 1.0;
    kprof_begin("block_solve", st);
#define SIM_LAUNCH_R(CT, RR) \
    launch_cl<CT, RR>(P, js, in_slot, out_slot, d_sigma, d_factor_ptrs, d_grp, ng, Ccl, pl, g_err, st)
    if (precision == SIM_FP64) {
        if (pl.R == 8) SIM_LAUNCH_R(double2, 8);
        else if (pl.R == 4) SIM_LAUNCH_R(double2, 4);
        else if (pl.R == 2) SIM_LAUNCH_R(double2, 2);
        else SIM_LAUNCH_R(double2, 1);
    } else {
        if (pl.R == 8) SIM_LAUNCH_R(float2, 8);
        else if (pl.R == 4) SIM_LAUNCH_R(float2, 4);
        else if (pl.R == 2) SIM_LAUNCH_R(float2, 2);
        else SIM_LAUNCH_R(float2, 1);
    }
#undef SIM_LAUNCH_R
    // algorithmic bytes: each group reads the factor once, and 4 vectors per job
    kprof_end("block_solve", st, ng * blocks * TT * cs + (double)active.size() * 4.0 * P.n * sizeof(double2),
              (double)active.size() * 8.0 * blocks * TT);
    return true;
}

int block_solve_error() {
    if (!g_err) return 0;
    int e = 0;
    cudaMemcpy(&e, g_err, sizeof(int), cudaMemcpyDeviceToHost);
    return e;
}

}  // namespace sim
