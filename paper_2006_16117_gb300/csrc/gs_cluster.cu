// Batched classical Gram–Schmidt, applied twice (CGS2) or with the
// Daniel–Gragg–Kaufman–Stewart test for the second pass, in one launch: the
// orthogonalisation of w against the cnt basis vectors of its job, the norm,
// the Arnoldi breakdown test and the normalisation (Sec. 3.1's Arnoldi
// process; the inner FGMRES uses the same step).
//
// One thread-block cluster per job.  CTA q of the cluster owns rows
// [q*256*E, (q+1)*256*E) and keeps its piece of w in shared memory (E values
// per thread, two CTAs per SM), so w is read once and written once; every
// pass over the basis is one streaming read.  The complex multiply-adds are
// FP64 and on this GPU the FP64 pipe, not HBM, bounds the step; the update
// streams all basis vectors per element so that many loads are in flight.  The dot products and norms are summed in the CTA
// (shuffles, then shared memory) and across the cluster by reading each peer
// CTA's partials through distributed shared memory, in rank order — every
// CTA forms the same totals and takes the same decisions.  The only waits are
// the hardware cluster barriers.
#include <cooperative_groups.h>

#include "gs.h"

namespace cg = cooperative_groups;

namespace sim {

namespace {

constexpr int GC_THREADS = 256;
constexpr int GC_WARPS = GC_THREADS / 32;
constexpr int GC_MAXV = 64;  // basis vectors per call (cnt), plus two norm slots below

struct GcShared {
    double2 red[GC_WARPS][GC_MAXV + 2];  // per-warp sums
    double2 part[GC_MAXV + 2];           // this CTA's sums (read by the peers)
    double2 tot[GC_MAXV + 2];            // cluster totals
    double2 h1[GC_MAXV];                 // first-pass coefficients
    double fro[GC_WARPS];
};

// Sum V values (each thread's contribution in v(i), i < V) over the CTA and
// the cluster; the totals land in S.tot[0..V).
template <class F>
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, GcShared& S, int V, F v) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < V; ++i) {
        const double2 x = warp_sum(v(i));
        if (lane == 0) S.red[warp][i] = x;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < V; i += GC_THREADS) {
        double2 s = S.red[0][i];
        for (int w = 1; w < GC_WARPS; ++w) s = cadd(s, S.red[w][i]);
        S.part[i] = s;
    }
    cl.sync();  // every CTA's partials are written
    const int nr = (int)cl.num_blocks();
    for (int i = threadIdx.x; i < V; i += GC_THREADS) {
        double2 s = make_double2(0.0, 0.0);
        for (int r = 0; r < nr; ++r) s = cadd(s, cl.map_shared_rank(S.part, r)[i]);
        S.tot[i] = s;
    }
    cl.sync();  // the peers have read our partials; the totals are visible
}

template <int E>
__global__ void __launch_bounds__(GC_THREADS, 2) k_gs_cluster(GSArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int Cg = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int job = a.active[blockIdx.x / Cg];
    const int tid = threadIdx.x;
    __shared__ GcShared S;
    extern __shared__ double2 wsm[];  // [E][GC_THREADS]: this CTA's rows of w
    const double2* B = a.basis + (size_t)job * a.bstride;
    double2* w = a.w + (size_t)job * a.wstride;
    const int64_t base = (int64_t)q * GC_THREADS * E + tid;
    const int cnt = a.cnt;

#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t r = base + (int64_t)e * GC_THREADS;
        wsm[e * GC_THREADS + tid] = r < a.n ? w[r] : make_double2(0.0, 0.0);
    }
    auto sq = [&]() {
        double s = 0.0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const double2 v = wsm[e * GC_THREADS + tid];
            s += v.x * v.x + v.y * v.y;
        }
        return make_double2(s, 0.0);
    };
    // h_i = conj(q_i) . w for i < cnt (and ||w||^2 in slot cnt if `with_norm`)
    auto dots = [&](bool with_norm) {
        cluster_sum(cl, S, cnt + (with_norm ? 1 : 0), [&](int i) -> double2 {
            if (i == cnt) return sq();
            const double2* qv = B + (size_t)i * a.n;
            double2 acc = make_double2(0.0, 0.0), acc2 = make_double2(0.0, 0.0);
#pragma unroll 10
            for (int e = 0; e < E; ++e) {
                const int64_t r = base + (int64_t)e * GC_THREADS;
                if (r < a.n) {
                    const double2 x = qv[r];
                    const double2 v = wsm[e * GC_THREADS + tid];
                    double2& c = (e & 1) ? acc2 : acc;
                    c.x = fma(x.x, v.x, c.x);
                    c.x = fma(x.y, v.y, c.x);
                    c.y = fma(x.x, v.y, c.y);
                    c.y = fma(-x.y, v.x, c.y);
                }
            }
            return cadd(acc, acc2);
        });
    };
    // w -= sum_i q_i h_i with h in S.tot[0..cnt): per element, all i
    auto update = [&]() {
#pragma unroll 2
        for (int e = 0; e < E; ++e) {
            const int64_t r = base + (int64_t)e * GC_THREADS;
            if (r >= a.n) continue;
            double2 v = wsm[e * GC_THREADS + tid];
            const double2* qv = B + r;
            for (int i = 0; i < cnt; ++i) {
                const double2 x = qv[(size_t)i * a.n];
                const double2 hi = S.tot[i];
                v.x = fma(-x.x, hi.x, v.x);
                v.x = fma(x.y, hi.y, v.x);
                v.y = fma(-x.x, hi.y, v.y);
                v.y = fma(-x.y, hi.x, v.y);
            }
            wsm[e * GC_THREADS + tid] = v;
        }
    };

    double nn = 0.0;  // ||w||^2 after the last pass
    if (cnt == 0) {
        cluster_sum(cl, S, 1, [&](int) { return sq(); });
        nn = S.tot[0].x;
    } else {
        dots(a.dgks != 0);
        const double nb = a.dgks ? S.tot[cnt].x : 0.0;  // ||w||^2 before the first pass
        for (int i = tid; i < cnt; i += GC_THREADS) S.h1[i] = S.tot[i];
        update();
        // the barriers in cluster_sum order S.h1's writes before its reads below
        bool second = !a.single;
        if (a.dgks || a.single) {
            cluster_sum(cl, S, 1, [&](int) { return sq(); });
            nn = S.tot[0].x;
            if (a.dgks && !a.single) second = !(nn > 0.5 * nb);
        }
        if (second) {
            dots(false);
            // S.tot now holds the second-pass coefficients
            for (int i = tid; i < cnt; i += GC_THREADS) S.h1[i] = cadd(S.h1[i], S.tot[i]);
            update();
            cluster_sum(cl, S, 1, [&](int) { return sq(); });
            nn = S.tot[0].x;
        }
        __syncthreads();  // S.h1 complete
    }
    const double hn = sqrt(nn);
    bool broken = !(hn > 0.0);
    if (a.Hfull) {
        // ||H(0:j, 0:j)||_F, column j being the coefficients just computed
        const double2* H = a.Hfull + (size_t)job * a.Hstride;
        const int jj = a.j, rows = a.j + 1;
        double f = 0.0;
        for (int idx = tid; idx < jj * rows; idx += GC_THREADS) f += cabs2(H[(size_t)(idx / rows) * a.Hld + idx % rows]);
        for (int r = tid; r < rows; r += GC_THREADS) f += cabs2(S.h1[r]);
        f = warp_sum(f);
        if ((tid & 31) == 0) S.fro[tid >> 5] = f;
        __syncthreads();
        double ft = 0.0;
        for (int w2 = 0; w2 < GC_WARPS; ++w2) ft += S.fro[w2];
        if (hn <= a.btol * sqrt(ft)) broken = true;
    }
    if (q == 0) {
        double2* hc = a.hcol + (size_t)job * a.hstride;
        for (int i = tid; i < cnt; i += GC_THREADS) hc[i] = S.h1[i];
        if (tid == 0) {
            hc[cnt] = make_double2((broken && a.Hfull) ? 0.0 : hn, 0.0);
            if (broken && a.meff) a.meff[job] = a.j + 1;
            if (broken && a.istat) a.istat[job * IS_N + IS_BROKEN] = 1;
        }
    }
    const double inv = broken ? 1.0 : 1.0 / hn;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int64_t r = base + (int64_t)e * GC_THREADS;
        const double2 v = wsm[e * GC_THREADS + tid];
        if (r < a.n) w[r] = broken ? v : cscale(v, inv);
    }
}

template <int E>
void launch_gc(const GSArgs& a, int nactive, int Cg, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nactive * Cg);
    cfg.blockDim = dim3(GC_THREADS);
    cfg.dynamicSmemBytes = (size_t)E * GC_THREADS * sizeof(double2);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Cg;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    static bool smem_set = false;  // per instantiation
    if (!smem_set) {
        SIM_CUDA(cudaFuncSetAttribute(k_gs_cluster<E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)cfg.dynamicSmemBytes));
        smem_set = true;
    }
    SIM_CUDA(cudaLaunchKernelEx(&cfg, k_gs_cluster<E>, a));
    SIM_LAUNCH_CHECK();
}

}  // namespace

bool gs_cluster(const GSArgs& a, int nactive, cudaStream_t st) {
    if (nactive <= 0) return true;
    if (a.cnt < 0 || a.cnt > GC_MAXV) return false;
    static const int Es[] = {4, 8, 12, 16, 20};
    int E = 0;
    for (int e : Es)
        if ((int64_t)GC_THREADS * e * 8 >= a.n) {
            E = e;
            break;
        }
    if (E == 0) return false;
    const int Cg = cdiv_up(a.n, (int64_t)GC_THREADS * E);
    // algorithmic bytes: w read and written once; the basis streamed once per
    // pass (two passes with the selective test in its usual outcome, four for CGS2)
    const double passes = a.cnt == 0 ? 0.0 : ((a.dgks || a.single) ? 2.0 : 4.0);
    kprof_begin("gram_schmidt", st);
    switch (E) {
        case 4: launch_gc<4>(a, nactive, Cg, st); break;
        case 8: launch_gc<8>(a, nactive, Cg, st); break;
        case 12: launch_gc<12>(a, nactive, Cg, st); break;
        case 16: launch_gc<16>(a, nactive, Cg, st); break;
        default: launch_gc<20>(a, nactive, Cg, st); break;
    }
    kprof_end("gram_schmidt", st, nactive * (passes * a.cnt + 2.0) * a.n * sizeof(double2),
              nactive * 8.0 * (passes * a.cnt + 1.0) * a.n);
    return true;
}

}  // namespace sim
