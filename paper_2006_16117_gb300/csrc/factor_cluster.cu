// Block Thomas factorisation of A - σB on thread-block clusters.
//
// Same factors as k_factor (krylov.cu): Dinv_k = D_k^{-1} with
// D_k = A_kk - σB_kk - L_k E_{k-1}, and E_k = Dinv_k U_k, plus the shifted
// values of the couplings L_k.  Here a cluster of Cf CTAs factors one shift;
// each CTA keeps a slice of Tc = ceil(T/Cf) rows of D_k in shared memory.
// Gauss–Jordan with partial pivoting runs without physical row swaps: at
// column p every CTA proposes its largest unused |re|+|im| entry, the proposals
// meet in every CTA through distributed shared memory, the owner of the winning
// row scales it and broadcasts it, and every CTA eliminates column p from its
// rows.  Two cluster barriers per pivot.  The in-place scheme leaves the
// inverse with rows and columns permuted; each CTA gathers its output rows
// from the owners' slices when writing Dinv_k.
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.h"
#include "factor_cluster.h"

namespace cg = cooperative_groups;

namespace sim {

namespace {

template <class C> __device__ __forceinline__ C zc();
template <> __device__ __forceinline__ double2 zc<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 zc<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 sval(const Pencil& P, int64_t e, double2 sg) {
    const double2 a = P.Ka[e], b = P.Kb[e];
    return make_double2(a.x - (sg.x * b.x - sg.y * b.y), a.y - (sg.x * b.y + sg.y * b.x));
}

// pivot magnitude |re| + |im| in the factor's own precision (float for complex64:
// FP64 on this GPU is slow and the pivot search is on every pivot's critical path)
template <class C> __device__ __forceinline__ auto m1(C a) -> decltype(a.x) { return fabs(a.x) + fabs(a.y); }

}  // namespace

template <class C>
__global__ void __launch_bounds__(256, 1) k_factor_cl(Pencil P, const int* shift_list, const double2* sigma,
                                                      void* const* fptrs, int* err) {
    cg::cluster_group cl = cg::this_cluster();
    const int Cf = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int T = P.T, nb = P.nb;
    const int s = shift_list[blockIdx.x / Cf];
    C* Dinv = reinterpret_cast<C*>(fptrs[s]);
    C* E = Dinv + (size_t)nb * T * T;
    C* Lval = Dinv + factor_lval_offset(P);
    const double2 sg = sigma[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int Tc = (T + Cf - 1) / Cf;
    const int r0 = min(T, q * Tc), r1 = min(T, r0 + Tc);
    const int my = r1 - r0;

    extern __shared__ __align__(16) unsigned char raw[];
    C* S = reinterpret_cast<C*>(raw);            // [Tc][T]
    C* prow = S + (size_t)Tc * T;                // [T]
    int* piv_row = reinterpret_cast<int*>(prow + T);  // [T] pivot row of column p (all CTAs)
    int* step_of = piv_row + T;                  // [T] column at which row r was the pivot
    int* used = step_of + T;                     // [Tc]
    using Mt = decltype(zc<C>().x);
    Mt* cand_v = reinterpret_cast<Mt*>(used + Tc + (Tc & 1) + 2);        // [8]
    int* cand_i = reinterpret_cast<int*>(cand_v + 8);                    // [8]
    Mt* red_v = reinterpret_cast<Mt*>(cand_i + 8);                       // [8 warps]
    int* red_i = reinterpret_cast<int*>(red_v + 8);                      // [8 warps]

    for (int64_t e = tid + (int64_t)q * blockDim.x; e < P.nnzL; e += (int64_t)blockDim.x * Cf)
        Lval[e] = from_c128<C>(sval(P, P.Lidx[e], sg));
    {
        C* L0val = Dinv + factor_l0_offset(P);
        for (int64_t g = tid + (int64_t)q * blockDim.x; g < P.n; g += (int64_t)blockDim.x * Cf) {
            const int e0 = P.Lptr[g];
            L0val[g] = from_c128<C>(P.Lptr[g + 1] > e0 ? sval(P, P.Lidx[e0], sg) : make_double2(0.0, 0.0));
        }
    }
    cl.sync();

    for (int k = 0; k < nb; ++k) {
        const int64_t g0 = (int64_t)k * T;
        C* Dk = Dinv + (size_t)k * T * T;
        // 1. my rows of D_k = K_kk - L_k E_{k-1}
        for (int i = warp; i < my; i += nw) {
            const int64_t g = g0 + r0 + i;
            C* Si = S + (size_t)i * T;
            for (int c = lane; c < T; c += 32) Si[c] = zc<C>();
            __syncwarp();
            if (g < P.n) {
                for (int64_t e = P.rp[g] + lane; e < P.rp[g + 1]; e += 32) {
                    const int64_t j = P.ci[e];
                    if (j >= g0 && j < g0 + T) Si[j - g0] = from_c128<C>(sval(P, e, sg));
                }
                __syncwarp();
                if (k > 0) {
                    const C* Ep = E + (size_t)(k - 1) * T * T;
                    const int e0 = P.Lptr[g], e1 = P.Lptr[g + 1];
                    for (int c = lane; c < T; c += 32) {
                        C acc = zc<C>();
                        for (int e = e0; e < e1; ++e) acc = cfma(Lval[e], Ep[(size_t)P.Lcol[e] * T + c], acc);
                        Si[c] = csub(Si[c], acc);
                    }
                }
            } else if (lane == 0) {
                Si[r0 + i] = from_c128<C>(make_double2(1.0, 0.0));
            }
        }
        for (int i = tid; i < my; i += blockDim.x) used[i] = 0;
        __syncthreads();
        // 2. Gauss–Jordan with implicit partial pivoting
        for (int p = 0; p < T; ++p) {
            Mt bv = Mt(-1);
            int bi = T;
            for (int i = tid; i < my; i += blockDim.x) {
                if (used[i]) continue;
                const Mt v = m1(S[(size_t)i * T + p]);
                if (v > bv || (v == bv && r0 + i < bi)) {
                    bv = v;
                    bi = r0 + i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const Mt ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                red_v[warp] = bv;
                red_i[warp] = bi;
            }
            __syncthreads();
            if (tid < Cf) {
                Mt v = red_v[0];
                int ii = red_i[0];
                for (int w = 1; w < nw; ++w)
                    if (red_v[w] > v || (red_v[w] == v && red_i[w] < ii)) {
                        v = red_v[w];
                        ii = red_i[w];
                    }
                *cl.map_shared_rank(cand_v + q, tid) = v;
                *cl.map_shared_rank(cand_i + q, tid) = ii;
            }
            cl.sync();
            Mt v = cand_v[0];
            int rs = cand_i[0];
            for (int w = 1; w < Cf; ++w)
                if (cand_v[w] > v || (cand_v[w] == v && cand_i[w] < rs)) {
                    v = cand_v[w];
                    rs = cand_i[w];
                }
            if (!(v > Mt(0)) && tid == 0 && q == 0) atomicExch(err, 1);  // singular Schur complement
            if (tid == 0) {
                piv_row[p] = rs;
                step_of[rs] = p;
            }
            const int owner = rs / Tc;
            if (owner == q) {
                const int li = rs - r0;
                C pv = S[(size_t)li * T + p];
                if (pv.x == 0 && pv.y == 0) pv.x = (decltype(pv.x))1e-30;
                const C inv = cdiv(from_c128<C>(make_double2(1.0, 0.0)), pv);
                __syncthreads();  // every thread has the pivot before its column is overwritten
                for (int c = tid; c < T; c += blockDim.x) {
                    const C val = (c == p) ? inv : cmul(S[(size_t)li * T + c], inv);
                    S[(size_t)li * T + c] = val;
                    for (int qq = 0; qq < Cf; ++qq) *cl.map_shared_rank(prow + c, qq) = val;
                }
                if (tid == 0) used[li] = 1;
            }
            cl.sync();
            for (int i = warp; i < my; i += nw) {
                if (r0 + i == rs) continue;
                C* Si = S + (size_t)i * T;
                const C f = Si[p];
                __syncwarp();  // every lane has f before lane p % 32 overwrites Si[p]
                for (int c = lane; c < T; c += 32) {
                    C base = (c == p) ? zc<C>() : Si[c];
                    const C rp = prow[c];
                    base.x -= f.x * rp.x - f.y * rp.y;
                    base.y -= f.x * rp.y + f.y * rp.x;
                    Si[c] = base;
                }
            }
            __syncthreads();
        }
        cl.sync();  // every CTA finished its last elimination before slices are read remotely
        // 3. gather my output rows: Dinv_k[p][c] = S_all[piv_row[p]][step_of[c]]
        for (int i = warp; i < my; i += nw) {
            const int p = r0 + i;
            const int src = piv_row[p];
            const C* row = cl.map_shared_rank(S + (size_t)(src - (src / Tc) * Tc) * T, src / Tc);
            for (int c = lane; c < T; c += 32) Dk[(size_t)p * T + c] = row[step_of[c]];
        }
        cl.sync();  // remote slices read; S may be overwritten
        // 4. my rows of E_k = Dinv_k U_k
        if (k < nb - 1) {
            C* Ek = E + (size_t)k * T * T;
            const int32_t* cp = P.up_ptr + (size_t)k * (T + 1);
            for (int i = warp; i < my; i += nw) {
                const int p = r0 + i;
                for (int c = lane; c < T; c += 32) {
                    C acc = zc<C>();
                    for (int qq = cp[c]; qq < cp[c + 1]; ++qq)
                        acc = cfma(Dk[(size_t)p * T + P.up_row[qq]], from_c128<C>(sval(P, P.up_idx[qq], sg)), acc);
                    Ek[(size_t)p * T + c] = acc;
                }
            }
        }
        cl.sync();  // E_k complete before the next block reads it
    }
}

namespace {
int* g_ferr = nullptr;

size_t smem_for(int T, int Cf, size_t cs) {
    const int Tc = (T + Cf - 1) / Cf;
    return (size_t)Tc * T * cs + T * cs + (size_t)(3 * T + Tc + 4) * sizeof(int) + 40 * sizeof(double) + 64;
}

template <class C>
void launch(const Pencil& P, const int* d_list, int count, const double2* d_sigma, void* const* fptrs, int Cf,
            size_t smem, cudaStream_t st) {
    auto kern = k_factor_cl<C>;
    SIM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(count * Cf);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = Cf;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SIM_CUDA(cudaLaunchKernelEx(&cfg, kern, P, d_list, d_sigma, fptrs, g_ferr));
    SIM_LAUNCH_CHECK();
}
}  // namespace

bool factor_shifts_cluster(const Pencil& P, int precision, const int* d_shift_list, int count,
                           const double2* d_sigma, void* const* d_factor_ptrs, cudaStream_t st) {
    if (count <= 0) return true;
    const size_t cs = precision == SIM_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t budget = 220 * 1024;
    // the fewest CTAs per shift whose slice fits, then more while the GPU has room
    int Cf = 1;
    while (Cf <= 8 && smem_for(P.T, Cf, cs) > budget) Cf *= 2;
    if (Cf > 8 || P.T < 2) return false;
    while (Cf < 8 && (int64_t)2 * Cf * count <= 152) Cf *= 2;
    Cf = std::min(Cf, P.T);
    if (!g_ferr) {
        SIM_CUDA(cudaMalloc(&g_ferr, sizeof(int)));
        SIM_CUDA(cudaMemset(g_ferr, 0, sizeof(int)));
    }
    const size_t smem = smem_for(P.T, Cf, cs);
    kprof_begin("factor", st);
    if (precision == SIM_FP64) launch<double2>(P, d_shift_list, count, d_sigma, d_factor_ptrs, Cf, smem, st);
    else launch<float2>(P, d_shift_list, count, d_sigma, d_factor_ptrs, Cf, smem, st);
    const double TT = (double)P.T * P.T;
    kprof_end("factor", st, count * (2.0 * P.nb * TT * cs), count * 8.0 * P.nb * TT * P.T);
    return true;
}

}  // namespace sim
