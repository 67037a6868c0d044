// Krylov side of SIM-M on the GPU: the Cayley transform's shifted operator
// (A - σB) and its inverse, and the Arnoldi process for M = (A - σB)^{-1} B
// (Sec. 2, Eqs. AzBxf, IMxb, eq:arnoldi).
//
//  * factor_shifts  : block-tridiagonal (block Thomas) factorisation of A - σB
//                     for many shifts at once, one CTA per shift; each
//                     diagonal Schur complement D_k is inverted by Gauss–Jordan
//                     with partial pivoting.  Storage: Dinv_k = D_k^{-1} and
//                     E_k = Dinv_k U_k, both dense T×T, in complex128 (FP64
//                     mode) or complex64 (mixed mode).
//  * (the solve x = (A - σB)^{-1} r through those factors is the cluster
//    kernel of solve_cluster.cu)
//  * inner_solve    : batched FGMRES(k) in FP64 with the factorisation as right
//                     preconditioner, CGS2 on its basis, Givens rotations and an
//                     explicit residual check per cycle.  In mixed mode this is
//                     GMRES-based iterative refinement of a complex64 solve.
//  * arnoldi        : m steps of w = M v_j = (A - σB)^{-1} B v_j with classical
//                     Gram–Schmidt applied twice (CGS2) in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <stdexcept>
#include <vector>

#include "internal.h"
#include "levels.h"
#include "gs.h"
#include "autotune.h"
#include "separable.h"
#include "solve_cluster.h"

namespace sim {

// ---------------------------------------------------------------------------
// block-tridiagonal factorisation
// ---------------------------------------------------------------------------
template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ double2 shifted_val(const Pencil& P, int64_t e, double2 sg) {
    double2 a = P.Ka[e], b = P.Kb[e];
    return make_double2(a.x - (sg.x * b.x - sg.y * b.y), a.y - (sg.x * b.y + sg.y * b.x));
}

template <class C> __device__ __forceinline__ double mag1(C a) { return fabs((double)a.x) + fabs((double)a.y); }

constexpr int FACTOR_THREADS = 512;

template <class C>
__global__ void __launch_bounds__(FACTOR_THREADS) k_factor(Pencil P, const int* shift_list, const double2* sigma,
                                                           void* const* fptrs, int* err) {
    const int T = P.T, nb = P.nb;
    const int s = shift_list[blockIdx.x];
    C* Dinv = reinterpret_cast<C*>(fptrs[s]);
    C* E = Dinv + (size_t)nb * T * T;
    const double2 sg = sigma[s];
    extern __shared__ unsigned char smem_raw[];
    C* rowp = reinterpret_cast<C*>(smem_raw);
    C* colp = rowp + T;
    int* piv = reinterpret_cast<int*>(colp + T);
    double* redv = reinterpret_cast<double*>(piv + T + (T & 1));
    int* redi = reinterpret_cast<int*>(redv + 32);
    const int tid = threadIdx.x, bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = bd >> 5;
    const size_t TT = (size_t)T * T;

    {
        C* Lval = Dinv + factor_lval_offset(P);
        for (int64_t e = tid; e < P.nnzL; e += bd) Lval[e] = from_c128<C>(shifted_val(P, P.Lidx[e], sg));
        C* L0val = Dinv + factor_l0_offset(P);
        for (int64_t g = tid; g < P.n; g += bd) {
            const int e0 = P.Lptr[g];
            L0val[g] = P.Lptr[g + 1] > e0 ? from_c128<C>(shifted_val(P, P.Lidx[e0], sg)) : czero<C>();
        }
    }
    for (int k = 0; k < nb; ++k) {
        C* D = Dinv + (size_t)k * TT;
        const int64_t g0 = (int64_t)k * T;
        for (int i = warp; i < T; i += nw)
            for (int c = lane; c < T; c += 32) D[(size_t)i * T + c] = czero<C>();
        __syncthreads();
        for (int i = tid; i < T; i += bd) {
            int64_t g = g0 + i;
            if (g < P.n) {
                for (int64_t e = P.rp[g]; e < P.rp[g + 1]; ++e) {
                    int64_t j = P.ci[e];
                    if (j >= g0 && j < g0 + T) D[(size_t)i * T + (j - g0)] = from_c128<C>(shifted_val(P, e, sg));
                }
            } else {
                D[(size_t)i * T + i] = from_c128<C>(make_double2(1.0, 0.0));
            }
        }
        __syncthreads();
        if (k > 0) {
            const C* Ep = E + (size_t)(k - 1) * TT;
            const C* Lval = Dinv + factor_lval_offset(P);
            for (int i = warp; i < T; i += nw) {
                const int64_t g = g0 + i;
                if (g >= P.n) continue;
                const int e0 = P.Lptr[g], e1 = P.Lptr[g + 1];
                for (int c = lane; c < T; c += 32) {
                    C acc = czero<C>();
                    for (int e = e0; e < e1; ++e) acc = cfma(Lval[e], Ep[(size_t)P.Lcol[e] * T + c], acc);
                    D[(size_t)i * T + c] = csub(D[(size_t)i * T + c], acc);
                }
            }
            __syncthreads();
        }
        // Gauss–Jordan inversion in place with partial pivoting (|re| + |im|)
        for (int p = 0; p < T; ++p) {
            double best = -1.0;
            int bi = p;
            for (int r = p + tid; r < T; r += bd) {
                double v = mag1(D[(size_t)r * T + p]);
                if (v > best) { best = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                double ov = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (lane == 0) { redv[warp] = best; redi[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                double b = redv[0];
                int i0 = redi[0];
                for (int w = 1; w < nw; ++w)
                    if (redv[w] > b || (redv[w] == b && redi[w] < i0)) { b = redv[w]; i0 = redi[w]; }
                piv[p] = i0;
                if (!(b > 0.0)) atomicExch(err, 1);  // singular Schur complement
            }
            __syncthreads();
            const int r = piv[p];
            if (r != p) {
                for (int c = tid; c < T; c += bd) {
                    C a = D[(size_t)p * T + c];
                    D[(size_t)p * T + c] = D[(size_t)r * T + c];
                    D[(size_t)r * T + c] = a;
                }
                __syncthreads();
            }
            C pv = D[(size_t)p * T + p];
            if (pv.x == 0 && pv.y == 0) pv.x = (decltype(pv.x))1e-30;  // singular: flagged above
            const C inv = cdiv(from_c128<C>(make_double2(1.0, 0.0)), pv);
            for (int c = tid; c < T; c += bd) {
                rowp[c] = (c == p) ? inv : cmul(D[(size_t)p * T + c], inv);
                colp[c] = D[(size_t)c * T + p];
            }
            __syncthreads();
            for (int i = warp; i < T; i += nw) {
                C* Di = D + (size_t)i * T;
                if (i == p) {
                    for (int c = lane; c < T; c += 32) Di[c] = rowp[c];
                } else {
                    const C f = colp[i];
                    for (int c = lane; c < T; c += 32) {
                        C base = (c == p) ? czero<C>() : Di[c];
                        const C rp = rowp[c];
                        base.x -= f.x * rp.x - f.y * rp.y;
                        base.y -= f.x * rp.y + f.y * rp.x;
                        Di[c] = base;
                    }
                }
            }
            __syncthreads();
        }
        for (int p = T - 1; p >= 0; --p) {
            const int r = piv[p];
            if (r != p) {
                for (int i = tid; i < T; i += bd) {
                    C a = D[(size_t)i * T + p];
                    D[(size_t)i * T + p] = D[(size_t)i * T + r];
                    D[(size_t)i * T + r] = a;
                }
                __syncthreads();
            }
        }
        // E_k = Dinv_k U_k, U_k = (A - σB)_{k,k+1} in column-compressed form
        if (k < nb - 1) {
            C* Ek = E + (size_t)k * TT;
            const int32_t* cp = P.up_ptr + (size_t)k * (T + 1);
            for (int rr = warp; rr < T; rr += nw)
                for (int c = lane; c < T; c += 32) {
                    C acc = czero<C>();
                    for (int q = cp[c]; q < cp[c + 1]; ++q)
                        acc = cfma(D[(size_t)rr * T + P.up_row[q]], from_c128<C>(shifted_val(P, P.up_idx[q], sg)), acc);
                    Ek[(size_t)rr * T + c] = acc;
                }
        }
        __syncthreads();
    }
}

static size_t factor_smem(int T, int precision) {
    size_t cs = precision == SIM_FP64 ? sizeof(double2) : sizeof(float2);
    return 2 * T * cs + (T + 2) * sizeof(int) + 32 * sizeof(double) + 32 * sizeof(int) + 16;
}

void factor_shifts(const Pencil& P, int precision, const int* d_shift_list, int count, const double2* d_sigma,
                   void* const* d_factor_ptrs, cudaStream_t st) {
    if (count <= 0) return;
    static int* d_err = nullptr;
    if (!d_err) SIM_CUDA(cudaMalloc(&d_err, sizeof(int)));
    SIM_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    size_t sm = factor_smem(P.T, precision);
    kprof_begin("factor", st);
    if (precision == SIM_FP64) {
        SIM_CUDA(cudaFuncSetAttribute(k_factor<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_factor<double2><<<count, FACTOR_THREADS, sm, st>>>(P, d_shift_list, d_sigma, d_factor_ptrs, d_err);
        SIM_LAUNCH_CHECK();
    } else {
        SIM_CUDA(cudaFuncSetAttribute(k_factor<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_factor<float2><<<count, FACTOR_THREADS, sm, st>>>(P, d_shift_list, d_sigma, d_factor_ptrs, d_err);
        SIM_LAUNCH_CHECK();
    }
    {
        const double cs = precision == SIM_FP64 ? sizeof(double2) : sizeof(float2);
        const double TT = (double)P.T * P.T;
        kprof_end("factor", st, count * (2.0 * P.nb * TT * cs), count * 8.0 * P.nb * TT * P.T);
    }
}

// ---------------------------------------------------------------------------
// sparse applies
// ---------------------------------------------------------------------------
// y = (A - σB) x, or y = rhs - (A - σB) x when rhs_slot >= 0, for SPMV_RJ
// active jobs per thread: a thread owns one row and reads its indices and
// values once for all of its jobs (the jobs' shifts differ only on B's
// entries), then gathers each job's x.  Every job's row sum runs over the
// row's entries in order, so the result does not depend on SPMV_RJ, which the
// autotuner picks per matrix (1, 2, 4 or 8).
template <int SPMV_RJ>
__global__ void __launch_bounds__(256) k_spmv_jobs(Pencil P, JobSpace js, int x_slot, int y_slot, int rhs_slot,
                                                   const double2* sigma, int nactive) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int jb = blockIdx.y * SPMV_RJ;
    if (g >= P.n) return;
    const int nj = min(SPMV_RJ, nactive - jb);
    const double2* x[SPMV_RJ];
    double2 sg[SPMV_RJ], acc[SPMV_RJ];
#pragma unroll
    for (int r = 0; r < SPMV_RJ; ++r) {
        const int job = js.d_active[jb + (r < nj ? r : 0)];
        sg[r] = sigma[js.d_jobshift[job]];
        x[r] = js.vec + (size_t)job * js.vstride + (size_t)x_slot * js.n;
        acc[r] = make_double2(0.0, 0.0);
    }
    const int64_t e0 = P.rp[g], e1 = P.rp[g + 1];
    if (P.b_kind <= 1) {
        // B = I or diagonal: A - σB differs from A on the diagonal only, where
        // σB_gg is subtracted (a select rather than a branch keeps the loads in flight)
        const double2 b = P.Bdiag[g];
        double2 sb[SPMV_RJ];
#pragma unroll
        for (int r = 0; r < SPMV_RJ; ++r) sb[r] = cmul(sg[r], b);
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t j = P.ci[e];
            const double2 a = P.Ka[e];
            const bool d = j == g;
#pragma unroll
            for (int r = 0; r < SPMV_RJ; ++r) {
                if (r < nj) {
                    const double2 v = make_double2(d ? a.x - sb[r].x : a.x, d ? a.y - sb[r].y : a.y);
                    acc[r] = cfma(v, x[r][j], acc[r]);
                }
            }
        }
    } else {
        for (int64_t e = e0; e < e1; ++e) {
            const int64_t j = P.ci[e];
            const double2 a = P.Ka[e], b = P.Kb[e];
#pragma unroll
            for (int r = 0; r < SPMV_RJ; ++r) {
                if (r < nj) acc[r] = cfma(csub(a, cmul(sg[r], b)), x[r][j], acc[r]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < SPMV_RJ; ++r) {
        if (r >= nj) break;
        const int job = js.d_active[jb + r];
        double2 v = acc[r];
        if (rhs_slot >= 0) v = csub(js.vec[(size_t)job * js.vstride + (size_t)rhs_slot * js.n + g], v);
        js.vec[(size_t)job * js.vstride + (size_t)y_slot * js.n + g] = v;
    }
}

static void spmv_launch_rj(int rj, const Pencil& P, const JobSpace& js, int nactive, int x_slot, int y_slot,
                           int rhs_slot, const double2* d_sigma, cudaStream_t st) {
    const dim3 grid(cdiv_up(P.n, 256), cdiv_up(nactive, rj));
    switch (rj) {
        case 1: k_spmv_jobs<1><<<grid, 256, 0, st>>>(P, js, x_slot, y_slot, rhs_slot, d_sigma, nactive); break;
        case 2: k_spmv_jobs<2><<<grid, 256, 0, st>>>(P, js, x_slot, y_slot, rhs_slot, d_sigma, nactive); break;
        case 8: k_spmv_jobs<8><<<grid, 256, 0, st>>>(P, js, x_slot, y_slot, rhs_slot, d_sigma, nactive); break;
        default: k_spmv_jobs<4><<<grid, 256, 0, st>>>(P, js, x_slot, y_slot, rhs_slot, d_sigma, nactive); break;
    }
    SIM_LAUNCH_CHECK();
}

// y = (A - σB)x (or rhs - (A - σB)x) for the active jobs of the inner solver, timed as "spmv":
// algorithmic bytes: the matrix (20·nnz + 4(n+1)) once per RJ jobs, and per
// job x and y (32n, +16n with rhs); 8·nnz flops per job.  Jobs per thread
// (RJ) autotuned per matrix and batch size class.
static void launch_spmv(const Pencil& P, const JobSpace& js, int nactive, int x_slot, int y_slot, int rhs_slot,
                        const double2* d_sigma, cudaStream_t st) {
    static const int rjs[4] = {1, 2, 4, 8};
    const int cls = nactive < 4 ? nactive : (nactive < 16 ? 4 : 16);
    const std::string key = "spmv:" + std::to_string(P.n) + ":" + std::to_string(P.nnz) + ":" + std::to_string(cls);
    bool timing = false;
    const int rj = nactive == 1 ? 1 : rjs[autotune_begin(key, 4, st, &timing)];
    kprof_begin("spmv", st);
    spmv_launch_rj(rj, P, js, nactive, x_slot, y_slot, rhs_slot, d_sigma, st);
    if (timing) autotune_end(key, st);
    kprof_end("spmv", st,
              cdiv_up(nactive, rj) * (20.0 * P.nnz + 4.0 * (P.n + 1)) + nactive * (rhs_slot >= 0 ? 48.0 : 32.0) * P.n,
              nactive * 8.0 * P.nnz);
}

void spmv_shifted_jobs(const Pencil& P, const JobSpace& js, int nactive, const double*, int x_slot, int y_slot,
                       const double2* d_sigma, cudaStream_t st) {
    if (nactive <= 0) return;
    // untimed: also the path of the no-allocation entry point
    spmv_launch_rj(4, P, js, nactive, x_slot, y_slot, -1, d_sigma, st);
}

__global__ void k_apply_B(Pencil P, const double2* x, double2* y) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    if (P.b_kind == 0) { y[g] = x[g]; return; }
    if (P.b_kind == 1) { y[g] = cmul(P.Bdiag[g], x[g]); return; }
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t e = P.rp[g]; e < P.rp[g + 1]; ++e) acc = cfma(P.Kb[e], x[P.ci[e]], acc);
    y[g] = acc;
}

void apply_B(const Pencil& P, const double2* x, double2* y, cudaStream_t st) {
    k_apply_B<<<cdiv_up(P.n, 256), 256, 0, st>>>(P, x, y);
    SIM_LAUNCH_CHECK();
}

// u_job = B v_{j, job}  for all active jobs (V slot j -> vec slot)
__global__ void k_apply_B_jobs(Pencil P, JobSpace js, int j, int y_slot) {
    const int job = js.d_active[blockIdx.y];
    const double2* x = js.V + ((size_t)job * (js.m + 1) + j) * js.n;
    double2* y = js.vec + (size_t)job * js.vstride + (size_t)y_slot * js.n;
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= P.n) return;
    if (P.b_kind == 0) { y[g] = x[g]; return; }
    if (P.b_kind == 1) { y[g] = cmul(P.Bdiag[g], x[g]); return; }
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t e = P.rp[g]; e < P.rp[g + 1]; ++e) acc = cfma(P.Kb[e], x[P.ci[e]], acc);
    y[g] = acc;
}

// ---------------------------------------------------------------------------
// batched classical Gram–Schmidt, applied twice (CGS2), FP64
// ---------------------------------------------------------------------------
__device__ __forceinline__ void block_reduce_vec(double2* red, int cnt, int nw) {
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        double2 s = red[i * nw];
        for (int w = 1; w < nw; ++w) s = cadd(s, red[i * nw + w]);
        red[i * nw] = s;
    }
}

constexpr int GS_PER = GS_CHUNK / GS_THREADS;

__device__ __forceinline__ void gs_partial_dots(const GSArgs& a, const double2* B, const double2 (&wv)[GS_PER],
                                                int64_t r0, double2* red, double2* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = 0; i < a.cnt; ++i) {
        const double2* q = B + (size_t)i * a.n;
        double2 acc = make_double2(0.0, 0.0);
#pragma unroll
        for (int t = 0; t < GS_PER; ++t) {
            int64_t r = r0 + threadIdx.x + t * GS_THREADS;
            if (r < a.n) {
                double2 qv = q[r];
                acc.x = fma(qv.x, wv[t].x, acc.x);
                acc.x = fma(qv.y, wv[t].y, acc.x);
                acc.y = fma(qv.x, wv[t].y, acc.y);
                acc.y = fma(-qv.y, wv[t].x, acc.y);
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) red[i * nw + warp] = acc;
    }
    if (a.dgks) {  // partial ||w||^2 as value cnt
        double nn = 0.0;
#pragma unroll
        for (int t = 0; t < GS_PER; ++t) nn += wv[t].x * wv[t].x + wv[t].y * wv[t].y;
        nn = warp_sum(nn);
        if (lane == 0) red[a.cnt * nw + warp] = make_double2(nn, 0.0);
    }
    __syncthreads();
    block_reduce_vec(red, a.cnt + (a.dgks ? 1 : 0), nw);
    __syncthreads();
    for (int i = threadIdx.x; i < a.cnt + (a.dgks ? 1 : 0); i += blockDim.x) out[i] = red[i * nw];
}

// pass-1 partial dot products  h_i = Σ_rows conj(q_i) w
__global__ void __launch_bounds__(GS_THREADS) k_gs_dots(GSArgs a) {
    const int job = a.active[blockIdx.y];
    const int chunk = blockIdx.x;
    const double2* B = a.basis + (size_t)job * a.bstride;
    const double2* w = a.w + (size_t)job * a.wstride;
    extern __shared__ double2 red[];
    const int64_t r0 = (int64_t)chunk * GS_CHUNK;
    double2 wv[GS_PER];
#pragma unroll
    for (int t = 0; t < GS_PER; ++t) {
        int64_t r = r0 + threadIdx.x + t * GS_THREADS;
        wv[t] = r < a.n ? w[r] : make_double2(0.0, 0.0);
    }
    gs_partial_dots(a, B, wv, r0, red, a.pout + ((size_t)job * a.nchunk + chunk) * a.pw);
}

// reduce pass partials -> h; w -= Σ q_i h_i; then either the next pass's
// partial dots (next_dots = 1) or the partial squared norm.  hcol = h or += h.
__global__ void __launch_bounds__(GS_THREADS) k_gs_update(GSArgs a, int accumulate, int next_dots) {
    const int job = a.active[blockIdx.y];
    const int chunk = blockIdx.x;
    const double2* B = a.basis + (size_t)job * a.bstride;
    double2* w = a.w + (size_t)job * a.wstride;
    extern __shared__ double2 sm[];
    double2* h = sm;                 // [cnt]
    double2* red = sm + a.cnt + 1;   // [cnt*nw]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double2* Pin = a.pin + (size_t)job * a.nchunk * a.pw;
    double2* out = a.pout + ((size_t)job * a.nchunk + chunk) * a.pw;
    if (a.dgks && accumulate) {
        // second pass: needed only if the first one lost more than half of ||w||^2
        __shared__ int s_skip;
        if (threadIdx.x == 0) {
            double na = 0.0;
            for (int c = 0; c < a.nchunk; ++c) na += Pin[(size_t)c * a.pw + a.cnt].x;
            const double nb = Pin[a.cnt + 1].x;
            s_skip = na > 0.5 * nb;
        }
        __syncthreads();
        if (s_skip) {
            if (threadIdx.x == 0) out[0] = Pin[(size_t)chunk * a.pw + a.cnt];  // this chunk's ||w||^2
            return;
        }
    }
    for (int i = threadIdx.x; i < a.cnt; i += blockDim.x) {
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < a.nchunk; ++c) s = cadd(s, Pin[(size_t)c * a.pw + i]);
        h[i] = s;
    }
    if (a.dgks && !accumulate && chunk == 0 && threadIdx.x == 0) {
        double nb = 0.0;
        for (int c = 0; c < a.nchunk; ++c) nb += Pin[(size_t)c * a.pw + a.cnt].x;
        out[a.cnt + 1] = make_double2(nb, 0.0);  // ||w||^2 before the first pass, for the test above
    }
    __syncthreads();
    if (chunk == 0) {
        double2* hc = a.hcol + (size_t)job * a.hstride;
        for (int i = threadIdx.x; i < a.cnt; i += blockDim.x) hc[i] = accumulate ? cadd(hc[i], h[i]) : h[i];
    }
    const int64_t r0 = (int64_t)chunk * GS_CHUNK;
    double2 wv[GS_PER];
#pragma unroll
    for (int t = 0; t < GS_PER; ++t) {
        int64_t r = r0 + threadIdx.x + t * GS_THREADS;
        wv[t] = r < a.n ? w[r] : make_double2(0.0, 0.0);
    }
    for (int i = 0; i < a.cnt; ++i) {
        const double2* q = B + (size_t)i * a.n;
        const double2 hi = h[i];
#pragma unroll
        for (int t = 0; t < GS_PER; ++t) {
            int64_t r = r0 + threadIdx.x + t * GS_THREADS;
            if (r < a.n) {
                double2 qv = q[r];
                wv[t].x = fma(-qv.x, hi.x, wv[t].x);
                wv[t].x = fma(qv.y, hi.y, wv[t].x);
                wv[t].y = fma(-qv.x, hi.y, wv[t].y);
                wv[t].y = fma(-qv.y, hi.x, wv[t].y);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < GS_PER; ++t) {
        int64_t r = r0 + threadIdx.x + t * GS_THREADS;
        if (r < a.n) w[r] = wv[t];
    }
    if (next_dots) {
        gs_partial_dots(a, B, wv, r0, red, out);
    } else {
        double acc = 0.0;
#pragma unroll
        for (int t = 0; t < GS_PER; ++t) acc += wv[t].x * wv[t].x + wv[t].y * wv[t].y;
        acc = warp_sum(acc);
        if (lane == 0) red[warp] = make_double2(acc, 0.0);
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w2 = 0; w2 < nw; ++w2) s += red[w2].x;
            out[0] = make_double2(s, 0.0);
        }
    }
}

// partial ||w||^2 of each chunk (w read only), into pout[chunk]
__global__ void __launch_bounds__(GS_THREADS) k_gs_norm_partial(GSArgs a) {
    const int job = a.active[blockIdx.y];
    const int chunk = blockIdx.x;
    const double2* w = a.w + (size_t)job * a.wstride;
    __shared__ double red[GS_THREADS / 32];
    const int64_t r0 = (int64_t)chunk * GS_CHUNK;
    double acc = 0.0;
    for (int t = 0; t < GS_PER; ++t) {
        const int64_t r = r0 + threadIdx.x + t * GS_THREADS;
        if (r < a.n) {
            const double2 v = w[r];
            acc += v.x * v.x + v.y * v.y;
        }
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int i = 0; i < GS_THREADS / 32; ++i) sum += red[i];
        a.pout[((size_t)job * a.nchunk + chunk) * a.pw] = make_double2(sum, 0.0);
    }
}

// reduce norm partials, write the subdiagonal entry and normalise w in place
// (Arnoldi: breakdown test h_{j+1,j} <= btol * ||H_{1:j+1,1:j+1}||_F).
__global__ void __launch_bounds__(GS_THREADS) k_gs_finish(GSArgs a) {
    const int job = a.active[blockIdx.y];
    const int chunk = blockIdx.x;
    double2* w = a.w + (size_t)job * a.wstride;
    __shared__ double s_hn;
    __shared__ int s_broken;
    if (threadIdx.x == 0) {
        const double2* Pin = a.pin + (size_t)job * a.nchunk * a.pw;
        double s = 0.0;
        for (int c = 0; c < a.nchunk; ++c) s += Pin[(size_t)c * a.pw].x;
        double hn = sqrt(s);
        int broken = !(hn > 0.0);
        if (a.Hfull) {
            const double2* H = a.Hfull + (size_t)job * a.Hstride;
            double f = 0.0;
            for (int c = 0; c <= a.j; ++c)
                for (int r = 0; r <= a.j; ++r) f += cabs2(H[(size_t)c * a.Hld + r]);
            if (hn <= a.btol * sqrt(f)) broken = 1;
        }
        s_hn = hn;
        s_broken = broken;
        if (chunk == 0) {
            double2* hc = a.hcol + (size_t)job * a.hstride;
            hc[a.cnt] = make_double2((broken && a.Hfull) ? 0.0 : hn, 0.0);
            if (broken && a.meff) a.meff[job] = a.j + 1;
            if (broken && a.istat) a.istat[job * IS_N + IS_BROKEN] = 1;
        }
    }
    __syncthreads();
    if (s_broken) return;
    const double inv = 1.0 / s_hn;
    const int64_t r0 = (int64_t)chunk * GS_CHUNK;
    for (int t = 0; t < GS_PER; ++t) {
        int64_t r = r0 + threadIdx.x + t * GS_THREADS;
        if (r < a.n) w[r] = cscale(w[r], inv);
    }
}

// one CGS2 step on the active jobs: partial buffers A = partial, B = partial + half
static void gs_run(GSArgs a, double2* partial, size_t half, int nactive, cudaStream_t st) {
    if (gs_cluster(a, nactive, st)) return;
    kprof_begin("gram_schmidt", st);
    dim3 grid(a.nchunk, nactive);
    const int nw = GS_THREADS / 32;
    size_t sm_dots = (size_t)(a.cnt + 2) * nw * sizeof(double2) + 64;
    size_t sm_upd = ((size_t)a.cnt + 1 + (size_t)(a.cnt + 2) * nw) * sizeof(double2) + 64;
    double2* A = partial;
    double2* Bf = partial + half;
    if (a.single) {  // one pass: dots, update with the norm, finish
        a.dgks = 0;
        a.pout = A;
        k_gs_dots<<<grid, GS_THREADS, sm_dots, st>>>(a);
        SIM_LAUNCH_CHECK();
        a.pin = A;
        a.pout = Bf;
        k_gs_update<<<grid, GS_THREADS, sm_upd, st>>>(a, 0, 0);
        SIM_LAUNCH_CHECK();
        a.pin = Bf;
        k_gs_finish<<<grid, GS_THREADS, 0, st>>>(a);
        SIM_LAUNCH_CHECK();
        kprof_end("gram_schmidt", st, nactive * (2.0 * a.cnt + 4.0) * a.n * sizeof(double2),
                  nactive * 16.0 * a.cnt * a.n);
        return;
    }
    a.pout = A;
    k_gs_dots<<<grid, GS_THREADS, sm_dots, st>>>(a);
    SIM_LAUNCH_CHECK();
    a.pin = A;
    a.pout = Bf;
    k_gs_update<<<grid, GS_THREADS, sm_upd, st>>>(a, 0, 1);
    SIM_LAUNCH_CHECK();
    a.pin = Bf;
    a.pout = A;
    k_gs_update<<<grid, GS_THREADS, sm_upd, st>>>(a, 1, 0);
    SIM_LAUNCH_CHECK();
    a.pin = A;
    k_gs_finish<<<grid, GS_THREADS, 0, st>>>(a);
    SIM_LAUNCH_CHECK();
    kprof_end("gram_schmidt", st, nactive * (4.0 * a.cnt + 6.0) * a.n * sizeof(double2), nactive * 32.0 * a.cnt * a.n);
}

// ---------------------------------------------------------------------------
// batched FGMRES(k) with the block factorisation as right preconditioner
// ---------------------------------------------------------------------------
__global__ void k_copy_slot(JobSpace js, int src, int dst) {
    const int job = js.d_active[blockIdx.y];
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    js.vec[(size_t)job * js.vstride + (size_t)dst * js.n + g] = js.vec[(size_t)job * js.vstride + (size_t)src * js.n + g];
}

__global__ void k_zero_slot(JobSpace js, int dst) {
    const int job = js.d_active[blockIdx.y];
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    js.vec[(size_t)job * js.vstride + (size_t)dst * js.n + g] = make_double2(0.0, 0.0);
}

// after the start vector's norm γ landed in g[0]: reset the cycle state
__global__ void k_gm_cycle_init(JobSpace js, int nactive, int first, double tol) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nactive) return;
    const int job = js.d_active[t];
    double2* g = js.g + (size_t)job * (js.k + 1);
    double* sc = js.scal + (size_t)job * SC_N;
    int* is = js.istat + (size_t)job * IS_N;
    const double gamma = g[0].x;
    for (int i = 1; i <= js.k; ++i) g[i] = make_double2(0.0, 0.0);
    if (first) {
        sc[SC_RNORM0] = gamma;
        is[IS_ITERS] = 0;
        is[IS_DONE] = 0;
        is[IS_STALL] = 0;
        is[IS_LOOSE] = 0;
    }
    sc[SC_GAMMA] = gamma;
    sc[SC_RES] = gamma;
    is[IS_STEPS] = 0;
    const int conv = !(gamma > tol * sc[SC_RNORM0]);
    is[IS_CYCLE_DONE] = conv;
    if (conv) is[IS_DONE] = 1;
}

// Givens update of Hessenberg column i; residual estimate |g_{i+1}|
__global__ void k_gm_givens(JobSpace js, int nactive, int i, double tol, int max_iter) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nactive) return;
    const int job = js.d_active[t];
    const int k = js.k;
    double2* col = js.Hg + (size_t)job * (k + 1) * k + (size_t)i * (k + 1);
    double2* cs = js.cs + (size_t)job * k;
    double2* sn = js.sn + (size_t)job * k;
    double2* g = js.g + (size_t)job * (k + 1);
    double* sc = js.scal + (size_t)job * SC_N;
    int* is = js.istat + (size_t)job * IS_N;
    const double hn = col[i + 1].x;
    for (int q = 0; q < i; ++q) {
        const double c = cs[q].x;
        const double2 s = sn[q];
        double2 a = col[q], b = col[q + 1];
        col[q] = cadd(cscale(a, c), cmul(s, b));
        col[q + 1] = csub(cscale(b, c), cconjmul(s, a));
    }
    double2 a = col[i], b = col[i + 1];
    const double na = cabsd(a), nbv = cabsd(b);
    double c;
    double2 s;
    if (na == 0.0) {
        c = 0.0;
        s = make_double2(1.0, 0.0);
    } else {
        const double nu = hypot(na, nbv);
        c = na / nu;
        const double2 ph = cscale(a, 1.0 / na);
        s = cscale(cmulc(ph, b), 1.0 / nu);  // (a/|a|) conj(b) / nu
    }
    cs[i] = make_double2(c, 0.0);
    sn[i] = s;
    col[i] = cadd(cscale(a, c), cmul(s, b));
    col[i + 1] = make_double2(0.0, 0.0);
    const double2 gi = g[i];
    g[i] = cscale(gi, c);
    g[i + 1] = make_double2(-(s.x * gi.x + s.y * gi.y), -(s.x * gi.y - s.y * gi.x));  // -conj(s) g_i
    const double res = cabsd(g[i + 1]);
    sc[SC_RES] = res;
    is[IS_STEPS] = i + 1;
    is[IS_ITERS] += 1;
    is[IS_CYCLE_DONE] = (res <= tol * sc[SC_RNORM0]) || !(hn > 0.0) || (i + 1 == k) || (is[IS_ITERS] >= max_iter);
}

// x += Z y with R y = g (R: the rotated Hessenberg, order = steps)
__global__ void k_gm_update_x(JobSpace js) {
    const int job = js.d_active[blockIdx.y];
    const int k = js.k;
    __shared__ double2 y[64];
    __shared__ int steps;
    if (threadIdx.x == 0) {
        const int* is = js.istat + (size_t)job * IS_N;
        steps = is[IS_STEPS];
        const double2* R = js.Hg + (size_t)job * (k + 1) * k;
        const double2* g = js.g + (size_t)job * (k + 1);
        for (int r = steps - 1; r >= 0; --r) {
            double2 acc = g[r];
            for (int c = r + 1; c < steps; ++c) acc = csub(acc, cmul(R[(size_t)c * (k + 1) + r], y[c]));
            double2 d = R[(size_t)r * (k + 1) + r];
            y[r] = (d.x == 0.0 && d.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(acc, d);
        }
    }
    __syncthreads();
    int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= js.n) return;
    double2* base = js.vec + (size_t)job * js.vstride;
    double2 x = base[(size_t)VS_X * js.n + gi];
    for (int q = 0; q < steps; ++q) x = cfma(base[(size_t)(vs_Z(k) + q) * js.n + gi], y[q], x);
    base[(size_t)VS_X * js.n + gi] = x;
}

// explicit residual norm from partials (buffer pin), and ||x|| (buffer pinx):
// done if <= tol * rnorm0
__global__ void k_gm_check(JobSpace js, int nactive, const double2* pin, const double2* pinx, int nchunk, int pw,
                           double tol, int max_iter, const double2* sigma, double anorm, double bnorm) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nactive) return;
    const int job = js.d_active[t];
    const double2* P = pin + (size_t)job * nchunk * pw;
    const double2* PX = pinx + (size_t)job * nchunk * pw;
    double s = 0.0, sx = 0.0;
    for (int c = 0; c < nchunk; ++c) {
        s += P[(size_t)c * pw].x;
        sx += PX[(size_t)c * pw].x;
    }
    double* sc = js.scal + (size_t)job * SC_N;
    int* is = js.istat + (size_t)job * IS_N;
    const double r = sqrt(s);
    const double rel = sc[SC_RNORM0] > 0 ? r / sc[SC_RNORM0] : 0.0;
    const double prev = sc[SC_GAMMA] > 0 && sc[SC_RNORM0] > 0 ? sc[SC_GAMMA] / sc[SC_RNORM0] : INFINITY;
    sc[SC_WORST] = rel;
    if (rel <= tol) {
        is[IS_DONE] = 1;
        return;
    }
    // The rounding floor of the explicit residual b - (A - σB)x in FP64: about
    // ε ||A - σB|| ||x|| / ||b|| (||A - σB|| <= ||A||_inf + |σ| ||B||_inf); near an
    // eigenvalue ||x|| / ||b|| is large and the floor rises above tol.
    const double2 sg = sigma[js.d_jobshift[job]];
    const double floor_rel = sc[SC_RNORM0] > 0
                                 ? 32.0 * 1.1102230246251565e-16 * (anorm + hypot(sg.x, sg.y) * bnorm) * sqrt(sx) /
                                       sc[SC_RNORM0]
                                 : 0.0;
    const double lim = fmax(tol, floor_rel);
    // A restart cycle that did not halve the residual has stagnated.  Stop early
    // only at the rounding floor: after one such cycle if the residual is already
    // within 10 max(tol, floor), else after two in a row.  An early stop (or the
    // iteration cap) accepts the solve within 100 max(tol, floor), counted as
    // loose, else fails.
    const int stall = rel > 0.5 * prev ? is[IS_STALL] + 1 : 0;
    is[IS_STALL] = stall;
    if (is[IS_ITERS] >= max_iter || (stall >= 1 && rel <= 10.0 * lim) || stall >= 2) {
        const int ok = rel <= 100.0 * lim;
        is[IS_DONE] = ok ? 1 : -1;
        is[IS_LOOSE] = ok;
    }
}

namespace {
struct Pinned {
    int* ist = nullptr;
    double* sc = nullptr;
    int* act = nullptr;
    int cap = 0;
    cudaEvent_t act_ev = nullptr;  // the last upload from `act`
    void ensure(int J) {
        if (J <= cap) return;
        if (ist) cudaFreeHost(ist);
        if (sc) cudaFreeHost(sc);
        if (act) cudaFreeHost(act);
        SIM_CUDA(cudaMallocHost(&ist, sizeof(int) * IS_N * J));
        SIM_CUDA(cudaMallocHost(&sc, sizeof(double) * SC_N * J));
        SIM_CUDA(cudaMallocHost(&act, sizeof(int) * J));
        cap = J;
    }
};
Pinned g_pin;

void upload_active(const JobSpace& js, const std::vector<int>& a, cudaStream_t st) {
    g_pin.ensure(js.J);
    // the previous upload must have left the pinned buffer before it is refilled
    if (g_pin.act_ev) SIM_CUDA(cudaEventSynchronize(g_pin.act_ev));
    else SIM_CUDA(cudaEventCreateWithFlags(&g_pin.act_ev, cudaEventDisableTiming));
    for (size_t i = 0; i < a.size(); ++i) g_pin.act[i] = a[i];
    SIM_CUDA(cudaMemcpyAsync(js.d_active, g_pin.act, sizeof(int) * a.size(), cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaEventRecord(g_pin.act_ev, st));
}

void read_state(const JobSpace& js, cudaStream_t st) {
    g_pin.ensure(js.J);
    SIM_CUDA(cudaMemcpyAsync(g_pin.ist, js.istat, sizeof(int) * IS_N * js.J, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaMemcpyAsync(g_pin.sc, js.scal, sizeof(double) * SC_N * js.J, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaStreamSynchronize(st));
}

// ||slot|| of active jobs into hcol[0] (stride), and scale slot by 1/||slot||
void norm_and_scale(const JobSpace& js, int nactive, double2* w_base, int64_t wstride, double2* hcol,
                    int64_t hstride, cudaStream_t st) {
    GSArgs a{};
    a.basis = nullptr;
    a.bstride = 0;
    a.w = w_base;
    a.wstride = wstride;
    a.hcol = hcol;
    a.hstride = hstride;
    a.cnt = 0;
    a.n = js.n;
    a.pw = js.pw;
    a.nchunk = js.nchunk;
    a.active = js.d_active;
    if (gs_cluster(a, nactive, st)) return;
    dim3 grid(js.nchunk, nactive);
    const int nw = GS_THREADS / 32;
    a.pout = js.partial;
    k_gs_update<<<grid, GS_THREADS, (size_t)(1 + nw) * sizeof(double2) + 64, st>>>(a, 0, 0);
    SIM_LAUNCH_CHECK();
    a.pin = js.partial;
    k_gs_finish<<<grid, GS_THREADS, 0, st>>>(a);
    SIM_LAUNCH_CHECK();
}
}  // namespace

bool inner_solve(const Pencil& P, const sim_options& opt, JobSpace& js, const std::vector<int>& jobs,
                 const double2* d_sigma, void* const* d_factor_ptrs, cudaStream_t st, InnerStats& stats) {
    if (jobs.empty()) return true;
    const int k = js.k;
    const dim3 rows_grid_1(cdiv_up(js.n, 256), 1);
    const size_t half = (size_t)js.J * js.nchunk * js.pw;
    auto rows_grid = [&](int na) { return dim3(cdiv_up(js.n, 256), na); };
    (void)rows_grid_1;
    std::vector<int> cyc = jobs;  // jobs that start a cycle
    upload_active(js, cyc, st);
    k_zero_slot<<<rows_grid((int)cyc.size()), 256, 0, st>>>(js, VS_X);
    SIM_LAUNCH_CHECK();
    k_copy_slot<<<rows_grid((int)cyc.size()), 256, 0, st>>>(js, VS_RHS, VS_R);
    SIM_LAUNCH_CHECK();
    bool first = true;
    bool ok = true;
    while (!cyc.empty()) {
        const int nc = (int)cyc.size();
        upload_active(js, cyc, st);
        k_copy_slot<<<rows_grid(nc), 256, 0, st>>>(js, VS_R, VS_Q0);
        SIM_LAUNCH_CHECK();
        norm_and_scale(js, nc, js.vec + (size_t)VS_Q0 * js.n, js.vstride, js.g, k + 1, st);
        k_gm_cycle_init<<<cdiv_up(nc, 128), 128, 0, st>>>(js, nc, first ? 1 : 0, opt.inner_tol);
        SIM_LAUNCH_CHECK();
        first = false;
        read_state(js, st);
        std::vector<int> act;
        for (int j : cyc)
            if (!g_pin.ist[j * IS_N + IS_CYCLE_DONE]) act.push_back(j);
        std::vector<int> in_cycle = act;
        for (int i = 0; i < k && !act.empty(); ++i) {
            const int na = (int)act.size();
            upload_active(js, act, st);
            if (P.sep)
                separable_apply(P.sep->S, opt.precision, js, act, VS_Q0 + i, vs_Z(k) + i, d_sigma, *P.sep->ar, st);
            else if (!js.h_jobshift ||
                     !block_solve_cluster(P, opt.precision, js, act, VS_Q0 + i, vs_Z(k) + i, d_sigma, d_factor_ptrs, st))
                throw std::runtime_error("LIMIT:block size " + std::to_string(P.T) +
                                         " too large for the cluster block solve's shared memory");
            launch_spmv(P, js, na, vs_Z(k) + i, VS_Q0 + i + 1, -1, d_sigma, st);
            GSArgs a{};
            a.basis = js.vec + (size_t)VS_Q0 * js.n;
            a.bstride = js.vstride;
            a.w = js.vec + (size_t)(VS_Q0 + i + 1) * js.n;
            a.wstride = js.vstride;
            a.hcol = js.Hg + (size_t)i * (k + 1);
            a.hstride = (int64_t)(k + 1) * k;
            a.cnt = i + 1;
            a.n = js.n;
            a.pw = js.pw;
            a.nchunk = js.nchunk;
            a.active = js.d_active;
            a.dgks = 1;
            gs_run(a, js.partial, half, na, st);
            k_gm_givens<<<cdiv_up(na, 128), 128, 0, st>>>(js, na, i, opt.inner_tol, opt.inner_max_iter);
            SIM_LAUNCH_CHECK();
            read_state(js, st);
            std::vector<int> next;
            for (int j : act)
                if (!g_pin.ist[j * IS_N + IS_CYCLE_DONE]) next.push_back(j);
            act.swap(next);
        }
        if (in_cycle.empty()) break;
        const int ni = (int)in_cycle.size();
        upload_active(js, in_cycle, st);
        k_gm_update_x<<<rows_grid(ni), 256, 0, st>>>(js);
        SIM_LAUNCH_CHECK();
        launch_spmv(P, js, ni, VS_X, VS_R, VS_RHS, d_sigma, st);
        {
            GSArgs a{};
            a.w = js.vec + (size_t)VS_R * js.n;
            a.wstride = js.vstride;
            a.cnt = 0;
            a.n = js.n;
            a.pw = js.pw;
            a.nchunk = js.nchunk;
            a.active = js.d_active;
            a.pout = js.partial;
            const int nw = GS_THREADS / 32;
            k_gs_update<<<dim3(js.nchunk, ni), GS_THREADS, (size_t)(1 + nw) * sizeof(double2) + 64, st>>>(a, 0, 0);
            SIM_LAUNCH_CHECK();
            // ||x||^2 partials into the second half, for the rounding floor
            a.w = js.vec + (size_t)VS_X * js.n;
            a.pout = js.partial + half;
            k_gs_norm_partial<<<dim3(js.nchunk, ni), GS_THREADS, 0, st>>>(a);
            SIM_LAUNCH_CHECK();
        }
        k_gm_check<<<cdiv_up(ni, 128), 128, 0, st>>>(js, ni, js.partial, js.partial + half, js.nchunk, js.pw,
                                                     opt.inner_tol, opt.inner_max_iter, d_sigma, P.anorm, P.bnorm);
        SIM_LAUNCH_CHECK();
        read_state(js, st);
        std::vector<int> again;
        for (int j : in_cycle) {
            int d = g_pin.ist[j * IS_N + IS_DONE];
            if (d == 0) again.push_back(j);
            if (d == -1) ok = false;
        }
        cyc.swap(again);
    }
    for (int j : jobs) {
        int it = g_pin.ist[j * IS_N + IS_ITERS];
        stats.solves += 1;
        stats.iters += it;
        stats.max_iters = std::max(stats.max_iters, it);
        stats.worst = std::max(stats.worst, g_pin.sc[j * SC_N + SC_WORST]);
        stats.loose += g_pin.ist[j * IS_N + IS_LOOSE];
        if (g_pin.ist[j * IS_N + IS_DONE] != 1) ok = false;
    }
    return ok;
}

// ---------------------------------------------------------------------------
// Arnoldi with CGS2 for all jobs of the space
// ---------------------------------------------------------------------------
__global__ void k_copy_to_V(JobSpace js, int src_slot, int j) {
    const int job = js.d_active[blockIdx.y];
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    js.V[((size_t)job * (js.m + 1) + j) * js.n + g] = js.vec[(size_t)job * js.vstride + (size_t)src_slot * js.n + g];
}

__global__ void k_arnoldi_init(JobSpace js, int nactive) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nactive) return;
    const int job = js.d_active[t];
    js.meff[job] = js.m;
    js.istat[job * IS_N + IS_BROKEN] = 0;
    double2* H = js.H + (size_t)job * (js.m + 1) * js.m;
    for (int e = 0; e < (js.m + 1) * js.m; ++e) H[e] = make_double2(0.0, 0.0);
}

__global__ void k_store_beta(JobSpace js, int nactive) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nactive) return;
    const int job = js.d_active[t];
    js.beta[job] = js.g[(size_t)job * (js.k + 1)].x;
}

bool arnoldi(const Pencil& P, const sim_options& opt, JobSpace& js, const double2* d_sigma,
             void* const* d_factor_ptrs, cudaStream_t st, InnerStats& stats, bool single_pass) {
    const int J = js.J, m = js.m;
    std::vector<int> all(J);
    for (int j = 0; j < J; ++j) all[j] = j;
    auto rows_grid = [&](int na) { return dim3(cdiv_up(js.n, 256), na); };
    bool ok = inner_solve(P, opt, js, all, d_sigma, d_factor_ptrs, st, stats);  // b = K^{-1} f
    upload_active(js, all, st);
    k_arnoldi_init<<<cdiv_up(J, 128), 128, 0, st>>>(js, J);
    SIM_LAUNCH_CHECK();
    k_copy_to_V<<<rows_grid(J), 256, 0, st>>>(js, VS_X, 0);
    SIM_LAUNCH_CHECK();
    // beta = ||b||, v_1 = b / beta   (the norm lands in g[job*(k+1)] as scratch)
    norm_and_scale(js, J, js.V, (int64_t)(m + 1) * js.n, js.g, js.k + 1, st);
    k_store_beta<<<cdiv_up(J, 128), 128, 0, st>>>(js, J);
    SIM_LAUNCH_CHECK();
    const size_t half = (size_t)js.J * js.nchunk * js.pw;
    std::vector<int> act = all;
    std::vector<int> broken(J, 0);
    for (int j = 0; j < m && !act.empty(); ++j) {
        const int na = (int)act.size();
        upload_active(js, act, st);
        k_apply_B_jobs<<<rows_grid(na), 256, 0, st>>>(P, js, j, VS_RHS);
        SIM_LAUNCH_CHECK();
        ok = inner_solve(P, opt, js, act, d_sigma, d_factor_ptrs, st, stats) && ok;
        upload_active(js, act, st);
        k_copy_to_V<<<rows_grid(na), 256, 0, st>>>(js, VS_X, j + 1);
        SIM_LAUNCH_CHECK();
        GSArgs a{};
        a.basis = js.V;
        a.bstride = (int64_t)(m + 1) * js.n;
        a.w = js.V + (size_t)(j + 1) * js.n;
        a.wstride = (int64_t)(m + 1) * js.n;
        a.hcol = js.H + (size_t)j * (m + 1);
        a.hstride = (int64_t)(m + 1) * m;
        a.cnt = j + 1;
        a.n = js.n;
        a.pw = js.pw;
        a.nchunk = js.nchunk;
        a.active = js.d_active;
        a.Hfull = js.H;
        a.Hstride = (int64_t)(m + 1) * m;
        a.Hld = m + 1;
        a.j = j;
        a.btol = opt.breakdown_tol;
        a.meff = js.meff;
        a.istat = js.istat;
        a.single = single_pass ? 1 : 0;
        gs_run(a, js.partial, half, na, st);
        read_state(js, st);
        std::vector<int> next;
        for (int q : act)
            if (!g_pin.ist[q * IS_N + IS_BROKEN]) next.push_back(q);
        act.swap(next);
    }
    SIM_CUDA(cudaStreamSynchronize(st));
    return ok;
}

int max_jobs_for_memory(int64_t n, int m, int k) {
    size_t fr = 0, tot = 0;
    SIM_CUDA(cudaMemGetInfo(&fr, &tot));
    const double per_job = (double)(vs_count(k) + m + 1 + 2) * (double)n * sizeof(double2);
    const double jobs = 0.4 * (double)tot / per_job;
    return (int)std::max(1.0, std::min(jobs, 1e6));
}

JobSpace make_jobspace(DeviceArena& ar, cudaStream_t st, int J, int k, int m, int64_t n, const std::string& tag) {
    JobSpace js;
    js.J = J;
    js.k = k;
    js.m = m;
    js.n = n;
    const int nv = vs_count(js.k);
    js.vstride = (int64_t)nv * js.n;
    js.vec = ar.get<double2>(tag + "vec", (int64_t)J * js.vstride);
    js.V = ar.get<double2>(tag + "V", (int64_t)J * (js.m + 1) * js.n);
    js.H = ar.get<double2>(tag + "H", (int64_t)J * (js.m + 1) * js.m);
    js.beta = ar.get<double>(tag + "beta", J);
    js.meff = ar.get<int>(tag + "meff", J);
    js.Hg = ar.get<double2>(tag + "Hg", (int64_t)J * (js.k + 1) * js.k);
    js.cs = ar.get<double2>(tag + "cs", (int64_t)J * js.k);
    js.sn = ar.get<double2>(tag + "sn", (int64_t)J * js.k);
    js.g = ar.get<double2>(tag + "g", (int64_t)J * (js.k + 1));
    js.scal = ar.get<double>(tag + "scal", (int64_t)J * SC_N);
    js.istat = ar.get<int>(tag + "istat", (int64_t)J * IS_N);
    js.nchunk = cdiv_up(js.n, GS_CHUNK);
    js.pw = std::max(js.m + 2, js.k + 2);
    js.partial = ar.get<double2>(tag + "partial", (int64_t)2 * J * js.nchunk * js.pw);
    js.d_jobshift = ar.get<int>(tag + "jobshift", J);
    js.d_active = ar.get<int>(tag + "active", J);
    SIM_CUDA(cudaMemsetAsync(js.istat, 0, sizeof(int) * J * IS_N, st));
    SIM_CUDA(cudaMemsetAsync(js.scal, 0, sizeof(double) * J * SC_N, st));
    return js;
}

}  // namespace sim
