// Ritz refinement of the located eigenvalues (Sec. 3.2, Eq. zjHm).
//
// H_m = P D P^{-1}: the eigenvalues d_i of a shift's Hessenberg matrix are
// Ritz values of the Cayley transform M = (A - σB)^{-1}B, whose eigenvalues
// are 1/(λ - σ), so λ_i = σ + 1/d_i.  For each located cluster the λ_i
// nearest its estimate replaces the estimate when it lies within
// 2·max(cluster radius, h0) of it.
//
// k_ritz: one warp per shift computes every eigenvalue of its m_eff × m_eff
// upper Hessenberg matrix (FP64) by the shifted QR algorithm: Wilkinson shift
// from the trailing 2×2 block, one sweep of Givens rotations over the active
// block, deflation where a subdiagonal entry falls below ε times its two
// diagonal neighbours, an exceptional shift after 10 sweeps without
// deflation, and at most 30·m_eff sweeps per matrix (else the shift is
// flagged).  Lane 0 forms the rotations; the lanes apply them along rows and
// columns.  k_ritz_pick: one thread per cluster.
#include <cfloat>

#include "hess.cuh"
#include "internal.h"
#include "ritz.h"

namespace sim {

namespace {

__device__ __forceinline__ double cabs_h(double2 a) { return hypot(a.x, a.y); }

// principal square root of a complex number, from sqrt(z) = sqrt((|z|+x)/2) + i sign(y) sqrt((|z|-x)/2)
__device__ __forceinline__ double2 csqrt_p(double2 z) {
    const double r = cabs_h(z);
    const double re = sqrt(fmax(0.0, 0.5 * (r + z.x)));
    const double im = sqrt(fmax(0.0, 0.5 * (r - z.x)));
    return make_double2(re, z.y < 0.0 ? -im : im);
}

__global__ void __launch_bounds__(32) k_ritz(const double2* Hall, int m, const int* meff_all, const int* list,
                                             double2* ritz, int* status) {
    const int s = list[blockIdx.x];
    const int n = meff_all[s];
    const double2* Hs = Hall + (size_t)s * (m + 1) * m;  // column-major, leading dimension m + 1
    extern __shared__ double2 A[];                         // [n][n] row-major, leading dimension m
    __shared__ double gc[64];
    __shared__ double2 gs[64];
    __shared__ double2 s_mu;
    __shared__ int s_l;
    const int lane = threadIdx.x;
    double2* out = ritz + (size_t)blockIdx.x * m;
    for (int idx = lane; idx < n * n; idx += 32) {
        const int r = idx / n, c = idx % n;
        A[r * m + c] = (r <= c + 1) ? Hs[(size_t)c * (m + 1) + r] : make_double2(0.0, 0.0);  // Hessenberg part only
    }
    // a scale for the deflation test when both diagonal neighbours vanish
    double nrm = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) nrm = fmax(nrm, cabs_h(A[(idx / n) * m + idx % n]));
    for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    __syncwarp();
    int hi = n - 1, its = 0, sweeps = 0, fail = 0;
    while (hi >= 0) {
        if (hi == 0) {
            if (lane == 0) out[0] = A[0];
            break;
        }
        if (lane == 0) {
            int l = hi;
            while (l > 0) {
                const double sub = cabs_h(A[l * m + l - 1]);
                double d = cabs_h(A[(l - 1) * m + l - 1]) + cabs_h(A[l * m + l]);
                if (d == 0.0) d = nrm;
                if (sub <= DBL_EPSILON * d) break;
                --l;
            }
            if (l > 0) A[l * m + l - 1] = make_double2(0.0, 0.0);
            s_l = l;
            if (l != hi) {
                // Wilkinson shift: the eigenvalue of the trailing 2×2 block nearer its last entry
                const double2 p = A[(hi - 1) * m + hi - 1], q = A[(hi - 1) * m + hi];
                const double2 r = A[hi * m + hi - 1], t = A[hi * m + hi];
                double2 mu = t;
                if (its > 0 && its % 10 == 0) {
                    mu.x += 0.75 * cabs_h(r);  // exceptional shift
                } else {
                    const double2 d = make_double2(0.5 * (p.x - t.x), 0.5 * (p.y - t.y));
                    const double2 qr = cmul(q, r);
                    const double2 disc = csqrt_p(cadd(cmul(d, d), qr));
                    const double2 den1 = cadd(d, disc), den2 = csub(d, disc);
                    const double2 den = cabs_h(den1) >= cabs_h(den2) ? den1 : den2;
                    if (cabs_h(den) > 0.0) mu = csub(t, cdiv(qr, den));
                }
                s_mu = mu;
            }
        }
        __syncwarp();
        const int l = s_l;
        if (l == hi) {
            if (lane == 0) out[hi] = A[hi * m + hi];
            --hi;
            its = 0;
            __syncwarp();
            continue;
        }
        if (++sweeps > 30 * n) {
            fail = 1;
            break;
        }
        ++its;
        const double2 mu = s_mu;
        for (int k = l + lane; k <= hi; k += 32) A[k * m + k] = csub(A[k * m + k], mu);
        __syncwarp();
        // rows: G_k zeroes A[k+1][k], applied to rows k, k+1 (columns k..hi)
        for (int k = l; k < hi; ++k) {
            if (lane == 0) {
                const double2 a = A[k * m + k], b = A[(k + 1) * m + k];
                const double na = cabs_h(a), nb = cabs_h(b);
                double c;
                double2 sn;
                if (nb == 0.0) {
                    c = 1.0;
                    sn = make_double2(0.0, 0.0);
                } else if (na == 0.0) {
                    c = 0.0;
                    sn = make_double2(b.x / nb, -b.y / nb);
                } else {
                    const double h = hypot(na, nb);
                    c = na / h;
                    const double2 ua = make_double2(a.x / na, a.y / na);  // a / |a|
                    sn = cmul(ua, make_double2(b.x / h, -b.y / h));     // (a/|a|) conj(b) / h
                }
                gc[k - l] = c;
                gs[k - l] = sn;
            }
            __syncwarp();
            const double c = gc[k - l];
            const double2 sn = gs[k - l];
            for (int j = k + lane; j <= hi; j += 32) {
                const double2 x = A[k * m + j], y = A[(k + 1) * m + j];
                A[k * m + j] = cadd(make_double2(c * x.x, c * x.y), cmul(sn, y));
                A[(k + 1) * m + j] = csub(make_double2(c * y.x, c * y.y), cmul(make_double2(sn.x, -sn.y), x));
            }
            __syncwarp();
        }
        // columns: R G_l^H ... G_{hi-1}^H
        for (int k = l; k < hi; ++k) {
            const double c = gc[k - l];
            const double2 sn = gs[k - l];
            const int rmax = min(k + 1, hi);
            for (int i = l + lane; i <= rmax; i += 32) {
                const double2 x = A[i * m + k], y = A[i * m + k + 1];
                A[i * m + k] = cadd(make_double2(c * x.x, c * x.y), cmul(make_double2(sn.x, -sn.y), y));
                A[i * m + k + 1] = csub(make_double2(c * y.x, c * y.y), cmul(sn, x));
            }
            __syncwarp();
        }
        for (int k = l + lane; k <= hi; k += 32) A[k * m + k] = cadd(A[k * m + k], mu);
        __syncwarp();
    }
    if (lane == 0) status[blockIdx.x] = fail;
}

__global__ void k_ritz_pick(int C, const double2* est, const double* radius, const int* cl_slot, const int* list,
                            const int* meff_all, const double2* sigma, const double2* ritz, int m, double h0,
                            double2* out, int* flag) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    const int b = cl_slot[c];
    const int s = list[b];
    const double2 e = est[c], sg = sigma[s];
    const double2* d = ritz + (size_t)b * m;
    double best = -1.0;
    double2 lam_best = e;
    for (int i = 0; i < meff_all[s]; ++i) {
        if (d[i].x == 0.0 && d[i].y == 0.0) continue;
        const double2 lam = cadd(sg, cdiv(make_double2(1.0, 0.0), d[i]));
        const double dist = cabs_h(csub(lam, e));
        if (best < 0.0 || dist < best) {
            best = dist;
            lam_best = lam;
        }
    }
    const bool ok = best >= 0.0 && best <= 2.0 * fmax(radius[c], h0);
    out[c] = ok ? lam_best : e;
    flag[c] = ok ? 1 : 0;
}


// Sec. 3.2, Eq. zjHm: the eigenvectors of H_m for its eigenvalues d_i (k_ritz),
// by one step of inverse iteration from e_1 — (H_m - d_i I) v = e_1 as
// (I - H_m/d_i) v = -e_1/d_i, the warp Hessenberg solve — normalised to unit
// length: the columns of P.  Then c_1 = P^{-1} e_1 (Gaussian elimination with
// partial pivoting) and, per eigenvalue, w_i = β e_m^T P e_i c_1[i] (so that
// e_m^T y = Σ_i w_i / (1 + (σ - z) d_i), Eq. rmLc1) and |c_1[i]|.
// One CTA of 4 warps per shift; P lives in global scratch (m × m per shift).
constexpr int EIG_WARPS = 4;

__global__ void __launch_bounds__(EIG_WARPS * 32) k_eigdec(const double2* Hall, int m, const int* meff_all,
                                                           const double* beta_all, const int* list,
                                                           const double2* ritz, double2* Pg, double2* w_out,
                                                           double* absc_out, int* status) {
    const int s = list[blockIdx.x];
    const int me = meff_all[s];
    const double2* H = Hall + (size_t)s * (m + 1) * m;
    extern __shared__ double2 sh[];
    double2* Hs = sh;                                   // [me][me]
    const int usz = me * (me + 1) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double2* U = Hs + (size_t)me * me + (size_t)warp * (usz + me);
    double2* ys = U + usz;
    double2* P = Pg + (size_t)blockIdx.x * m * m;       // row-major, leading dimension me
    const double2* d = ritz + (size_t)blockIdx.x * m;
    __shared__ int s_bad;
    if (threadIdx.x == 0) s_bad = 0;
    stage_H(H, m, me, Hs);
    __syncthreads();
    for (int i = warp; i < me; i += EIG_WARPS) {
        const double2 di = d[i];
        double ylast = 0.0, yn2 = 0.0;
        bool ok = false;
        for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
            // the second attempt moves the shift off an exactly singular pivot
            const double2 dd = attempt == 0 ? di : cscale(di, 1.0 + 1e-13);
            const double2 alpha = cdiv(make_double2(-1.0, 0.0), dd);
            warp_hess_solve(Hs, me, alpha, 1.0, U, ys, ylast, yn2);
            ok = yn2 > 0.0 && isfinite(yn2);
        }
        const double inv = ok ? 1.0 / sqrt(yn2) : 0.0;
        for (int r = lane; r < me; r += 32) P[(size_t)r * me + i] = cscale(ys[r], inv);
        if (!ok && lane == 0) s_bad = 1;
        __syncwarp();
    }
    __syncthreads();
    // c_1 = P^{-1} e_1: eliminate on a copy of P (in the per-warp scratch, 2·me·(me+1) >= me² + me entries)
    double2* M = Hs + (size_t)me * me;
    double2* rhs = M + (size_t)me * me;
    for (int e = threadIdx.x; e < me * me; e += blockDim.x) M[e] = P[e];
    for (int r = threadIdx.x; r < me; r += blockDim.x) rhs[r] = make_double2(r == 0 ? 1.0 : 0.0, 0.0);
    __shared__ int s_piv;
    __syncthreads();
    for (int k = 0; k < me; ++k) {
        if (threadIdx.x == 0) {
            int pr = k;
            double best = -1.0;
            for (int r = k; r < me; ++r) {
                const double v = fabs(M[(size_t)r * me + k].x) + fabs(M[(size_t)r * me + k].y);
                if (v > best) {
                    best = v;
                    pr = r;
                }
            }
            if (!(best > 0.0)) s_bad = 1;
            s_piv = pr;
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k) {
            for (int c = threadIdx.x; c < me; c += blockDim.x) {
                const double2 t = M[(size_t)k * me + c];
                M[(size_t)k * me + c] = M[(size_t)pr * me + c];
                M[(size_t)pr * me + c] = t;
            }
            if (threadIdx.x == 0) {
                const double2 t = rhs[k];
                rhs[k] = rhs[pr];
                rhs[pr] = t;
            }
        }
        __syncthreads();
        const double2 piv = M[(size_t)k * me + k];
        const bool zero = piv.x == 0.0 && piv.y == 0.0;
        for (int e = threadIdx.x; e < (me - k - 1) * (me - k); e += blockDim.x) {
            const int r = k + 1 + e / (me - k), c = k + e % (me - k);
            const double2 l = zero ? make_double2(0.0, 0.0) : cdiv(M[(size_t)r * me + k], piv);
            if (c == k) continue;  // column k is consumed by the factor l (read before it is cleared below)
            M[(size_t)r * me + c] = csub(M[(size_t)r * me + c], cmul(l, M[(size_t)k * me + c]));
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int r = k + 1; r < me; ++r) {
                const double2 l = zero ? make_double2(0.0, 0.0) : cdiv(M[(size_t)r * me + k], piv);
                rhs[r] = csub(rhs[r], cmul(l, rhs[k]));
                M[(size_t)r * me + k] = make_double2(0.0, 0.0);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int r = me - 1; r >= 0; --r) {
            double2 acc = rhs[r];
            for (int c = r + 1; c < me; ++c) acc = csub(acc, cmul(M[(size_t)r * me + c], rhs[c]));
            const double2 dg = M[(size_t)r * me + r];
            rhs[r] = (dg.x == 0.0 && dg.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(acc, dg);
        }
        status[blockIdx.x] = s_bad;
    }
    __syncthreads();
    const double beta = beta_all[s];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        if (i < me) {
            w_out[(size_t)blockIdx.x * m + i] = cscale(cmul(P[(size_t)(me - 1) * me + i], rhs[i]), beta);
            absc_out[(size_t)blockIdx.x * m + i] = cabs_h(rhs[i]);
        } else {
            w_out[(size_t)blockIdx.x * m + i] = make_double2(0.0, 0.0);
            absc_out[(size_t)blockIdx.x * m + i] = 0.0;
        }
    }
}

// e_m^T y and the β-relative residual of Eq. eq:error at points z (Eq. rmLc1)
__global__ void k_screen_points(int me, double hlast, double beta, double2 sigma, const double2* d, const double2* w,
                                const double2* z, int64_t count, double2* ym, double* rho) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const double2 alpha = csub(sigma, z[t]);
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < me; ++i)
        acc = cadd(acc, cdiv(w[i], make_double2(1.0 + (alpha.x * d[i].x - alpha.y * d[i].y),
                                                alpha.x * d[i].y + alpha.y * d[i].x)));
    ym[t] = acc;
    rho[t] = cabs_h(alpha) * hlast * cabs_h(acc) / beta;
}

}  // namespace

bool ritz_refine(const RitzInput& in, std::vector<double2>& out, std::vector<int>& flags) {
    const int C = (int)in.est.size();
    out.assign(in.est.begin(), in.est.end());
    flags.assign(C, 0);
    if (C == 0) return true;
    // the shifts that resolve clusters, and each cluster's slot among them
    std::vector<int> list, slot(C);
    std::vector<int> where(in.num_slots, -1);
    for (int c = 0; c < C; ++c) {
        const int s = in.shift[c];
        if (where[s] < 0) {
            where[s] = (int)list.size();
            list.push_back(s);
        }
        slot[c] = where[s];
    }
    const int S = (int)list.size();
    DeviceArena& ar = *in.arena;
    cudaStream_t st = in.st;
    const int m = in.m;
    int* d_list = ar.get<int>("rz_list", S);
    int* d_slot = ar.get<int>("rz_slot", C);
    int* d_status = ar.get<int>("rz_status", S);
    double2* d_ritz = ar.get<double2>("rz_ritz", (int64_t)S * m);
    double2* d_est = ar.get<double2>("rz_est", C);
    double* d_rad = ar.get<double>("rz_rad", C);
    double2* d_out = ar.get<double2>("rz_out", C);
    int* d_flag = ar.get<int>("rz_flag", C);
    SIM_CUDA(cudaMemcpyAsync(d_list, list.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_slot, slot.data(), sizeof(int) * C, cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_est, in.est.data(), sizeof(double2) * C, cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_rad, in.radius.data(), sizeof(double) * C, cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemsetAsync(d_ritz, 0, sizeof(double2) * S * m, st));
    const size_t smem = (size_t)m * m * sizeof(double2);
    k_ritz<<<S, 32, smem, st>>>(in.d_H, m, in.d_meff, d_list, d_ritz, d_status);
    SIM_LAUNCH_CHECK();
    k_ritz_pick<<<cdiv_up(C, 128), 128, 0, st>>>(C, d_est, d_rad, d_slot, d_list, in.d_meff, in.d_sigma, d_ritz, m,
                                                 in.h0, d_out, d_flag);
    SIM_LAUNCH_CHECK();
    std::vector<int> status(S);
    SIM_CUDA(cudaMemcpyAsync(status.data(), d_status, sizeof(int) * S, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaMemcpyAsync(out.data(), d_out, sizeof(double2) * C, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaMemcpyAsync(flags.data(), d_flag, sizeof(int) * C, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaStreamSynchronize(st));
    for (int v : status)
        if (v) return false;
    return true;
}

bool eig_decompose(const RitzInput& in, const std::vector<int>& list, EigDecomposition& out) {
    const int S = (int)list.size();
    if (S == 0) return true;
    DeviceArena& ar = *in.arena;
    cudaStream_t st = in.st;
    const int m = in.m;
    int* d_list = ar.get<int>("ed_list", S);
    int* d_status = ar.get<int>("ed_status", S);
    double2* d_ritz = ar.get<double2>("ed_ritz", (int64_t)S * m);
    double2* d_w = ar.get<double2>("ed_w", (int64_t)S * m);
    double* d_absc = ar.get<double>("ed_absc", (int64_t)S * m);
    out.d = d_ritz;
    out.w = d_w;
    out.absc = d_absc;
    double2* Pg = ar.get<double2>("ed_P", (int64_t)S * m * m);
    SIM_CUDA(cudaMemcpyAsync(d_list, list.data(), sizeof(int) * S, cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemsetAsync(d_ritz, 0, sizeof(double2) * S * m, st));
    k_ritz<<<S, 32, (size_t)m * m * sizeof(double2), st>>>(in.d_H, m, in.d_meff, d_list, d_ritz, d_status);
    SIM_LAUNCH_CHECK();
    std::vector<int> status(S), status2(S);
    SIM_CUDA(cudaMemcpyAsync(status.data(), d_status, sizeof(int) * S, cudaMemcpyDeviceToHost, st));
    const size_t smem = ((size_t)m * m + (size_t)EIG_WARPS * (m * (m + 1) / 2 + m)) * sizeof(double2);
    SIM_CUDA(cudaFuncSetAttribute(k_eigdec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_eigdec<<<S, EIG_WARPS * 32, smem, st>>>(in.d_H, m, in.d_meff, in.d_beta, d_list, d_ritz, Pg, d_w, d_absc,
                                             d_status);
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaMemcpyAsync(status2.data(), d_status, sizeof(int) * S, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < S; ++i)
        if (status[i] || status2[i]) return false;
    return true;
}

void screen_points(int me, double hlast, double beta, double2 sigma, const double2* d, const double2* w,
                   const double2* z, int64_t count, double2* ym, double* rho, cudaStream_t st) {
    if (count <= 0) return;
    k_screen_points<<<cdiv_up(count, 128), 128, 0, st>>>(me, hlast, beta, sigma, d, w, z, count, ym, rho);
    SIM_LAUNCH_CHECK();
}

}  // namespace sim
