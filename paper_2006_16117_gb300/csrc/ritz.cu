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

}  // namespace sim
