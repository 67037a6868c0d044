// Multiplicity step of SIM-M (Sec. 3.4): for every shift σ that resolves
// clusters, k random vectors f_i give k Krylov spaces K_m^σ(M; b_i) (one
// classical Gram-Schmidt pass per Arnoldi step unless mult_reorth); for each
// cluster, P f_i ≈ V_i Σ_j w_j y_ij on a circle around the cluster estimate
// (radius 2·max(cluster radius, h0), mult_nodes trapezoid nodes), and the
// multiplicity is the number of singular values of [P f_1 … P f_k] above
// mult_tol times the largest (from the eigenvalues of the k×k Gram matrix,
// FP64).  k doubles while the rank equals k, up to mult_kmax.
//
// Kernels: k_mult_proj (one CTA per (cluster, vector): 8 warps solve the
// projected systems at the nodes, 8 nodes per pass), k_mult_pf (P f_i for all
// clusters of a job, the job's basis staged in shared memory row block by row
// block), k_mult_gram (partial Gram matrices per row chunk), k_mult_rank (sum
// of the partials, cyclic Jacobi on the real 2k×2k embedding of the Hermitian
// Gram matrix, rank).
#include <algorithm>
#include <map>
#include <vector>

#include "hess.cuh"
#include "mult.h"

namespace sim {

struct MultArgs {
    JobSpace js;
    int k;                   // vectors per shift in this pass
    int m;
    int nodes;
    double h0;
    const int* cl_job0;      // [Cp] job index of vector 0 of the cluster's shift
    const double2* cl_est;   // [Cp]
    const double* cl_rad;    // [Cp]
    double2* u;              // [Cp][k][m]
    double2* P;              // [Cp][k][n]
    int Cp;
};

// u[c][i] = Σ_j (off_j / N) y_j,  y_j = β (I + (σ - z_j) H)^{-1} e1
__global__ void __launch_bounds__(256) k_mult_proj(MultArgs a, const double2* sigma) {
    const int c = blockIdx.x / a.k, i = blockIdx.x % a.k;
    const int job = a.cl_job0[c] + i;
    const JobSpace& js = a.js;
    const int m = a.m;
    const double2* H = js.H + (size_t)job * (m + 1) * m;
    const int meff = js.meff[job];
    const double beta = js.beta[job];
    const double2 sg = sigma[js.d_jobshift[job]];
    extern __shared__ unsigned char raw[];
    double2* Hs = reinterpret_cast<double2*>(raw);
    double2* U = Hs + (size_t)m * m;
    const int usz = meff * (meff + 1) / 2;
    double2* Y = U + (size_t)8 * (m * (m + 1) / 2);
    double2* acc = Y + (size_t)8 * m;
    const int warp = threadIdx.x >> 5;
    stage_H(H, m, meff, Hs);
    for (int q = threadIdx.x; q < m; q += blockDim.x) acc[q] = make_double2(0.0, 0.0);
    __syncthreads();
    const double rc = 2.0 * fmax(a.cl_rad[c], a.h0);
    const double2 e = a.cl_est[c];
    for (int base = 0; base < a.nodes; base += 8) {
        const int j = base + warp;
        double2 off = make_double2(0.0, 0.0);
        if (j < a.nodes) {
            double sn, cs;
            sincospi(2.0 * (double)j / (double)a.nodes, &sn, &cs);
            off = make_double2(rc * cs, rc * sn);
            const double2 z = make_double2(e.x + off.x, e.y + off.y);
            const double2 alpha = make_double2(sg.x - z.x, sg.y - z.y);
            double yl, yn;
            warp_hess_solve(Hs, meff, alpha, beta, U + (size_t)warp * usz, Y + (size_t)warp * m, yl, yn);
        }
        __syncthreads();
        for (int q = threadIdx.x; q < meff; q += blockDim.x) {
            double2 s = acc[q];
            for (int w = 0; w < 8 && base + w < a.nodes; ++w) {
                double sn, cs;
                sincospi(2.0 * (double)(base + w) / (double)a.nodes, &sn, &cs);
                const double2 wj = make_double2(rc * cs / a.nodes, rc * sn / a.nodes);
                s = cfma(wj, Y[(size_t)w * m + q], s);
            }
            acc[q] = s;
        }
        __syncthreads();
    }
    double2* out = a.u + ((size_t)c * a.k + i) * m;
    for (int q = threadIdx.x; q < m; q += blockDim.x) out[q] = q < meff ? acc[q] : make_double2(0.0, 0.0);
}

constexpr int PF_ROWS = 64;

// P[c][i][r] = Σ_t V_job[t][r] u[c][i][t] for every cluster c of the job's shift
__global__ void __launch_bounds__(256) k_mult_pf(MultArgs a, const int* job_cl_ptr, const int* job_cl) {
    const int job = blockIdx.y;  // job index (shift-major, vector-minor)
    const int i = job % a.k;
    const JobSpace& js = a.js;
    const int m = a.m;
    const int meff = js.meff[job];
    const int64_t r0 = (int64_t)blockIdx.x * PF_ROWS;
    extern __shared__ double2 vs[];  // [meff][PF_ROWS]
    const double2* V = js.V + (size_t)job * (m + 1) * js.n;
    for (int e = threadIdx.x; e < meff * PF_ROWS; e += blockDim.x) {
        int t = e / PF_ROWS, rr = e % PF_ROWS;
        int64_t r = r0 + rr;
        vs[e] = r < js.n ? V[(size_t)t * js.n + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int rr = threadIdx.x % PF_ROWS, grp = threadIdx.x / PF_ROWS, ngrp = blockDim.x / PF_ROWS;
    const int64_t r = r0 + rr;
    const int sh = job / a.k;
    for (int q = job_cl_ptr[sh] + grp; q < job_cl_ptr[sh + 1]; q += ngrp) {
        const int c = job_cl[q];
        const double2* uc = a.u + ((size_t)c * a.k + i) * m;
        double2 s = make_double2(0.0, 0.0);
        for (int t = 0; t < meff; ++t) s = cfma(vs[t * PF_ROWS + rr], uc[t], s);
        if (r < js.n) a.P[((size_t)c * a.k + i) * js.n + r] = s;
    }
}


// partial Gram matrices G[i][l] = Σ_r conj(P_i[r]) P_l[r] over a row chunk
__global__ void __launch_bounds__(256) k_mult_gram(MultArgs a, double2* gpart, int nchunk, int GR_ROWS) {
    const int c = blockIdx.y, chunk = blockIdx.x;
    const int k = a.k;
    const int64_t n = a.js.n;
    extern __shared__ double2 ps[];  // [k][GR_ROWS]
    const int64_t r0 = (int64_t)chunk * GR_ROWS;
    for (int e = threadIdx.x; e < k * GR_ROWS; e += blockDim.x) {
        int i = e / GR_ROWS, rr = e % GR_ROWS;
        int64_t r = r0 + rr;
        ps[e] = r < n ? a.P[((size_t)c * k + i) * n + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < k * k; p += blockDim.x) {
        const int i = p / k, l = p % k;
        double2 s = make_double2(0.0, 0.0);
        for (int rr = 0; rr < GR_ROWS; ++rr) {
            const double2 x = ps[i * GR_ROWS + rr], y = ps[l * GR_ROWS + rr];
            s.x = fma(x.x, y.x, fma(x.y, y.y, s.x));
            s.y = fma(x.x, y.y, fma(-x.y, y.x, s.y));
        }
        gpart[((size_t)c * nchunk + chunk) * k * k + p] = s;
    }
}

// sum the partials, eigenvalues of the Hermitian Gram matrix through its real
// symmetric embedding [[Re G, -Im G], [Im G, Re G]] (each eigenvalue twice) by
// cyclic Jacobi, rank = #{sqrt(λ) > tol * sqrt(λ_max)}
__global__ void k_mult_rank(MultArgs a, const double2* gpart, int nchunk, double* work, double tol, int* rank) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.Cp) return;
    const int k = a.k, N = 2 * k;
    double* A = work + (size_t)c * N * N;
    for (int i = 0; i < k; ++i)
        for (int l = 0; l < k; ++l) {
            double2 s = make_double2(0.0, 0.0);
            for (int ch = 0; ch < nchunk; ++ch) s = cadd(s, gpart[((size_t)c * nchunk + ch) * k * k + i * k + l]);
            A[i * N + l] = s.x;
            A[(i + k) * N + (l + k)] = s.x;
            A[(i + k) * N + l] = s.y;
            A[i * N + (l + k)] = -s.y;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < N; ++p) {
            diag += A[p * N + p] * A[p * N + p];
            for (int q = p + 1; q < N; ++q) off += A[p * N + q] * A[p * N + q];
        }
        if (off <= 1e-32 * diag || off == 0.0) break;
        for (int p = 0; p < N - 1; ++p)
            for (int q = p + 1; q < N; ++q) {
                const double apq = A[p * N + q];
                if (fabs(apq) < 1e-300) continue;
                const double tau = (A[q * N + q] - A[p * N + p]) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double cth = 1.0 / sqrt(1.0 + t * t), sth = t * cth;
                for (int r = 0; r < N; ++r) {
                    const double arp = A[r * N + p], arq = A[r * N + q];
                    A[r * N + p] = cth * arp - sth * arq;
                    A[r * N + q] = sth * arp + cth * arq;
                }
                for (int r = 0; r < N; ++r) {
                    const double apr = A[p * N + r], aqr = A[q * N + r];
                    A[p * N + r] = cth * apr - sth * aqr;
                    A[q * N + r] = sth * apr + cth * aqr;
                }
            }
    }
    double lmax = 0.0;
    for (int p = 0; p < N; ++p) lmax = fmax(lmax, A[p * N + p]);
    int cnt = 0;
    const double smax = sqrt(fmax(lmax, 0.0));
    for (int p = 0; p < N; ++p) {
        const double sv = sqrt(fmax(A[p * N + p], 0.0));
        if (smax > 0.0 && sv > tol * smax) ++cnt;
    }
    rank[c] = cnt / 2;
}

__global__ void k_mult_start(JobSpace js, int J, int k, const double2* F) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int job = blockIdx.y;
    if (g >= js.n || job >= J) return;
    js.vec[(size_t)job * js.vstride + (size_t)VS_RHS * js.n + g] = F[(size_t)(job % k) * js.n + g];
}

std::vector<int> multiplicities(const MultInput& in, bool& ok) {
    sim_options o = *in.opt;
    o.inner_tol = o.mult_inner_tol;  // these spaces feed only the rank test
    const int C = (int)in.est.size();
    std::vector<int> mult(C, 0);
    ok = true;
    if (C == 0) return mult;
    DeviceArena& ar = *in.arena;
    cudaStream_t st = in.st;
    const int64_t n = in.P->n;
    const int m = o.m;
    std::vector<int> pending(C);
    for (int c = 0; c < C; ++c) pending[c] = c;
    int k = o.mult_k;
    const int kin = std::max(1, std::min(o.inner_restart, 32));
    constexpr int JMAX = 512;  // jobs per batch: all shifts of a 64-vector pass at once up to 64 shifts
    while (!pending.empty()) {
        double2* F = ar.get<double2>("mu_F", (int64_t)k * n);
        random_vectors(o.mult_seed, n, k, 0, F, n, st);
        // group pending clusters by shift, batches of at most JMAX jobs
        std::map<int, std::vector<int>> by_shift;
        for (int c : pending) by_shift[in.shift[c]].push_back(c);
        std::vector<int> shifts;
        for (auto& kv : by_shift) shifts.push_back(kv.first);
        const int per = std::max(1, std::min(JMAX, max_jobs_for_memory(n, m, kin)) / k);
        std::vector<int> rank_of(C, -1);
        for (size_t b0 = 0; b0 < shifts.size(); b0 += per) {
            const int nsh = (int)std::min<size_t>(per, shifts.size() - b0);
            const int J = nsh * k;
            JobSpace js = make_jobspace(ar, st, J, kin, m, n, "mul_");
            std::vector<int> jobshift(J);
            std::vector<int> cl_list, cl_ptr(1, 0), cl_job0;
            std::vector<double2> cl_est;
            std::vector<double> cl_rad;
            std::vector<int> cl_id;
            for (int u = 0; u < nsh; ++u) {
                const int s = shifts[b0 + u];
                for (int i = 0; i < k; ++i) jobshift[u * k + i] = s;
                for (int c : by_shift[s]) {
                    cl_list.push_back((int)cl_id.size());
                    cl_id.push_back(c);
                    cl_job0.push_back(u * k);
                    cl_est.push_back(in.est[c]);
                    cl_rad.push_back(in.radius[c]);
                }
                cl_ptr.push_back((int)cl_list.size());
            }
            const int Cp = (int)cl_id.size();
            js.h_jobshift = jobshift.data();
            SIM_CUDA(cudaMemcpyAsync(js.d_jobshift, jobshift.data(), sizeof(int) * J, cudaMemcpyHostToDevice, st));
            dim3 g1(cdiv_up(n, 256), J);
            k_mult_start<<<g1, 256, 0, st>>>(js, J, k, F);
            SIM_LAUNCH_CHECK();
            ok = arnoldi(*in.P, o, js, in.d_sigma, in.d_fptrs, st, *in.inner, o.mult_reorth == 0) && ok;
            MultArgs a;
            a.js = js;
            a.k = k;
            a.m = m;
            a.nodes = o.mult_nodes;
            a.h0 = o.h0;
            a.Cp = Cp;
            int* d_job0 = ar.get<int>("mu_job0", Cp);
            double2* d_est = ar.get<double2>("mu_est", Cp);
            double* d_rad = ar.get<double>("mu_rad", Cp);
            int* d_clptr = ar.get<int>("mu_clptr", nsh + 1);
            int* d_cl = ar.get<int>("mu_cl", Cp);
            SIM_CUDA(cudaMemcpyAsync(d_job0, cl_job0.data(), sizeof(int) * Cp, cudaMemcpyHostToDevice, st));
            SIM_CUDA(cudaMemcpyAsync(d_est, cl_est.data(), sizeof(double2) * Cp, cudaMemcpyHostToDevice, st));
            SIM_CUDA(cudaMemcpyAsync(d_rad, cl_rad.data(), sizeof(double) * Cp, cudaMemcpyHostToDevice, st));
            SIM_CUDA(cudaMemcpyAsync(d_clptr, cl_ptr.data(), sizeof(int) * (nsh + 1), cudaMemcpyHostToDevice, st));
            SIM_CUDA(cudaMemcpyAsync(d_cl, cl_list.data(), sizeof(int) * Cp, cudaMemcpyHostToDevice, st));
            a.cl_job0 = d_job0;
            a.cl_est = d_est;
            a.cl_rad = d_rad;
            a.u = ar.get<double2>("mu_u", (int64_t)Cp * k * m);
            a.P = ar.get<double2>("mu_P", (int64_t)Cp * k * n);
            const size_t sm_proj = ((size_t)m * m + 8 * ((size_t)m * (m + 1) / 2) + 8 * (size_t)m + m) * sizeof(double2);
            SIM_CUDA(cudaFuncSetAttribute(k_mult_proj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_proj));
            k_mult_proj<<<Cp * k, 256, sm_proj, st>>>(a, in.d_sigma);
            SIM_LAUNCH_CHECK();
            const size_t sm_pf = (size_t)m * PF_ROWS * sizeof(double2);
            SIM_CUDA(cudaFuncSetAttribute(k_mult_pf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_pf));
            k_mult_pf<<<dim3(cdiv_up(n, PF_ROWS), J), 256, sm_pf, st>>>(a, d_clptr, d_cl);
            SIM_LAUNCH_CHECK();
            const int GR_ROWS = std::max(16, std::min(256, 12288 / k));  // k*GR_ROWS complex in shared memory
            const int nch = cdiv_up(n, GR_ROWS);
            double2* gpart = ar.get<double2>("mu_gpart", (int64_t)Cp * nch * k * k);
            const size_t sm_gr = (size_t)k * GR_ROWS * sizeof(double2);
            SIM_CUDA(cudaFuncSetAttribute(k_mult_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_gr));
            k_mult_gram<<<dim3(nch, Cp), 256, sm_gr, st>>>(a, gpart, nch, GR_ROWS);
            SIM_LAUNCH_CHECK();
            double* work = ar.get<double>("mu_work", (int64_t)Cp * 4 * k * k);
            int* d_rank = ar.get<int>("mu_rank", Cp);
            k_mult_rank<<<cdiv_up(Cp, 64), 64, 0, st>>>(a, gpart, nch, work, o.mult_tol, d_rank);
            SIM_LAUNCH_CHECK();
            std::vector<int> rk(Cp);
            SIM_CUDA(cudaMemcpyAsync(rk.data(), d_rank, sizeof(int) * Cp, cudaMemcpyDeviceToHost, st));
            SIM_CUDA(cudaStreamSynchronize(st));
            for (int q = 0; q < Cp; ++q) rank_of[cl_id[q]] = rk[q];
        }
        std::vector<int> next;
        for (int c : pending) {
            if (rank_of[c] < k || k >= o.mult_kmax) mult[c] = rank_of[c];
            else next.push_back(c);
        }
        pending.swap(next);
        k = std::min(2 * k, o.mult_kmax);
    }
    return mult;
}

bool projection_vector(const MultInput& in, const double2* d_f, int c, double2* h_out) {
    const sim_options& o = *in.opt;
    DeviceArena& ar = *in.arena;
    cudaStream_t st = in.st;
    const int64_t n = in.P->n;
    const int m = o.m;
    const int kin = std::max(1, std::min(o.inner_restart, 32));
    // one Krylov space: f at the cluster's resolving shift, CGS2 as for the location spaces
    JobSpace js = make_jobspace(ar, st, 1, kin, m, n, "pv_");
    const int jobshift = in.shift[c];
    js.h_jobshift = &jobshift;
    SIM_CUDA(cudaMemcpyAsync(js.d_jobshift, &jobshift, sizeof(int), cudaMemcpyHostToDevice, st));
    k_mult_start<<<dim3(cdiv_up(n, 256), 1), 256, 0, st>>>(js, 1, 1, d_f);
    SIM_LAUNCH_CHECK();
    bool ok = arnoldi(*in.P, o, js, in.d_sigma, in.d_fptrs, st, *in.inner, false);
    MultArgs a;
    a.js = js;
    a.k = 1;
    a.m = m;
    a.nodes = o.mult_nodes;
    a.h0 = o.h0;
    a.Cp = 1;
    const int zero = 0, ptr[2] = {0, 1};
    const double2 est = in.est[c];
    const double rad = in.radius[c];
    int* d_job0 = ar.get<int>("pv_job0", 1);
    double2* d_est = ar.get<double2>("pv_est", 1);
    double* d_rad = ar.get<double>("pv_rad", 1);
    int* d_clptr = ar.get<int>("pv_clptr", 2);
    int* d_cl = ar.get<int>("pv_cl", 1);
    SIM_CUDA(cudaMemcpyAsync(d_job0, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_est, &est, sizeof(double2), cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_rad, &rad, sizeof(double), cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_clptr, ptr, sizeof(int) * 2, cudaMemcpyHostToDevice, st));
    SIM_CUDA(cudaMemcpyAsync(d_cl, &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    a.cl_job0 = d_job0;
    a.cl_est = d_est;
    a.cl_rad = d_rad;
    a.u = ar.get<double2>("pv_u", m);
    a.P = ar.get<double2>("pv_P", n);
    const size_t sm_proj = ((size_t)m * m + 8 * ((size_t)m * (m + 1) / 2) + 8 * (size_t)m + m) * sizeof(double2);
    SIM_CUDA(cudaFuncSetAttribute(k_mult_proj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_proj));
    k_mult_proj<<<1, 256, sm_proj, st>>>(a, in.d_sigma);
    SIM_LAUNCH_CHECK();
    const size_t sm_pf = (size_t)m * PF_ROWS * sizeof(double2);
    SIM_CUDA(cudaFuncSetAttribute(k_mult_pf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_pf));
    k_mult_pf<<<dim3(cdiv_up(n, PF_ROWS), 1), 256, sm_pf, st>>>(a, d_clptr, d_cl);
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaMemcpyAsync(h_out, a.P, sizeof(double2) * n, cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaStreamSynchronize(st));
    return ok;
}

}  // namespace sim
