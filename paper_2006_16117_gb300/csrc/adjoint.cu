// Kernels of the gradient calls (the adjoint path): quadrature sums of node
// solutions, norms and bilinear forms, and the gradient on the matrices'
// stored entries.
//
// The projection of Sec. 2 (Eq. XLXf) on a circle: x = Σ_j w_j x_j with
// (A - z_j B) x_j = f.  For Φ = ||x||² the adjoint solves
// (A - z_j B)^H μ_j = conj(w_j) x give, per stored entry (p, q),
//   ∂Φ/∂Re + i ∂Φ/∂Im:   A: -2 Σ_j μ_j[p] conj(x_j[q]),   B: 2 Σ_j conj(z_j) μ_j[p] conj(x_j[q]);
// for a simple eigenvalue with eigenvectors x, y: dλ/dA_pq = conj(y_p) x_q / (y^H B x),
// dλ/dB_pq = -λ conj(y_p) x_q / (y^H B x).
#include "adjoint.h"

namespace sim {

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 512;

// out = Σ_j c_j X_j  (c conjugated when conj_c), X: [N][n]
__global__ void k_combine(const double2* X, int N, int64_t n, const double2* c, int conj_c, double2* out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
        double2 cj = c[j];
        if (conj_c) cj.y = -cj.y;
        acc = cfma(cj, X[(size_t)j * n + g], acc);
    }
    out[g] = acc;
}

// R_j = conj(c_j) x for j < N, R: [N][n]
__global__ void k_scaled_copies(const double2* x, int N, int64_t n, const double2* c, double2* R) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    const double2 v = x[g];
    for (int j = 0; j < N; ++j) R[(size_t)j * n + g] = cmul(make_double2(c[j].x, -c[j].y), v);
}

// per-block partial sums of conj(u_g) v_g (or of |u_g|² when v == nullptr)
__global__ void __launch_bounds__(RED_THREADS) k_dot_partial(const double2* u, const double2* v, int64_t n,
                                                               double2* part) {
    __shared__ double2 sh[RED_THREADS / 32];
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
        const double2 a = u[g];
        if (v) acc = cadd(acc, cconjmul(a, v[g]));
        else acc.x += a.x * a.x + a.y * a.y;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = sh[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) s = cadd(s, sh[w]);
        part[blockIdx.x] = s;
    }
}

// per-block partial sums of conj(u[row_e]) val_e v[col_e] over stored entries
// (val_e = vals[map_e]; all ones when vals == nullptr)
__global__ void __launch_bounds__(RED_THREADS) k_form_partial(const int32_t* row, const int32_t* col,
                                                                const int32_t* map, const double2* vals, int64_t nnz,
                                                                const double2* u, const double2* v, double2* part) {
    __shared__ double2 sh[RED_THREADS / 32];
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        double2 t = v[col[e]];
        if (vals) t = cmul(vals[map[e]], t);
        acc = cadd(acc, cconjmul(u[row[e]], t));
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 s = sh[0];
        for (int w = 1; w < RED_THREADS / 32; ++w) s = cadd(s, sh[w]);
        part[blockIdx.x] = s;
    }
}

__global__ void k_sum_partials(const double2* part, int np, double2* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i < np; ++i) s = cadd(s, part[i]);
    *out = s;
}

// out_e = Σ_j a_j U_j[row_e] conj(V_j[col_e])   (mode 0: the projection-norm gradient)
// out_e = a_0 conj(U_0[row_e]) V_0[col_e]          (mode 1: the eigenvalue gradient)
__global__ void k_entry_grad(const int32_t* row, const int32_t* col, int64_t nnz, const double2* U, const double2* V,
                             int N, int64_t n, const double2* a, int mode, double2* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const int64_t p = row[e], q = col[e];
    double2 acc = make_double2(0.0, 0.0);
    if (mode == 0) {
        for (int j = 0; j < N; ++j) acc = cfma(a[j], cmulc(U[(size_t)j * n + p], V[(size_t)j * n + q]), acc);
    } else {
        acc = cmul(a[0], cconjmul(U[p], V[q]));
    }
    out[e] = acc;
}

}  // namespace

void combine_nodes(const double2* X, int N, int64_t n, const double2* d_c, bool conj_c, double2* out, cudaStream_t st) {
    k_combine<<<cdiv_up(n, 256), 256, 0, st>>>(X, N, n, d_c, conj_c ? 1 : 0, out);
    SIM_LAUNCH_CHECK();
}

void scaled_copies(const double2* x, int N, int64_t n, const double2* d_c, double2* R, cudaStream_t st) {
    k_scaled_copies<<<cdiv_up(n, 256), 256, 0, st>>>(x, N, n, d_c, R);
    SIM_LAUNCH_CHECK();
}

void dot(const double2* u, const double2* v, int64_t n, double2* part, double2* d_out, cudaStream_t st) {
    const int nb = (int)std::min<int64_t>(RED_BLOCKS, std::max<int64_t>(1, cdiv_up(n, RED_THREADS)));
    k_dot_partial<<<nb, RED_THREADS, 0, st>>>(u, v, n, part);
    SIM_LAUNCH_CHECK();
    k_sum_partials<<<1, 32, 0, st>>>(part, nb, d_out);
    SIM_LAUNCH_CHECK();
}

void entry_form(const EntryList& E, const double2* vals, const double2* u, const double2* v, double2* part,
                double2* d_out, cudaStream_t st) {
    const int nb = (int)std::min<int64_t>(RED_BLOCKS, std::max<int64_t>(1, cdiv_up(E.nnz, RED_THREADS)));
    k_form_partial<<<nb, RED_THREADS, 0, st>>>(E.row, E.col, E.map, vals, E.nnz, u, v, part);
    SIM_LAUNCH_CHECK();
    k_sum_partials<<<1, 32, 0, st>>>(part, nb, d_out);
    SIM_LAUNCH_CHECK();
}

void entry_grad(const EntryList& E, const double2* U, const double2* V, int N, int64_t n, const double2* d_a,
                int mode, double2* out, cudaStream_t st) {
    if (E.nnz <= 0) return;
    k_entry_grad<<<cdiv_up(E.nnz, 256), 256, 0, st>>>(E.row, E.col, E.nnz, U, V, N, n, d_a, mode, out);
    SIM_LAUNCH_CHECK();
}

int dot_partials() { return RED_BLOCKS; }

}  // namespace sim
