// Internal declarations shared by the translation units of libsim.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sim.h"
#include "common.cuh"

namespace sim {

// The pencil stored once on the device: the union sparsity pattern of A and
// B in CSR form with A's and B's values on it (Ka, Kb; zero where absent), so
// that (A - σB)_ij = Ka - σ Kb.  Block-tridiagonal view: blocks of side T,
// nb = ceil(n / T) block rows; entries of block row k fall in block columns
// k-1, k, k+1 only (T >= the band half-width).
struct SepCtx;  // separable.h: fast-diagonalisation preconditioner and its arena

struct Pencil {
    int64_t n = 0;
    int64_t nnz = 0;
    int T = 1;
    int nb = 1;
    int b_kind = 0;            // 0: B = I, 1: B diagonal, 2: general
    const int32_t* rp = nullptr;
    const int32_t* ci = nullptr;
    const double2* Ka = nullptr;
    const double2* Kb = nullptr;
    const double2* Bdiag = nullptr;  // b_kind == 1: B's diagonal (complex128[n])
    // couplings to block row k+1 in column-compressed form, one segment per
    // block row: for block k, entries [up_ptr[k*(T+1)+c], up_ptr[k*(T+1)+c+1])
    // hold (row-in-block, value index) of column c of the block (k, k+1).
    const int32_t* up_ptr = nullptr;
    const int32_t* up_row = nullptr;
    const int32_t* up_idx = nullptr;
    // couplings to block row k-1, per row g: entries [Lptr[g], Lptr[g+1]) with
    // column Lcol (relative to the start of block k-1) and value index Lidx.
    // Each shift's factor stores the shifted values Lval (after E).
    const int32_t* Lptr = nullptr;
    const int32_t* Lcol = nullptr;
    const int32_t* Lidx = nullptr;
    int64_t nnzL = 0;
    // per row g: Lcol of its first coupling, -1 if it has none (a solve can
    // load it, and the shift's first value L0val[g], without reading Lptr first)
    const int32_t* L0col = nullptr;
    // host pointer: when set, the inner solver's preconditioner is the
    // fast-diagonalisation inverse of the pencil's separable part instead of
    // the block factorisation (nothing is factored per shift)
    SepCtx* sep = nullptr;
    // ||A||_inf and ||B||_inf (row sums of |entries|): the rounding floor of a
    // shifted residual is about ε (||A|| + |σ| ||B||) ||x||
    double anorm = 0.0, bnorm = 0.0;
};

// Offset (in elements of the factor type) of Lval inside a shift's factor.
__host__ __device__ inline size_t factor_lval_offset(const Pencil& P) { return (size_t)2 * P.nb * P.T * P.T; }
// Offset of L0val (n values: the first coupling's shifted value of each row, 0 if none).
__host__ __device__ inline size_t factor_l0_offset(const Pencil& P) { return factor_lval_offset(P) + (size_t)P.nnzL; }

// Workspace of a batch of Krylov jobs (one job = one Arnoldi process for
// one shift and one starting vector).  All vectors are complex128 of length n,
// job j's vector v at base + j*stride + v*n.
struct JobSpace {
    int J = 0;                 // slots
    int k = 8;                 // GMRES restart length
    int m = 50;                // Arnoldi dimension
    int64_t n = 0;
    double2* vec = nullptr;    // [J][NV][n]
    int64_t vstride = 0;       // NV * n
    double2* V = nullptr;      // [J][m+1][n] Arnoldi bases
    double2* H = nullptr;      // [J][(m+1)*m] column-major Arnoldi Hessenberg
    double* beta = nullptr;    // [J]
    int* meff = nullptr;       // [J]
    // GMRES small state
    double2* Hg = nullptr;     // [J][(k+1)*k] column-major
    double2* cs = nullptr;     // [J][k] rotation: c (real part used) and s
    double2* sn = nullptr;     // [J][k]
    double2* g = nullptr;      // [J][k+1]
    double* scal = nullptr;    // [J][8]: rnorm0, res_est, res_true, ...
    int* istat = nullptr;      // [J][8]: steps in cycle, total iters, flags
    double2* partial = nullptr;  // [J][nchunk][max(m+2, k+2)] partial dot products
    int nchunk = 0;
    int pstride = 0;           // per-job partial stride = nchunk * pw
    int pw = 0;                // partial width
    int* d_jobshift = nullptr; // [J] shift id of each slot
    int* d_active = nullptr;   // [J] active slot list
    const int* h_jobshift = nullptr;  // [J] the same ids in host memory (owned by the caller)
};

// vector slots inside vec
enum { VS_RHS = 0, VS_X = 1, VS_R = 2, VS_W = 3, VS_Q0 = 4 };  // then Q[0..k], Z[0..k-1]
__host__ __device__ inline int vs_Z(int k) { return VS_Q0 + k + 1; }
__host__ __device__ inline int vs_count(int k) { return VS_Q0 + 2 * k + 1; }

// scal / istat fields
enum { SC_RNORM0 = 0, SC_RES = 1, SC_GAMMA = 2, SC_WORST = 3, SC_N = 8 };
enum { IS_STEPS = 0, IS_ITERS = 1, IS_DONE = 2, IS_CYCLE_DONE = 3, IS_BROKEN = 4, IS_STALL = 5, IS_LOOSE = 6, IS_N = 8 };

constexpr int GS_CHUNK = 4096;   // rows per CTA in the Gram–Schmidt kernels (16 per thread)
constexpr int GS_THREADS = 256;

// ---- krylov.cu ------------------------------------------------------------
// Factor A - σB for the listed shifts into block form Dinv_k = D_k^{-1},
// E_k = Dinv_k U_k (block Thomas).  factors[s] points to 2*nb*T*T entries of C.
void factor_shifts(const Pencil& P, int precision, const int* d_shift_list, int count,
                   const double2* d_sigma, void* const* d_factor_ptrs, cudaStream_t st);

// Batched FGMRES for (A - σB) x = rhs on the jobs listed on the host; x in
// VS_X.  Returns false if some job hit the iteration cap.
struct InnerStats {
    int64_t solves = 0, iters = 0;
    int64_t loose = 0;  // solves accepted above inner_tol (within 100x) after stagnating
    int max_iters = 0;
    double worst = 0.0;
};
bool inner_solve(const Pencil& P, const sim_options& opt, JobSpace& js, const std::vector<int>& jobs,
                 const double2* d_sigma, void* const* d_factor_ptrs, cudaStream_t st, InnerStats& stats);

// y = (A - σ_s B) x for active jobs, vector slots.
void spmv_shifted_jobs(const Pencil& P, const JobSpace& js, int nactive, const double* dummy, int x_slot,
                       int y_slot, const double2* d_sigma, cudaStream_t st);

// Arnoldi for all jobs: b = K^{-1} start (start vectors in VS_RHS on entry),
// beta, V, H, meff.  Classical Gram-Schmidt applied twice (CGS2), or once if
// single_pass (the printed algorithm of Sec. 2).
bool arnoldi(const Pencil& P, const sim_options& opt, JobSpace& js, const double2* d_sigma,
             void* const* d_factor_ptrs, cudaStream_t st, InnerStats& stats, bool single_pass = false);

void apply_B(const Pencil& P, const double2* x, double2* y, cudaStream_t st);

class DeviceArena;
JobSpace make_jobspace(DeviceArena& ar, cudaStream_t st, int J, int k, int m, int64_t n, const std::string& tag);
// Krylov jobs whose job spaces (vectors, basis, preconditioner work vectors)
// fit 40% of the device's memory: the batch size of the shift and
// multiplicity builds (at least 1).
int max_jobs_for_memory(int64_t n, int m, int k);

// ---- philox.cu ---------------------------------------------------------------
void random_vectors(uint64_t seed, int64_t n, int k, int first, double2* out, int64_t ld, cudaStream_t st);

}  // namespace sim
