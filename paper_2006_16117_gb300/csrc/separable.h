// Fast-diagonalisation preconditioner for pencils with a separable part.
//
// The paper applies (A - σB)^{-1} without naming a solver (Sec. 2, Eqs.
// AzBxf, IMxb).  For operators whose principal part is a Kronecker sum of
// one-dimensional tridiagonal Toeplitz operators,
//     A_s = Σ_d I ⊗ … ⊗ T_d ⊗ … ⊗ I   (axis 0 fastest),   B = b I,
// the inverse of A_s - σB is known in closed form (fast diagonalisation,
// Lynch, Rice & Thomas 1964): T_d = S_d Λ_d S_d^{-1} with
//     S_d = D_d Q_d,  D_d = diag(ρ_d^j),  ρ_d = sqrt(sub_d / sup_d),
//     Q_d[j][k] = sqrt(2/(N+1)) sin((j+1)(k+1)π/(N+1))   (symmetric, orthogonal),
//     λ_{d,k} = diag_d + 2 sup_d ρ_d cos((k+1)π/(N+1)),
// so (A_s - σB)^{-1} = (⊗S_d) (Σ_d Λ_d - σb)^{-1} (⊗S_d^{-1}), applied as
// dense mode products along each axis.  It is exact for constant-coefficient
// convection–diffusion and leaves only the non-separable remainder (reaction
// terms) to the flexible GMRES around it.  Memory is O(n) per job and O(N_d²)
// per axis, independent of the shift: no factorisation per shift.
#pragma once

#include "internal.h"

namespace sim {

struct Separable {
    int ndim = 0;
    int64_t dims[3] = {1, 1, 1};
    double2 axis[3][3] = {};  // (sub, diag, sup) per axis
    double2 b = {1.0, 0.0};   // B = b I
    // per axis, device: Q (N×N row-major) in FP64 and FP32; ρ^j and ρ^{-j}; λ_k
    double* Q64[3] = {nullptr, nullptr, nullptr};
    float* Q32[3] = {nullptr, nullptr, nullptr};
    double2* rho[3] = {nullptr, nullptr, nullptr};
    double2* irho[3] = {nullptr, nullptr, nullptr};
    double2* lam[3] = {nullptr, nullptr, nullptr};
    // Q split for the tensor cores: Q = Qh + Ql, Qh exact in TF32 (FP32 tables)
    float* Qh[3] = {nullptr, nullptr, nullptr};
    float* Ql[3] = {nullptr, nullptr, nullptr};
    bool tc = false;  // complex64 mode products on the tensor cores (separable_tc.cu)
    // per element, for the complex64 path: Π_d ρ_d^{-j_d} and Π_d ρ_d^{j_d} rounded
    // from FP64, and Σ_d λ_{d,k_d} in FP64 (so the denominator's cancellation
    // against σb still happens in FP64)
    float2* sin32 = nullptr;
    float2* sout32 = nullptr;
    double2* lsum = nullptr;
};

struct SepCtx {
    Separable S;
    DeviceArena* ar = nullptr;  // the handle's arena (work vectors of the applies)
};

// Builds the per-axis tables on the device (arena buffers tag + "ax*").
void separable_setup(Separable& S, DeviceArena& ar, cudaStream_t st, const std::string& tag = "sep_");

// One mode product of na complex64 vectors on the tensor cores (3xTF32),
// Y = X ×_axis Q for an axis of length N with inner stride P (separable_tc.cu).
bool sep_mode_tc(const float2* cur, float2* nxt, const float* Qhi, const float* Qlo, int N, int64_t P, int64_t rows,
                 int64_t n, int na, cudaStream_t st);
void sep_split_tables(const double* Q64, int N, float* Qhi, float* Qlo, cudaStream_t st);

// z_job = (A_s - σ_job b I)^{-1} q_job for the active jobs (vector slots
// in_slot -> out_slot): the transforms in complex64 in mixed precision
// (complex128 otherwise), the division in FP64.
void separable_apply(const Separable& S, int precision, const JobSpace& js, const std::vector<int>& active,
                     int in_slot, int out_slot, const double2* d_sigma, DeviceArena& ar, cudaStream_t st);

}  // namespace sim
