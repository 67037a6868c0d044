// Ritz refinement of located eigenvalues (ritz.cu).
#pragma once

#include <vector>

#include "internal.h"
#include "levels.h"

namespace sim {

struct RitzInput {
    DeviceArena* arena = nullptr;
    cudaStream_t st = nullptr;
    int m = 50;
    int num_slots = 0;               // shift-table slots
    const double2* d_H = nullptr;    // shift table: H per slot, column-major, leading dimension m + 1
    const int* d_meff = nullptr;
    const double2* d_sigma = nullptr;
    const double* d_beta = nullptr;
    double h0 = 1e-6;
    std::vector<double2> est;        // cluster estimates
    std::vector<int> shift;          // resolving shift per cluster
    std::vector<double> radius;      // cluster radius
};

// Refined values (the estimate where no Ritz value qualifies) and flags (1 =
// refined).  Returns false if the QR iteration of a Hessenberg matrix did not
// converge within its sweep limit.
bool ritz_refine(const RitzInput& in, std::vector<double2>& out, std::vector<int>& flags);

// Sec. 3.2: the eigendecomposition H_m = P D P^{-1} of the listed shifts'
// Hessenberg matrices, as the data of the O(m) formula of Eq. rmLc1: per
// listed shift (row b of each array, m entries) the eigenvalues d_i, the
// weights w_i = β (e_m^T P e_i) c_1[i] with c_1 = P^{-1} e_1 (P's columns of
// unit length), and |c_1[i]|.  Device arrays in the arena (valid until the
// next call).  False if an eigenvalue or eigenvector computation failed.
struct EigDecomposition {
    const double2* d = nullptr;
    const double2* w = nullptr;
    const double* absc = nullptr;
};
bool eig_decompose(const RitzInput& in, const std::vector<int>& list, EigDecomposition& out);

// e_m^T y = Σ_i w_i / (1 + (σ - z) d_i) and |σ - z| h_{m+1,m} |e_m^T y| / β
// for `count` points z (device arrays).
void screen_points(int me, double hlast, double beta, double2 sigma, const double2* d, const double2* w,
                   const double2* z, int64_t count, double2* ym, double* rho, cudaStream_t st);

}  // namespace sim
