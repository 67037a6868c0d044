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
    double h0 = 1e-6;
    std::vector<double2> est;        // cluster estimates
    std::vector<int> shift;          // resolving shift per cluster
    std::vector<double> radius;      // cluster radius
};

// Refined values (the estimate where no Ritz value qualifies) and flags (1 =
// refined).  Returns false if the QR iteration of a Hessenberg matrix did not
// converge within its sweep limit.
bool ritz_refine(const RitzInput& in, std::vector<double2>& out, std::vector<int>& flags);

}  // namespace sim
