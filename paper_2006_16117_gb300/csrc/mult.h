// Multiplicity step (Sec. 3.4) declarations.
#pragma once

#include <vector>

#include "internal.h"
#include "levels.h"

namespace sim {

struct MultInput {
    const Pencil* P = nullptr;
    const sim_options* opt = nullptr;
    cudaStream_t st = nullptr;
    DeviceArena* arena = nullptr;
    const double2* d_sigma = nullptr;
    void* const* d_fptrs = nullptr;
    std::vector<double2> est;    // cluster estimates (sorted)
    std::vector<int> shift;      // resolving shift per cluster
    std::vector<double> radius;  // cluster radius
    InnerStats* inner = nullptr;
};

std::vector<int> multiplicities(const MultInput& in, bool& ok);

// P f of cluster c into h_out (n complex values, host): the trapezoid rule on
// the mult_nodes-node circle of radius 2·max(radius, h0) around its estimate,
// through the Krylov space of f at its resolving shift (rebuilt, CGS2).
// Returns false if an inner solve did not converge.
bool projection_vector(const MultInput& in, const double2* d_f, int c, double2* h_out);

}  // namespace sim
