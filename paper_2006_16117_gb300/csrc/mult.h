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

}  // namespace sim
