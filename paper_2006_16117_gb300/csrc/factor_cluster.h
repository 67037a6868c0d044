// Cluster-parallel block Thomas factorisation (factor_cluster.cu).
#pragma once

#include "internal.h"

namespace sim {

// Factor A - σB for the listed shifts, one thread-block cluster per shift.
// Returns false (nothing launched) when a row slice does not fit in shared
// memory for any cluster size up to 8; the caller then uses factor_shifts().
bool factor_shifts_cluster(const Pencil& P, int precision, const int* d_shift_list, int count,
                           const double2* d_sigma, void* const* d_factor_ptrs, cudaStream_t st);

}  // namespace sim
