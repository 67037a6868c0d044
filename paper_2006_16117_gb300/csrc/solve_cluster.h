// Cluster-based block Thomas solve (solve_cluster.cu).
#pragma once

#include <vector>

#include "internal.h"

namespace sim {

// z_job = (A - σB)^{-1} q_job for the active jobs (vector slots in_slot ->
// out_slot).  Jobs of the same shift that are adjacent in `active` share one
// pass over the factors.  Returns false (nothing launched) when the block size
// does not fit the kernel's shared memory (T above about 2,800 in complex128).
bool block_solve_cluster(const Pencil& P, int precision, const JobSpace& js, const std::vector<int>& active,
                         int in_slot, int out_slot, const double2* d_sigma, void* const* d_factor_ptrs,
                         cudaStream_t st);

// Nonzero if a cluster solve recorded a failed wait (an mbarrier poll limit).
int block_solve_error();

}  // namespace sim
