// Batched Gram–Schmidt arguments (krylov.cu, gs_cluster.cu).
#pragma once

#include "internal.h"

namespace sim {

// Vectors of job `job`: basis vector i at basis + job*bstride + i*n; w at
// w + job*wstride.  Coefficients go to hcol + job*hstride (+= for the second
// pass), the norm to hcol[cnt].  Partial sums of one pass are written to
// pout and read by the next kernel from pin (two buffers, since every CTA of
// a job reads all of that job's partials).
struct GSArgs {
    const double2* basis;
    int64_t bstride;
    double2* w;
    int64_t wstride;
    double2* hcol;
    int64_t hstride;
    int cnt;
    int64_t n;
    const double2* pin;   // [job][chunk][pw]
    double2* pout;
    int pw;
    int nchunk;
    const int* active;
    // Arnoldi breakdown test (optional): H base / stride / ld and column j
    const double2* Hfull;
    int64_t Hstride;
    int Hld;
    int j;
    double btol;
    int* meff;      // per job (optional)
    int* istat;     // per job IS_N ints (optional): IS_BROKEN flag
    // selective reorthogonalisation (Daniel-Gragg-Kaufman-Stewart): the second
    // pass runs only if the first one cut the norm of w below 1/sqrt(2) of it
    int dgks;
    // one pass only (the classical Gram-Schmidt printed in Sec. 2); overrides dgks
    int single;
};

// The whole CGS2 step of gs_run in one cluster launch per call (gs_cluster.cu):
// a cluster of up to 8 CTAs per job keeps w in registers and sums the dot
// products through distributed shared memory.  Same results up to rounding
// order; returns false (nothing launched) when n or cnt is beyond its range.
bool gs_cluster(const GSArgs& a, int nactive, cudaStream_t st);

}  // namespace sim
