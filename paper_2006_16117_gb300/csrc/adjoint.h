// Kernels of the gradient calls (adjoint.cu).
#pragma once

#include <algorithm>

#include "internal.h"

namespace sim {

// A matrix's own stored entries: row, column and position in the pencil's
// union pattern (device arrays of length nnz).
struct EntryList {
    const int32_t* row = nullptr;
    const int32_t* col = nullptr;
    const int32_t* map = nullptr;
    int64_t nnz = 0;
};

// out = Σ_j c_j X_j (conj(c_j) when conj_c); X: [N][n], c: device [N].
void combine_nodes(const double2* X, int N, int64_t n, const double2* d_c, bool conj_c, double2* out, cudaStream_t st);
// R_j = conj(c_j) x, R: [N][n].
void scaled_copies(const double2* x, int N, int64_t n, const double2* d_c, double2* R, cudaStream_t st);
// *d_out = u^H v (or ||u||² when v == nullptr); part: dot_partials() scratch entries.
void dot(const double2* u, const double2* v, int64_t n, double2* part, double2* d_out, cudaStream_t st);
// *d_out = Σ_e conj(u[row_e]) vals[map_e] v[col_e] (vals == nullptr: all ones).
void entry_form(const EntryList& E, const double2* vals, const double2* u, const double2* v, double2* part,
                double2* d_out, cudaStream_t st);
// mode 0: out_e = Σ_j a_j U_j[row_e] conj(V_j[col_e]); mode 1: out_e = a_0 conj(U[row_e]) V[col_e].
void entry_grad(const EntryList& E, const double2* U, const double2* V, int N, int64_t n, const double2* d_a,
                int mode, double2* out, cudaStream_t st);
int dot_partials();

}  // namespace sim
