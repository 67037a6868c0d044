/*
 * sim.h — C ABI of the GB300 SIM-M library (libsim.so).
 *
 * SIM-M (Huang, Sun, Yang, "A Multilevel Spectral Indicator Method for
 * Eigenvalues of Large Non-Hermitian Matrices") finds every eigenvalue of the
 * pencil A x = λ B x inside a region R of the complex plane (Sec. 1, Eq.
 * AxLambdaBx) to a precision h0, together with its multiplicity (Sec. 3.4).
 * The calls follow the algorithm's signature SIM-M(A, B, R, f, h0, ε, δ0, m, n0)
 * of Sec. 3.5:
 *
 *   sim_create        — A, B (steps' inputs)                         Sec. 3.5
 *   sim_set_region    — R and f; steps 1-3 (first shift, initial
 *                       squares, shift association with new Krylov
 *                       spaces)                                        Sec. 3.5
 *   sim_solve_level   — one pass of step 5 (one level of Sec. 3.3)
 *   sim_eigenvalues   — step 6-7 (merge, output)
 *   sim_multiplicity  — Sec. 3.4
 *
 * and, optional after sim_eigenvalues:
 *
 *   sim_refine        — Ritz refinement of the eigenvalues      Sec. 3.2
 *   sim_projection    — P f of one eigenvalue (an eigenvector)  Remark 3.5
 *
 * Conventions shared by every call:
 *  - Complex numbers are complex128 stored as interleaved (re, im) doubles.
 *  - Every call returns a sim_status and never throws; a handle's last error
 *    message is available from sim_last_error().
 *  - The library copies what it needs (A, B, f) into its own device memory;
 *    the caller keeps ownership of every pointer it passes and may free it
 *    when the call returns.  Outputs go to caller-allocated host arrays.
 *  - All device work is issued on the CUDA stream given to sim_create (NULL
 *    means the legacy default stream).  Calls return when their outputs are
 *    ready.
 *  - The handle is a state machine: create -> set_region -> solve_level (until
 *    done) -> eigenvalues -> multiplicity.  A call out of order returns
 *    SIM_ERR_BAD_STATE; sim_set_region may be called again to start over.
 *  - One handle must not be used by two host threads at once.
 */
#ifndef SIM_GB300_H
#define SIM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sim_ctx* sim_handle;

typedef enum {
    SIM_OK = 0,
    SIM_ERR_INVALID_ARG = 1,    /* bad pointer, size, CSR structure or option */
    SIM_ERR_BAD_STATE = 2,      /* call out of order */
    SIM_ERR_CUDA = 3,           /* a CUDA runtime call failed (message names it) */
    SIM_ERR_OOM = 4,            /* device allocation failed */
    SIM_ERR_NOT_CONVERGED = 5,  /* an inner solve hit its iteration cap */
    SIM_ERR_CAPACITY = 6,       /* output buffer too small; *count holds the size needed */
    SIM_ERR_LIMIT = 7           /* a level would exceed max_squares, or too many shifts */
} sim_status;

typedef enum {
    SIM_FP64 = 0,   /* factorisation, inner solves and Krylov bases in complex128 */
    SIM_MIXED = 1   /* complex64 factorisation with FP64 GMRES refinement of each
                       shifted solve; FP64 Gram–Schmidt, Hessenberg solves and tests */
} sim_precision;

/* A square sparse matrix in CSR form: row_ptr[n+1], col_idx[nnz] (0-based,
 * each row's columns strictly increasing), values[2*nnz] (complex128).
 * on_device != 0 means the three arrays are device pointers. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const double* values;
    int32_t on_device;
} sim_csr;

/* Parameters of Sec. 3.5 plus the readings this library fixes.  Get the
 * defaults from sim_default_options() and change fields as needed. */
typedef struct {
    int32_t m;                /* Krylov dimension (Sec. 3.5: 50) */
    int32_t n0;               /* coarse quadrature rule size; the fine rule has 2*n0
                                 nodes.  Only n0 = 4 is supported. */
    double delta0;            /* indicator threshold δ0 (Sec. 3.1: 1/20) */
    double eps;               /* residual tolerance ε of Def. 3.1 (1e-8) */
    double h0;                /* precision: the final squares have side <= h0 (1e-6) */
    double init_side;         /* side of the initial squares; 0 => min(width, height) of R */
    double shift_sep;         /* min separation, in initial sides, of shifts made in one round (4) */
    int32_t max_shift_rounds; /* rounds of step 3 (16) */
    int32_t max_shifts;       /* capacity for Krylov spaces (256) */
    double breakdown_tol;     /* Arnoldi stops when h_{j+1,j} <= tol * ||H||_F (1e-14) */
    double merge_radius;      /* clusters whose estimates are closer are joined (0) */
    int32_t mult_k;           /* random vectors for multiplicity (8); doubled while rank == k */
    int32_t mult_kmax;        /* upper limit of k (64) */
    double mult_tol;          /* singular values > mult_tol * largest count toward the rank (1e-6) */
    int32_t mult_nodes;       /* quadrature nodes on a cluster's circle (16) */
    uint64_t mult_seed;       /* Philox4x64-10 key word 0 for the multiplicity vectors */
    int32_t residual_scale;   /* 0: residual relative to ||y|| (default); 1: relative to beta */
    int64_t max_squares;      /* a level holding more squares is an error (4,000,000) */
    sim_precision precision;  /* SIM_FP64 (default) or SIM_MIXED */
    double inner_tol;         /* relative residual target of each shifted solve (1e-12) */
    int32_t inner_restart;    /* GMRES restart length (8) */
    int32_t inner_max_iter;   /* GMRES iteration cap per solve (64) */
    double mult_inner_tol;    /* inner tolerance for the multiplicity step's Krylov spaces,
                                 which feed only a rank test at mult_tol (1e-10; 1e-8 was measured
                                 to count simple eigenvalues of the 2-D reaction workload twice) */
    int32_t mult_reorth;      /* Gram-Schmidt of the multiplicity step's Arnoldi: 0 (default) one
                                 classical pass, as printed in Sec. 2; 1: applied twice (CGS2), as
                                 for the location spaces */
    int32_t new_shifts_in_levels; /* 0 (default, as printed): shifts are made only by the rounds of
                                 step 3; 1: at every level, squares no shift resolves get new Krylov
                                 spaces at their centres (at least shift_sep·side apart, up to
                                 max_shift_rounds rounds) and the level is evaluated again */
    int32_t level_solver;     /* projected solves of the levels (Eqs. eq:many, eq:error): 1 (default)
                                 the complex Schur form H_m = Z T Z^H of each shift (computed once)
                                 and one triangular solve per node, with the direct solve for the
                                 squares their own shift leaves unresolved; 0: Gaussian elimination
                                 with partial pivoting of I + (σ - z) H_m at every node */
    int32_t separable_tensor_cores; /* mixed precision with sim_set_separable: 1 (default) the mode
                                 products on the tensor cores (tcgen05, TF32 with hi/lo splitting to
                                 FP32 accuracy); 0: FP32 CUDA-core GEMMs */
} sim_options;

/* Counters of the last set_region .. multiplicity sequence. */
typedef struct {
    int64_t n, nnz_A, nnz_B;
    int32_t block_size, num_blocks;      /* block-tridiagonal layout of A - σB */
    int32_t num_shifts;
    int32_t levels_total, levels_done;
    int64_t squares_evaluated;           /* summed over levels */
    int64_t projected_solves;            /* Hessenberg solves (quadrature points) */
    int64_t inner_solves;                /* shifted solves (A - σB) x = r completed */
    int64_t gmres_iterations;            /* summed over inner solves */
    int32_t max_gmres_iterations;        /* worst single inner solve */
    int64_t unresolvable_final;          /* final squares not resolvable (warnings of step 6) */
    int64_t final_squares;
    int64_t clusters;
    double max_inner_residual;           /* worst relative residual of an inner solve */
    double t_factor_ms, t_krylov_ms, t_levels_ms, t_merge_ms, t_mult_ms;
    int64_t loose_inner_solves;          /* inner solves that stagnated above inner_tol and were
                                            accepted within 100·inner_tol */
    int64_t unresolvable_last_level;     /* squares of the last solved level no shift resolved */
    int64_t shift_retries;               /* evaluations against a second, third, ... shift (summed) */
    int64_t direct_level_evaluations;    /* squares evaluated by direct solves (all of them with
                                            level_solver 0; those the Schur path leaves with 1) */
} sim_stats_t;

/* Fills *opt with the defaults listed above.  opt must not be NULL. */
void sim_default_options(sim_options* opt);

/* Creates a handle for the pencil (A, B).  B == NULL means B = I.  A and B must
 * have the same n; B may be any CSR (a diagonal B is detected and stored as a
 * vector).  The library determines the band half-width w = max |i - j| over the
 * nonzeros of A and B and stores A - σB for each shift as a block tridiagonal
 * matrix with blocks of side w; its memory per shift is about 2·n·w complex
 * numbers.  stream is a cudaStream_t (NULL = default stream).
 * Errors: SIM_ERR_INVALID_ARG (NULL pointers, n < 1, unsorted or out-of-range
 * columns, options out of range), SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_create(const sim_csr* A, const sim_csr* B, const sim_options* opt,
                      void* stream, sim_handle* out);

/* Optional, between sim_create and sim_set_region: replaces the inner
 * solver's preconditioner for (A - σB).  The paper leaves the solver of the
 * shifted systems open (Sec. 2, Eqs. AzBxf, IMxb); by default this library
 * factors A - σB per shift as a block-tridiagonal matrix, whose memory grows
 * as n times the band width.  Pencils whose principal part is separable —
 *   A ≈ A_s = Σ_d I ⊗ … ⊗ T_d ⊗ … ⊗ I   (axis 0 fastest, n = Π dims[d]),
 *   T_d = tridiag(sub_d, diag_d, sup_d) Toeplitz of order dims[d],  B = b·I,
 * e.g. finite-difference convection–diffusion–reaction on a box — can use the
 * fast-diagonalisation inverse (Lynch, Rice, Thomas 1964) of A_s - σB as the
 * preconditioner instead: O(n) memory per Krylov job, O(Σ dims[d]²) per
 * pencil, nothing factored per shift.  The flexible GMRES around it corrects
 * for A - A_s (reaction terms), so the results do not depend on the choice;
 * only the iteration count does.  axes: complex128 (sub, diag, sup) per axis,
 * i.e. 6·ndim doubles.  The handle's previous region (if any) is discarded.
 * Errors: SIM_ERR_INVALID_ARG (ndim outside 1..3, a length outside 1..8192,
 * Π dims != n, B not a multiple of I, a zero off-diagonal, non-finite
 * entries), SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_set_separable(sim_handle h, int32_t ndim, const int64_t* dims, const double* axes);

/* Sets the search region R = [re_lo, re_hi] × [im_lo, im_hi] and the random
 * vector f (complex128[n]; f_on_device selects host or device memory; f ==
 * NULL draws f from Philox4x64-10 with key (seed, 0x53494D4D), vector index 0).
 * Runs steps 1-3 of Sec. 3.5: the first shift at the centre of R, the initial
 * squares (side init_side tiling R's bounding box from its lower-left corner,
 * row-major), and shift rounds: each round tests every unresolved square
 * against every shift nearest-first, then builds new Krylov spaces at the
 * centres of unresolved squares spaced at least
 * max(shift_sep·side, ρ) apart, ρ being the distance from the first shift to
 * the nearest square it does not resolve.
 * Errors: SIM_ERR_INVALID_ARG (empty region, bad f), SIM_ERR_LIMIT (more than
 * max_shifts shifts), SIM_ERR_NOT_CONVERGED, SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_set_region(sim_handle h, double re_lo, double re_hi, double im_lo, double im_hi,
                          const double* f, int32_t f_on_device, uint64_t seed);

/* Evaluates every square of the current level at once (Sec. 3.3, step 5):
 * the 8 quadrature nodes on each square's circumscribed circle, the projected
 * solves (I + (σ - z)H_m) y = β e1 (Eq. eq:many) with the residual of Eq.
 * eq:error, resolvability (Def. 3.1; an unresolvable square retries the other
 * shifts nearest-first), the indicator of Eq. DeltaSm and the mark
 * (Ĩ > δ0, or unresolvable).  Marked squares are split into four children for
 * the next level.  *n_marked receives the number of marked squares, *done is
 * set to 1 after the last level (side <= h0).
 * Errors: SIM_ERR_BAD_STATE (no region, or already done), SIM_ERR_LIMIT. */
sim_status sim_solve_level(sim_handle h, int64_t* n_marked, int32_t* done);

/* Step 6-7: merges the final squares into clusters (8-connected components;
 * estimate = mean of member centres; estimates closer than merge_radius
 * joined), keeps clusters whose estimate lies in the closed region, sorts by
 * (Re, Im) and writes 2*count doubles (re, im) to out.  capacity is in
 * eigenvalues; capacity 0 (out may be NULL) only returns *count.
 * Errors: SIM_ERR_BAD_STATE (levels not finished), SIM_ERR_CAPACITY. */
sim_status sim_eigenvalues(sim_handle h, double* out, int64_t capacity, int64_t* count);

/* Sec. 3.4: the multiplicity of every eigenvalue returned by sim_eigenvalues
 * (same order): for each shift that resolves clusters, k random vectors
 * (Philox4x64-10, key (mult_seed, 0x53494D4D), vector indices 1..k), their k
 * Krylov spaces, P f_i on a mult_nodes-point circle of radius
 * 2·max(cluster radius, h0) around each estimate, and the number of singular
 * values of [P f_1 … P f_k] above mult_tol times the largest; k doubles while
 * the rank equals k, up to mult_kmax.
 * Errors: SIM_ERR_BAD_STATE (sim_eigenvalues not called), SIM_ERR_CAPACITY. */
sim_status sim_multiplicity(sim_handle h, int32_t* out, int64_t capacity, int64_t* count);

/* The spectral projection P f of the region's vector f onto the eigenspace
 * of located eigenvalue c (index into sim_eigenvalues' output): the
 * trapezoid rule of Sec. 2 (Eq. XLXf) on a mult_nodes-node circle of radius
 * 2·max(cluster radius, h0) around the estimate, through the Krylov space of
 * f at the cluster's resolving shift (rebuilt, one set of inner solves).  For
 * a simple eigenvalue this is a right eigenvector (Remark 3.5), unnormalised.
 * out: complex128[n], caller-allocated.  Valid after sim_eigenvalues until
 * the next sim_set_region.  Errors: SIM_ERR_BAD_STATE, SIM_ERR_INVALID_ARG
 * (c out of range, NULL out), SIM_ERR_NOT_CONVERGED. */
sim_status sim_projection(sim_handle h, int64_t c, double* out);

/* Ritz refinement of the located eigenvalues (Sec. 3.2, Eq. zjHm: the
 * eigenvalues d_i of a shift's Hessenberg matrix H_m are Ritz values of the
 * Cayley transform M = (A - σB)^{-1}B, so λ_i = σ + 1/d_i).  For each
 * eigenvalue of sim_eigenvalues (same order), the λ_i of its resolving shift
 * nearest the estimate replaces it when within 2·max(cluster radius, h0), the
 * radius of the multiplicity circle; refined[c] is then 1, else 0 and out[c]
 * is the estimate.  out: complex128[count] (capacity entries); refined:
 * int32[count] or NULL.  capacity == 0 only sets *count.  Valid after
 * sim_eigenvalues until the next sim_set_region; may be called any number
 * of times.  Errors: SIM_ERR_BAD_STATE, SIM_ERR_CAPACITY,
 * SIM_ERR_NOT_CONVERGED (a Hessenberg QR iteration hit its sweep limit). */
sim_status sim_refine(sim_handle h, double* out, int32_t* refined, int64_t capacity, int64_t* count);

/* ---- Batches of pencils ------------------------------------------------------
 * Many independent pencils, each with its own region, located together: the
 * squares of every pencil's current level are evaluated in one launch (the
 * level-synchronous evaluation of all squares that Sec. 3.3 makes the
 * parallel axis), and subdivided by one compaction.  Each pencil's shifts,
 * Krylov spaces, merge and multiplicity stay its own; a square only uses its
 * own pencil's shifts.  Pencils may differ in size; their regions must give
 * the same number of levels (same initial side and h0).  A batch owns one
 * sim_handle per pencil (sim_batch_handle), all on the given stream. */
typedef struct sim_batch_ctx* sim_batch;

/* count pencils A[p] (and B[p]; B == NULL means B = I for all), one set of
 * options.  Errors as sim_create (the message of sim_batch_last_error(NULL)
 * names the pencil). */
sim_status sim_batch_create(int32_t count, const sim_csr* A, const sim_csr* B, const sim_options* opt, void* stream,
                            sim_batch* out);
/* sim_set_separable for pencil p. */
sim_status sim_batch_set_separable(sim_batch b, int32_t p, int32_t ndim, const int64_t* dims, const double* axes);
/* Steps 1-3 of Sec. 3.5 for every pencil: regions[4p..4p+3] = (re_lo, re_hi,
 * im_lo, im_hi); f[p] = host complex128[n_p] or f == NULL (Philox, key word 0
 * = seed + p).  Errors: as sim_set_region; SIM_ERR_INVALID_ARG when the
 * regions need different numbers of levels. */
sim_status sim_batch_set_regions(sim_batch b, const double* regions, const double* const* f, uint64_t seed);
/* One level of every pencil in one evaluation launch (Sec. 3.3, step 5);
 * *n_marked: marked squares over all pencils; *done = 1 after the last level.
 * Then sim_batch_eigenvalues / sim_batch_multiplicity per pencil. */
sim_status sim_batch_solve_level(sim_batch b, int64_t* n_marked, int32_t* done);
sim_status sim_batch_eigenvalues(sim_batch b, int32_t p, double* out, int64_t capacity, int64_t* count);
sim_status sim_batch_multiplicity(sim_batch b, int32_t p, int32_t* out, int64_t capacity, int64_t* count);
/* Pencil p's handle (owned by the batch): for sim_stats, sim_refine, ... */
sim_handle sim_batch_handle(sim_batch b, int32_t p);
const char* sim_batch_last_error(sim_batch b);
void sim_batch_destroy(sim_batch b);

/* ---- Differentiation -------------------------------------------------------
 * Gradients of spectral functionals with respect to the values of A's and B's
 * stored entries (the order of the CSR arrays given to sim_create), through
 * adjoint shifted solves with (A - zB)^H.  The paper defines the spectral
 * projection these functionals are built on (Sec. 2, Eq. XLXf) but does not
 * differentiate it.  The shifted systems are solved by the inner solver
 * (FGMRES with the handle's preconditioner: a block factorisation per node,
 * or the separable one of sim_set_separable).  These calls do not depend on
 * the region state and leave it alone. */

/* Φ = ||P f||² with P f = Σ_j w_j (A - z_j B)^{-1} f, the trapezoid rule of
 * Eq. XLXf on the circle z_j = c + r e^{2πij/N}, w_j = (z_j - c)/N (j < N =
 * nodes, 4..64).  f: complex128[n], host or device (f_on_device).  keep != 0
 * keeps the N node solutions on the device for sim_projection_norm_grad
 * (N·n·16 bytes); keep == 0 frees them, and the gradient call solves for them
 * again (less memory, N more solves).  Errors: SIM_ERR_INVALID_ARG,
 * SIM_ERR_NOT_CONVERGED, SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_projection_norm(sim_handle h, double c_re, double c_im, double radius, int32_t nodes, const double* f,
                               int32_t f_on_device, int32_t keep, double* phi);

/* The gradient of the last sim_projection_norm's Φ: with the adjoint solves
 * (A - z_j B)^H μ_j = conj(w_j) P f,
 *   grad_A[e] = -2 Σ_j μ_j[p] conj(x_j[q]),   grad_B[e] = 2 Σ_j conj(z_j) μ_j[p] conj(x_j[q])
 * for stored entry e at (p, q), where x_j = (A - z_j B)^{-1} f; each value is
 * ∂Φ/∂Re(entry) + i ∂Φ/∂Im(entry) (complex128, nnz_A resp. nnz_B values).
 * grad_B may be NULL (and is ignored when B = I).  out_on_device selects
 * device or host output arrays.  Errors: SIM_ERR_BAD_STATE (no forward call),
 * SIM_ERR_INVALID_ARG, SIM_ERR_NOT_CONVERGED, SIM_ERR_CUDA. */
sim_status sim_projection_norm_grad(sim_handle h, double* grad_A, double* grad_B, int32_t out_on_device);

/* A simple eigenvalue λ inside the circle (c, r) and its derivatives
 * dλ/dA[e] = conj(y_p) x_q / (y^H B x), dλ/dB[e] = -λ conj(y_p) x_q / (y^H B x)
 * (complex128 per stored entry; λ is holomorphic in the entries).  x and y
 * are the right and left eigenvectors from the same quadrature as above: x =
 * Σ_j w_j (A - z_j B)^{-1} v and y = Σ_j conj(w_j) (A - z_j B)^{-H} B^H u for
 * Philox4x64-10 vectors v, u (key (seed, 0x53494D4D), indices 0 and 1);
 * lambda (2 doubles) = y^H A x / y^H B x.  The circle must hold exactly one
 * eigenvalue, simple; the quadrature error is about (r/d)^N for the nearest
 * other eigenvalue at distance d from c.  dl_dB may be NULL.
 * Errors: SIM_ERR_INVALID_ARG (bad argument, or no eigenvalue inside),
 * SIM_ERR_NOT_CONVERGED, SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_eigenvalue_grad(sim_handle h, double c_re, double c_im, double radius, int32_t nodes, uint64_t seed,
                               double* lambda, double* dl_dA, double* dl_dB, int32_t out_on_device);

/* Replaces the values of A's (a_values, nnz_A complex128) and/or B's
 * (b_values, nnz_B) stored entries, keeping the sparsity patterns given to
 * sim_create; either may be NULL.  The handle returns to its created state
 * (region, shifts and factorisations discarded); a separable preconditioner
 * stays (B must remain a multiple of I).  Errors: SIM_ERR_INVALID_ARG
 * (non-finite values, b_values with B = I), SIM_ERR_OOM, SIM_ERR_CUDA. */
sim_status sim_update_values(sim_handle h, const double* a_values, const double* b_values, int32_t on_device);

/* Copies the counters into *out (size = sizeof(sim_stats_t)). */
sim_status sim_stats(sim_handle h, sim_stats_t* out, size_t size);

/* Per-handle message of the last failed call ("" if none).  Valid until the
 * next call on the handle.  h == NULL returns the message of the last failed
 * sim_create. */
const char* sim_last_error(sim_handle h);

/* Frees every device and host resource of the handle.  NULL is a no-op. */
void sim_destroy(sim_handle h);

/* ---- Component entry points (the same kernels the pipeline uses) ---------
 * These expose single steps for parity tests.  All pointers are DEVICE
 * pointers unless stated; stream may be NULL.  They allocate only the small
 * scratch they need and free it before returning. */

/* Number of shifts built by the last sim_set_region, and shift s's Krylov data:
 * sigma (2 doubles), H ((m+1)·m complex128, column-major, leading dim m+1,
 * HOST memory), beta, and m_eff (< m after an Arnoldi breakdown). */
sim_status sim_shift_count(sim_handle h, int32_t* count);
sim_status sim_get_shift(sim_handle h, int32_t s, double* sigma, double* H_host, double* beta,
                         int32_t* m_eff);

/* Batched projected solves and indicator (Eqs. eq:many, eq:error, DeltaSm)
 * for `count` squares against one Krylov space given explicitly:
 * H: (m+1)·m complex128 column-major (ld m+1), sigma = sig_re + i sig_im,
 * centers: complex128[count], sides: double[count].  Outputs indicator[count]
 * and rho[count] (the largest residual over the 8 nodes, scaled as
 * residual_scale says).  1 <= m_eff <= m <= 64. */
sim_status sim_eval_squares(const double* H, int32_t m, int32_t m_eff, double beta, double sig_re,
                            double sig_im, const double* centers, const double* sides, int64_t count,
                            int32_t residual_scale, double* indicator, double* rho, void* stream);

/* Sec. 3.2, Eqs. zjHm and rmLc1: with the eigendecomposition H_m = P D P^{-1}
 * of shift s's Hessenberg matrix (computed on the GPU: QR eigenvalues, one
 * step of inverse iteration per eigenvector, c_1 = P^{-1} e_1), the last
 * entry of the projected solution at each point z_j costs O(m):
 *   e_m^T y_j = β r_m (I + (σ - z_j) D)^{-1} c_1,   r_m = e_m^T P,
 * and so does the residual |σ - z_j| h_{m+1,m} |e_m^T y_j| / β of Eq. eq:error
 * (relative to β).  z: count complex128 points (host); ym: complex128[count]
 * and rho: double[count] (host outputs).  Exact for a diagonalisable H_m; the
 * rounding grows with the condition of P.  Valid after sim_set_region.
 * Errors: SIM_ERR_BAD_STATE, SIM_ERR_INVALID_ARG, SIM_ERR_NOT_CONVERGED. */
sim_status sim_residual_screen(sim_handle h, int32_t s, const double* z, int64_t count, double* ym, double* rho);

/* y = (A - σB) x for the handle's pencil (complex128[n] vectors). */
sim_status sim_apply_shifted(sim_handle h, double sig_re, double sig_im, const double* x, double* y);

/* x = (A - σB)^{-1} r by the handle's inner solver (factorisation in the
 * handle's precision + FP64 GMRES); *iters and *relres report the solve. */
sim_status sim_shifted_solve(sim_handle h, double sig_re, double sig_im, const double* r, double* x,
                             int32_t* iters, double* relres);

/* y = (A - σB) x like sim_apply_shifted, for callers that must not allocate
 * device memory: a process whose GPU memory is owned by another allocator (a
 * framework's caching pool that reserved it), where a cudaMalloc would fail or
 * fragment that pool, or a latency-critical loop that cannot afford the device
 * synchronisation cudaMalloc/cudaFree may cause.  The paper has no counterpart:
 * this is a deployment variant of the sparse apply.  It stages x and y in one
 * file-scope device array (n <= 262,144 complex128 per vector, about 8 MiB)
 * and calls no cudaMalloc, cudaFree or other allocating routine.  The CUDA
 * runtime reserves the array on a device when it loads the library's module
 * there: with the default lazy module loading, during the first call made on
 * that device (with CUDA_MODULE_LOADING=EAGER, at context creation).  Make
 * that first call, or set CUDA_MODULE_LOADING=EAGER, before another allocator
 * reserves the GPU; the device keeps the array until the process exits.  The
 * first call on each device also looks up the array's device address (make it
 * before any stream capture).  Calls share the array: each call fully
 * overwrites what it reads, and calls that overlap on the GPU race.  The call
 * is synchronous: it returns once y is written.
 * Errors: SIM_ERR_LIMIT when n exceeds 262,144; SIM_ERR_INVALID_ARG;
 * SIM_ERR_OOM when loading the array fails for lack of device memory;
 * SIM_ERR_CUDA. */
sim_status sim_apply_shifted_noalloc(sim_handle h, double sig_re, double sig_im, const double* x, double* y);

/* Philox4x64-10 complex Gaussian vectors: out[v*n + e] for v < k is element e
 * of random vector (first + v) with key (seed, 0x53494D4D); complex128. */
sim_status sim_random_vectors(uint64_t seed, int64_t n, int32_t k, int32_t first, double* out,
                              void* stream);

/* ---- Instrumentation ------------------------------------------------------
 * Not part of the method: counters used by the benchmark.
 * sim_kernel_timing(1) resets and turns on per-kernel CUDA-event timing of the
 * library's main kernels ("block_solve", "factor", "gram_schmidt",
 * "eval_level", "spmv"); 0 turns it off.  Process-wide, not thread-safe.
 * sim_kernel_stats fills the accumulated device time (ms), algorithmic bytes
 * and flops and launch count of one of them; returns 0 if it never ran.
 * sim_launch_count returns the number of kernel launches the library has made
 * in this process. */
void sim_kernel_timing(int32_t enable);
/* A measured arithmetic peak of the current device, for the benchmark's
 * rooflines: which = 0 FP64 fused multiply-add throughput, 1 FP32; writes
 * TFLOP/s (2 flops per FMA) to *tflops.  Runs one short register-only kernel. */
sim_status sim_measure_fma_peak(int32_t which, double* tflops);
int32_t sim_kernel_stats(const char* name, double* ms, double* bytes, double* flops, int64_t* launches);
int64_t sim_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SIM_GB300_H */
