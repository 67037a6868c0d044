// C ABI of the SIM-M library and the host-side drivers that sequence the
// kernels: pencil upload, Krylov spaces per shift, the shift rounds of
// Sec. 3.5 step 3, one level per sim_solve_level (Sec. 3.3), the merge
// (step 6) and the multiplicity step (Sec. 3.4).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"
#include "factor_cluster.h"
#include "levels.h"
#include "mult.h"
#include "adjoint.h"
#include "ritz.h"
#include "separable.h"

using namespace sim;

namespace {

enum State { ST_CREATED = 0, ST_REGION = 1, ST_LEVELS_DONE = 2, ST_EIGS = 3 };

struct Timer {
    cudaStream_t st;
    std::chrono::steady_clock::time_point t0;
    explicit Timer(cudaStream_t s) : st(s) { t0 = std::chrono::steady_clock::now(); }
    double ms() {
        cudaStreamSynchronize(st);
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

std::string g_create_error;

}  // namespace

struct sim_ctx {
    cudaStream_t st = nullptr;
    sim_options opt{};
    std::string err;
    int state = ST_CREATED;
    Pencil P;
    DeviceArena arena;
    // shifts
    int S = 0;
    int cap = 0;
    std::vector<double2> h_sigma;
    std::vector<void*> factors;
    double2* d_sigma = nullptr;
    double2* d_H = nullptr;
    double* d_beta = nullptr;
    int* d_meff = nullptr;
    // Schur forms of the Hessenberg matrices (schur.cu)
    double2* d_schT = nullptr;
    double2* d_schC = nullptr;
    double2* d_schQ = nullptr;
    int* d_schOK = nullptr;
    void** d_fptrs = nullptr;
    size_t factor_bytes = 0;
    // input vector
    double2* d_f = nullptr;
    // region and levels
    double re_lo = 0, re_hi = 0, im_lo = 0, im_hi = 0, s1 = 1;
    int64_t cols = 1, rows = 1;
    int K = 1, level = 1;
    int64_t nsq = 0;
    int cur = 0;
    int64_t nfinal = 0;
    double s_final = 1;
    // clusters (sorted, inside R)
    std::vector<double2> eig;
    std::vector<int> cl_shift, cl_size, cl_flag;
    std::vector<double> cl_radius;
    std::vector<int> mult;
    sim_stats_t stats{};
    InnerStats inner;
    // B = b_value·I (identity, or a diagonal with one value): the separable
    // preconditioner needs it
    bool b_scalar = false;
    double2 b_value = {1.0, 0.0};
    std::unique_ptr<SepCtx> sep;
    // the pencil's union pattern on the host (for the adjoint pencil and value
    // updates), and A's / B's own entries: row, column, position in the union
    std::vector<int32_t> u_rp, u_ci;
    std::vector<double2> u_Ka, u_Kb, u_bd;
    bool has_B = false;
    int64_t nnzA = 0, nnzB = 0;
    int32_t *d_arow = nullptr, *d_acol = nullptr, *d_amap = nullptr;
    int32_t *d_brow = nullptr, *d_bcol = nullptr, *d_bmap = nullptr;
    std::vector<int32_t> h_amap, h_bmap;
    // adjoint pencil (A^H, B^H), built on first use by the gradient calls
    Pencil Padj;
    bool adj_built = false;
    std::unique_ptr<SepCtx> sep_adj;
    // node solves of the gradient calls: per direction (0 forward, 1 adjoint)
    // a shift table of the quadrature nodes and, for the band preconditioner,
    // a factorisation per node
    double2* d_nsig[2] = {nullptr, nullptr};
    void** d_nfptrs[2] = {nullptr, nullptr};
    std::vector<void*> nfactors[2];
    // forward state of sim_projection_norm for sim_projection_norm_grad
    bool pn_valid = false, pn_kept = false;
    std::vector<double2> pn_z, pn_w;
    double2* d_pn_X = nullptr;  // [N][n] node solutions (when kept)
    double2* d_pn_x = nullptr;  // [n] P f
    double2* d_pn_f = nullptr;  // [n] f

    ~sim_ctx() {
        for (void* p : factors)
            if (p) cudaFree(p);
        for (auto& v : nfactors)
            for (void* p : v)
                if (p) cudaFree(p);
    }
};

// ---------------------------------------------------------------------------
namespace {

sim_status fail(sim_ctx* h, sim_status s, const std::string& msg) {
    if (h) h->err = msg;
    else g_create_error = msg;
    return s;
}

template <class F> sim_status guarded(sim_ctx* h, F&& f) {
    try {
        if (h) h->err.clear();
        return f();
    } catch (const CudaError& e) {
        return fail(h, e.code == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA, e.what);
    } catch (const std::bad_alloc&) {
        return fail(h, SIM_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        const std::string w = e.what();
        if (w.rfind("LIMIT:", 0) == 0) return fail(h, SIM_ERR_LIMIT, w.substr(6));
        return fail(h, SIM_ERR_CUDA, w);
    }
}

void* up_buf(sim_ctx* h, const std::string& name, const void* src, size_t bytes) {
    void* d = h->arena.get<unsigned char>(name, (int64_t)bytes);
    if (bytes) SIM_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, h->st));
    return d;
}

struct HostCsr {
    int64_t n = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double2> v;
};

bool fetch_csr(const sim_csr* A, HostCsr& out, std::string& why) {
    if (!A || A->n < 1 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->values))) {
        why = "CSR: NULL pointer or bad size";
        return false;
    }
    out.n = A->n;
    out.rp.resize(A->n + 1);
    out.ci.resize(A->nnz);
    out.v.resize(A->nnz);
    auto kind = A->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    SIM_CUDA(cudaMemcpy(out.rp.data(), A->row_ptr, sizeof(int32_t) * (A->n + 1), kind));
    if (A->nnz) {
        SIM_CUDA(cudaMemcpy(out.ci.data(), A->col_idx, sizeof(int32_t) * A->nnz, kind));
        SIM_CUDA(cudaMemcpy(out.v.data(), A->values, sizeof(double2) * A->nnz, kind));
    }
    if (out.rp[0] != 0 || out.rp[A->n] != A->nnz) {
        why = "CSR: row_ptr[0] must be 0 and row_ptr[n] must equal nnz";
        return false;
    }
    for (int64_t i = 0; i < A->n; ++i) {
        if (out.rp[i + 1] < out.rp[i]) {
            why = "CSR: row_ptr not monotone";
            return false;
        }
        for (int64_t e = out.rp[i]; e < out.rp[i + 1]; ++e) {
            if (out.ci[e] < 0 || out.ci[e] >= A->n) {
                why = "CSR: column index out of range";
                return false;
            }
            if (e > out.rp[i] && out.ci[e] <= out.ci[e - 1]) {
                why = "CSR: columns of a row must be strictly increasing";
                return false;
            }
            if (!std::isfinite(out.v[e].x) || !std::isfinite(out.v[e].y)) {
                why = "CSR: non-finite value";
                return false;
            }
        }
    }
    return true;
}

// Band layout and device arrays of a pencil given on its union pattern (rows
// rp/ci, A's values Ka and B's values Kb on it, B's kind and diagonal).
void upload_pencil(DeviceArena& ar, cudaStream_t st, Pencil& P, const std::vector<int32_t>& rp,
                   const std::vector<int32_t>& ci, const std::vector<double2>& Ka, const std::vector<double2>& Kb,
                   int b_kind, const std::vector<double2>& bd, const std::string& tag) {
    const int64_t n = (int64_t)rp.size() - 1;
    int64_t kl = 0, ku = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            kl = std::max<int64_t>(kl, i - ci[e]);
            ku = std::max<int64_t>(ku, ci[e] - i);
        }
    P.n = n;
    P.nnz = (int64_t)ci.size();
    P.T = (int)std::max<int64_t>(2, std::max(kl, ku));
    P.T += P.T & 1;  // even: block rows stay 16-byte aligned in complex64
    P.nb = (int)((n + P.T - 1) / P.T);
    P.b_kind = b_kind;
    // couplings to the next block row, column-compressed per block
    const int T = P.T, nb = P.nb;
    std::vector<int32_t> up_ptr((size_t)nb * (T + 1), 0), up_row, up_idx;
    {
        std::vector<std::vector<std::pair<int32_t, int32_t>>> cols(T);
        for (int k = 0; k + 1 < nb; ++k) {
            for (auto& c : cols) c.clear();
            for (int i = 0; i < T; ++i) {
                int64_t g = (int64_t)k * T + i;
                if (g >= n) break;
                for (int64_t e = rp[g]; e < rp[g + 1]; ++e) {
                    int64_t j = ci[e];
                    if (j >= (int64_t)(k + 1) * T) cols[j - (int64_t)(k + 1) * T].push_back({i, (int32_t)e});
                }
            }
            size_t base = (size_t)k * (T + 1);
            up_ptr[base] = (int32_t)up_row.size();
            for (int c = 0; c < T; ++c) {
                for (auto& pr : cols[c]) {
                    up_row.push_back(pr.first);
                    up_idx.push_back(pr.second);
                }
                up_ptr[base + c + 1] = (int32_t)up_row.size();
            }
        }
    }
    // couplings to the previous block row
    std::vector<int32_t> Lptr(n + 1, 0), Lcol, Lidx;
    for (int64_t g = 0; g < n; ++g) {
        const int64_t k = g / T;
        for (int64_t e = rp[g]; e < rp[g + 1]; ++e) {
            const int64_t j = ci[e];
            if (k > 0 && j < k * T && j >= (k - 1) * T) {
                Lcol.push_back((int32_t)(j - (k - 1) * T));
                Lidx.push_back((int32_t)e);
            }
        }
        Lptr[g + 1] = (int32_t)Lcol.size();
    }
    auto up = [&](const char* name, const void* src, size_t bytes) -> void* {
        void* d = ar.get<unsigned char>(tag + name, (int64_t)bytes);
        if (bytes) SIM_CUDA(cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st));
        return d;
    };
    P.rp = (const int32_t*)up("rp", rp.data(), sizeof(int32_t) * rp.size());
    P.ci = (const int32_t*)up("ci", ci.data(), sizeof(int32_t) * ci.size());
    P.Ka = (const double2*)up("Ka", Ka.data(), sizeof(double2) * Ka.size());
    P.Kb = (const double2*)up("Kb", Kb.data(), sizeof(double2) * Kb.size());
    P.Bdiag = (const double2*)up("Bd", bd.data(), sizeof(double2) * bd.size());
    P.up_ptr = (const int32_t*)up("upp", up_ptr.data(), sizeof(int32_t) * up_ptr.size());
    P.up_row = (const int32_t*)up("upr", up_row.data(), sizeof(int32_t) * up_row.size());
    P.up_idx = (const int32_t*)up("upi", up_idx.data(), sizeof(int32_t) * up_idx.size());
    P.Lptr = (const int32_t*)up("Lptr", Lptr.data(), sizeof(int32_t) * Lptr.size());
    P.Lcol = (const int32_t*)up("Lcol", Lcol.data(), sizeof(int32_t) * Lcol.size());
    P.Lidx = (const int32_t*)up("Lidx", Lidx.data(), sizeof(int32_t) * Lidx.size());
    P.nnzL = (int64_t)Lcol.size();
    std::vector<int32_t> L0col(n);
    for (int64_t g = 0; g < n; ++g) L0col[g] = Lptr[g + 1] > Lptr[g] ? Lcol[Lptr[g]] : -1;
    P.L0col = (const int32_t*)up("L0col", L0col.data(), sizeof(int32_t) * L0col.size());
    P.anorm = P.bnorm = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double ra = 0.0, rb = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            ra += std::hypot(Ka[e].x, Ka[e].y);
            rb += std::hypot(Kb[e].x, Kb[e].y);
        }
        P.anorm = std::max(P.anorm, ra);
        P.bnorm = std::max(P.bnorm, rb);
    }
    SIM_CUDA(cudaStreamSynchronize(st));
}

void ensure_shift_capacity(sim_ctx* h) {
    if (h->cap) return;
    const int cap = h->opt.max_shifts + 1;  // last slot: scratch for component calls
    const int m = h->opt.m;
    h->d_sigma = h->arena.get<double2>("sigma", cap);
    h->d_H = h->arena.get<double2>("H", (int64_t)cap * (m + 1) * m);
    h->d_beta = h->arena.get<double>("beta", cap);
    h->d_meff = h->arena.get<int>("meff", cap);
    h->d_schT = h->arena.get<double2>("schT", (int64_t)cap * m * m);
    h->d_schC = h->arena.get<double2>("schC", (int64_t)cap * m);
    h->d_schQ = h->arena.get<double2>("schQ", (int64_t)cap * m);
    h->d_schOK = h->arena.get<int>("schOK", cap);
    SIM_CUDA(cudaMemsetAsync(h->d_schOK, 0, sizeof(int) * cap, h->st));
    h->d_fptrs = h->arena.get<void*>("fptrs", cap);
    h->factors.assign(cap, nullptr);
    h->h_sigma.assign(cap, make_double2(0, 0));
    h->cap = cap;
}

void* factor_storage(sim_ctx* h, int s) {
    if (!h->factors[s]) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, h->factor_bytes);
        if (e != cudaSuccess)
            throw CudaError{e, "cudaMalloc of a shift factorisation (" + std::to_string(h->factor_bytes) + " bytes)"};
        h->factors[s] = p;
        SIM_CUDA(cudaMemcpyAsync(h->d_fptrs + s, &h->factors[s], sizeof(void*), cudaMemcpyHostToDevice, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
    }
    return h->factors[s];
}

JobSpace make_jobspace(sim_ctx* h, int J, const std::string& tag) {
    return sim::make_jobspace(h->arena, h->st, J, std::max(1, std::min(h->opt.inner_restart, 32)), h->opt.m, h->P.n, tag);
}

__global__ void k_copy_start(JobSpace js, int J, const double2* f) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int job = blockIdx.y;
    if (g >= js.n || job >= J) return;
    js.vec[(size_t)job * js.vstride + (size_t)VS_RHS * js.n + g] = f[g];
}

__global__ void k_store_space(JobSpace js, int J, const int* job_shift, double2* H, double* beta, int* meff, int m) {
    int job = blockIdx.x;
    if (job >= J) return;
    int s = job_shift[job];
    for (int e = threadIdx.x; e < (m + 1) * m; e += blockDim.x) H[(size_t)s * (m + 1) * m + e] = js.H[(size_t)job * (m + 1) * m + e];
    if (threadIdx.x == 0) {
        beta[s] = js.beta[job];
        meff[s] = js.meff[job];
    }
}

// Build Krylov spaces for new shifts at the given centres (Sec. 2: factor
// A - σB, b = (A - σB)^{-1} f, m Arnoldi steps).  Returns false on non-convergence.
bool build_shifts(sim_ctx* h, const std::vector<double2>& sig) {
    if (sig.empty()) return true;
    const int Jall = (int)sig.size();
    if (h->S + Jall > h->opt.max_shifts) throw std::runtime_error("LIMIT:too many shifts (max_shifts)");
    // Krylov jobs per batch: as many as fit the device memory budget of job spaces
    const int Jmax = max_jobs_for_memory(h->P.n, h->opt.m, std::max(1, std::min(h->opt.inner_restart, 32)));
    bool ok = true;
    for (int b0 = 0; b0 < Jall; b0 += Jmax) {
        const int J = std::min(Jmax, Jall - b0);
        std::vector<int> ids(J);
        for (int j = 0; j < J; ++j) {
            ids[j] = h->S + j;
            h->h_sigma[ids[j]] = sig[b0 + j];
        }
        SIM_CUDA(cudaMemcpyAsync(h->d_sigma + h->S, sig.data() + b0, sizeof(double2) * J, cudaMemcpyHostToDevice,
                                 h->st));
        if (!h->P.sep) {
            for (int s : ids) factor_storage(h, s);
            int* d_list = h->arena.get<int>("shift_list", J);
            SIM_CUDA(cudaMemcpyAsync(d_list, ids.data(), sizeof(int) * J, cudaMemcpyHostToDevice, h->st));
            Timer tf(h->st);
            if (!factor_shifts_cluster(h->P, h->opt.precision, d_list, J, h->d_sigma, h->d_fptrs, h->st))
                factor_shifts(h->P, h->opt.precision, d_list, J, h->d_sigma, h->d_fptrs, h->st);
            h->stats.t_factor_ms += tf.ms();
        }
        Timer tk(h->st);
        JobSpace js = make_jobspace(h, J, "loc_");
        js.h_jobshift = ids.data();
        SIM_CUDA(cudaMemcpyAsync(js.d_jobshift, ids.data(), sizeof(int) * J, cudaMemcpyHostToDevice, h->st));
        dim3 grid(cdiv_up(h->P.n, 256), J);
        k_copy_start<<<grid, 256, 0, h->st>>>(js, J, h->d_f);
        SIM_LAUNCH_CHECK();
        ok = arnoldi(h->P, h->opt, js, h->d_sigma, h->d_fptrs, h->st, h->inner) && ok;
        k_store_space<<<J, 256, 0, h->st>>>(js, J, js.d_jobshift, h->d_H, h->d_beta, h->d_meff, h->opt.m);
        SIM_LAUNCH_CHECK();
        schur_shifts(h->d_H, h->opt.m, h->d_meff, h->d_beta, h->S, J, h->d_schT, h->d_schC, h->d_schQ, h->d_schOK,
                     h->st);
        SIM_CUDA(cudaStreamSynchronize(h->st));
        h->S += J;
        h->stats.t_krylov_ms += tk.ms();
    }
    return ok;
}

ShiftTable shift_table(sim_ctx* h) {
    ShiftTable t;
    t.H = h->d_H;
    t.beta = h->d_beta;
    t.meff = h->d_meff;
    t.sigma = h->d_sigma;
    t.S = h->S;
    t.m = h->opt.m;
    t.scale = h->opt.residual_scale;
    t.eps = h->opt.eps;
    t.delta0 = h->opt.delta0;
    t.schT = h->d_schT;
    t.schC = h->d_schC;
    t.schQ = h->d_schQ;
    t.schOK = h->d_schOK;
    return t;
}

// One evaluation of a level (mode 0): with level_solver 1 the Schur forms
// evaluate every square against its own shift, then the squares left against
// every shift of their pencil (smax: the most shifts a pencil has), and the
// direct evaluation runs only where a zero pivot or a missing Schur form
// stops them; with 0 the direct evaluation runs for all.  Returns the number
// of squares evaluated directly.
int64_t evaluate_level(const ShiftTable& t, LevelArgs la, int level_solver, int smax, DeviceArena& ar,
                       int64_t* bsum, int64_t* tot, cudaStream_t st) {
    if (level_solver == 1 && t.schT && la.count > 0) {
        uint8_t* todo = ar.get<uint8_t>("lvl_todo", la.count);
        eval_level_schur(t, la, todo, st);
        const int64_t left = count_marked(todo, la.count, bsum, tot, ar.host_i64(), st);
        if (left == 0) return 0;
        eval_level_schur_retries(t, la, todo, left, smax, ar, st);
        const int64_t direct = count_marked(todo, la.count, bsum, tot, ar.host_i64(), st);
        if (direct == 0) return 0;
        la.todo = todo;
        eval_level(t, la, 0, st);
        return direct;
    }
    eval_level(t, la, 0, st);
    return la.count;
}

double2 center_of(const sim_ctx* h, double s, int64_t ix, int64_t iy) {
    return make_double2(h->re_lo + ((double)ix + 0.5) * s, h->im_lo + ((double)iy + 0.5) * s);
}

int num_levels(double s1, double h0) { return s1 > h0 ? (int)std::ceil(std::log2(s1 / h0)) + 1 : 1; }

void sync_stats(sim_ctx* h) {
    h->stats.num_shifts = h->S;
    h->stats.inner_solves = h->inner.solves;
    h->stats.gmres_iterations = h->inner.iters;
    h->stats.max_gmres_iterations = h->inner.max_iters;
    h->stats.max_inner_residual = h->inner.worst;
    h->stats.loose_inner_solves = h->inner.loose;
}


// ---------------------------------------------------------------------------
// node solves for the gradient calls
// ---------------------------------------------------------------------------
EntryList entries_A(sim_ctx* h) { return EntryList{h->d_arow, h->d_acol, h->d_amap, h->nnzA}; }
EntryList entries_B(sim_ctx* h) { return EntryList{h->d_brow, h->d_bcol, h->d_bmap, h->nnzB}; }

// The adjoint pencil (A^H, B^H) on the transposed union pattern, and its
// separable part (the conjugate transposes of the axis factors) if any.
void ensure_adjoint(sim_ctx* h) {
    if (h->adj_built) return;
    const int64_t n = h->P.n;
    const std::vector<int32_t>& rp = h->u_rp;
    const std::vector<int32_t>& ci = h->u_ci;
    std::vector<int32_t> rpt(n + 1, 0), cit(ci.size());
    std::vector<double2> Kat(ci.size()), Kbt(ci.size());
    for (int32_t c : ci) ++rpt[c + 1];
    for (int64_t i = 0; i < n; ++i) rpt[i + 1] += rpt[i];
    std::vector<int32_t> pos(rpt.begin(), rpt.end() - 1);
    for (int64_t i = 0; i < n; ++i)  // rows in increasing order: each transposed row's columns stay sorted
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t d = pos[ci[e]]++;
            cit[d] = (int32_t)i;
            Kat[d] = make_double2(h->u_Ka[e].x, -h->u_Ka[e].y);
            Kbt[d] = make_double2(h->u_Kb[e].x, -h->u_Kb[e].y);
        }
    std::vector<double2> bdt(n);
    for (int64_t i = 0; i < n; ++i) bdt[i] = make_double2(h->u_bd[i].x, -h->u_bd[i].y);
    upload_pencil(h->arena, h->st, h->Padj, rpt, cit, Kat, Kbt, h->P.b_kind, bdt, "Padj_");
    if (h->sep) {
        auto sa = std::make_unique<SepCtx>();
        sa->S = h->sep->S;
        for (int d = 0; d < sa->S.ndim; ++d) {
            const double2 sub = h->sep->S.axis[d][0], dg = h->sep->S.axis[d][1], sup = h->sep->S.axis[d][2];
            sa->S.axis[d][0] = make_double2(sup.x, -sup.y);
            sa->S.axis[d][1] = make_double2(dg.x, -dg.y);
            sa->S.axis[d][2] = make_double2(sub.x, -sub.y);
        }
        sa->S.b = make_double2(h->sep->S.b.x, -h->sep->S.b.y);
        sa->ar = &h->arena;
        separable_setup(sa->S, h->arena, h->st, "sepadj_");
        h->sep_adj = std::move(sa);
        h->Padj.sep = h->sep_adj.get();
    }
    h->adj_built = true;
}

__global__ void k_nodes_in(JobSpace js, int J, const double2* rhs, int64_t stride) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (g >= js.n || j >= J) return;
    js.vec[(size_t)j * js.vstride + (size_t)VS_RHS * js.n + g] = rhs[(size_t)j * stride + g];
}

__global__ void k_nodes_out(JobSpace js, int J, double2* out) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (g >= js.n || j >= J) return;
    out[(size_t)j * js.n + g] = js.vec[(size_t)j * js.vstride + (size_t)VS_X * js.n + g];
}

// out_j = (A - z_j B)^{-1} rhs_j (dir 0) or (A - z_j B)^{-H} rhs_j (dir 1) for
// j < N, by the inner solver (FGMRES with the handle's preconditioner at each
// node); rhs_j = rhs + j * rhs_stride, out: [N][n].  False on non-convergence.
bool solve_nodes(sim_ctx* h, int dir, const std::vector<double2>& z, const double2* rhs, int64_t rhs_stride,
                 double2* out) {
    const int N = (int)z.size();
    if (dir) ensure_adjoint(h);
    const Pencil& P = dir ? h->Padj : h->P;
    std::vector<double2> zs(N);
    for (int j = 0; j < N; ++j) zs[j] = dir ? make_double2(z[j].x, -z[j].y) : z[j];
    const std::string tag = dir ? "nadj_" : "nfwd_";
    h->d_nsig[dir] = h->arena.get<double2>(tag + "sig", 64);
    h->d_nfptrs[dir] = h->arena.get<void*>(tag + "fptrs", 64);
    SIM_CUDA(cudaMemcpyAsync(h->d_nsig[dir], zs.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, h->st));
    std::vector<int> ids(N);
    for (int j = 0; j < N; ++j) ids[j] = j;
    if (!P.sep) {
        auto& fac = h->nfactors[dir];
        if ((int)fac.size() < N) fac.resize(N, nullptr);
        for (int j = 0; j < N; ++j)
            if (!fac[j]) {
                cudaError_t e = cudaMalloc(&fac[j], h->factor_bytes);
                if (e != cudaSuccess) throw CudaError{e, "cudaMalloc of a node factorisation"};
            }
        SIM_CUDA(cudaMemcpyAsync(h->d_nfptrs[dir], fac.data(), sizeof(void*) * N, cudaMemcpyHostToDevice, h->st));
        int* d_list = h->arena.get<int>(tag + "list", N);
        SIM_CUDA(cudaMemcpyAsync(d_list, ids.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->st));
        if (!factor_shifts_cluster(P, h->opt.precision, d_list, N, h->d_nsig[dir], h->d_nfptrs[dir], h->st))
            factor_shifts(P, h->opt.precision, d_list, N, h->d_nsig[dir], h->d_nfptrs[dir], h->st);
    }
    JobSpace js = sim::make_jobspace(h->arena, h->st, N, std::max(1, std::min(h->opt.inner_restart, 32)), 1, P.n,
                                     tag);
    js.h_jobshift = ids.data();
    SIM_CUDA(cudaMemcpyAsync(js.d_jobshift, ids.data(), sizeof(int) * N, cudaMemcpyHostToDevice, h->st));
    const dim3 grid(cdiv_up(P.n, 256), N);
    k_nodes_in<<<grid, 256, 0, h->st>>>(js, N, rhs, rhs_stride);
    SIM_LAUNCH_CHECK();
    bool ok = inner_solve(P, h->opt, js, ids, h->d_nsig[dir], h->d_nfptrs[dir], h->st, h->inner);
    k_nodes_out<<<grid, 256, 0, h->st>>>(js, N, out);
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaStreamSynchronize(h->st));
    return ok;
}

// z_j = c + r e^{2πij/N} and the normalised trapezoid weights (z_j - c)/N
void circle_nodes(double2 c, double r, int N, std::vector<double2>& z, std::vector<double2>& w) {
    z.resize(N);
    w.resize(N);
    for (int j = 0; j < N; ++j) {
        const double a = 2.0 * M_PI * j / N;
        const double ox = r * std::cos(a), oy = r * std::sin(a);
        z[j] = make_double2(c.x + ox, c.y + oy);
        w[j] = make_double2(ox / N, oy / N);
    }
}

void copy_out(void* dst, const void* src, size_t bytes, int on_device, cudaStream_t st) {
    SIM_CUDA(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
}

}  // namespace


// ---------------------------------------------------------------------------
// batches of pencils: every pencil's squares of a level in one evaluation
// ---------------------------------------------------------------------------
struct sim_batch_ctx {
    cudaStream_t st = nullptr;
    std::string err;
    std::vector<sim_ctx*> h;
    DeviceArena arena;
    bool region = false;
    int K = 1, level = 1, cur = 0;
    int64_t nsq = 0;
    std::vector<int> sb;         // first global shift id of each pencil (+ total at the end)
    std::vector<double> re_lo, im_lo, s1;
    int64_t squares_evaluated = 0;
    ~sim_batch_ctx() {
        for (sim_ctx* x : h) delete x;
    }
};

namespace {

sim_status bfail(sim_batch_ctx* b, sim_status s, const std::string& msg) {
    if (b) b->err = msg;
    return s;
}

template <class F> sim_status bguarded(sim_batch_ctx* b, F&& f) {
    try {
        b->err.clear();
        return f();
    } catch (const CudaError& e) {
        return bfail(b, e.code == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA, e.what);
    } catch (const std::bad_alloc&) {
        return bfail(b, SIM_ERR_OOM, "host allocation failed");
    } catch (const std::exception& e) {
        const std::string w = e.what();
        if (w.rfind("LIMIT:", 0) == 0) return bfail(b, SIM_ERR_LIMIT, w.substr(6));
        return bfail(b, SIM_ERR_CUDA, w);
    }
}

__global__ void k_add_offset(const int* in, int* out, int64_t n, int off) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] + off;
}

__global__ void k_fill_int(int* out, int64_t n, int v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = v;
}


// The batch's shift table from every pencil's current shifts: H, β, m_eff, σ
// and the pencil id at each pencil's offset b->sb[p] (recomputed here).
void batch_build_table(sim_batch_ctx* b) {
    const int P = (int)b->h.size();
    b->sb.assign(1, 0);
    for (int p = 0; p < P; ++p) b->sb.push_back(b->sb.back() + b->h[p]->S);
    const int S = b->sb.back();
    const int m = b->h[0]->opt.m;
    double2* H = b->arena.get<double2>("H", (int64_t)S * (m + 1) * m);
    double* beta = b->arena.get<double>("beta", S);
    int* meff = b->arena.get<int>("meff", S);
    double2* sigma = b->arena.get<double2>("sigma", S);
    int* pen = b->arena.get<int>("pencil_of", S);
    double2* sT = b->arena.get<double2>("schT", (int64_t)S * m * m);
    double2* sC = b->arena.get<double2>("schC", (int64_t)S * m);
    double2* sQ = b->arena.get<double2>("schQ", (int64_t)S * m);
    int* sOK = b->arena.get<int>("schOK", S);
    for (int p = 0; p < P; ++p) {
        sim_ctx* h = b->h[p];
        const int o = b->sb[p], Sp = h->S;
        SIM_CUDA(cudaMemcpyAsync(H + (size_t)o * (m + 1) * m, h->d_H, sizeof(double2) * Sp * (m + 1) * m,
                                 cudaMemcpyDeviceToDevice, b->st));
        SIM_CUDA(cudaMemcpyAsync(beta + o, h->d_beta, sizeof(double) * Sp, cudaMemcpyDeviceToDevice, b->st));
        SIM_CUDA(cudaMemcpyAsync(meff + o, h->d_meff, sizeof(int) * Sp, cudaMemcpyDeviceToDevice, b->st));
        SIM_CUDA(cudaMemcpyAsync(sigma + o, h->d_sigma, sizeof(double2) * Sp, cudaMemcpyDeviceToDevice, b->st));
        SIM_CUDA(cudaMemcpyAsync(sT + (size_t)o * m * m, h->d_schT, sizeof(double2) * Sp * m * m,
                                 cudaMemcpyDeviceToDevice, b->st));
        SIM_CUDA(cudaMemcpyAsync(sC + (size_t)o * m, h->d_schC, sizeof(double2) * Sp * m, cudaMemcpyDeviceToDevice,
                                 b->st));
        SIM_CUDA(cudaMemcpyAsync(sQ + (size_t)o * m, h->d_schQ, sizeof(double2) * Sp * m, cudaMemcpyDeviceToDevice,
                                 b->st));
        SIM_CUDA(cudaMemcpyAsync(sOK + o, h->d_schOK, sizeof(int) * Sp, cudaMemcpyDeviceToDevice, b->st));
        k_fill_int<<<cdiv_up(Sp, 256), 256, 0, b->st>>>(pen + o, Sp, p);
        SIM_LAUNCH_CHECK();
    }
    std::vector<int> psb(b->sb.begin(), b->sb.end() - 1), pse(b->sb.begin() + 1, b->sb.end());
    SIM_CUDA(cudaMemcpyAsync(b->arena.get<int>("p_sb", P), psb.data(), sizeof(int) * P, cudaMemcpyHostToDevice, b->st));
    SIM_CUDA(cudaMemcpyAsync(b->arena.get<int>("p_se", P), pse.data(), sizeof(int) * P, cudaMemcpyHostToDevice, b->st));
    SIM_CUDA(cudaStreamSynchronize(b->st));
}

}  // namespace

// Accessors for sim_apply_shifted_noalloc (noalloc.cu).
namespace sim {
struct NoallocView {
    const Pencil* P;
    double2* d_sigma;
    int scratch_slot;
    cudaStream_t st;
};
bool noalloc_view(sim_handle h, NoallocView* v) {
    if (!h || !h->d_sigma || h->cap < 1) return false;
    v->P = &h->P;
    v->d_sigma = h->d_sigma;
    v->scratch_slot = h->cap - 1;
    v->st = h->st;
    return true;
}
void noalloc_fail(sim_handle h, const std::string& msg) {
    if (h) h->err = msg;
}
}  // namespace sim

// ---------------------------------------------------------------------------
extern "C" {

void sim_default_options(sim_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->m = 50;
    o->n0 = 4;
    o->delta0 = 0.05;
    o->eps = 1e-8;
    o->h0 = 1e-6;
    o->init_side = 0.0;
    o->shift_sep = 4.0;
    o->max_shift_rounds = 16;
    o->max_shifts = 256;
    o->breakdown_tol = 1e-14;
    o->merge_radius = 0.0;
    o->mult_k = 8;
    o->mult_kmax = 64;
    o->mult_tol = 1e-6;
    o->mult_nodes = 16;
    o->mult_seed = 0x5EED;
    o->residual_scale = 0;
    o->max_squares = 4000000;
    o->precision = SIM_FP64;
    o->inner_tol = 1e-12;
    o->inner_restart = 8;
    o->inner_max_iter = 64;
    o->mult_inner_tol = 1e-10;
    o->mult_reorth = 0;
    o->new_shifts_in_levels = 0;
    o->level_solver = 1;
    o->separable_tensor_cores = 1;
}

sim_status sim_create(const sim_csr* A, const sim_csr* B, const sim_options* opt, void* stream, sim_handle* out) {
    if (!out) return fail(nullptr, SIM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    std::unique_ptr<sim_ctx> h(new sim_ctx());
    sim_status s = guarded(nullptr, [&]() -> sim_status {
        h->st = (cudaStream_t)stream;
        if (opt) h->opt = *opt;
        else sim_default_options(&h->opt);
        const sim_options& o = h->opt;
        if (o.m < 2 || eval_smem_bytes(o.m) > 220 * 1024 || o.n0 != 4 || !(o.delta0 > 0) || !(o.eps > 0) ||
            !(o.h0 > 0) || o.max_shifts < 1 || o.max_shifts > SIM_MAX_SHIFTS - 1 || o.mult_k < 1 ||
            o.mult_kmax < o.mult_k || o.mult_kmax > 64 || o.mult_nodes < 4 || o.mult_nodes > 64 ||
            !(o.inner_tol > 0) || !(o.mult_inner_tol > 0) || o.inner_restart < 1 || o.inner_restart > 32 || o.inner_max_iter < 1 ||
            (o.precision != SIM_FP64 && o.precision != SIM_MIXED) || o.max_squares < 1 ||
            (o.residual_scale != 0 && o.residual_scale != 1) || (o.mult_reorth != 0 && o.mult_reorth != 1) ||
            (o.new_shifts_in_levels != 0 && o.new_shifts_in_levels != 1) ||
            (o.level_solver != 0 && o.level_solver != 1) ||
            (o.separable_tensor_cores != 0 && o.separable_tensor_cores != 1))
            return fail(nullptr, SIM_ERR_INVALID_ARG, "options out of range (m must be <= 52, n0 must be 4)");
        HostCsr a, b;
        std::string why;
        if (!fetch_csr(A, a, why)) return fail(nullptr, SIM_ERR_INVALID_ARG, "A: " + why);
        const bool hasB = B != nullptr;
        if (hasB) {
            if (!fetch_csr(B, b, why)) return fail(nullptr, SIM_ERR_INVALID_ARG, "B: " + why);
            if (b.n != a.n) return fail(nullptr, SIM_ERR_INVALID_ARG, "A and B differ in size");
        }
        const int64_t n = a.n;
        // union pattern with A's and B's values
        std::vector<int32_t> rp(n + 1, 0), ci;
        std::vector<double2> Ka, Kb;
        ci.reserve(a.ci.size() + (hasB ? b.ci.size() : n));
        bool bdiag = true;
        std::vector<double2> bd(n, make_double2(hasB ? 0.0 : 1.0, 0.0));
        std::vector<int32_t> amap(a.ci.size()), bmap(hasB ? b.ci.size() : 0);
        for (int64_t i = 0; i < n; ++i) {
            int64_t ea = a.rp[i], eb = hasB ? b.rp[i] : 0;
            const int64_t fa = a.rp[i + 1], fb = hasB ? b.rp[i + 1] : 0;
            bool diag_done = hasB;  // B = I contributes the diagonal
            while (ea < fa || (hasB && eb < fb) || !diag_done) {
                int64_t ja = ea < fa ? a.ci[ea] : INT64_MAX;
                int64_t jb = hasB ? (eb < fb ? b.ci[eb] : INT64_MAX) : (diag_done ? INT64_MAX : i);
                int64_t j = std::min(ja, jb);
                double2 va = make_double2(0, 0), vb = make_double2(0, 0);
                if (ja == j) {
                    amap[ea] = (int32_t)ci.size();
                    va = a.v[ea++];
                }
                if (jb == j) {
                    if (hasB) {
                        bmap[eb] = (int32_t)ci.size();
                        vb = b.v[eb++];
                    }
                    else {
                        vb = make_double2(1.0, 0.0);
                        diag_done = true;
                    }
                }
                if (hasB && jb == j) {
                    if (j != i && (vb.x != 0 || vb.y != 0)) bdiag = false;
                    if (j == i) bd[i] = vb;
                }
                ci.push_back((int32_t)j);
                Ka.push_back(va);
                Kb.push_back(vb);
            }
            rp[i + 1] = (int32_t)ci.size();
        }
        Pencil& P = h->P;
        upload_pencil(h->arena, h->st, P, rp, ci, Ka, Kb, hasB ? (bdiag ? 1 : 2) : 0, bd, "P_");
        const int T = P.T, nb = P.nb;
        h->u_rp = std::move(rp);
        h->u_ci = std::move(ci);
        h->u_Ka = std::move(Ka);
        h->u_Kb = std::move(Kb);
        h->u_bd = bd;
        h->has_B = hasB;
        {
            // rows, columns and union positions of A's (and B's) own entries
            std::vector<int32_t> row(a.ci.size());
            for (int64_t i = 0; i < n; ++i)
                for (int64_t e = a.rp[i]; e < a.rp[i + 1]; ++e) row[e] = (int32_t)i;
            h->nnzA = (int64_t)a.ci.size();
            h->d_arow = (int32_t*)up_buf(h.get(), "A_row", row.data(), sizeof(int32_t) * row.size());
            h->d_acol = (int32_t*)up_buf(h.get(), "A_col", a.ci.data(), sizeof(int32_t) * a.ci.size());
            h->d_amap = (int32_t*)up_buf(h.get(), "A_map", amap.data(), sizeof(int32_t) * amap.size());
            h->h_amap = amap;
            if (hasB) {
                std::vector<int32_t> brow(b.ci.size());
                for (int64_t i = 0; i < n; ++i)
                    for (int64_t e = b.rp[i]; e < b.rp[i + 1]; ++e) brow[e] = (int32_t)i;
                h->nnzB = (int64_t)b.ci.size();
                h->d_brow = (int32_t*)up_buf(h.get(), "B_row", brow.data(), sizeof(int32_t) * brow.size());
                h->d_bcol = (int32_t*)up_buf(h.get(), "B_col", b.ci.data(), sizeof(int32_t) * b.ci.size());
                h->d_bmap = (int32_t*)up_buf(h.get(), "B_map", bmap.data(), sizeof(int32_t) * bmap.size());
                h->h_bmap = bmap;
            }
        }
        SIM_CUDA(cudaStreamSynchronize(h->st));
        const size_t cs = o.precision == SIM_FP64 ? sizeof(double2) : sizeof(float2);
        h->factor_bytes = ((size_t)2 * nb * (size_t)T * T + (size_t)P.nnzL + (size_t)n + 16) * cs;
        ensure_shift_capacity(h.get());
        h->d_f = h->arena.get<double2>("f", n);
        h->stats.n = n;
        h->stats.nnz_A = (int64_t)a.ci.size();
        h->stats.nnz_B = hasB ? (int64_t)b.ci.size() : n;
        h->stats.block_size = T;
        h->stats.num_blocks = nb;
        if (P.b_kind == 0) {
            h->b_scalar = true;
            h->b_value = make_double2(1.0, 0.0);
        } else if (P.b_kind == 1) {
            h->b_scalar = true;
            h->b_value = bd[0];
            for (int64_t i = 1; i < n && h->b_scalar; ++i)
                h->b_scalar = bd[i].x == bd[0].x && bd[i].y == bd[0].y;
        }
        return SIM_OK;
    });
    if (s != SIM_OK) return s;
    *out = h.release();
    return SIM_OK;
}

sim_status sim_set_region(sim_handle h, double re_lo, double re_hi, double im_lo, double im_hi, const double* f,
                          int32_t f_on_device, uint64_t seed) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!(re_hi > re_lo) || !(im_hi > im_lo) || !std::isfinite(re_lo) || !std::isfinite(re_hi) ||
            !std::isfinite(im_lo) || !std::isfinite(im_hi))
            return fail(h, SIM_ERR_INVALID_ARG, "empty or non-finite region");
        const sim_options& o = h->opt;
        // reset the state of any previous region
        for (int s = 0; s < h->cap - 1; ++s) {
            if (h->factors[s]) {
                cudaFree(h->factors[s]);
                h->factors[s] = nullptr;
            }
        }
        h->S = 0;
        h->eig.clear();
        h->mult.clear();
        h->state = ST_CREATED;
        sim_stats_t keep = h->stats;
        h->stats = sim_stats_t{};
        h->stats.n = keep.n;
        h->stats.nnz_A = keep.nnz_A;
        h->stats.nnz_B = keep.nnz_B;
        h->stats.block_size = keep.block_size;
        h->stats.num_blocks = keep.num_blocks;
        h->inner = InnerStats{};
        const int64_t n = h->P.n;
        if (f) {
            SIM_CUDA(cudaMemcpyAsync(h->d_f, f, sizeof(double2) * n,
                                     f_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
        } else {
            random_vectors(seed, n, 1, 0, h->d_f, n, h->st);
        }
        h->re_lo = re_lo;
        h->re_hi = re_hi;
        h->im_lo = im_lo;
        h->im_hi = im_hi;
        const double W = re_hi - re_lo, Hh = im_hi - im_lo;
        h->s1 = o.init_side > 0 ? o.init_side : std::min(W, Hh);
        h->cols = std::max<int64_t>(1, (int64_t)std::ceil(W / h->s1 - 1e-12));
        h->rows = std::max<int64_t>(1, (int64_t)std::ceil(Hh / h->s1 - 1e-12));
        const int64_t N0 = h->cols * h->rows;
        if (N0 > o.max_squares) return fail(h, SIM_ERR_LIMIT, "initial tiling exceeds max_squares");
        h->K = num_levels(h->s1, o.h0);
        // lattice coordinates at the last level must fit the merge's 64-bit key
        {
            const double nx = (double)h->cols * std::ldexp(1.0, h->K - 1), ny = (double)h->rows * std::ldexp(1.0, h->K - 1);
            if (nx * ny > 9.0e18) return fail(h, SIM_ERR_LIMIT, "region too large for h0 (lattice key overflow)");
        }
        std::vector<int64_t> ix(N0), iy(N0);
        for (int64_t r = 0; r < h->rows; ++r)
            for (int64_t c = 0; c < h->cols; ++c) {
                ix[r * h->cols + c] = c;
                iy[r * h->cols + c] = r;
            }
        int64_t* d_ix = h->arena.get<int64_t>("L0_ix", N0);
        int64_t* d_iy = h->arena.get<int64_t>("L0_iy", N0);
        int* d_sid = h->arena.get<int>("L0_sid", N0);
        SIM_CUDA(cudaMemcpyAsync(d_ix, ix.data(), sizeof(int64_t) * N0, cudaMemcpyHostToDevice, h->st));
        SIM_CUDA(cudaMemcpyAsync(d_iy, iy.data(), sizeof(int64_t) * N0, cudaMemcpyHostToDevice, h->st));
        SIM_CUDA(cudaMemsetAsync(d_sid, 0, sizeof(int) * N0, h->st));
        // step 1: the centre of R is the first shift
        bool ok = build_shifts(h, {make_double2(0.5 * (re_lo + re_hi), 0.5 * (im_lo + im_hi))});
        // step 3 in rounds
        std::vector<uint8_t> resolved(N0, 0);
        std::vector<int> sid(N0, 0);
        std::vector<uint8_t> hflag(N0);
        uint8_t* d_todo = h->arena.get<uint8_t>("L0_todo", N0);
        uint8_t* d_flag = h->arena.get<uint8_t>("L0_flag", N0);
        double sep = -1.0;
        Timer tl(h->st);
        for (int round = 0; round < o.max_shift_rounds; ++round) {
            std::vector<uint8_t> todo(N0);
            for (int64_t q = 0; q < N0; ++q) todo[q] = !resolved[q];
            SIM_CUDA(cudaMemcpyAsync(d_todo, todo.data(), N0, cudaMemcpyHostToDevice, h->st));
            SIM_CUDA(cudaMemcpyAsync(d_sid, sid.data(), sizeof(int) * N0, cudaMemcpyHostToDevice, h->st));
            LevelArgs la;
            la.ix = d_ix;
            la.iy = d_iy;
            la.sid = d_sid;
            la.todo = d_todo;
            la.flag = d_flag;
            la.count = N0;
            la.re_lo = re_lo;
            la.im_lo = im_lo;
            la.side = h->s1;
            eval_level(shift_table(h), la, 1, h->st);
            SIM_CUDA(cudaMemcpyAsync(hflag.data(), d_flag, N0, cudaMemcpyDeviceToHost, h->st));
            SIM_CUDA(cudaMemcpyAsync(sid.data(), d_sid, sizeof(int) * N0, cudaMemcpyDeviceToHost, h->st));
            SIM_CUDA(cudaStreamSynchronize(h->st));
            h->stats.projected_solves += 8 * (int64_t)std::count(todo.begin(), todo.end(), 1);
            std::vector<int64_t> un;
            for (int64_t q = 0; q < N0; ++q) {
                if (todo[q] && hflag[q] == 0) resolved[q] = 1;
                if (!resolved[q]) un.push_back(q);
            }
            if (un.empty()) break;
            if (sep < 0) {
                double rho = INFINITY;
                const double2 s0 = h->h_sigma[0];
                for (int64_t q : un) {
                    double2 c = center_of(h, h->s1, ix[q], iy[q]);
                    rho = std::min(rho, std::hypot(c.x - s0.x, c.y - s0.y));
                }
                sep = std::max(o.shift_sep * h->s1, rho);
            }
            std::vector<int64_t> picked;
            for (int64_t q : un) {
                double2 c = center_of(h, h->s1, ix[q], iy[q]);
                bool far = true;
                for (int64_t p : picked) {
                    double2 d = center_of(h, h->s1, ix[p], iy[p]);
                    if (std::hypot(c.x - d.x, c.y - d.y) < sep) {
                        far = false;
                        break;
                    }
                }
                if (far) picked.push_back(q);
            }
            std::vector<double2> cen;
            for (size_t t = 0; t < picked.size(); ++t) {
                cen.push_back(center_of(h, h->s1, ix[picked[t]], iy[picked[t]]));
                sid[picked[t]] = h->S + (int)t;
            }
            ok = build_shifts(h, cen) && ok;
        }
        SIM_CUDA(cudaMemcpyAsync(d_sid, sid.data(), sizeof(int) * N0, cudaMemcpyHostToDevice, h->st));
        h->stats.t_levels_ms += tl.ms();
        h->nsq = N0;
        h->cur = 0;
        h->level = 1;
        h->stats.levels_total = h->K;
        h->state = ST_REGION;
        sync_stats(h);
        if (!ok) return fail(h, SIM_ERR_NOT_CONVERGED, "an inner shifted solve did not converge");
        return SIM_OK;
    });
}

sim_status sim_solve_level(sim_handle h, int64_t* n_marked, int32_t* done) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (h->state != ST_REGION || h->level > h->K) return fail(h, SIM_ERR_BAD_STATE, "no level to solve");
        Timer tl(h->st);
        const int k = h->level;
        const double side = h->s1 / std::ldexp(1.0, k - 1);
        const std::string a = "L" + std::to_string(h->cur) + "_", b = "L" + std::to_string(1 - h->cur) + "_";
        const int64_t N = h->nsq;
        int64_t* ix = h->arena.get<int64_t>(a + "ix", N);
        int64_t* iy = h->arena.get<int64_t>(a + "iy", N);
        int* sid = h->arena.get<int>(a + "sid", N);
        uint8_t* mark = h->arena.get<uint8_t>("mark", N);
        uint8_t* flag = h->arena.get<uint8_t>("flag", N);
        double* ind = h->arena.get<double>("ind", N);
        LevelArgs la;
        la.ix = ix;
        la.iy = iy;
        la.sid = sid;
        la.mark = mark;
        la.flag = flag;
        la.ind = ind;
        la.count = N;
        la.re_lo = h->re_lo;
        la.im_lo = h->im_lo;
        la.side = side;
        la.retries = h->arena.get<unsigned long long>("retries", 1);
        const int nbk = cdiv_up(std::max<int64_t>(N, 1), 1024);
        int64_t* bsum = h->arena.get<int64_t>("bsum", nbk + 1);
        int64_t* tot = h->arena.get<int64_t>("tot", 1);
        bool level_ok = true;
        for (int round = 0;; ++round) {
            SIM_CUDA(cudaMemsetAsync(la.retries, 0, sizeof(unsigned long long), h->st));
            h->stats.direct_level_evaluations +=
                evaluate_level(shift_table(h), la, h->opt.level_solver, h->S, h->arena, bsum, tot, h->st);
            h->stats.squares_evaluated += N;
            h->stats.unresolvable_last_level = count_marked(flag, N, bsum, tot, h->arena.host_i64(), h->st);
            unsigned long long rt = 0;
            SIM_CUDA(cudaMemcpyAsync(&rt, la.retries, sizeof(rt), cudaMemcpyDeviceToHost, h->st));
            SIM_CUDA(cudaStreamSynchronize(h->st));
            h->stats.shift_retries += (int64_t)rt;
            h->stats.projected_solves += 8 * (N + (int64_t)rt);
            if (!h->opt.new_shifts_in_levels || h->stats.unresolvable_last_level == 0 ||
                round >= h->opt.max_shift_rounds)
                break;
            // step 3's rounds at this level: new Krylov spaces at the centres of the
            // unresolved squares (list order, at least shift_sep·side apart), then the
            // whole level again (resolved squares give the same result)
            std::vector<uint8_t> hf(N);
            std::vector<int64_t> hx(N), hy(N);
            SIM_CUDA(cudaMemcpyAsync(hf.data(), flag, N, cudaMemcpyDeviceToHost, h->st));
            SIM_CUDA(cudaMemcpyAsync(hx.data(), ix, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, h->st));
            SIM_CUDA(cudaMemcpyAsync(hy.data(), iy, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, h->st));
            SIM_CUDA(cudaStreamSynchronize(h->st));
            const double sep = h->opt.shift_sep * side;
            std::vector<double2> cen;
            for (int64_t q = 0; q < N; ++q) {
                if (!hf[q]) continue;
                const double2 c = center_of(h, side, hx[q], hy[q]);
                bool far = true;
                for (const double2& d : cen)
                    if (std::hypot(c.x - d.x, c.y - d.y) < sep) {
                        far = false;
                        break;
                    }
                if (far) cen.push_back(c);
            }
            level_ok = build_shifts(h, cen) && level_ok;
            sync_stats(h);
        }
        if (!level_ok) return fail(h, SIM_ERR_NOT_CONVERGED, "an inner shifted solve did not converge");
        const int64_t cnt = count_marked(mark, N, bsum, tot, h->arena.host_i64(), h->st);
        const bool last = (k == h->K);
        if (!last) {
            if (4 * cnt > h->opt.max_squares)
                return fail(h, SIM_ERR_LIMIT, "level " + std::to_string(k + 1) + " would hold " +
                                                  std::to_string(4 * cnt) + " squares (> max_squares)");
            int64_t* nix = h->arena.get<int64_t>(b + "ix", 4 * cnt);
            int64_t* niy = h->arena.get<int64_t>(b + "iy", 4 * cnt);
            int* nsid = h->arena.get<int>(b + "sid", 4 * cnt);
            emit_marked(mark, flag, ix, iy, sid, N, bsum, 0, nix, niy, nsid, nullptr, h->st);
            h->cur = 1 - h->cur;
            h->nsq = 4 * cnt;
        } else {
            int64_t* fix = h->arena.get<int64_t>("F_ix", cnt);
            int64_t* fiy = h->arena.get<int64_t>("F_iy", cnt);
            int* fsid = h->arena.get<int>("F_sid", cnt);
            uint8_t* ffl = h->arena.get<uint8_t>("F_flag", cnt);
            emit_marked(mark, flag, ix, iy, sid, N, bsum, 1, fix, fiy, fsid, ffl, h->st);
            h->nfinal = cnt;
            h->s_final = side;
            h->state = ST_LEVELS_DONE;
        }
        SIM_CUDA(cudaStreamSynchronize(h->st));
        h->stats.t_levels_ms += tl.ms();
        h->stats.levels_done = k;
        h->level = k + 1;
        if (n_marked) *n_marked = cnt;
        if (done) *done = last ? 1 : 0;
        return SIM_OK;
    });
}

sim_status sim_eigenvalues(sim_handle h, double* out, int64_t capacity, int64_t* count) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (h->state < ST_LEVELS_DONE) return fail(h, SIM_ERR_BAD_STATE, "levels not finished");
        if (h->state == ST_LEVELS_DONE) {
            Timer tm(h->st);
            const int64_t N = h->nfinal;
            h->eig.clear();
            h->cl_shift.clear();
            h->cl_size.clear();
            h->cl_flag.clear();
            h->cl_radius.clear();
            if (N > 0) {
                const int64_t nx = h->cols << (h->K - 1), ny = h->rows << (h->K - 1);
                MergeResult R = merge_final(h->arena.get<int64_t>("F_ix", N), h->arena.get<int64_t>("F_iy", N),
                                            h->arena.get<int>("F_sid", N), h->arena.get<uint8_t>("F_flag", N), N, nx,
                                            ny, h->re_lo, h->re_hi, h->im_lo, h->im_hi, h->s_final,
                                            h->opt.merge_radius, h->arena, h->st);
                std::vector<double2> est(R.C);
                std::vector<int> size(R.C), nfl(R.C), shift(R.C), rank(R.C);
                std::vector<double> rad(R.C);
                SIM_CUDA(cudaMemcpyAsync(est.data(), R.est, sizeof(double2) * R.C, cudaMemcpyDeviceToHost, h->st));
                SIM_CUDA(cudaMemcpyAsync(size.data(), R.size, sizeof(int) * R.C, cudaMemcpyDeviceToHost, h->st));
                SIM_CUDA(cudaMemcpyAsync(nfl.data(), R.nflag, sizeof(int) * R.C, cudaMemcpyDeviceToHost, h->st));
                SIM_CUDA(cudaMemcpyAsync(shift.data(), R.shift, sizeof(int) * R.C, cudaMemcpyDeviceToHost, h->st));
                SIM_CUDA(cudaMemcpyAsync(rank.data(), R.rank, sizeof(int) * R.C, cudaMemcpyDeviceToHost, h->st));
                SIM_CUDA(cudaMemcpyAsync(rad.data(), R.radius, sizeof(double) * R.C, cudaMemcpyDeviceToHost, h->st));
                SIM_CUDA(cudaStreamSynchronize(h->st));
                h->eig.assign(R.inside, make_double2(0, 0));
                h->cl_shift.assign(R.inside, 0);
                h->cl_size.assign(R.inside, 0);
                h->cl_flag.assign(R.inside, 0);
                h->cl_radius.assign(R.inside, 0.0);
                int64_t unres = 0;
                for (int c = 0; c < R.C; ++c) {
                    if (rank[c] < 0) continue;
                    h->eig[rank[c]] = est[c];
                    h->cl_shift[rank[c]] = shift[c];
                    h->cl_size[rank[c]] = size[c];
                    h->cl_flag[rank[c]] = nfl[c];
                    h->cl_radius[rank[c]] = rad[c];
                }
                std::vector<uint8_t> ff(N);
                SIM_CUDA(cudaMemcpy(ff.data(), h->arena.get<uint8_t>("F_flag", N), N, cudaMemcpyDeviceToHost));
                for (auto v : ff) unres += v;
                h->stats.unresolvable_final = unres;
            }
            h->stats.final_squares = N;
            h->stats.clusters = (int64_t)h->eig.size();
            h->stats.t_merge_ms += tm.ms();
            h->state = ST_EIGS;
        }
        const int64_t C = (int64_t)h->eig.size();
        if (count) *count = C;
        if (capacity == 0) return SIM_OK;
        if (capacity < C || !out) return fail(h, SIM_ERR_CAPACITY, "output capacity too small");
        std::memcpy(out, h->eig.data(), sizeof(double2) * C);
        return SIM_OK;
    });
}

sim_status sim_multiplicity(sim_handle h, int32_t* out, int64_t capacity, int64_t* count) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (h->state != ST_EIGS) return fail(h, SIM_ERR_BAD_STATE, "call sim_eigenvalues first");
        const int64_t C = (int64_t)h->eig.size();
        if (h->mult.size() != (size_t)C) {
            Timer tm(h->st);
            MultInput mi;
            mi.P = &h->P;
            mi.opt = &h->opt;
            mi.st = h->st;
            mi.arena = &h->arena;
            mi.d_sigma = h->d_sigma;
            mi.d_fptrs = h->d_fptrs;
            mi.est = h->eig;
            mi.shift = h->cl_shift;
            mi.radius = h->cl_radius;
            mi.inner = &h->inner;
            bool ok = true;
            h->mult = multiplicities(mi, ok);
            h->stats.t_mult_ms += tm.ms();
            sync_stats(h);
            if (!ok) return fail(h, SIM_ERR_NOT_CONVERGED, "an inner shifted solve did not converge");
        }
        if (count) *count = C;
        if (capacity == 0) return SIM_OK;
        if (capacity < C || !out) return fail(h, SIM_ERR_CAPACITY, "output capacity too small");
        for (int64_t c = 0; c < C; ++c) out[c] = h->mult[c];
        return SIM_OK;
    });
}

sim_status sim_projection(sim_handle h, int64_t c, double* out) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (h->state != ST_EIGS) return fail(h, SIM_ERR_BAD_STATE, "call sim_eigenvalues first");
        if (c < 0 || c >= (int64_t)h->eig.size()) return fail(h, SIM_ERR_INVALID_ARG, "no such eigenvalue");
        if (!out) return fail(h, SIM_ERR_INVALID_ARG, "NULL output");
        MultInput mi;
        mi.P = &h->P;
        mi.opt = &h->opt;
        mi.st = h->st;
        mi.arena = &h->arena;
        mi.d_sigma = h->d_sigma;
        mi.d_fptrs = h->d_fptrs;
        mi.est = h->eig;
        mi.shift = h->cl_shift;
        mi.radius = h->cl_radius;
        mi.inner = &h->inner;
        if (!projection_vector(mi, h->d_f, (int)c, reinterpret_cast<double2*>(out)))
            return fail(h, SIM_ERR_NOT_CONVERGED, "an inner shifted solve did not converge");
        return SIM_OK;
    });
}

sim_status sim_refine(sim_handle h, double* out, int32_t* refined, int64_t capacity, int64_t* count) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (h->state != ST_EIGS) return fail(h, SIM_ERR_BAD_STATE, "call sim_eigenvalues first");
        const int64_t C = (int64_t)h->eig.size();
        if (count) *count = C;
        if (capacity == 0) return SIM_OK;
        if (capacity < C || !out) return fail(h, SIM_ERR_CAPACITY, "output capacity too small");
        RitzInput ri;
        ri.arena = &h->arena;
        ri.st = h->st;
        ri.m = h->opt.m;
        ri.num_slots = h->cap;
        ri.d_H = h->d_H;
        ri.d_meff = h->d_meff;
        ri.d_sigma = h->d_sigma;
        ri.h0 = h->opt.h0;
        ri.est = h->eig;
        ri.shift = h->cl_shift;
        ri.radius = h->cl_radius;
        std::vector<double2> vals;
        std::vector<int> flags;
        if (!ritz_refine(ri, vals, flags))
            return fail(h, SIM_ERR_NOT_CONVERGED, "the QR iteration of a Hessenberg matrix did not converge");
        std::memcpy(out, vals.data(), sizeof(double2) * C);
        if (refined)
            for (int64_t c = 0; c < C; ++c) refined[c] = flags[c];
        return SIM_OK;
    });
}

sim_status sim_stats(sim_handle h, sim_stats_t* out, size_t size) {
    if (!h || !out) return fail(h, SIM_ERR_INVALID_ARG, "NULL argument");
    sync_stats(h);
    std::memcpy(out, &h->stats, std::min(size, sizeof(sim_stats_t)));
    return SIM_OK;
}

const char* sim_last_error(sim_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void sim_destroy(sim_handle h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    delete h;
}

sim_status sim_shift_count(sim_handle h, int32_t* count) {
    if (!h || !count) return fail(h, SIM_ERR_INVALID_ARG, "NULL argument");
    *count = h->S;
    return SIM_OK;
}

sim_status sim_get_shift(sim_handle h, int32_t s, double* sigma, double* H_host, double* beta, int32_t* m_eff) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (s < 0 || s >= h->S) return fail(h, SIM_ERR_INVALID_ARG, "shift index out of range");
        const int m = h->opt.m;
        if (sigma) {
            sigma[0] = h->h_sigma[s].x;
            sigma[1] = h->h_sigma[s].y;
        }
        if (H_host)
            SIM_CUDA(cudaMemcpy(H_host, h->d_H + (size_t)s * (m + 1) * m, sizeof(double2) * (m + 1) * m,
                                cudaMemcpyDeviceToHost));
        if (beta) SIM_CUDA(cudaMemcpy(beta, h->d_beta + s, sizeof(double), cudaMemcpyDeviceToHost));
        if (m_eff) SIM_CUDA(cudaMemcpy(m_eff, h->d_meff + s, sizeof(int), cudaMemcpyDeviceToHost));
        return SIM_OK;
    });
}

sim_status sim_eval_squares(const double* H, int32_t m, int32_t m_eff, double beta, double sig_re, double sig_im,
                            const double* centers, const double* sides, int64_t count, int32_t residual_scale,
                            double* indicator, double* rho, void* stream) {
    return guarded(nullptr, [&]() -> sim_status {
        if (!H || !centers || !sides || !indicator || !rho || count < 0 || m < 1 || m_eff < 1 || m_eff > m ||
            eval_smem_bytes(m) > 220 * 1024)
            return fail(nullptr, SIM_ERR_INVALID_ARG, "sim_eval_squares: bad argument (m <= 52)");
        eval_explicit((const double2*)H, m, m_eff, beta, make_double2(sig_re, sig_im), (const double2*)centers, sides,
                      count, residual_scale, indicator, rho, (cudaStream_t)stream);
        SIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return SIM_OK;
    });
}

sim_status sim_apply_shifted(sim_handle h, double sig_re, double sig_im, const double* x, double* y) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!x || !y) return fail(h, SIM_ERR_INVALID_ARG, "NULL vector");
        const int sc = h->cap - 1;
        const double2 sg = make_double2(sig_re, sig_im);
        SIM_CUDA(cudaMemcpyAsync(h->d_sigma + sc, &sg, sizeof(double2), cudaMemcpyHostToDevice, h->st));
        JobSpace js = make_jobspace(h, 1, "cmp_");
        SIM_CUDA(cudaMemcpyAsync(js.d_jobshift, &sc, sizeof(int), cudaMemcpyHostToDevice, h->st));
        const int zero = 0;
        SIM_CUDA(cudaMemcpyAsync(js.d_active, &zero, sizeof(int), cudaMemcpyHostToDevice, h->st));
        SIM_CUDA(cudaMemcpyAsync(js.vec + (size_t)VS_X * js.n, x, sizeof(double2) * js.n, cudaMemcpyDeviceToDevice, h->st));
        spmv_shifted_jobs(h->P, js, 1, nullptr, VS_X, VS_W, h->d_sigma, h->st);
        SIM_CUDA(cudaMemcpyAsync(y, js.vec + (size_t)VS_W * js.n, sizeof(double2) * js.n, cudaMemcpyDeviceToDevice, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
        return SIM_OK;
    });
}

sim_status sim_shifted_solve(sim_handle h, double sig_re, double sig_im, const double* r, double* x, int32_t* iters,
                             double* relres) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!r || !x) return fail(h, SIM_ERR_INVALID_ARG, "NULL vector");
        const int sc = h->cap - 1;
        const double2 sg = make_double2(sig_re, sig_im);
        h->h_sigma[sc] = sg;
        SIM_CUDA(cudaMemcpyAsync(h->d_sigma + sc, &sg, sizeof(double2), cudaMemcpyHostToDevice, h->st));
        if (!h->P.sep) {
            factor_storage(h, sc);
            int* d_list = h->arena.get<int>("cmp_list", 1);
            SIM_CUDA(cudaMemcpyAsync(d_list, &sc, sizeof(int), cudaMemcpyHostToDevice, h->st));
            if (!factor_shifts_cluster(h->P, h->opt.precision, d_list, 1, h->d_sigma, h->d_fptrs, h->st))
                factor_shifts(h->P, h->opt.precision, d_list, 1, h->d_sigma, h->d_fptrs, h->st);
        }
        JobSpace js = make_jobspace(h, 1, "cmp_");
        js.h_jobshift = &sc;
        SIM_CUDA(cudaMemcpyAsync(js.d_jobshift, &sc, sizeof(int), cudaMemcpyHostToDevice, h->st));
        SIM_CUDA(cudaMemcpyAsync(js.vec + (size_t)VS_RHS * js.n, r, sizeof(double2) * js.n, cudaMemcpyDeviceToDevice,
                                 h->st));
        InnerStats is;
        bool ok = inner_solve(h->P, h->opt, js, {0}, h->d_sigma, h->d_fptrs, h->st, is);
        SIM_CUDA(cudaMemcpyAsync(x, js.vec + (size_t)VS_X * js.n, sizeof(double2) * js.n, cudaMemcpyDeviceToDevice, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
        if (iters) *iters = (int32_t)is.iters;
        if (relres) *relres = is.worst;
        if (!ok) return fail(h, SIM_ERR_NOT_CONVERGED, "shifted solve did not converge");
        return SIM_OK;
    });
}

sim_status sim_set_separable(sim_handle h, int32_t ndim, const int64_t* dims, const double* axes) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (ndim < 1 || ndim > 3 || !dims || !axes) return fail(h, SIM_ERR_INVALID_ARG, "ndim must be 1..3");
        int64_t prod = 1;
        for (int d = 0; d < ndim; ++d) {
            if (dims[d] < 1 || dims[d] > 8192) return fail(h, SIM_ERR_INVALID_ARG, "axis length out of range (1..8192)");
            prod *= dims[d];
        }
        if (prod != h->P.n) return fail(h, SIM_ERR_INVALID_ARG, "the axis lengths' product differs from n");
        if (!h->b_scalar) return fail(h, SIM_ERR_INVALID_ARG, "B is not a multiple of the identity");
        auto sep = std::make_unique<SepCtx>();
        sep->S.ndim = ndim;
        sep->S.b = h->b_value;
        for (int d = 0; d < ndim; ++d) {
            sep->S.dims[d] = dims[d];
            for (int e = 0; e < 3; ++e) {
                const double re = axes[6 * d + 2 * e], im = axes[6 * d + 2 * e + 1];
                if (!std::isfinite(re) || !std::isfinite(im)) return fail(h, SIM_ERR_INVALID_ARG, "non-finite axis entry");
                sep->S.axis[d][e] = make_double2(re, im);
            }
            const double2 sub = sep->S.axis[d][0], sup = sep->S.axis[d][2];
            if (dims[d] > 1 && ((sub.x == 0 && sub.y == 0) || (sup.x == 0 && sup.y == 0)))
                return fail(h, SIM_ERR_INVALID_ARG, "an axis with a zero off-diagonal is not diagonalisable");
        }
        sep->S.tc = h->opt.separable_tensor_cores != 0;
        sep->ar = &h->arena;
        separable_setup(sep->S, h->arena, h->st);
        // the factorisations of an earlier region are no longer used
        for (int s = 0; s < h->cap; ++s) {
            if (h->factors[s]) {
                cudaFree(h->factors[s]);
                h->factors[s] = nullptr;
            }
        }
        h->sep = std::move(sep);
        h->P.sep = h->sep.get();
        h->S = 0;
        h->state = ST_CREATED;
        return SIM_OK;
    });
}

sim_status sim_projection_norm(sim_handle h, double c_re, double c_im, double radius, int32_t nodes, const double* f,
                               int32_t f_on_device, int32_t keep, double* phi) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!f || !phi || !(radius > 0) || !std::isfinite(radius) || nodes < 4 || nodes > 64 || !std::isfinite(c_re) ||
            !std::isfinite(c_im))
            return fail(h, SIM_ERR_INVALID_ARG, "bad argument (radius > 0, 4 <= nodes <= 64, f and phi non-NULL)");
        const int64_t n = h->P.n;
        h->pn_valid = false;
        circle_nodes(make_double2(c_re, c_im), radius, nodes, h->pn_z, h->pn_w);
        h->d_pn_f = h->arena.get<double2>("pn_f", n);
        h->d_pn_x = h->arena.get<double2>("pn_x", n);
        SIM_CUDA(cudaMemcpyAsync(h->d_pn_f, f, sizeof(double2) * n,
                                 f_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st));
        double2* X = h->arena.get<double2>("pn_X", (int64_t)nodes * n);
        if (!solve_nodes(h, 0, h->pn_z, h->d_pn_f, 0, X)) return fail(h, SIM_ERR_NOT_CONVERGED, "node solve did not converge");
        double2* d_w = h->arena.get<double2>("pn_w", 64);
        SIM_CUDA(cudaMemcpyAsync(d_w, h->pn_w.data(), sizeof(double2) * nodes, cudaMemcpyHostToDevice, h->st));
        combine_nodes(X, nodes, n, d_w, false, h->d_pn_x, h->st);
        double2* part = h->arena.get<double2>("red_part", dot_partials());
        double2* d_s = h->arena.get<double2>("red_out", 4);
        dot(h->d_pn_x, nullptr, n, part, d_s, h->st);
        double2 s;
        SIM_CUDA(cudaMemcpyAsync(&s, d_s, sizeof(double2), cudaMemcpyDeviceToHost, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
        *phi = s.x;
        h->pn_kept = keep != 0;
        if (!h->pn_kept) h->arena.release("pn_X");
        h->pn_valid = true;
        return SIM_OK;
    });
}

sim_status sim_projection_norm_grad(sim_handle h, double* grad_A, double* grad_B, int32_t out_on_device) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!h->pn_valid) return fail(h, SIM_ERR_BAD_STATE, "call sim_projection_norm first");
        if (!grad_A) return fail(h, SIM_ERR_INVALID_ARG, "grad_A is NULL");
        const int64_t n = h->P.n;
        const int N = (int)h->pn_z.size();
        double2* X = h->arena.get<double2>("pn_X", (int64_t)N * n);
        if (!h->pn_kept) {  // recompute the node solutions instead of having kept them
            if (!solve_nodes(h, 0, h->pn_z, h->d_pn_f, 0, X))
                return fail(h, SIM_ERR_NOT_CONVERGED, "node solve did not converge");
        }
        double2* d_w = h->arena.get<double2>("pn_w", 64);
        SIM_CUDA(cudaMemcpyAsync(d_w, h->pn_w.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, h->st));
        double2* R = h->arena.get<double2>("pn_R", (int64_t)N * n);
        scaled_copies(h->d_pn_x, N, n, d_w, R, h->st);
        double2* Mu = h->arena.get<double2>("pn_Mu", (int64_t)N * n);
        if (!solve_nodes(h, 1, h->pn_z, R, n, Mu)) return fail(h, SIM_ERR_NOT_CONVERGED, "adjoint solve did not converge");
        std::vector<double2> aA(N), aB(N);
        for (int j = 0; j < N; ++j) {
            aA[j] = make_double2(-2.0, 0.0);
            aB[j] = make_double2(2.0 * h->pn_z[j].x, -2.0 * h->pn_z[j].y);
        }
        double2* d_a = h->arena.get<double2>("pn_a", 128);
        SIM_CUDA(cudaMemcpyAsync(d_a, aA.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, h->st));
        SIM_CUDA(cudaMemcpyAsync(d_a + 64, aB.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, h->st));
        double2* gA = h->arena.get<double2>("pn_gA", h->nnzA);
        entry_grad(entries_A(h), Mu, X, N, n, d_a, 0, gA, h->st);
        copy_out(grad_A, gA, sizeof(double2) * h->nnzA, out_on_device, h->st);
        if (grad_B && h->has_B) {
            double2* gB = h->arena.get<double2>("pn_gB", h->nnzB);
            entry_grad(entries_B(h), Mu, X, N, n, d_a + 64, 0, gB, h->st);
            copy_out(grad_B, gB, sizeof(double2) * h->nnzB, out_on_device, h->st);
        }
        SIM_CUDA(cudaStreamSynchronize(h->st));
        h->arena.release("pn_R");
        h->arena.release("pn_Mu");
        if (!h->pn_kept) h->arena.release("pn_X");
        return SIM_OK;
    });
}

sim_status sim_eigenvalue_grad(sim_handle h, double c_re, double c_im, double radius, int32_t nodes, uint64_t seed,
                               double* lambda, double* dl_dA, double* dl_dB, int32_t out_on_device) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!lambda || !dl_dA || !(radius > 0) || !std::isfinite(radius) || nodes < 4 || nodes > 64 ||
            !std::isfinite(c_re) || !std::isfinite(c_im))
            return fail(h, SIM_ERR_INVALID_ARG, "bad argument (radius > 0, 4 <= nodes <= 64, lambda and dl_dA non-NULL)");
        const int64_t n = h->P.n;
        std::vector<double2> z, w;
        circle_nodes(make_double2(c_re, c_im), radius, nodes, z, w);
        double2* vu = h->arena.get<double2>("eg_vu", 2 * n);  // v (right start), u (left start)
        random_vectors(seed, n, 2, 0, vu, n, h->st);
        double2* X = h->arena.get<double2>("eg_X", (int64_t)nodes * n);
        if (!solve_nodes(h, 0, z, vu, 0, X)) return fail(h, SIM_ERR_NOT_CONVERGED, "node solve did not converge");
        double2* d_w = h->arena.get<double2>("eg_w", 64);
        SIM_CUDA(cudaMemcpyAsync(d_w, w.data(), sizeof(double2) * nodes, cudaMemcpyHostToDevice, h->st));
        double2* x = h->arena.get<double2>("eg_x", n);
        double2* y = h->arena.get<double2>("eg_y", n);
        double2* t = h->arena.get<double2>("eg_t", n);
        combine_nodes(X, nodes, n, d_w, false, x, h->st);
        ensure_adjoint(h);
        apply_B(h->Padj, vu + n, t, h->st);  // B^H u
        if (!solve_nodes(h, 1, z, t, 0, X)) return fail(h, SIM_ERR_NOT_CONVERGED, "adjoint solve did not converge");
        combine_nodes(X, nodes, n, d_w, true, y, h->st);
        h->arena.release("eg_X");
        // y^H A x and y^H B x
        double2* part = h->arena.get<double2>("red_part", dot_partials());
        double2* d_s = h->arena.get<double2>("red_out", 4);
        entry_form(entries_A(h), h->P.Ka, y, x, part, d_s, h->st);
        apply_B(h->P, x, t, h->st);
        dot(y, t, n, part, d_s + 1, h->st);
        double2 s[2];
        SIM_CUDA(cudaMemcpyAsync(s, d_s, sizeof(s), cudaMemcpyDeviceToHost, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
        const double2 yAx = s[0], yBx = s[1];
        if (!(cabsd(yBx) > 0.0)) return fail(h, SIM_ERR_INVALID_ARG, "no eigenvalue inside the circle (y^H B x = 0)");
        const double2 lam = cdiv(yAx, yBx);
        lambda[0] = lam.x;
        lambda[1] = lam.y;
        const double2 inv = cdiv(make_double2(1.0, 0.0), yBx);
        const double2 a[2] = {inv, make_double2(-(lam.x * inv.x - lam.y * inv.y), -(lam.x * inv.y + lam.y * inv.x))};
        double2* d_a = h->arena.get<double2>("eg_a", 2);
        SIM_CUDA(cudaMemcpyAsync(d_a, a, sizeof(a), cudaMemcpyHostToDevice, h->st));
        double2* gA = h->arena.get<double2>("eg_gA", h->nnzA);
        entry_grad(entries_A(h), y, x, 1, n, d_a, 1, gA, h->st);
        copy_out(dl_dA, gA, sizeof(double2) * h->nnzA, out_on_device, h->st);
        if (dl_dB && h->has_B) {
            double2* gB = h->arena.get<double2>("eg_gB", h->nnzB);
            entry_grad(entries_B(h), y, x, 1, n, d_a + 1, 1, gB, h->st);
            copy_out(dl_dB, gB, sizeof(double2) * h->nnzB, out_on_device, h->st);
        }
        SIM_CUDA(cudaStreamSynchronize(h->st));
        return SIM_OK;
    });
}

sim_status sim_update_values(sim_handle h, const double* a_values, const double* b_values, int32_t on_device) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (!a_values && !b_values) return fail(h, SIM_ERR_INVALID_ARG, "no values given");
        if (b_values && !h->has_B) return fail(h, SIM_ERR_INVALID_ARG, "the handle has B = I");
        const auto kind = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        std::vector<double2> va, vb;
        if (a_values) {
            va.resize(h->nnzA);
            SIM_CUDA(cudaMemcpy(va.data(), a_values, sizeof(double2) * h->nnzA, kind));
        }
        if (b_values) {
            vb.resize(h->nnzB);
            SIM_CUDA(cudaMemcpy(vb.data(), b_values, sizeof(double2) * h->nnzB, kind));
        }
        for (const auto& v : va)
            if (!std::isfinite(v.x) || !std::isfinite(v.y)) return fail(h, SIM_ERR_INVALID_ARG, "non-finite value");
        for (const auto& v : vb)
            if (!std::isfinite(v.x) || !std::isfinite(v.y)) return fail(h, SIM_ERR_INVALID_ARG, "non-finite value");
        std::vector<double2> Ka = h->u_Ka, Kb = h->u_Kb;
        for (size_t i = 0; i < va.size(); ++i) Ka[h->h_amap[i]] = va[i];
        for (size_t i = 0; i < vb.size(); ++i) Kb[h->h_bmap[i]] = vb[i];
        // B's kind (identity, diagonal, general) and diagonal from the new values
        const int64_t n = h->P.n;
        int b_kind = 0;
        std::vector<double2> bd(n, make_double2(h->has_B ? 0.0 : 1.0, 0.0));
        if (h->has_B) {
            b_kind = 1;
            for (int64_t i = 0; i < n; ++i)
                for (int64_t e = h->u_rp[i]; e < h->u_rp[i + 1]; ++e) {
                    if (h->u_ci[e] == i) bd[i] = Kb[e];
                    else if (Kb[e].x != 0 || Kb[e].y != 0) b_kind = 2;
                }
        }
        bool b_scalar = b_kind == 0;
        if (b_kind == 1) {
            b_scalar = true;
            for (int64_t i = 1; i < n && b_scalar; ++i) b_scalar = bd[i].x == bd[0].x && bd[i].y == bd[0].y;
        }
        if (h->sep && !b_scalar) return fail(h, SIM_ERR_INVALID_ARG, "the separable preconditioner needs B = b I");
        SepCtx* sep = h->P.sep;
        upload_pencil(h->arena, h->st, h->P, h->u_rp, h->u_ci, Ka, Kb, b_kind, bd, "P_");
        h->P.sep = sep;
        h->u_Ka.swap(Ka);
        h->u_Kb.swap(Kb);
        h->u_bd.swap(bd);
        h->b_scalar = b_scalar;
        h->b_value = b_kind == 0 ? make_double2(1.0, 0.0) : h->u_bd[0];
        if (h->sep && (h->sep->S.b.x != h->b_value.x || h->sep->S.b.y != h->b_value.y)) {
            h->sep->S.b = h->b_value;
        }
        // everything derived from the old values is stale
        h->adj_built = false;
        h->sep_adj.reset();
        h->Padj.sep = nullptr;
        h->pn_valid = false;
        for (int s = 0; s < h->cap; ++s) {
            if (h->factors[s]) {
                cudaFree(h->factors[s]);
                h->factors[s] = nullptr;
            }
        }
        h->S = 0;
        h->state = ST_CREATED;
        return SIM_OK;
    });
}

// ---- batches of pencils -------------------------------------------------------
sim_status sim_batch_create(int32_t count, const sim_csr* A, const sim_csr* B, const sim_options* opt, void* stream,
                            sim_batch* out) {
    if (!out) return SIM_ERR_INVALID_ARG;
    *out = nullptr;
    if (count < 1 || !A) return SIM_ERR_INVALID_ARG;
    std::unique_ptr<sim_batch_ctx> b(new sim_batch_ctx());
    b->st = (cudaStream_t)stream;
    for (int p = 0; p < count; ++p) {
        sim_handle h = nullptr;
        const sim_status s = sim_create(&A[p], B ? &B[p] : nullptr, opt, stream, &h);
        if (s != SIM_OK) {
            g_create_error = "pencil " + std::to_string(p) + ": " + g_create_error;
            return s;
        }
        b->h.push_back(h);
    }
    *out = b.release();
    return SIM_OK;
}

sim_status sim_batch_set_separable(sim_batch b, int32_t p, int32_t ndim, const int64_t* dims, const double* axes) {
    if (!b) return SIM_ERR_INVALID_ARG;
    if (p < 0 || p >= (int)b->h.size()) return bfail(b, SIM_ERR_INVALID_ARG, "pencil index out of range");
    const sim_status s = sim_set_separable(b->h[p], ndim, dims, axes);
    if (s != SIM_OK) b->err = "pencil " + std::to_string(p) + ": " + b->h[p]->err;
    b->region = false;
    return s;
}

sim_status sim_batch_set_regions(sim_batch b, const double* regions, const double* const* f, uint64_t seed) {
    if (!b) return SIM_ERR_INVALID_ARG;
    return bguarded(b, [&]() -> sim_status {
        if (!regions) return bfail(b, SIM_ERR_INVALID_ARG, "regions is NULL");
        const int P = (int)b->h.size();
        b->region = false;
        b->sb.assign(1, 0);
        b->re_lo.clear();
        b->im_lo.clear();
        b->s1.clear();
        for (int p = 0; p < P; ++p) {
            sim_ctx* h = b->h[p];
            const double* r = regions + 4 * p;
            const sim_status s = sim_set_region(h, r[0], r[1], r[2], r[3], f ? f[p] : nullptr, 0, seed + p);
            if (s != SIM_OK) return bfail(b, s, "pencil " + std::to_string(p) + ": " + h->err);
            if (p > 0 && h->K != b->h[0]->K)
                return bfail(b, SIM_ERR_INVALID_ARG, "the pencils' regions need the same number of levels");
            b->sb.push_back(b->sb.back() + h->S);
            b->re_lo.push_back(h->re_lo);
            b->im_lo.push_back(h->im_lo);
            b->s1.push_back(h->s1);
        }
        batch_build_table(b);
        int64_t N = 0;
        for (int p = 0; p < P; ++p) N += b->h[p]->nsq;
        int64_t* ix = b->arena.get<int64_t>("L0_ix", N);
        int64_t* iy = b->arena.get<int64_t>("L0_iy", N);
        int* sid = b->arena.get<int>("L0_sid", N);
        int64_t at = 0;
        for (int p = 0; p < P; ++p) {
            sim_ctx* h = b->h[p];
            const int o = b->sb[p];
            const int64_t n0 = h->nsq;
            SIM_CUDA(cudaMemcpyAsync(ix + at, h->arena.get<int64_t>("L0_ix", n0), sizeof(int64_t) * n0,
                                     cudaMemcpyDeviceToDevice, b->st));
            SIM_CUDA(cudaMemcpyAsync(iy + at, h->arena.get<int64_t>("L0_iy", n0), sizeof(int64_t) * n0,
                                     cudaMemcpyDeviceToDevice, b->st));
            k_add_offset<<<cdiv_up(n0, 256), 256, 0, b->st>>>(h->arena.get<int>("L0_sid", n0), sid + at, n0, o);
            SIM_LAUNCH_CHECK();
            at += n0;
        }
        SIM_CUDA(cudaMemcpyAsync(b->arena.get<double>("p_re_lo", P), b->re_lo.data(), sizeof(double) * P,
                                 cudaMemcpyHostToDevice, b->st));
        SIM_CUDA(cudaMemcpyAsync(b->arena.get<double>("p_im_lo", P), b->im_lo.data(), sizeof(double) * P,
                                 cudaMemcpyHostToDevice, b->st));
        SIM_CUDA(cudaStreamSynchronize(b->st));
        b->K = b->h[0]->K;
        b->level = 1;
        b->cur = 0;
        b->nsq = N;
        b->squares_evaluated = 0;
        b->region = true;
        return SIM_OK;
    });
}

sim_status sim_batch_solve_level(sim_batch b, int64_t* n_marked, int32_t* done) {
    if (!b) return SIM_ERR_INVALID_ARG;
    return bguarded(b, [&]() -> sim_status {
        if (!b->region || b->level > b->K) return bfail(b, SIM_ERR_BAD_STATE, "no level to solve");
        const int P = (int)b->h.size();
        const int k = b->level;
        const sim_ctx* h0 = b->h[0];
        std::vector<double> side(P);
        for (int p = 0; p < P; ++p) side[p] = b->s1[p] / std::ldexp(1.0, k - 1);
        double* d_side = b->arena.get<double>("p_side", P);
        SIM_CUDA(cudaMemcpyAsync(d_side, side.data(), sizeof(double) * P, cudaMemcpyHostToDevice, b->st));
        ShiftTable t;
        t.H = b->arena.get<double2>("H", 1);
        t.beta = b->arena.get<double>("beta", 1);
        t.meff = b->arena.get<int>("meff", 1);
        t.sigma = b->arena.get<double2>("sigma", 1);
        t.S = b->sb.back();
        t.m = h0->opt.m;
        t.scale = h0->opt.residual_scale;
        t.eps = h0->opt.eps;
        t.delta0 = h0->opt.delta0;
        t.pencil_of = b->arena.get<int>("pencil_of", 1);
        t.p_re_lo = b->arena.get<double>("p_re_lo", 1);
        t.p_im_lo = b->arena.get<double>("p_im_lo", 1);
        t.p_side = d_side;
        t.p_sb = b->arena.get<int>("p_sb", 1);
        t.p_se = b->arena.get<int>("p_se", 1);
        t.schT = b->arena.get<double2>("schT", 1);
        t.schC = b->arena.get<double2>("schC", 1);
        t.schQ = b->arena.get<double2>("schQ", 1);
        t.schOK = b->arena.get<int>("schOK", 1);
        const std::string a = "L" + std::to_string(b->cur) + "_", c = "L" + std::to_string(1 - b->cur) + "_";
        const int64_t N = b->nsq;
        int64_t* ix = b->arena.get<int64_t>(a + "ix", N);
        int64_t* iy = b->arena.get<int64_t>(a + "iy", N);
        int* sid = b->arena.get<int>(a + "sid", N);
        uint8_t* mark = b->arena.get<uint8_t>("mark", N);
        uint8_t* flag = b->arena.get<uint8_t>("flag", N);
        LevelArgs la;
        la.ix = ix;
        la.iy = iy;
        la.sid = sid;
        la.mark = mark;
        la.flag = flag;
        la.ind = b->arena.get<double>("ind", N);
        la.count = N;
        const int nbk = cdiv_up(std::max<int64_t>(N, 1), 1024);
        int64_t* bsum = b->arena.get<int64_t>("bsum", nbk + 1);
        int64_t* tot = b->arena.get<int64_t>("tot", 1);
        for (int round = 0;; ++round) {
            int smax = 0;
            for (int p = 0; p < P; ++p) smax = std::max(smax, b->sb[p + 1] - b->sb[p]);
            evaluate_level(t, la, h0->opt.level_solver, smax, b->arena, bsum, tot, b->st);
            b->squares_evaluated += N;
            if (!h0->opt.new_shifts_in_levels || round >= h0->opt.max_shift_rounds) break;
            const int64_t un = count_marked(flag, N, bsum, tot, b->arena.host_i64(), b->st);
            if (un == 0) break;
            // new Krylov spaces at the centres of each pencil's unresolved squares
            // (as for one pencil), the batch's table rebuilt, and the squares' shift
            // ids moved to the pencils' new offsets
            std::vector<uint8_t> hf(N);
            std::vector<int64_t> hx(N), hy(N);
            std::vector<int> hs(N);
            SIM_CUDA(cudaMemcpyAsync(hf.data(), flag, N, cudaMemcpyDeviceToHost, b->st));
            SIM_CUDA(cudaMemcpyAsync(hx.data(), ix, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, b->st));
            SIM_CUDA(cudaMemcpyAsync(hy.data(), iy, sizeof(int64_t) * N, cudaMemcpyDeviceToHost, b->st));
            SIM_CUDA(cudaMemcpyAsync(hs.data(), sid, sizeof(int) * N, cudaMemcpyDeviceToHost, b->st));
            SIM_CUDA(cudaStreamSynchronize(b->st));
            const std::vector<int> old_sb = b->sb;
            auto pencil_of = [&](int g) {
                return (int)(std::upper_bound(old_sb.begin(), old_sb.end(), g) - old_sb.begin()) - 1;
            };
            std::vector<std::vector<double2>> cen(P);
            for (int64_t q = 0; q < N; ++q) {
                if (!hf[q]) continue;
                const int p = pencil_of(hs[q]);
                const double2 c = center_of(b->h[p], side[p], hx[q], hy[q]);
                bool far = true;
                for (const double2& d : cen[p])
                    if (std::hypot(c.x - d.x, c.y - d.y) < h0->opt.shift_sep * side[p]) {
                        far = false;
                        break;
                    }
                if (far) cen[p].push_back(c);
            }
            bool ok = true;
            for (int p = 0; p < P; ++p)
                if (!cen[p].empty()) ok = build_shifts(b->h[p], cen[p]) && ok;
            if (!ok) return bfail(b, SIM_ERR_NOT_CONVERGED, "an inner shifted solve did not converge");
            batch_build_table(b);
            for (int64_t q = 0; q < N; ++q) {
                const int p = pencil_of(hs[q]);
                hs[q] = hs[q] - old_sb[p] + b->sb[p];
            }
            SIM_CUDA(cudaMemcpyAsync(sid, hs.data(), sizeof(int) * N, cudaMemcpyHostToDevice, b->st));
            t.H = b->arena.get<double2>("H", 1);
            t.beta = b->arena.get<double>("beta", 1);
            t.meff = b->arena.get<int>("meff", 1);
            t.sigma = b->arena.get<double2>("sigma", 1);
            t.pencil_of = b->arena.get<int>("pencil_of", 1);
            t.p_sb = b->arena.get<int>("p_sb", 1);
            t.p_se = b->arena.get<int>("p_se", 1);
            t.schT = b->arena.get<double2>("schT", 1);
            t.schC = b->arena.get<double2>("schC", 1);
            t.schQ = b->arena.get<double2>("schQ", 1);
            t.schOK = b->arena.get<int>("schOK", 1);
            t.S = b->sb.back();
        }
        const int64_t cnt = count_marked(mark, N, bsum, tot, b->arena.host_i64(), b->st);
        const bool last = k == b->K;
        if (!last) {
            if (4 * cnt > h0->opt.max_squares)
                return bfail(b, SIM_ERR_LIMIT, "level " + std::to_string(k + 1) + " would hold " +
                                                   std::to_string(4 * cnt) + " squares (> max_squares)");
            emit_marked(mark, flag, ix, iy, sid, N, bsum, 0, b->arena.get<int64_t>(c + "ix", 4 * cnt),
                        b->arena.get<int64_t>(c + "iy", 4 * cnt), b->arena.get<int>(c + "sid", 4 * cnt), nullptr,
                        b->st);
            b->cur = 1 - b->cur;
            b->nsq = 4 * cnt;
        } else {
            // the final squares, pencil by pencil (the list stays in pencil order),
            // go to each pencil's handle with its own shift ids
            int64_t* fix = b->arena.get<int64_t>("F_ix", cnt);
            int64_t* fiy = b->arena.get<int64_t>("F_iy", cnt);
            int* fsid = b->arena.get<int>("F_sid", cnt);
            uint8_t* ffl = b->arena.get<uint8_t>("F_flag", cnt);
            emit_marked(mark, flag, ix, iy, sid, N, bsum, 1, fix, fiy, fsid, ffl, b->st);
            std::vector<int> hs(cnt);
            if (cnt) SIM_CUDA(cudaMemcpyAsync(hs.data(), fsid, sizeof(int) * cnt, cudaMemcpyDeviceToHost, b->st));
            SIM_CUDA(cudaStreamSynchronize(b->st));
            int64_t at = 0;
            for (int p = 0; p < P; ++p) {
                sim_ctx* h = b->h[p];
                int64_t e = at;
                while (e < cnt && hs[e] < b->sb[p + 1]) ++e;
                const int64_t np = e - at;
                if (np) {
                    SIM_CUDA(cudaMemcpyAsync(h->arena.get<int64_t>("F_ix", np), fix + at, sizeof(int64_t) * np,
                                             cudaMemcpyDeviceToDevice, b->st));
                    SIM_CUDA(cudaMemcpyAsync(h->arena.get<int64_t>("F_iy", np), fiy + at, sizeof(int64_t) * np,
                                             cudaMemcpyDeviceToDevice, b->st));
                    SIM_CUDA(cudaMemcpyAsync(h->arena.get<uint8_t>("F_flag", np), ffl + at, np,
                                             cudaMemcpyDeviceToDevice, b->st));
                    k_add_offset<<<cdiv_up(np, 256), 256, 0, b->st>>>(fsid + at, h->arena.get<int>("F_sid", np), np,
                                                                      -b->sb[p]);
                    SIM_LAUNCH_CHECK();
                }
                h->nfinal = np;
                h->s_final = b->s1[p] / std::ldexp(1.0, k - 1);
                h->level = k + 1;
                h->stats.levels_done = k;
                h->state = ST_LEVELS_DONE;
                at = e;
            }
            SIM_CUDA(cudaStreamSynchronize(b->st));
            b->region = false;
        }
        b->level = k + 1;
        if (n_marked) *n_marked = cnt;
        if (done) *done = last ? 1 : 0;
        return SIM_OK;
    });
}

sim_status sim_batch_eigenvalues(sim_batch b, int32_t p, double* out, int64_t capacity, int64_t* count) {
    if (!b) return SIM_ERR_INVALID_ARG;
    if (p < 0 || p >= (int)b->h.size()) return bfail(b, SIM_ERR_INVALID_ARG, "pencil index out of range");
    const sim_status s = sim_eigenvalues(b->h[p], out, capacity, count);
    if (s != SIM_OK) b->err = b->h[p]->err;
    return s;
}

sim_status sim_batch_multiplicity(sim_batch b, int32_t p, int32_t* out, int64_t capacity, int64_t* count) {
    if (!b) return SIM_ERR_INVALID_ARG;
    if (p < 0 || p >= (int)b->h.size()) return bfail(b, SIM_ERR_INVALID_ARG, "pencil index out of range");
    const sim_status s = sim_multiplicity(b->h[p], out, capacity, count);
    if (s != SIM_OK) b->err = b->h[p]->err;
    return s;
}

sim_handle sim_batch_handle(sim_batch b, int32_t p) {
    if (!b || p < 0 || p >= (int)b->h.size()) return nullptr;
    return b->h[p];
}

const char* sim_batch_last_error(sim_batch b) { return b ? b->err.c_str() : g_create_error.c_str(); }

void sim_batch_destroy(sim_batch b) { delete b; }

sim_status sim_residual_screen(sim_handle h, int32_t s, const double* z, int64_t count, double* ym, double* rho) {
    if (!h) return fail(nullptr, SIM_ERR_INVALID_ARG, "NULL handle");
    return guarded(h, [&]() -> sim_status {
        if (h->state < ST_REGION || h->S < 1) return fail(h, SIM_ERR_BAD_STATE, "no Krylov spaces (call sim_set_region)");
        if (s < 0 || s >= h->S) return fail(h, SIM_ERR_INVALID_ARG, "shift index out of range");
        if (count < 0 || (count > 0 && (!z || !ym || !rho))) return fail(h, SIM_ERR_INVALID_ARG, "bad points");
        const int m = h->opt.m;
        RitzInput in;
        in.arena = &h->arena;
        in.st = h->st;
        in.m = m;
        in.num_slots = h->cap;
        in.d_H = h->d_H;
        in.d_meff = h->d_meff;
        in.d_sigma = h->d_sigma;
        in.d_beta = h->d_beta;
        EigDecomposition dec;
        if (!eig_decompose(in, {s}, dec))
            return fail(h, SIM_ERR_NOT_CONVERGED, "eigendecomposition of the Hessenberg matrix failed");
        int me = 0;
        double beta = 0.0;
        SIM_CUDA(cudaMemcpyAsync(&me, h->d_meff + s, sizeof(int), cudaMemcpyDeviceToHost, h->st));
        SIM_CUDA(cudaMemcpyAsync(&beta, h->d_beta + s, sizeof(double), cudaMemcpyDeviceToHost, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
        double2 hl;
        SIM_CUDA(cudaMemcpy(&hl, h->d_H + (size_t)s * (m + 1) * m + (size_t)(me - 1) * (m + 1) + me, sizeof(double2),
                            cudaMemcpyDeviceToHost));
        if (count == 0) return SIM_OK;
        double2* dz = h->arena.get<double2>("scr_z", count);
        double2* dy = h->arena.get<double2>("scr_y", count);
        double* dr = h->arena.get<double>("scr_r", count);
        SIM_CUDA(cudaMemcpyAsync(dz, z, sizeof(double2) * count, cudaMemcpyHostToDevice, h->st));
        screen_points(me, std::hypot(hl.x, hl.y), beta, h->h_sigma[s], dec.d, dec.w, dz, count, dy, dr, h->st);
        SIM_CUDA(cudaMemcpyAsync(ym, dy, sizeof(double2) * count, cudaMemcpyDeviceToHost, h->st));
        SIM_CUDA(cudaMemcpyAsync(rho, dr, sizeof(double) * count, cudaMemcpyDeviceToHost, h->st));
        SIM_CUDA(cudaStreamSynchronize(h->st));
        return SIM_OK;
    });
}

void sim_kernel_timing(int32_t enable) {
    kprof_reset();
    kprof_enable(enable != 0);
}

int32_t sim_kernel_stats(const char* name, double* ms, double* bytes, double* flops, int64_t* launches) {
    if (!name) return 0;
    return kprof_query(name, ms, bytes, flops, launches) ? 1 : 0;
}

int64_t sim_launch_count(void) { return launch_counter(); }

sim_status sim_random_vectors(uint64_t seed, int64_t n, int32_t k, int32_t first, double* out, void* stream) {
    return guarded(nullptr, [&]() -> sim_status {
        if (!out || n < 0 || k < 0 || first < 0) return fail(nullptr, SIM_ERR_INVALID_ARG, "bad argument");
        random_vectors(seed, n, k, first, (double2*)out, n, (cudaStream_t)stream);
        SIM_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
        return SIM_OK;
    });
}

}  // extern "C"
