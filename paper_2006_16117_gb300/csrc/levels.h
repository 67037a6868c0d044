// Level-side declarations (projected solves, marks, compaction, merge) and a
// small named device-memory arena used by the host drivers.
#pragma once

#include <map>
#include <string>

#include "internal.h"

namespace sim {

constexpr int SIM_MAX_SHIFTS = 1024;

struct ShiftTable {
    const double2* H = nullptr;     // [S][(m+1)*m] column-major
    const double* beta = nullptr;   // [S]
    const int* meff = nullptr;      // [S]
    const double2* sigma = nullptr; // [S]
    int S = 0;
    int m = 50;
    int scale = 0;                  // 0: residual / ||y||, 1: residual / beta
    double eps = 1e-8;
    double delta0 = 0.05;
    // batches of pencils (sim_batch_*): shift s belongs to pencil pencil_of[s],
    // whose squares have their own origin and side (this level) and may only
    // use that pencil's shifts [p_sb[p], p_se[p]).  nullptr for one pencil.
    const int* pencil_of = nullptr;
    const double* p_re_lo = nullptr;
    const double* p_im_lo = nullptr;
    const double* p_side = nullptr;
    const int* p_sb = nullptr;
    const int* p_se = nullptr;
    // complex Schur form H_m = Z T Z^H of each shift (schur.cu): T [S][m][m]
    // row-major upper triangle, c = β Z^H e_1 [S][m], last row of Z [S][m],
    // and whether the QR iteration converged [S].  nullptr: not available.
    const double2* schT = nullptr;
    const double2* schC = nullptr;
    const double2* schQ = nullptr;
    const int* schOK = nullptr;
};

struct LevelArgs {
    const int64_t* ix = nullptr;
    const int64_t* iy = nullptr;
    int* sid = nullptr;
    const uint8_t* todo = nullptr;  // squares to evaluate (all if nullptr in level mode)
    uint8_t* mark = nullptr;
    uint8_t* flag = nullptr;
    double* ind = nullptr;
    unsigned long long* retries = nullptr;  // optional: += evaluations beyond the first shift
    int64_t count = 0;
    double re_lo = 0, im_lo = 0, side = 1;
};

// Named, grow-only device buffers.
class DeviceArena {
public:
    template <class T> T* get(const std::string& name, int64_t count) {
        size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
        auto it = bufs_.find(name);
        if (it != bufs_.end() && it->second.bytes >= bytes) return reinterpret_cast<T*>(it->second.ptr);
        if (it != bufs_.end()) {
            cudaFree(it->second.ptr);
            bufs_.erase(it);
        }
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) throw CudaError{e, "cudaMalloc(" + name + ", " + std::to_string(bytes) + " bytes)"};
        bufs_[name] = Buf{p, bytes};
        total_ += bytes;
        return reinterpret_cast<T*>(p);
    }
    int64_t* host_i64() {
        if (!h64_) SIM_CUDA(cudaMallocHost(&h64_, sizeof(int64_t) * 8));
        return h64_;
    }
    void release(const std::string& name) {
        auto it = bufs_.find(name);
        if (it != bufs_.end()) {
            cudaFree(it->second.ptr);
            bufs_.erase(it);
        }
    }
    ~DeviceArena() {
        for (auto& kv : bufs_) cudaFree(kv.second.ptr);
        if (h64_) cudaFreeHost(h64_);
    }
    size_t total() const { return total_; }

private:
    struct Buf {
        void* ptr;
        size_t bytes;
    };
    std::map<std::string, Buf> bufs_;
    int64_t* h64_ = nullptr;
    size_t total_ = 0;
};

struct MergeResult {
    int C = 0;          // clusters before the region filter
    int inside = 0;     // clusters inside R
    double2* est = nullptr;
    int* size = nullptr;
    int* nflag = nullptr;
    int* shift = nullptr;
    double* radius = nullptr;
    int* rank = nullptr;  // output position, -1 if outside R
};

// Schur forms of shifts s0 .. s0+count-1 (one warp each).
void schur_shifts(const double2* H, int m, const int* meff, const double* beta, int s0, int count, double2* T,
                  double2* C, double2* Q, int* ok, cudaStream_t st);
// Mode-0 evaluation of every square against its own shift through the Schur
// forms; todo[q] = 1 for the squares left to eval_level (unresolved by their
// own shift, or a zero pivot / no Schur form), 0 for those written.
void eval_level_schur(const ShiftTable& st, const LevelArgs& a, uint8_t* todo, cudaStream_t stream);
// The ntodo squares it left: every shift of their pencil (at most smax) through
// the Schur forms at once, then the shift the direct evaluation's order would
// pick; todo[q] stays 1 only where a zero pivot or a missing Schur form needs
// the direct evaluation.
void eval_level_schur_retries(const ShiftTable& st, const LevelArgs& a, uint8_t* todo, int64_t ntodo, int smax,
                              DeviceArena& ar, cudaStream_t stream);

size_t eval_smem_bytes(int m);
void eval_level(const ShiftTable& st, const LevelArgs& a, int mode, cudaStream_t stream);
void eval_explicit(const double2* H, int m, int meff, double beta, double2 sigma, const double2* centers,
                   const double* sides, int64_t count, int scale, double* ind, double* rho, cudaStream_t stream);
int64_t count_marked(const uint8_t* mark, int64_t count, int64_t* d_bsum, int64_t* d_total, int64_t* h_total,
                     cudaStream_t st);
void emit_marked(const uint8_t* mark, const uint8_t* flag, const int64_t* ix, const int64_t* iy, const int* sid,
                 int64_t count, const int64_t* d_bsum, int final_level, int64_t* oix, int64_t* oiy, int* osid,
                 uint8_t* oflag, cudaStream_t st);
MergeResult merge_final(const int64_t* d_ix, const int64_t* d_iy, const int* d_sid, const uint8_t* d_flag, int64_t N,
                        int64_t nx, int64_t ny, double re_lo, double re_hi, double im_lo, double im_hi, double s,
                        double merge_radius, DeviceArena& arena, cudaStream_t st);

}  // namespace sim
