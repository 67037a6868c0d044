// Level side of SIM-M on the GPU: the projected shifted solves at the
// quadrature nodes of every square of a level, the residual test of
// resolvability, the indicator and the marks (Sec. 3.1-3.3, Eqs. eq:many,
// eq:error, DeltaSm, Defs. 3.1-3.2), the subdivision of marked squares as a
// device-side compaction, and the merge of the final squares into clusters
// (Sec. 3.5 step 6).
//
// Direct projected solve (option level_solver 0, and the squares the Schur
// path of schur.cu cannot take): one warp per quadrature node.  T = I + (σ - z) H_m is upper
// Hessenberg, so Gaussian elimination with partial pivoting only ever compares
// the carried pivot row with the next original row; the warp keeps the carried
// row in registers (two columns per lane), writes the rows of U to shared
// memory and finishes with a column-oriented back substitution.  FP64
// throughout.  One CTA (8 warps) evaluates the 8 nodes of one square, so the
// indicator's two quadrature sums are reduced inside the CTA.
#include <cmath>

#include "internal.h"
#include "levels.h"
#include "hess.cuh"

namespace sim {

// Evaluate one square (centre c, side s) against one shift, by the whole CTA
// (8 warps, one per node).  Returns indicator and max residual (CTA-uniform).
struct EvalSmem {
    double2* Hs;   // m*m
    double2* U;    // 8 * m(m+1)/2
    double2* Y;    // 8 * m
    double* rho;   // 8
    double* red;   // 2 * 8
};

__device__ void eval_square(const double2* H, int m, int meff, double beta, double2 sigma, double2 c, double s,
                            int scale, const EvalSmem& sm, double& ind, double& rho_max) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    stage_H(H, m, meff, sm.Hs);
    __syncthreads();
    const double hlast = cabsd(H[(size_t)(meff - 1) * (m + 1) + meff]);
    const int Usz = meff * (meff + 1) / 2;
    {
        const int j = warp;  // node
        const double2 off = node_offset(j, s);
        const double2 z = make_double2(__dadd_rn(c.x, off.x), __dadd_rn(c.y, off.y));
        const double2 alpha = make_double2(__dsub_rn(sigma.x, z.x), __dsub_rn(sigma.y, z.y));
        double ylast, yn2;
        warp_hess_solve(sm.Hs, meff, alpha, beta, sm.U + (size_t)j * Usz, sm.Y + (size_t)j * meff, ylast, yn2);
        if (lane == 0) {
            const double num = cabsd(alpha) * hlast * ylast;
            const double den = scale == 0 ? sqrt(yn2) : beta;
            double r = num / den;
            if (!(r == r) || isinf(r)) r = INFINITY;
            if (num == 0.0) r = 0.0;
            sm.rho[j] = r;
        }
    }
    __syncthreads();
    // quadrature sums Y8 = Σ_j (off_j/8) y_j, Y4 = Σ_{j even} (off_j/4) y_j
    double n8 = 0.0, n4 = 0.0;
    for (int q = threadIdx.x; q < meff; q += blockDim.x) {
        double2 y8 = make_double2(0.0, 0.0), y4 = make_double2(0.0, 0.0);
        for (int j = 0; j < 8; ++j) {
            const double2 off = node_offset(j, s);
            const double2 yj = sm.Y[(size_t)j * meff + q];
            y8 = cadd(y8, cmul(cscale(off, 0.125), yj));
            if ((j & 1) == 0) y4 = cadd(y4, cmul(cscale(off, 0.25), yj));
        }
        n8 += cabs2(y8);
        n4 += cabs2(y4);
    }
    n8 = warp_sum(n8);
    n4 = warp_sum(n4);
    if (lane == 0) {
        sm.red[warp] = n8;
        sm.red[8 + warp] = n4;
    }
    __syncthreads();
    double s8 = 0.0, s4 = 0.0, rm = 0.0;
    for (int w = 0; w < 8; ++w) {
        s8 += sm.red[w];
        s4 += sm.red[8 + w];
        rm = fmax(rm, sm.rho[w]);
        if (sm.rho[w] != sm.rho[w]) rm = INFINITY;
    }
    s8 = sqrt(s8);
    s4 = sqrt(s4);
    ind = s4 > 0.0 ? s8 / s4 : (s8 > 0.0 ? INFINITY : 0.0);
    rho_max = rm;
    __syncthreads();
}

size_t eval_smem_bytes(int m) {
    const size_t usz = (size_t)m * (m + 1) / 2;
    return ((size_t)m * m + 8 * usz + 8 * (size_t)m) * sizeof(double2) + 8 * sizeof(double) + 16 * sizeof(double) + 64;
}

__device__ __forceinline__ EvalSmem carve(unsigned char* raw, int m) {
    EvalSmem sm;
    const size_t usz = (size_t)m * (m + 1) / 2;
    sm.Hs = reinterpret_cast<double2*>(raw);
    sm.U = sm.Hs + (size_t)m * m;
    sm.Y = sm.U + 8 * usz;
    sm.rho = reinterpret_cast<double*>(sm.Y + 8 * (size_t)m);
    sm.red = sm.rho + 8;
    return sm;
}

// choose the nearest untried shift in [lo, hi) to c (ties: lower id); -1 if none.
__device__ int next_shift(const ShiftTable& st, double2 c, const uint32_t* tried, double* sred, int* sidx, int lo,
                          int hi) {
    double best = INFINITY;
    int bi = -1;
    for (int s = lo + threadIdx.x; s < hi; s += blockDim.x) {
        if (tried[(s - lo) >> 5] & (1u << ((s - lo) & 31))) continue;
        double d = hypot(st.sigma[s].x - c.x, st.sigma[s].y - c.y);
        if (d < best || (d == best && s < bi)) { best = d; bi = s; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi >= 0 && (bi < 0 || ob < best || (ob == best && oi < bi))) { best = ob; bi = oi; }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sred[warp] = best; sidx[warp] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = sred[0];
        int i0 = sidx[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            int oi = sidx[w];
            if (oi >= 0 && (i0 < 0 || sred[w] < b || (sred[w] == b && oi < i0))) { b = sred[w]; i0 = oi; }
        }
        sidx[0] = i0;
    }
    __syncthreads();
    const int r = sidx[0];
    __syncthreads();
    return r;
}

// mode 0 (level): own shift first, then the others nearest-first; writes mark,
//   flag, indicator and the (possibly new) shift id.
// mode 1 (association): only squares with todo[q] != 0; every shift
//   nearest-first; writes resolved (flag = 0) / unresolved (flag = 1) and sid.
__global__ void __launch_bounds__(256) k_eval_level(ShiftTable st, LevelArgs a, int mode) {
    extern __shared__ unsigned char raw[];
    const EvalSmem sm = carve(raw, st.m);
    __shared__ uint32_t tried[SIM_MAX_SHIFTS / 32];
    __shared__ double sred[8];
    __shared__ int sidx[8];
    for (int64_t q = blockIdx.x; q < a.count; q += gridDim.x) {
        if (a.todo && !a.todo[q]) continue;
        // one pencil: the level's origin and side; a batch: those of the
        // pencil that owns the square's shift, and only its shifts
        double re_lo = a.re_lo, im_lo = a.im_lo, side = a.side;
        int lo = 0, hi = st.S;
        if (st.pencil_of && mode == 0) {
            const int p = st.pencil_of[a.sid[q]];
            re_lo = st.p_re_lo[p];
            im_lo = st.p_im_lo[p];
            side = st.p_side[p];
            lo = st.p_sb[p];
            hi = st.p_se[p];
        }
        const double2 c = square_center(re_lo, im_lo, side, a.ix[q], a.iy[q]);
        for (int w = threadIdx.x; w < SIM_MAX_SHIFTS / 32; w += blockDim.x) tried[w] = 0u;
        __syncthreads();
        int s = (mode == 0) ? a.sid[q] : next_shift(st, c, tried, sred, sidx, lo, hi);
        double ind0 = 0.0, ind = 0.0;
        bool res = false;
        int first = s;
        int used = s;
        for (int attempt = 0; s >= 0 && attempt < hi - lo; ++attempt) {
            double ii, rr;
            eval_square(st.H + (size_t)s * (st.m + 1) * st.m, st.m, st.meff[s], st.beta[s], st.sigma[s], c, side,
                        st.scale, sm, ii, rr);
            if (attempt == 0) ind0 = ii;
            if (threadIdx.x == 0) tried[(s - lo) >> 5] |= 1u << ((s - lo) & 31);
            __syncthreads();
            if (rr <= st.eps) {
                res = true;
                ind = ii;
                used = s;
                break;
            }
            s = next_shift(st, c, tried, sred, sidx, lo, hi);
        }
        if (threadIdx.x == 0) {
            if (a.retries) {
                unsigned int tried_n = 0;
                for (int w = 0; w < SIM_MAX_SHIFTS / 32; ++w) tried_n += __popc(tried[w]);
                if (tried_n > 1) atomicAdd(a.retries, (unsigned long long)(tried_n - 1));
            }
            if (!res) {
                ind = ind0;
                used = first;
            }
            if (mode == 0) {
                a.ind[q] = ind;
                a.mark[q] = res ? (ind > st.delta0 ? 1 : 0) : 1;
                a.flag[q] = res ? 0 : 1;
                a.sid[q] = used;
            } else {
                a.flag[q] = res ? 0 : 1;
                if (res) a.sid[q] = used;
            }
        }
        __syncthreads();
    }
}

void eval_level(const ShiftTable& st, const LevelArgs& a, int mode, cudaStream_t stream) {
    if (a.count <= 0) return;
    const size_t sm = eval_smem_bytes(st.m);
    SIM_CUDA(cudaFuncSetAttribute(k_eval_level, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int grid = (int)std::min<int64_t>(a.count, 152 * 64);
    kprof_begin("eval_level", stream);
    k_eval_level<<<grid, 256, sm, stream>>>(st, a, mode);
    SIM_LAUNCH_CHECK();
    kprof_end("eval_level", stream, 0.0, a.count * 8.0 * 8.0 * st.m * st.m);
}

// explicit squares against one explicit Krylov space (component entry point)
__global__ void __launch_bounds__(256) k_eval_explicit(const double2* H, int m, int meff, double beta, double2 sigma,
                                                       const double2* centers, const double* sides, int64_t count,
                                                       int scale, double* ind, double* rho) {
    extern __shared__ unsigned char raw[];
    const EvalSmem sm = carve(raw, m);
    for (int64_t q = blockIdx.x; q < count; q += gridDim.x) {
        double ii, rr;
        eval_square(H, m, meff, beta, sigma, centers[q], sides[q], scale, sm, ii, rr);
        if (threadIdx.x == 0) {
            ind[q] = ii;
            rho[q] = rr;
        }
    }
}

void eval_explicit(const double2* H, int m, int meff, double beta, double2 sigma, const double2* centers,
                   const double* sides, int64_t count, int scale, double* ind, double* rho, cudaStream_t stream) {
    if (count <= 0) return;
    const size_t sm = eval_smem_bytes(m);
    SIM_CUDA(cudaFuncSetAttribute(k_eval_explicit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int grid = (int)std::min<int64_t>(count, 152 * 64);
    k_eval_explicit<<<grid, 256, sm, stream>>>(H, m, meff, beta, sigma, centers, sides, count, scale, ind, rho);
    SIM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// subdivision: stable compaction of marked squares into children (SW, SE, NW,
// NE) or, at the last level, into the final list
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024;

__device__ __forceinline__ int block_excl_scan(int v, int* wsum, int& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    total = wsum[nw - 1];
    int excl = x - v + (warp > 0 ? wsum[warp - 1] : 0);
    __syncthreads();
    return excl;
}

__global__ void k_count_marks(const uint8_t* mark, int64_t count, int64_t* bsum) {
    __shared__ int wsum[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    int v = (i < count && mark[i]) ? 1 : 0;
    int total;
    block_excl_scan(v, wsum, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_bsums(int64_t* bsum, int nblocks, int64_t* total_out) {
    // single CTA, sequential over chunks of blockDim
    __shared__ int64_t carry;
    __shared__ int64_t tmp[SCAN_T];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += blockDim.x) {
        int i = base + threadIdx.x;
        int64_t v = i < nblocks ? bsum[i] : 0;
        tmp[threadIdx.x] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t run = carry;
            int lim = min((int)blockDim.x, nblocks - base);
            for (int t = 0; t < lim; ++t) {
                int64_t x = tmp[t];
                tmp[t] = run;
                run += x;
            }
            carry = run;
        }
        __syncthreads();
        if (i < nblocks) bsum[i] = tmp[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_emit(const uint8_t* mark, const uint8_t* flag, const int64_t* ix, const int64_t* iy, const int* sid,
                       int64_t count, const int64_t* boff, int final_level, int64_t* oix, int64_t* oiy, int* osid,
                       uint8_t* oflag) {
    __shared__ int wsum[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    int v = (i < count && mark[i]) ? 1 : 0;
    int total;
    int ex = block_excl_scan(v, wsum, total);
    if (!v) return;
    const int64_t pos = boff[blockIdx.x] + ex;
    if (final_level) {
        oix[pos] = ix[i];
        oiy[pos] = iy[i];
        osid[pos] = sid[i];
        oflag[pos] = flag[i];
    } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            oix[4 * pos + c] = 2 * ix[i] + (c & 1);
            oiy[4 * pos + c] = 2 * iy[i] + (c >> 1);
            osid[4 * pos + c] = sid[i];
        }
    }
}

int64_t count_marked(const uint8_t* mark, int64_t count, int64_t* d_bsum, int64_t* d_total, int64_t* h_total,
                     cudaStream_t st) {
    if (count <= 0) return 0;
    const int nb = cdiv_up(count, SCAN_T);
    k_count_marks<<<nb, SCAN_T, 0, st>>>(mark, count, d_bsum);
    SIM_LAUNCH_CHECK();
    k_scan_bsums<<<1, SCAN_T, 0, st>>>(d_bsum, nb, d_total);
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaMemcpyAsync(h_total, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaStreamSynchronize(st));
    return *h_total;
}

void emit_marked(const uint8_t* mark, const uint8_t* flag, const int64_t* ix, const int64_t* iy, const int* sid,
                 int64_t count, const int64_t* d_bsum, int final_level, int64_t* oix, int64_t* oiy, int* osid,
                 uint8_t* oflag, cudaStream_t st) {
    if (count <= 0) return;
    const int nb = cdiv_up(count, SCAN_T);
    k_emit<<<nb, SCAN_T, 0, st>>>(mark, flag, ix, iy, sid, count, d_bsum, final_level, oix, oiy, osid, oflag);
    SIM_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// merge: 8-connected components of the final squares (union–find with a hash
// of lattice coordinates), cluster statistics in member order, optional join
// of clusters closer than merge_radius, filter to R and sort by (Re, Im)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t hmix(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__global__ void k_hash_insert(const int64_t* ix, const int64_t* iy, int64_t N, int64_t ny, unsigned long long* keys,
                              int* vals, int64_t cap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned long long key = (unsigned long long)(ix[i] * ny + iy[i]) + 1ull;
    uint64_t h = hmix(key) & (uint64_t)(cap - 1);
    for (int64_t probe = 0; probe < cap; ++probe) {
        unsigned long long prev = atomicCAS(&keys[h], 0ull, key);
        if (prev == 0ull || prev == key) {
            vals[h] = (int)i;
            return;
        }
        h = (h + 1) & (uint64_t)(cap - 1);
    }
}

__device__ int hash_find(const unsigned long long* keys, const int* vals, int64_t cap, unsigned long long key) {
    uint64_t h = hmix(key) & (uint64_t)(cap - 1);
    for (int64_t probe = 0; probe < cap; ++probe) {
        unsigned long long k = keys[h];
        if (k == key) return vals[h];
        if (k == 0ull) return -1;
        h = (h + 1) & (uint64_t)(cap - 1);
    }
    return -1;
}

__device__ int uf_find(int* parent, int a) {
    int p = parent[a];
    while (p != a) {
        int gp = parent[p];
        if (gp != p) parent[a] = gp;  // path halving (benign race)
        a = p;
        p = parent[a];
    }
    return a;
}

__device__ void uf_union(int* parent, int a, int b) {
    for (int iter = 0; iter < 1 << 20; ++iter) {
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        if (a < b) { int t = a; a = b; b = t; }  // link the larger root below the smaller
        if (atomicCAS(&parent[a], a, b) == a) return;
    }
}

__global__ void k_uf_init(int* parent, int64_t N) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) parent[i] = (int)i;
}

__global__ void k_uf_neighbours(const int64_t* ix, const int64_t* iy, int64_t N, int64_t nx, int64_t ny,
                                const unsigned long long* keys, const int* vals, int64_t cap, int* parent) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy) {
            if (dx == 0 && dy == 0) continue;
            const int64_t x = ix[i] + dx, y = iy[i] + dy;
            if (x < 0 || y < 0 || x >= nx || y >= ny) continue;
            const int j = hash_find(keys, vals, cap, (unsigned long long)(x * ny + y) + 1ull);
            if (j >= 0) uf_union(parent, (int)i, j);
        }
}

__global__ void k_uf_flatten(int* parent, int64_t N) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) parent[i] = uf_find(parent, (int)i);
}

// root flags -> dense cluster ids in root (= first member) order
__global__ void k_root_flags(const int* parent, int64_t N, uint8_t* isroot) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) isroot[i] = parent[i] == (int)i;
}

__global__ void k_root_ids(const uint8_t* isroot, int64_t N, const int64_t* boff, int* cid_of_root) {
    __shared__ int wsum[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_T + threadIdx.x;
    int v = (i < N && isroot[i]) ? 1 : 0;
    int total;
    int ex = block_excl_scan(v, wsum, total);
    if (i < N) cid_of_root[i] = v ? (int)(boff[blockIdx.x] + ex) : -1;
}

__global__ void k_labels(const int* parent, const int* cid_of_root, int64_t N, int* label) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) label[i] = cid_of_root[parent[i]];
}

// one warp per cluster: sums of member centres in member (index) order,
// member count, flagged count, first member; then the radius.
__global__ void k_cluster_stats(const int* label, const int64_t* ix, const int64_t* iy, const uint8_t* flag,
                                const int* sid, int64_t N, int C, double re_lo, double im_lo, double s, double2* est,
                                int* size, int* nflag, int* shift, double* radius) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= C) return;
    double sx = 0.0, sy = 0.0;
    int cnt = 0, nf = 0, firstm = -1;
    for (int64_t b = 0; b < N; b += 32) {
        const int64_t i = b + lane;
        const bool mem = i < N && label[i] == warp;
        const unsigned bal = __ballot_sync(0xffffffffu, mem);
        double2 cc = mem ? square_center(re_lo, im_lo, s, ix[i], iy[i]) : make_double2(0.0, 0.0);
        int fl = mem ? (int)flag[i] : 0;
        unsigned bb = bal;
        while (bb) {
            const int src = __ffs(bb) - 1;
            bb &= bb - 1;
            const double x = __shfl_sync(0xffffffffu, cc.x, src);
            const double y = __shfl_sync(0xffffffffu, cc.y, src);
            const int f = __shfl_sync(0xffffffffu, fl, src);
            sx = __dadd_rn(sx, x);
            sy = __dadd_rn(sy, y);
            nf += f;
            if (cnt == 0) firstm = (int)(b + src);
            cnt += 1;
        }
    }
    const double2 e = make_double2(sx / cnt, sy / cnt);
    double rad = 0.0;
    for (int64_t b = 0; b < N; b += 32) {
        const int64_t i = b + lane;
        if (i < N && label[i] == warp) {
            double2 cc = square_center(re_lo, im_lo, s, ix[i], iy[i]);
            rad = fmax(rad, hypot(cc.x - e.x, cc.y - e.y) + s * SQRT1_2);
        }
    }
    for (int o = 16; o > 0; o >>= 1) rad = fmax(rad, __shfl_xor_sync(0xffffffffu, rad, o));
    if (lane == 0) {
        est[warp] = e;
        size[warp] = cnt;
        nflag[warp] = nf;
        shift[warp] = sid[firstm];
        radius[warp] = rad;
    }
}

// join clusters whose estimates are closer than r: union over cluster ids,
// expressed on the member squares' union–find (roots are first members)
__global__ void k_join_close(const double2* est, const int* root_of_cluster, int C, double r, int* parent) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= C) return;
    for (int b = a + 1; b < C; ++b) {
        if (hypot(est[a].x - est[b].x, est[a].y - est[b].y) < r) uf_union(parent, root_of_cluster[a], root_of_cluster[b]);
    }
}

__global__ void k_root_of_cluster(const int* cid_of_root, int64_t N, int* root_of_cluster) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && cid_of_root[i] >= 0) root_of_cluster[cid_of_root[i]] = (int)i;
}

// keep clusters in the closed region; rank by (Re, Im, id); scatter
__global__ void k_select_sort(const double2* est, int C, double re_lo, double re_hi, double im_lo, double im_hi,
                              int* out_rank, int* n_inside) {
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= C) return;
    auto inside = [&](int q) {
        return est[q].x >= re_lo && est[q].x <= re_hi && est[q].y >= im_lo && est[q].y <= im_hi;
    };
    if (!inside(a)) {
        out_rank[a] = -1;
        return;
    }
    int rank = 0;
    for (int b = 0; b < C; ++b) {
        if (b == a || !inside(b)) continue;
        bool less = est[b].x < est[a].x || (est[b].x == est[a].x && (est[b].y < est[a].y || (est[b].y == est[a].y && b < a)));
        rank += less;
    }
    out_rank[a] = rank;
    atomicAdd(n_inside, 1);
}

// ---- host driver of the merge ----------------------------------------------
MergeResult merge_final(const int64_t* d_ix, const int64_t* d_iy, const int* d_sid, const uint8_t* d_flag, int64_t N,
                        int64_t nx, int64_t ny, double re_lo, double re_hi, double im_lo, double im_hi, double s,
                        double merge_radius, DeviceArena& arena, cudaStream_t st) {
    MergeResult R;
    if (N <= 0) return R;
    int64_t cap = 1;
    while (cap < 2 * N) cap <<= 1;
    auto* keys = arena.get<unsigned long long>("m_keys", cap);
    auto* vals = arena.get<int>("m_vals", cap);
    auto* parent = arena.get<int>("m_parent", N);
    auto* isroot = arena.get<uint8_t>("m_isroot", N);
    auto* cidr = arena.get<int>("m_cidr", N);
    auto* label = arena.get<int>("m_label", N);
    const int nb = cdiv_up(N, SCAN_T);
    auto* bsum = arena.get<int64_t>("m_bsum", nb + 1);
    auto* total = arena.get<int64_t>("m_total", 1);
    int64_t* h_total = arena.host_i64();
    SIM_CUDA(cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * cap, st));
    const int g = cdiv_up(N, 256);
    k_hash_insert<<<g, 256, 0, st>>>(d_ix, d_iy, N, ny, keys, vals, cap);
    SIM_LAUNCH_CHECK();
    k_uf_init<<<g, 256, 0, st>>>(parent, N);
    SIM_LAUNCH_CHECK();
    k_uf_neighbours<<<g, 256, 0, st>>>(d_ix, d_iy, N, nx, ny, keys, vals, cap, parent);
    SIM_LAUNCH_CHECK();
    k_uf_flatten<<<g, 256, 0, st>>>(parent, N);
    SIM_LAUNCH_CHECK();
    for (int pass = 0; pass < 2; ++pass) {
        k_root_flags<<<g, 256, 0, st>>>(parent, N, isroot);
        SIM_LAUNCH_CHECK();
        const int64_t C = count_marked(isroot, N, bsum, total, h_total, st);
        k_root_ids<<<nb, SCAN_T, 0, st>>>(isroot, N, bsum, cidr);
        SIM_LAUNCH_CHECK();
        k_labels<<<g, 256, 0, st>>>(parent, cidr, N, label);
        SIM_LAUNCH_CHECK();
        R.C = (int)C;
        R.est = arena.get<double2>("m_est", C);
        R.size = arena.get<int>("m_size", C);
        R.nflag = arena.get<int>("m_nflag", C);
        R.shift = arena.get<int>("m_shift", C);
        R.radius = arena.get<double>("m_radius", C);
        k_cluster_stats<<<cdiv_up(C * 32, 256), 256, 0, st>>>(label, d_ix, d_iy, d_flag, d_sid, N, (int)C, re_lo, im_lo,
                                                             s, R.est, R.size, R.nflag, R.shift, R.radius);
        SIM_LAUNCH_CHECK();
        if (pass == 1 || !(merge_radius > 0.0) || C < 2) break;
        auto* roc = arena.get<int>("m_roc", C);
        k_root_of_cluster<<<g, 256, 0, st>>>(cidr, N, roc);
        SIM_LAUNCH_CHECK();
        k_join_close<<<cdiv_up(C, 128), 128, 0, st>>>(R.est, roc, (int)C, merge_radius, parent);
        SIM_LAUNCH_CHECK();
        k_uf_flatten<<<g, 256, 0, st>>>(parent, N);
        SIM_LAUNCH_CHECK();
    }
    R.rank = arena.get<int>("m_rank", R.C);
    auto* nin = arena.get<int>("m_nin", 1);
    SIM_CUDA(cudaMemsetAsync(nin, 0, sizeof(int), st));
    k_select_sort<<<cdiv_up(R.C, 128), 128, 0, st>>>(R.est, R.C, re_lo, re_hi, im_lo, im_hi, R.rank, nin);
    SIM_LAUNCH_CHECK();
    int h_nin = 0;
    SIM_CUDA(cudaMemcpyAsync(&h_nin, nin, sizeof(int), cudaMemcpyDeviceToHost, st));
    SIM_CUDA(cudaStreamSynchronize(st));
    R.inside = h_nin;
    return R;
}

}  // namespace sim
