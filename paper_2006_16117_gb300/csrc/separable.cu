// Fast-diagonalisation preconditioner (see separable.h for the formulas).
//
// One apply, for every active job at once:
//   1. w = D^{-1} q            (⊗ρ_d^{-j} scaling; complex64 in mixed mode)
//   2. w = (⊗Q_d) w            (one dense mode product per axis)
//   3. w = w / (Σ_d λ_{d,k_d} - σ b)   (denominators in FP64; the quotient in
//      FP32 in mixed mode, from per-element tables of Σ_d λ and of the scales)
//   4. w = (⊗Q_d) w
//   5. z = D w                 (to complex128)
// A mode product along axis d is a GEMM over the rows r = (p, q) of the
// vector viewed as [q][j][p] with p < P = Π_{e<d} N_e and j < N_d:
//   out(p, k, q) = Σ_j Q_d[k][j] in(p, j, q)      (Q_d symmetric).
// Tiles of 64 or 128 rows × as many outputs (autotuned), 16 reduction steps
// per stage, each thread 4 × 4 or 8 × 8 outputs; loads and stores are
// coalesced along rows for axes d > 0 (consecutive p) and along j / k for
// axis 0 (contiguous fibres).
#include <algorithm>
#include <cmath>
#include <vector>

#include "autotune.h"
#include "levels.h"
#include "separable.h"

namespace sim {

namespace {

// Q (both precisions), ρ^j, ρ^{-j} and λ_k of one axis.
__global__ void k_sep_tables(int N, double2 sub, double2 dg, double2 sup, double* Q64, float* Q32, double2* rho,
                             double2* irho, double2* lam) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t NN = (int64_t)N * N;
    if (t < NN) {
        const int64_t j = t / N, k = t % N;
        // sin((j+1)(k+1)π/(N+1)) with the integer argument reduced exactly mod 2(N+1)
        const int64_t a = ((j + 1) * (k + 1)) % (2 * (int64_t)(N + 1));
        const double v = sqrt(2.0 / (N + 1)) * sinpi((double)a / (double)(N + 1));
        Q64[t] = v;
        Q32[t] = (float)v;
    }
    if (t < N) {
        // ρ = sqrt(sub / sup) (principal branch); ρ^j = |r|^{j/2} e^{i j arg(r)/2}
        const double2 r = cdiv(sub, sup);
        const double lr = log(hypot(r.x, r.y)), ar = atan2(r.y, r.x);
        const double j = (double)t;
        const double mag = exp(0.5 * j * lr), ang = 0.5 * j * ar;
        rho[t] = make_double2(mag * cos(ang), mag * sin(ang));
        irho[t] = make_double2(cos(ang) / mag, -sin(ang) / mag);
        const double m1 = exp(0.5 * lr), a1 = 0.5 * ar;
        const double2 rho1 = make_double2(m1 * cos(a1), m1 * sin(a1));
        const double2 g = cmul(sup, rho1);  // sup·ρ = sqrt(sub·sup)
        const double c = 2.0 * cospi((double)(t + 1) / (double)(N + 1));
        lam[t] = make_double2(dg.x + c * g.x, dg.y + c * g.y);
    }
}

struct Axes {
    int ndim;
    int64_t N0, N1, N2;
    const double2 *t0, *t1, *t2;  // per-axis tables (ρ^j, ρ^{-j} or λ)
};

__device__ __forceinline__ double2 axes_product(const Axes& a, int64_t idx) {
    const int64_t i0 = idx % a.N0;
    double2 v = a.t0[i0];
    if (a.ndim > 1) {
        const int64_t i1 = (idx / a.N0) % a.N1;
        v = cmul(v, a.t1[i1]);
        if (a.ndim > 2) v = cmul(v, a.t2[idx / (a.N0 * a.N1)]);
    }
    return v;
}

__device__ __forceinline__ double2 axes_sum(const Axes& a, int64_t idx) {
    const int64_t i0 = idx % a.N0;
    double2 v = a.t0[i0];
    if (a.ndim > 1) {
        const int64_t i1 = (idx / a.N0) % a.N1;
        v = cadd(v, a.t1[i1]);
        if (a.ndim > 2) v = cadd(v, a.t2[idx / (a.N0 * a.N1)]);
    }
    return v;
}

// per-element tables of the complex64 path, formed in FP64 once
__global__ void k_sep_elem_tables(int64_t n, Axes irho, Axes rho, Axes lam, float2* sin32, float2* sout32,
                                  double2* lsum) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    sin32[g] = from_c128<float2>(axes_product(irho, g));
    sout32[g] = from_c128<float2>(axes_product(rho, g));
    lsum[g] = axes_sum(lam, g);
}

// complex64 path: w = x D^{-1} with the per-element scale in FP32 (the input
// rounded to FP32 first: FP64 arithmetic is scarce on this GPU)
__global__ void k_sep_in32(JobSpace js, int in_slot, float2* W, const float2* __restrict__ sc) {
    const int z = blockIdx.y;
    const int job = js.d_active[z];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    const float2 x = from_c128<float2>(js.vec[(size_t)job * js.vstride + (size_t)in_slot * js.n + g]);
    const float2 s = sc[g];
    W[(size_t)z * js.n + g] = make_float2(x.x * s.x - x.y * s.y, x.x * s.y + x.y * s.x);
}

// complex64 path: out = in / (Σ_d λ - σb), the denominator formed in FP64 from
// the FP64 sum table and rounded once, the quotient in FP32
__global__ void k_sep_div32(JobSpace js, const float2* in, float2* out, const double2* __restrict__ lsum,
                            const double2* sigma, double2 b) {
    const int z = blockIdx.y;
    const int job = js.d_active[z];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    const double2 s = sigma[js.d_jobshift[job]];
    const float2 d = from_c128<float2>(csub(lsum[g], cmul(s, b)));
    const float2 v = in[(size_t)z * js.n + g];
    const float inv = 1.0f / (d.x * d.x + d.y * d.y);
    out[(size_t)z * js.n + g] = make_float2((v.x * d.x + v.y * d.y) * inv, (v.y * d.x - v.x * d.y) * inv);
}

// complex64 path: z = D w, the scale in FP32, the result stored in FP64
__global__ void k_sep_out32(JobSpace js, int out_slot, const float2* W, const float2* __restrict__ sc) {
    const int z = blockIdx.y;
    const int job = js.d_active[z];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    const float2 w = W[(size_t)z * js.n + g], s = sc[g];
    js.vec[(size_t)job * js.vstride + (size_t)out_slot * js.n + g] =
        to_c128(make_float2(w.x * s.x - w.y * s.y, w.x * s.y + w.y * s.x));
}

template <class CW>
__global__ void k_sep_in(JobSpace js, int in_slot, CW* W, Axes irho) {
    const int z = blockIdx.y;
    const int job = js.d_active[z];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    const double2 x = js.vec[(size_t)job * js.vstride + (size_t)in_slot * js.n + g];
    W[(size_t)z * js.n + g] = from_c128<CW>(cmul(x, axes_product(irho, g)));
}

// out = in / (Σ_d λ_{d,k_d} - σ b), the denominators and the quotient in FP64
template <class CI, class CO>
__global__ void k_sep_div(JobSpace js, const CI* in, CO* out, Axes lam, const double2* sigma, double2 b) {
    const int z = blockIdx.y;
    const int job = js.d_active[z];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    const double2 s = sigma[js.d_jobshift[job]];
    const double2 d = csub(axes_sum(lam, g), cmul(s, b));
    out[(size_t)z * js.n + g] = from_c128<CO>(cdiv(to_c128(in[(size_t)z * js.n + g]), d));
}

template <class CW>
__global__ void k_sep_out(JobSpace js, int out_slot, const CW* W, Axes rho) {
    const int z = blockIdx.y;
    const int job = js.d_active[z];
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= js.n) return;
    js.vec[(size_t)job * js.vstride + (size_t)out_slot * js.n + g] =
        cmul(to_c128(W[(size_t)z * js.n + g]), axes_product(rho, g));
}

constexpr int MP_BJ = 16, MP_THREADS = 256;

// Y = mode product of X along an axis of length N with inner stride P
// (rows r = p + P q, element (r, j) at p + P(j + N q)); Q symmetric N×N.
// Tile TB rows × TB outputs (TB = 64: 4×4 per thread; TB = 128, complex64
// only: 8×8 per thread, fewer shared-memory loads per multiply-add).  Every output sums its
// j in the same order in both shapes, so they give bit-identical results and
// the autotuner picks between them.
template <class R, bool AXIS0, int TB>
__global__ void __launch_bounds__(MP_THREADS) k_sep_mode(const cplx<R>* __restrict__ Xall, cplx<R>* __restrict__ Yall,
                                                         const R* __restrict__ Q, int N, int64_t P, int64_t rows,
                                                         int64_t n) {
    using CW = cplx<R>;
    constexpr int MP_BR = TB, MP_BK = TB, PT = TB / 16;  // PT rows and PT outputs per thread
    __shared__ CW As[MP_BJ][MP_BR + 1];
    __shared__ R Qs[MP_BJ][MP_BK + 1];
    const CW* X = Xall + (size_t)blockIdx.z * n;
    CW* Y = Yall + (size_t)blockIdx.z * n;
    const int t = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * MP_BR;
    const int k0 = blockIdx.y * MP_BK;
    // compute mapping: axis 0 spreads threads over outputs k, other axes over rows
    const int tr = AXIS0 ? t / 16 : t % 16;
    const int tk = AXIS0 ? t % 16 : t / 16;
    const int64_t PN = P * (int64_t)N;
    CW acc[PT][PT];
#pragma unroll
    for (int i = 0; i < PT; ++i)
#pragma unroll
        for (int c = 0; c < PT; ++c) acc[i][c] = mk(R(0), R(0));
    for (int j0 = 0; j0 < N; j0 += MP_BJ) {
#pragma unroll
        for (int i = 0; i < (MP_BJ * MP_BR) / MP_THREADS; ++i) {
            const int e = t + MP_THREADS * i;
            const int jj = AXIS0 ? e % MP_BJ : e / MP_BR;
            const int rr = AXIS0 ? e / MP_BJ : e % MP_BR;
            const int64_t r = r0 + rr;
            const int j = j0 + jj;
            CW v = mk(R(0), R(0));
            if (r < rows && j < N) v = X[(r % P) + PN * (r / P) + P * (int64_t)j];
            As[jj][rr] = v;
            const int kk = e % MP_BK, jq = e / MP_BK;
            const int k = k0 + kk, jr = j0 + jq;
            Qs[jq][kk] = (k < N && jr < N) ? Q[(size_t)jr * N + k] : R(0);
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < MP_BJ; ++jj) {
            CW a[PT];
            R q[PT];
#pragma unroll
            for (int i = 0; i < PT; ++i) a[i] = As[jj][tr + 16 * i];
#pragma unroll
            for (int c = 0; c < PT; ++c) q[c] = Qs[jj][tk + 16 * c];
#pragma unroll
            for (int i = 0; i < PT; ++i)
#pragma unroll
                for (int c = 0; c < PT; ++c) {
                    acc[i][c].x = fma(a[i].x, q[c], acc[i][c].x);
                    acc[i][c].y = fma(a[i].y, q[c], acc[i][c].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < PT; ++i) {
        const int64_t r = r0 + tr + 16 * i;
        if (r >= rows) continue;
        const int64_t base = (r % P) + PN * (r / P);
#pragma unroll
        for (int c = 0; c < PT; ++c) {
            const int k = k0 + tk + 16 * c;
            if (k < N) Y[base + P * (int64_t)k] = acc[i][c];
        }
    }
}

Axes axes_of(const Separable& S, double2* const* tab) {
    Axes a;
    a.ndim = S.ndim;
    a.N0 = S.dims[0];
    a.N1 = S.dims[1];
    a.N2 = S.dims[2];
    a.t0 = tab[0];
    a.t1 = S.ndim > 1 ? tab[1] : tab[0];
    a.t2 = S.ndim > 2 ? tab[2] : tab[0];
    return a;
}

template <class R, int TB>
void launch_mode(const cplx<R>* cur, cplx<R>* nxt, const R* Q, int N, int64_t P, int64_t rows, int64_t n, int na,
                 cudaStream_t st) {
    const dim3 grid(cdiv_up(rows, TB), cdiv_up(N, TB), na);
    if (P == 1) k_sep_mode<R, true, TB><<<grid, MP_THREADS, 0, st>>>(cur, nxt, Q, N, P, rows, n);
    else k_sep_mode<R, false, TB><<<grid, MP_THREADS, 0, st>>>(cur, nxt, Q, N, P, rows, n);
    SIM_LAUNCH_CHECK();
}

// the mode products along every axis, ping-ponging between two buffers;
// returns the buffer that holds the result.  Tile shape autotuned per axis.
template <class R>
cplx<R>* run_modes(const Separable& S, int64_t n, int na, cplx<R>* cur, cplx<R>* nxt, cudaStream_t st) {
    int64_t P = 1;
    // instrumentation: the mode products alone (a part of "separable")
    kprof_begin(sizeof(R) == 4 && S.tc ? "sep_mode_tc" : "sep_mode", st);
    double flops = 0.0;
    for (int d = 0; d < S.ndim; ++d) flops += 4.0 * (double)n * (double)S.dims[d] * na;
    for (int d = 0; d < S.ndim; ++d) {
        const int N = (int)S.dims[d];
        const int64_t rows = n / N;
        const R* Q = sizeof(R) == 4 ? reinterpret_cast<const R*>(S.Q32[d]) : reinterpret_cast<const R*>(S.Q64[d]);
        if (sizeof(R) == 4 && S.tc &&
            sep_mode_tc(reinterpret_cast<const float2*>(cur), reinterpret_cast<float2*>(nxt), S.Qh[d], S.Ql[d], N, P,
                        rows, n, na, st)) {
            std::swap(cur, nxt);
            P *= N;
            continue;
        }
        const std::string key = std::string("sep_mode:") + (sizeof(R) == 4 ? "f:" : "d:") + std::to_string(N) + ":" +
                                std::to_string(P) + ":" + std::to_string(rows) + ":" + std::to_string(na < 4 ? na : 4);
        bool timing = false;
        // FP64 keeps the 64-wide tile (8 × 8 complex128 accumulators exceed the register file)
        const int c = sizeof(R) == 4 ? autotune_begin(key, 2, st, &timing) : 0;
        if (c == 0) launch_mode<R, 64>(cur, nxt, Q, N, P, rows, n, na, st);
        else launch_mode<float, 128>(reinterpret_cast<const float2*>(cur), reinterpret_cast<float2*>(nxt),
                                     reinterpret_cast<const float*>(Q), N, P, rows, n, na, st);
        if (timing) autotune_end(key, st);
        std::swap(cur, nxt);
        P *= N;
    }
    kprof_end(sizeof(R) == 4 && S.tc ? "sep_mode_tc" : "sep_mode", st, 2.0 * S.ndim * (double)na * n * sizeof(cplx<R>),
              flops);
    return cur;
}

// forward transform S^{-1} in RF, inverse transform S in RB (the division
// between them in FP64).  Mixed mode runs both transforms in FP32: an FP64
// inverse transform was measured to leave the inner iteration counts of the
// 3-D workload unchanged at six times the cost.
template <class RF, class RB>
void apply_t(const Separable& S, const JobSpace& js, int na, int in_slot, int out_slot, const double2* d_sigma,
             DeviceArena& ar, cudaStream_t st) {
    using CF = cplx<RF>;
    using CB = cplx<RB>;
    const int64_t n = js.n;
    CF* F0 = ar.get<CF>(sizeof(RF) == 4 ? "sep_w0_f" : "sep_w0_d", (int64_t)na * n);
    CF* F1 = ar.get<CF>(sizeof(RF) == 4 ? "sep_w1_f" : "sep_w1_d", (int64_t)na * n);
    CB* B0 = ar.get<CB>(sizeof(RB) == 4 ? "sep_w0_f" : "sep_w0_d", (int64_t)na * n);
    CB* B1 = ar.get<CB>(sizeof(RB) == 4 ? "sep_w1_f" : "sep_w1_d", (int64_t)na * n);
    const dim3 eg(cdiv_up(n, 256), na);
    constexpr bool c64 = sizeof(RF) == 4 && sizeof(RB) == 4;
    if constexpr (c64) k_sep_in32<<<eg, 256, 0, st>>>(js, in_slot, F0, S.sin32);
    else k_sep_in<CF><<<eg, 256, 0, st>>>(js, in_slot, F0, axes_of(S, S.irho));
    SIM_LAUNCH_CHECK();
    CF* f = run_modes<RF>(S, n, na, F0, F1, st);
    CB* bout = (void*)f == (void*)B0 ? B1 : B0;  // same buffers in both passes: do not overwrite the input
    if constexpr (c64) k_sep_div32<<<eg, 256, 0, st>>>(js, f, bout, S.lsum, d_sigma, S.b);
    else k_sep_div<CF, CB><<<eg, 256, 0, st>>>(js, f, bout, axes_of(S, S.lam), d_sigma, S.b);
    SIM_LAUNCH_CHECK();
    CB* other = bout == B0 ? B1 : B0;
    CB* b = run_modes<RB>(S, n, na, bout, other, st);
    if constexpr (c64) k_sep_out32<<<eg, 256, 0, st>>>(js, out_slot, b, S.sout32);
    else k_sep_out<CB><<<eg, 256, 0, st>>>(js, out_slot, b, axes_of(S, S.rho));
    SIM_LAUNCH_CHECK();
}

}  // namespace

void separable_setup(Separable& S, DeviceArena& ar, cudaStream_t st, const std::string& prefix) {
    for (int d = 0; d < S.ndim; ++d) {
        const int64_t N = S.dims[d];
        const std::string tag = prefix + "ax" + std::to_string(d) + "_";
        S.Q64[d] = ar.get<double>(tag + "Q64", N * N);
        S.Q32[d] = ar.get<float>(tag + "Q32", N * N);
        S.rho[d] = ar.get<double2>(tag + "rho", N);
        S.irho[d] = ar.get<double2>(tag + "irho", N);
        S.lam[d] = ar.get<double2>(tag + "lam", N);
        S.Qh[d] = ar.get<float>(tag + "Qh", N * N);
        S.Ql[d] = ar.get<float>(tag + "Ql", N * N);
        k_sep_tables<<<cdiv_up(N * N, 256), 256, 0, st>>>((int)N, S.axis[d][0], S.axis[d][1], S.axis[d][2], S.Q64[d],
                                                         S.Q32[d], S.rho[d], S.irho[d], S.lam[d]);
        SIM_LAUNCH_CHECK();
        sep_split_tables(S.Q64[d], (int)N, S.Qh[d], S.Ql[d], st);
    }
    int64_t n = 1;
    for (int d = 0; d < S.ndim; ++d) n *= S.dims[d];
    S.sin32 = ar.get<float2>(prefix + "sin32", n);
    S.sout32 = ar.get<float2>(prefix + "sout32", n);
    S.lsum = ar.get<double2>(prefix + "lsum", n);
    k_sep_elem_tables<<<cdiv_up(n, 256), 256, 0, st>>>(n, axes_of(S, S.irho), axes_of(S, S.rho), axes_of(S, S.lam),
                                                      S.sin32, S.sout32, S.lsum);
    SIM_LAUNCH_CHECK();
    SIM_CUDA(cudaStreamSynchronize(st));
}

void separable_apply(const Separable& S, int precision, const JobSpace& js, const std::vector<int>& active,
                     int in_slot, int out_slot, const double2* d_sigma, DeviceArena& ar, cudaStream_t st) {
    const int na = (int)active.size();
    if (na <= 0) return;
    // the active list is already on the device (js.d_active) in this order
    kprof_begin("separable", st);
    if (precision == SIM_FP64) apply_t<double, double>(S, js, na, in_slot, out_slot, d_sigma, ar, st);
    else apply_t<float, float>(S, js, na, in_slot, out_slot, d_sigma, ar, st);
    double flops = 0.0;
    for (int d = 0; d < S.ndim; ++d) flops += 2.0 * 4.0 * (double)js.n * (double)S.dims[d];  // 2 passes, 2 FMA
    const double cw = precision == SIM_FP64 ? 16.0 : 8.0;
    // per job: the complex128 input and output, and each pass's read and write
    const double bytes = 32.0 * js.n + (2.0 * S.ndim + 1.0) * 2.0 * cw * js.n;
    kprof_end("separable", st, na * bytes, na * flops);
}

}  // namespace sim
