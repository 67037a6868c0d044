// Schur form of each shift's Hessenberg matrix and the level evaluation
// built on it (Sec. 3.2, Eqs. zjHm, rmLc1; Sec. 3.3, Eqs. eq:many, eq:error,
// DeltaSm).
//
// The projected solves of a square all use one H_m: at node z_j,
//     (I + α_j H_m) y_j = β e_1,   α_j = σ - z_j.
// With the complex Schur form H_m = Z T Z^H (T upper triangular, Z unitary),
// computed once per shift,
//     (I + α_j T) x_j = c,   c = β Z^H e_1,   y_j = Z x_j,
// so a node costs one triangular solve, and everything the level needs is
// available without forming y_j:  e_m^T y_j = z_m^T x_j (z_m^T the last row
// of Z) for the residual of Eq. eq:error, ||y_j|| = ||x_j||, and the norms of
// the two quadrature sums Σ_j w_j y_j = Z Σ_j w_j x_j of Eq. DeltaSm.  The
// paper's own formula (the eigendecomposition H_m = P D P^{-1}) gives the same
// quantities; the Schur form is its unitary, backward-stable counterpart.
//
// k_schur: one warp per shift, the shifted QR algorithm of k_ritz applied to
// whole rows and columns with the rotations accumulated into the two rows of Z
// the level needs (the first and the last: a row of Z evolves on its own
// under the column rotations).
// k_eval_schur: one lane per quadrature node (a warp holds the 8 nodes of 4
// squares), so every FP64 instruction does useful work in all lanes; T's
// entries are warp-uniform loads when the 4 squares share a shift (children
// of one square do).  The squares their own shift does not resolve are then
// evaluated against every shift of their pencil at once (square-shift pairs
// as items) and k_pick_shift takes the shift the direct evaluation's order
// would.  Only a zero pivot or a shift without a Schur form sends a square to
// the direct evaluation (k_eval_level).
#include <cfloat>

#include "hess.cuh"
#include "internal.h"
#include "levels.h"

namespace sim {

namespace {

__device__ __forceinline__ double cabs_s(double2 a) { return hypot(a.x, a.y); }

__device__ __forceinline__ double2 csqrt_s(double2 z) {
    const double r = cabs_s(z);
    const double re = sqrt(fmax(0.0, 0.5 * (r + z.x)));
    const double im = sqrt(fmax(0.0, 0.5 * (r - z.x)));
    return make_double2(re, z.y < 0.0 ? -im : im);
}

__device__ __forceinline__ double2 conj_s(double2 a) { return make_double2(a.x, -a.y); }

}  // namespace

// Shared memory: A [m][m] row-major, then rows 0 and n-1 of Z.
__global__ void __launch_bounds__(32) k_schur(const double2* Hall, int m, const int* meff_all, const double* beta_all,
                                              int s0, double2* Tall, double2* Call, double2* Qall, int* ok_all) {
    const int s = s0 + blockIdx.x;
    const int n = meff_all[s];
    const double2* Hs = Hall + (size_t)s * (m + 1) * m;  // column-major, leading dimension m + 1
    extern __shared__ double2 sh_schur[];
    double2* A = sh_schur;
    double2* Z0 = sh_schur + (size_t)m * m;  // row 0 of Z
    double2* Zl = Z0 + m;                    // row n-1 of Z
    __shared__ double gc[64];
    __shared__ double2 gs[64];
    __shared__ double2 s_mu;
    __shared__ int s_l;
    const int lane = threadIdx.x;
    for (int idx = lane; idx < n * n; idx += 32) {
        const int r = idx / n, c = idx % n;
        A[r * m + c] = (r <= c + 1) ? Hs[(size_t)c * (m + 1) + r] : make_double2(0.0, 0.0);
    }
    for (int c = lane; c < n; c += 32) {
        Z0[c] = make_double2(c == 0 ? 1.0 : 0.0, 0.0);
        Zl[c] = make_double2(c == n - 1 ? 1.0 : 0.0, 0.0);
    }
    double nrm = 0.0;
    for (int idx = lane; idx < n * n; idx += 32) nrm = fmax(nrm, cabs_s(A[(idx / n) * m + idx % n]));
    for (int o = 16; o > 0; o >>= 1) nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
    __syncwarp();
    int hi = n - 1, its = 0, sweeps = 0, fail = (n < 1 || n > 64) ? 1 : 0;
    while (!fail && hi > 0) {
        if (lane == 0) {
            int l = hi;
            while (l > 0) {
                const double sub = cabs_s(A[l * m + l - 1]);
                double d = cabs_s(A[(l - 1) * m + l - 1]) + cabs_s(A[l * m + l]);
                if (d == 0.0) d = nrm;
                if (sub <= DBL_EPSILON * d) break;
                --l;
            }
            if (l > 0) A[l * m + l - 1] = make_double2(0.0, 0.0);
            s_l = l;
            if (l != hi) {
                // Wilkinson shift from the trailing 2×2 block, exceptional every 10 sweeps
                const double2 p = A[(hi - 1) * m + hi - 1], q = A[(hi - 1) * m + hi];
                const double2 r = A[hi * m + hi - 1], t = A[hi * m + hi];
                double2 mu = t;
                if (its > 0 && its % 10 == 0) {
                    mu.x += 0.75 * cabs_s(r);
                } else {
                    const double2 d = make_double2(0.5 * (p.x - t.x), 0.5 * (p.y - t.y));
                    const double2 qr = cmul(q, r);
                    const double2 disc = csqrt_s(cadd(cmul(d, d), qr));
                    const double2 den1 = cadd(d, disc), den2 = csub(d, disc);
                    const double2 den = cabs_s(den1) >= cabs_s(den2) ? den1 : den2;
                    if (cabs_s(den) > 0.0) mu = csub(t, cdiv(qr, den));
                }
                s_mu = mu;
            }
        }
        __syncwarp();
        const int l = s_l;
        if (l == hi) {
            --hi;
            its = 0;
            __syncwarp();
            continue;
        }
        if (++sweeps > 30 * n) {
            fail = 1;
            break;
        }
        ++its;
        const double2 mu = s_mu;
        for (int k = l + lane; k <= hi; k += 32) A[k * m + k] = csub(A[k * m + k], mu);
        __syncwarp();
        // left: G_k zeroes A[k+1][k] of the active block; applied to whole rows k, k+1
        for (int k = l; k < hi; ++k) {
            if (lane == 0) {
                const double2 a = A[k * m + k], b = A[(k + 1) * m + k];
                const double na = cabs_s(a), nb = cabs_s(b);
                double c;
                double2 sn;
                if (nb == 0.0) {
                    c = 1.0;
                    sn = make_double2(0.0, 0.0);
                } else if (na == 0.0) {
                    c = 0.0;
                    sn = make_double2(b.x / nb, -b.y / nb);
                } else {
                    const double h = hypot(na, nb);
                    c = na / h;
                    const double2 ua = make_double2(a.x / na, a.y / na);
                    sn = cmul(ua, make_double2(b.x / h, -b.y / h));
                }
                gc[k - l] = c;
                gs[k - l] = sn;
            }
            __syncwarp();
            const double c = gc[k - l];
            const double2 sn = gs[k - l];
            for (int j = k + lane; j < n; j += 32) {
                const double2 x = A[k * m + j], y = A[(k + 1) * m + j];
                A[k * m + j] = cadd(make_double2(c * x.x, c * x.y), cmul(sn, y));
                A[(k + 1) * m + j] = csub(make_double2(c * y.x, c * y.y), cmul(conj_s(sn), x));
            }
            __syncwarp();
        }
        // right: columns k, k+1 of every row above the active block's subdiagonal, and of Z
        for (int k = l; k < hi; ++k) {
            const double c = gc[k - l];
            const double2 sn = gs[k - l];
            const int rmax = min(k + 1, hi);
            for (int i = lane; i <= rmax; i += 32) {
                const double2 x = A[i * m + k], y = A[i * m + k + 1];
                A[i * m + k] = cadd(make_double2(c * x.x, c * x.y), cmul(conj_s(sn), y));
                A[i * m + k + 1] = csub(make_double2(c * y.x, c * y.y), cmul(sn, x));
            }
            if (lane < 2) {
                double2* Zr = lane == 0 ? Z0 : Zl;
                const double2 x = Zr[k], y = Zr[k + 1];
                Zr[k] = cadd(make_double2(c * x.x, c * x.y), cmul(conj_s(sn), y));
                Zr[k + 1] = csub(make_double2(c * y.x, c * y.y), cmul(sn, x));
            }
            __syncwarp();
        }
        for (int k = l + lane; k <= hi; k += 32) A[k * m + k] = cadd(A[k * m + k], mu);
        __syncwarp();
    }
    double2* T = Tall + (size_t)s * m * m;
    const double beta = beta_all[s];
    if (!fail) {
        for (int idx = lane; idx < n * n; idx += 32) {
            const int r = idx / n, c = idx % n;
            T[r * m + c] = c >= r ? A[r * m + c] : make_double2(0.0, 0.0);
        }
        for (int i = lane; i < n; i += 32) {
            const double2 z0 = Z0[i];
            Call[(size_t)s * m + i] = make_double2(beta * z0.x, -beta * z0.y);
            Qall[(size_t)s * m + i] = Zl[i];
        }
    }
    if (lane == 0) ok_all[s] = fail ? 0 : 1;
}

// 8 nodes per square, 4 squares per warp, SE_WARPS warps per CTA; x_j of every
// lane in shared memory as [i][lane] (conflict-free 16-byte accesses).
constexpr int SE_WARPS = 4;

// ALL = false: item t is square t against its own shift; a square it resolves
//   gets its results, the others todo[q] = 1.
// ALL = true: item t = (i, o) is square list[i] against shift lo + o of its
//   pencil's range [lo, hi), o < smax; the indicator, the largest node
//   residual and the zero-pivot / no-Schur-form flag go to rind, rrho, rbad.
template <bool ALL>
__global__ void __launch_bounds__(SE_WARPS * 32) k_eval_schur(ShiftTable st, LevelArgs a, uint8_t* todo,
                                                              const int64_t* list, int smax, int64_t nitems,
                                                              double* rind, double* rrho, uint8_t* rbad) {
    const double2* Tall = st.schT;
    const double2* Call = st.schC;
    const double2* Qall = st.schQ;
    const int* ok_all = st.schOK;
    extern __shared__ double2 sh_x[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = st.m;
    double2* xs = sh_x + (size_t)warp * m * 32;
    const int j = lane & 7;  // node
    const int64_t nwarps = (int64_t)gridDim.x * SE_WARPS;
    for (int64_t t0 = ((int64_t)blockIdx.x * SE_WARPS + warp) * 4; t0 < nitems; t0 += nwarps * 4) {
        const int64_t t = t0 + (lane >> 3);
        int64_t q = t;
        bool active = t < nitems;
        int s = 0, n = 0;
        if (ALL && active) {
            q = list[t / smax];
            int lo = 0, hi = st.S;
            if (st.pencil_of) {
                const int p = st.pencil_of[a.sid[q]];
                lo = st.p_sb[p];
                hi = st.p_se[p];
            }
            s = lo + (int)(t % smax);
            active = s < hi;
        }
        double re_lo = a.re_lo, im_lo = a.im_lo, side = a.side;
        bool good = false;
        if (active) {
            if (!ALL) s = a.sid[q];
            if (st.pencil_of) {
                const int p = st.pencil_of[s];
                re_lo = st.p_re_lo[p];
                im_lo = st.p_im_lo[p];
                side = st.p_side[p];
            }
            good = ok_all[s] != 0;
            n = good ? st.meff[s] : 0;
        }
        const double2 c = square_center(re_lo, im_lo, side, active ? a.ix[q] : 0, active ? a.iy[q] : 0);
        const double2 off = node_offset(j, side);
        const double2 z = make_double2(__dadd_rn(c.x, off.x), __dadd_rn(c.y, off.y));
        const double2 sig = active ? st.sigma[s] : make_double2(0.0, 0.0);
        const double2 alpha = make_double2(__dsub_rn(sig.x, z.x), __dsub_rn(sig.y, z.y));
        const double2 w8 = cscale(off, 0.125), w4 = (j & 1) == 0 ? cscale(off, 0.25) : make_double2(0.0, 0.0);
        const double2* T = Tall + (size_t)s * m * m;
        const double2* Cv = Call + (size_t)s * m;
        const double2* Qv = Qall + (size_t)s * m;
        int nmax = n;
        for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
        double2 yl = make_double2(0.0, 0.0);
        double yn2 = 0.0, n8 = 0.0, n4 = 0.0;
        for (int i = nmax - 1; i >= 0; --i) {
            double2 xi = make_double2(0.0, 0.0);
            if (i < n) {
                // x_i = (c_i - α Σ_{k>i} T_ik x_k) / (1 + α T_ii)
                double2 acc = make_double2(0.0, 0.0);
                const double2* Ti = T + (size_t)i * m;
                int k = i + 1;
                for (; k + 1 < n; k += 2) {
                    const double2 t0 = __ldg(Ti + k), t1 = __ldg(Ti + k + 1);
                    const double2 x0 = xs[(size_t)k * 32 + lane], x1 = xs[(size_t)(k + 1) * 32 + lane];
                    acc.x = fma(t0.x, x0.x, acc.x);
                    acc.x = fma(-t0.y, x0.y, acc.x);
                    acc.y = fma(t0.x, x0.y, acc.y);
                    acc.y = fma(t0.y, x0.x, acc.y);
                    acc.x = fma(t1.x, x1.x, acc.x);
                    acc.x = fma(-t1.y, x1.y, acc.x);
                    acc.y = fma(t1.x, x1.y, acc.y);
                    acc.y = fma(t1.y, x1.x, acc.y);
                }
                if (k < n) {
                    const double2 t0 = __ldg(Ti + k);
                    const double2 x0 = xs[(size_t)k * 32 + lane];
                    acc.x = fma(t0.x, x0.x, acc.x);
                    acc.x = fma(-t0.y, x0.y, acc.x);
                    acc.y = fma(t0.x, x0.y, acc.y);
                    acc.y = fma(t0.y, x0.x, acc.y);
                }
                const double2 tii = __ldg(Ti + i);
                double2 den = cmul(alpha, tii);
                den.x += 1.0;
                const double2 rhs = csub(__ldg(Cv + i), cmul(alpha, acc));
                if (den.x == 0.0 && den.y == 0.0) good = false;
                else xi = cdiv(rhs, den);
                xs[(size_t)i * 32 + lane] = xi;
                const double2 ql = __ldg(Qv + i);
                yl = cadd(yl, cmul(ql, xi));
                yn2 += cabs2(xi);
            }
            // the two quadrature sums of component i over the square's 8 lanes
            double2 p8 = cmul(w8, xi), p4 = cmul(w4, xi);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                p8.x += __shfl_xor_sync(0xffffffffu, p8.x, o);
                p8.y += __shfl_xor_sync(0xffffffffu, p8.y, o);
                p4.x += __shfl_xor_sync(0xffffffffu, p4.x, o);
                p4.y += __shfl_xor_sync(0xffffffffu, p4.y, o);
            }
            n8 += cabs2(p8);
            n4 += cabs2(p4);
        }
        __syncwarp();
        // residual of Eq. eq:error at this node, as the direct evaluation forms it
        double r = 0.0;
        if (active && good && n > 0) {
            const double hlast = cabsd(st.H[(size_t)s * (m + 1) * m + (size_t)(n - 1) * (m + 1) + n]);
            const double num = cabsd(alpha) * hlast * cabsd(yl);
            const double den = st.scale == 0 ? sqrt(yn2) : st.beta[s];
            r = num / den;
            if (!(r == r) || isinf(r)) r = INFINITY;
            if (num == 0.0) r = 0.0;
        }
        int bad = (active && (!good || n == 0)) ? 1 : 0;
        double rmax = r;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        if (ALL && t < nitems && j == 0) {
            const double s8 = sqrt(n8), s4 = sqrt(n4);
            rind[t] = s4 > 0.0 ? s8 / s4 : (s8 > 0.0 ? INFINITY : 0.0);
            rrho[t] = active ? rmax : INFINITY;
            rbad[t] = active ? (uint8_t)bad : (uint8_t)0;
        }
        if (!ALL && active && j == 0) {
            const double s8 = sqrt(n8), s4 = sqrt(n4);
            const double ind = s4 > 0.0 ? s8 / s4 : (s8 > 0.0 ? INFINITY : 0.0);
            if (!bad && rmax <= st.eps) {
                a.ind[q] = ind;
                a.mark[q] = ind > st.delta0 ? 1 : 0;
                a.flag[q] = 0;
                todo[q] = 0;
            } else {
                todo[q] = 1;
            }
        }
    }
}

void schur_shifts(const double2* H, int m, const int* meff, const double* beta, int s0, int count, double2* T,
                  double2* C, double2* Q, int* ok, cudaStream_t st) {
    if (count <= 0) return;
    const size_t sm = ((size_t)m * m + 2 * (size_t)m) * sizeof(double2);
    SIM_CUDA(cudaFuncSetAttribute(k_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_schur<<<count, 32, sm, st>>>(H, m, meff, beta, s0, T, C, Q, ok);
    SIM_LAUNCH_CHECK();
}

// The squares their own shift left (todo != 0), listed in any order.
__global__ void k_list_todo(const uint8_t* todo, int64_t count, int64_t* list, unsigned long long* n) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < count && todo[q]) list[atomicAdd(n, 1ull)] = (int64_t)q;
}

// One thread per listed square: the result the direct evaluation's shift order
// gives (own shift first, then the others nearest-first by |σ - c|, ties by the
// lower id; the first that resolves the square is used; if none does, the own
// shift's indicator and "unresolvable").  A square with any zero pivot or
// missing Schur form among its shifts stays todo for the direct evaluation.
__global__ void k_pick_shift(ShiftTable st, LevelArgs a, const int64_t* list, int64_t ntodo, int smax,
                             const double* rind, const double* rrho, const uint8_t* rbad, uint8_t* todo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntodo) return;
    const int64_t q = list[i];
    const int own = a.sid[q];
    int lo = 0, hi = st.S;
    double re_lo = a.re_lo, im_lo = a.im_lo, side = a.side;
    if (st.pencil_of) {
        const int p = st.pencil_of[own];
        lo = st.p_sb[p];
        hi = st.p_se[p];
        re_lo = st.p_re_lo[p];
        im_lo = st.p_im_lo[p];
        side = st.p_side[p];
    }
    const int64_t r0 = i * (int64_t)smax;
    for (int s = lo; s < hi; ++s)
        if (rbad[r0 + (s - lo)]) return;  // left to the direct evaluation
    const double2 c = square_center(re_lo, im_lo, side, a.ix[q], a.iy[q]);
    int used = own, tried = 1;
    bool res = rrho[r0 + (own - lo)] <= st.eps;
    if (!res) {
        double bd = INFINITY;
        int best = -1;
        for (int s = lo; s < hi; ++s) {
            if (s == own || !(rrho[r0 + (s - lo)] <= st.eps)) continue;
            const double d = hypot(st.sigma[s].x - c.x, st.sigma[s].y - c.y);
            if (d < bd || (d == bd && s < best)) {
                bd = d;
                best = s;
            }
        }
        if (best >= 0) {
            res = true;
            used = best;
            for (int s = lo; s < hi; ++s) {
                if (s == own) continue;
                const double d = hypot(st.sigma[s].x - c.x, st.sigma[s].y - c.y);
                if (d < bd || (d == bd && s <= best)) ++tried;
            }
        } else {
            tried = hi - lo;
        }
    }
    if (a.retries && tried > 1) atomicAdd(a.retries, (unsigned long long)(tried - 1));
    const double ind = res ? rind[r0 + (used - lo)] : rind[r0 + (own - lo)];
    a.ind[q] = ind;
    a.mark[q] = res ? (ind > st.delta0 ? 1 : 0) : 1;
    a.flag[q] = res ? 0 : 1;
    a.sid[q] = used;
    todo[q] = 0;
}

void eval_level_schur(const ShiftTable& st, const LevelArgs& a, uint8_t* todo, cudaStream_t stream) {
    if (a.count <= 0) return;
    const size_t sm = (size_t)SE_WARPS * st.m * 32 * sizeof(double2);
    SIM_CUDA(cudaFuncSetAttribute(k_eval_schur<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t warps = (a.count + 3) / 4;
    const int grid = (int)std::min<int64_t>((warps + SE_WARPS - 1) / SE_WARPS, 152 * 16);
    kprof_begin("eval_level_schur", stream);
    k_eval_schur<false><<<grid, SE_WARPS * 32, sm, stream>>>(st, a, todo, nullptr, 1, a.count, nullptr, nullptr,
                                                             nullptr);
    SIM_LAUNCH_CHECK();
    // per square: 8 triangular solves of order m (m²/2 complex multiply-adds each)
    kprof_end("eval_level_schur", stream, 0.0, a.count * 8.0 * 4.0 * st.m * st.m);
}

void eval_level_schur_retries(const ShiftTable& st, const LevelArgs& a, uint8_t* todo, int64_t ntodo, int smax,
                              DeviceArena& ar, cudaStream_t stream) {
    if (ntodo <= 0 || smax <= 0) return;
    int64_t* list = ar.get<int64_t>("lvl_list", ntodo);
    unsigned long long* cnt = ar.get<unsigned long long>("lvl_list_n", 1);
    const int64_t nitems = ntodo * (int64_t)smax;
    double* rind = ar.get<double>("lvl_rind", nitems);
    double* rrho = ar.get<double>("lvl_rrho", nitems);
    uint8_t* rbad = ar.get<uint8_t>("lvl_rbad", nitems);
    SIM_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), stream));
    k_list_todo<<<cdiv_up(a.count, 256), 256, 0, stream>>>(todo, a.count, list, cnt);
    SIM_LAUNCH_CHECK();
    const size_t sm = (size_t)SE_WARPS * st.m * 32 * sizeof(double2);
    SIM_CUDA(cudaFuncSetAttribute(k_eval_schur<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const int64_t warps = (nitems + 3) / 4;
    const int grid = (int)std::min<int64_t>((warps + SE_WARPS - 1) / SE_WARPS, 152 * 16);
    kprof_begin("eval_level_schur", stream);
    k_eval_schur<true><<<grid, SE_WARPS * 32, sm, stream>>>(st, a, todo, list, smax, nitems, rind, rrho, rbad);
    SIM_LAUNCH_CHECK();
    k_pick_shift<<<cdiv_up(ntodo, 128), 128, 0, stream>>>(st, a, list, ntodo, smax, rind, rrho, rbad, todo);
    SIM_LAUNCH_CHECK();
    kprof_end("eval_level_schur", stream, 0.0, nitems * 8.0 * 4.0 * st.m * st.m);
}

}  // namespace sim
