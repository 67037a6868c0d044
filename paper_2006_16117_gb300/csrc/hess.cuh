// Device helpers shared by the level kernels and the multiplicity kernels:
// quadrature node offsets, square centres, staging of a Hessenberg matrix and
// the warp-level Hessenberg solve (I + alpha H) y = beta e1.
#pragma once

#include "common.cuh"

namespace sim {

constexpr double SQRT1_2 = 0.70710678118654752440;

__device__ __forceinline__ double mag1(double2 a) { return fabs(a.x) + fabs(a.y); }

// node offsets z_j - c on the circle circumscribing a square of side s, j = 0..7
__device__ __forceinline__ double2 node_offset(int j, double s) {
    const double r = __dmul_rn(s, SQRT1_2);
    const double hs = 0.5 * s;
    switch (j) {
        case 0: return make_double2(r, 0.0);
        case 1: return make_double2(hs, hs);
        case 2: return make_double2(0.0, r);
        case 3: return make_double2(-hs, hs);
        case 4: return make_double2(-r, 0.0);
        case 5: return make_double2(-hs, -hs);
        case 6: return make_double2(0.0, -r);
        default: return make_double2(hs, -hs);
    }
}

__device__ __forceinline__ double2 square_center(double re_lo, double im_lo, double s, int64_t ix, int64_t iy) {
    return make_double2(__dadd_rn(re_lo, __dmul_rn((double)ix + 0.5, s)),
                        __dadd_rn(im_lo, __dmul_rn((double)iy + 0.5, s)));
}

// Stage shift s's Hessenberg (column-major (m+1) x m in global) row-major into
// Hs[r*m + c] (r < m) and return h_{m+1,m}.
__device__ __forceinline__ void stage_H(const double2* H, int m, int meff, double2* Hs) {
    for (int e = threadIdx.x; e < meff * meff; e += blockDim.x) {
        int r = e / meff, c = e % meff;
        Hs[r * meff + c] = (r <= c + 1) ? H[(size_t)c * (m + 1) + r] : make_double2(0.0, 0.0);
    }
}

// One warp solves (I + alpha H) y = beta e1 (order m, H row-major in Hs with
// leading dimension m) and leaves y in ys[0..m).  U: packed upper-triangular
// scratch of m(m+1)/2 entries.  Returns |y_{m-1}| and ||y||^2 (warp-uniform).
__device__ __forceinline__ void warp_hess_solve(const double2* Hs, int m, double2 alpha, double beta, double2* U, double2* ys,
                                double& ylast, double& ynorm2) {
    const int lane = threadIdx.x & 31;
    const int c0 = lane, c1 = lane + 32;
    auto trow = [&](int r, int c) -> double2 {
        if (c >= m) return make_double2(0.0, 0.0);
        double2 h = Hs[r * m + c];
        double2 v = cmul(alpha, h);
        if (r == c) v.x += 1.0;
        return v;
    };
    double2 a0 = trow(0, c0), a1 = trow(0, c1);
    double2 arhs = make_double2(beta, 0.0);
    for (int k = 0; k < m - 1; ++k) {
        double2 b0 = (c0 >= k) ? trow(k + 1, c0) : make_double2(0.0, 0.0);
        double2 b1 = (c1 >= k) ? trow(k + 1, c1) : make_double2(0.0, 0.0);
        double2 brhs = make_double2(0.0, 0.0);
        const int src = k & 31;
        const bool hi = k >= 32;
        double2 ak, bk;
        ak.x = __shfl_sync(0xffffffffu, hi ? a1.x : a0.x, src);
        ak.y = __shfl_sync(0xffffffffu, hi ? a1.y : a0.y, src);
        bk.x = __shfl_sync(0xffffffffu, hi ? b1.x : b0.x, src);
        bk.y = __shfl_sync(0xffffffffu, hi ? b1.y : b0.y, src);
        if (mag1(bk) > mag1(ak)) {
            double2 t;
            t = a0; a0 = b0; b0 = t;
            t = a1; a1 = b1; b1 = t;
            t = arhs; arhs = brhs; brhs = t;
            t = ak; ak = bk; bk = t;
        }
        // U row k
        const int ofs = k * m - (k * (k - 1)) / 2;
        if (c0 >= k && c0 < m) U[ofs + (c0 - k)] = a0;
        if (c1 >= k && c1 < m) U[ofs + (c1 - k)] = a1;
        if (lane == 0) ys[k] = arhs;  // transformed right-hand side
        double2 l = (ak.x == 0.0 && ak.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(bk, ak);
        if (c0 > k) b0 = csub(b0, cmul(l, a0));
        if (c1 > k) b1 = csub(b1, cmul(l, a1));
        brhs = csub(brhs, cmul(l, arhs));
        a0 = b0;
        a1 = b1;
        arhs = brhs;
    }
    {
        const int k = m - 1;
        const int ofs = k * m - (k * (k - 1)) / 2;
        if (c0 == k) U[ofs] = a0;
        if (c1 == k) U[ofs] = a1;
        if (lane == 0) ys[k] = arhs;
    }
    __syncwarp();
    // column-oriented back substitution: lane owns rows lane and lane+32
    double2 r0 = (c0 < m) ? ys[c0] : make_double2(0.0, 0.0);
    double2 r1 = (c1 < m) ? ys[c1] : make_double2(0.0, 0.0);
    __syncwarp();
    double nrm = 0.0;
    double last = 0.0;
    for (int j = m - 1; j >= 0; --j) {
        const int ofsj = j * m - (j * (j - 1)) / 2;
        const double2 ujj = U[ofsj];
        const bool hi = j >= 32;
        double2 rj;
        rj.x = __shfl_sync(0xffffffffu, hi ? r1.x : r0.x, j & 31);
        rj.y = __shfl_sync(0xffffffffu, hi ? r1.y : r0.y, j & 31);
        const double2 yj = (ujj.x == 0.0 && ujj.y == 0.0) ? make_double2(0.0, 0.0) : cdiv(rj, ujj);
        if (lane == 0) ys[j] = yj;
        if (j == m - 1) last = cabsd(yj);
        nrm += cabs2(yj);
        if (c0 < j) r0 = csub(r0, cmul(U[c0 * m - (c0 * (c0 - 1)) / 2 + (j - c0)], yj));
        if (c1 < j) r1 = csub(r1, cmul(U[c1 * m - (c1 * (c1 - 1)) / 2 + (j - c1)], yj));
    }
    __syncwarp();
    ylast = last;
    ynorm2 = nrm;
}


}  // namespace sim
