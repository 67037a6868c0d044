// Counter-based random vectors for SIM-M: the random f of Sec. 3.5 (when the
// caller passes none) and the k random vectors of the multiplicity step
// (Sec. 3.4).  Philox4x64-10 as published by Salmon, Moraes, Dror and Shaw
// ("Parallel random numbers: as easy as 1, 2, 3", SC'11): per round two
// 64x64->128-bit products with multipliers 0xD2E7470EE14C6C93 and
// 0xCA5A826395121157, Weyl key increments 0x9E3779B97F4A7C15 and
// 0xBB67AE8584CAA73B.  Element e of vector v under seed s uses counter
// (e, v, 0, 0) and key (s, 0x53494D4D); output words 0 and 1 become uniforms
// u = (x >> 11) 2^-53 and Box–Muller gives sqrt(-2 ln(1-u0)) e^{2πi u1}/sqrt(2).
#include "internal.h"

namespace sim {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0;
        c[1] = n1;
        c[2] = n2;
        c[3] = n3;
        k0 += W0;
        k1 += W1;
    }
}

__global__ void k_random_vectors(uint64_t seed, int64_t n, int k, int first, double2* out, int64_t ld) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y;
    if (e >= n || v >= k) return;
    uint64_t c[4] = {(uint64_t)e, (uint64_t)(first + v), 0ull, 0ull};
    philox4x64_10(c, seed, 0x53494D4Dull);
    const double u0 = (double)(c[0] >> 11) * 0x1.0p-53;
    const double u1 = (double)(c[1] >> 11) * 0x1.0p-53;
    const double r = sqrt(-2.0 * log1p(-u0));
    double sn, cs;
    sincospi(2.0 * u1, &sn, &cs);
    const double s2 = 0.70710678118654752440;
    out[(size_t)v * ld + e] = make_double2(r * cs * s2, r * sn * s2);
}

void random_vectors(uint64_t seed, int64_t n, int k, int first, double2* out, int64_t ld, cudaStream_t st) {
    if (n <= 0 || k <= 0) return;
    dim3 grid(cdiv_up(n, 256), k);
    k_random_vectors<<<grid, 256, 0, st>>>(seed, n, k, first, out, ld);
    SIM_LAUNCH_CHECK();
}

}  // namespace sim
