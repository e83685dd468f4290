// philox.cuh -- Philox4x32-10 counter-based generator (Salmon, Moraes, Dror
// and Shaw, SC'11) and the Vasicek zero-coupon price, shared by the nested
// valuation and the surrogate's query sampler.
#pragma once

#include <cstdint>

namespace rsv {

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t (&out)[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// Conditional forward discount curve of the Vasicek model at each node (the
// expectation of the inner loop): vbar_tau = P((tau+1) dt | r) / P(tau dt | r)
// with the zero-coupon price P(T | r) = A(T) exp(-B(T) r) (Vasicek 1977).
__device__ __forceinline__ double vasicek_lnP(double T, double r, double a, double b, double sigma) {
    const double B = -expm1(-a * T) / a;
    return (B - T) * (a * a * b - 0.5 * sigma * sigma) / (a * a) - sigma * sigma * B * B / (4.0 * a) - B * r;
}

}  // namespace rsv
