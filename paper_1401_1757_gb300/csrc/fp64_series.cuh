// fp64_series.cuh -- short FP64 series for arguments known to be small.
#pragma once

#include <cuda_runtime.h>

namespace rsv {

// e^x in FP64: |x| < 2^-6 by its Taylor series to x^6, |x| < 1/16 to x^8
// (remainders below 5e-17 relative either way; a month's integrated rate,
// about 0.003, takes the short one), exp() beyond.
__device__ __forceinline__ double exp_small(double x) {
    const double ax = fabs(x);
    if (ax < 0.015625) {
        double p = __fma_rn(x, 1.0 / 720.0, 1.0 / 120.0);
        p = __fma_rn(x, p, 1.0 / 24.0);
        p = __fma_rn(x, p, 1.0 / 6.0);
        p = __fma_rn(x, p, 0.5);
        p = __fma_rn(x, p, 1.0);
        return __fma_rn(x, p, 1.0);
    }
    if (!(ax < 0.0625)) return exp(x);
    double p = __fma_rn(x, 1.0 / 40320.0, 1.0 / 5040.0);
    p = __fma_rn(x, p, 1.0 / 720.0);
    p = __fma_rn(x, p, 1.0 / 120.0);
    p = __fma_rn(x, p, 1.0 / 24.0);
    p = __fma_rn(x, p, 1.0 / 6.0);
    p = __fma_rn(x, p, 0.5);
    p = __fma_rn(x, p, 1.0);
    return __fma_rn(x, p, 1.0);
}

}  // namespace rsv
