// Variants of the deflated recurrence kernel and the deflator plane.
#include "defl_kernel.cuh"

namespace rsv {

// (policies per warp P, scenarios per lane M, valuing warps per CTA NW (plus
// one staging warp), staged blocks in flight NBUF, minimum resident CTAs per
// SM, arithmetic: 0 scalar, 1 packed pairs, 2 packed pairs with each chain's
// double-float sum in tensor memory, 3 the same folded once per 32-step
// block).  One CTA per SM: each of an SM's four schedulers has a quarter of
// the register file, so NW + 1 = 12 warps leave 168 registers a thread, 16
// warps 128 (which the packed accumulators fit only with the sums in tensor
// memory).
static const DeflVariant kDefl[] = {
    // the tuned best on the headline workload first: the default before tuning
    RSV_DEFL_VARIANT(4, 4, 15, 6, 1, 3, "deflated P4xM4 nw15 buf6 x2 tm2"),
    RSV_DEFL_VARIANT(4, 4, 15, 8, 1, 2, "deflated P4xM4 nw15 buf8 x2 tm"),
    RSV_DEFL_VARIANT(4, 4, 11, 8, 1, 1, "deflated P4xM4 nw11 buf8 x2"),
    RSV_DEFL_VARIANT(4, 4, 11, 8, 1, 0, "deflated P4xM4 nw11 buf8"),
    RSV_DEFL_VARIANT(4, 4, 11, 4, 1, 0, "deflated P4xM4 nw11 buf4"),
    RSV_DEFL_VARIANT(4, 2, 15, 8, 1, 0, "deflated P4xM2 nw15 buf8"),
    RSV_DEFL_VARIANT(4, 2, 15, 8, 1, 1, "deflated P4xM2 nw15 buf8 x2"),
    RSV_DEFL_VARIANT(4, 4, 10, 8, 1, 1, "deflated P4xM4 nw10 buf8 x2"),
    RSV_DEFL_VARIANT(4, 4, 7, 8, 1, 0, "deflated P4xM4 nw7 buf8"),
    RSV_DEFL_VARIANT(4, 4, 7, 8, 1, 1, "deflated P4xM4 nw7 buf8 x2"),
    RSV_DEFL_VARIANT(2, 4, 15, 6, 1, 0, "deflated P2xM4 nw15 buf6"),
    RSV_DEFL_VARIANT(2, 4, 15, 6, 1, 1, "deflated P2xM4 nw15 buf6 x2"),
};

const DeflVariant* variants_defl(int* n) {
    *n = (int)(sizeof(kDefl) / sizeof(kDefl[0]));
    return kDefl;
}

size_t defl_smem_extra(const DeflVariant& v) {
    const size_t CH = 32 * (size_t)v.M;
    return (size_t)v.NBUF * DEFL_G * CH * sizeof(float4) + (size_t)2 * v.NW * CH * sizeof(float2) +
           (size_t)2 * v.NW * v.P * sizeof(DeflSlot) + (size_t)v.NBUF * sizeof(DeflBlock) +
           (size_t)2 * v.NBUF * sizeof(uint64_t);
}

// The deflator plane: D_{t+1} = v_0 v_1 ... v_t of every scenario column as an
// FP64 running product (the discount-factor products over long terms), stored
// rounded to FP32 as rows of four steps, out[g][s] = (D_{4g+1}, .., D_{4g+4});
// rows at or beyond n_steps hold 0.  One thread per scenario column.
__global__ void defl_plane_kernel(const double* __restrict__ v, int n_steps, int s_pad, int n_groups,
                                  float4* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s_pad) return;
    double D = 1.0;
    for (int g = 0; g < n_groups; ++g) {
        float r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int t = 4 * g + j;
            if (t < n_steps) {
                D = __dmul_rn(D, v[(size_t)t * s_pad + s]);
                r[j] = __double2float_rn(D);
            } else {
                r[j] = 0.0f;
            }
        }
        out[(size_t)g * s_pad + s] = make_float4(r[0], r[1], r[2], r[3]);
    }
}

cudaError_t launch_defl_plane(const double* v64, int n_steps, int s_pad, int n_groups, float4* out,
                              cudaStream_t st) {
    defl_plane_kernel<<<(s_pad + 127) / 128, 128, 0, st>>>(v64, n_steps, s_pad, n_groups, out);
    return cudaGetLastError();
}

}  // namespace rsv
