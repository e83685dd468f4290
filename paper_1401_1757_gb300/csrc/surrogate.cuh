// surrogate.cuh -- queries, per-policy data and kernels of the reserve surrogate.
#pragma once

#include <cstdint>

#include "mlp.cuh"

struct rsv_ctx;

namespace rsv {

struct PolSur {   // per policy: what the sampler, the labeller and the features need
    int32_t product, age1, age2, S, lim1, lim2, tab1, tab2;   // lim = length of each life's table
    double amount, rho;
};

struct SurQuery {  // a policy in a reduced state at a node month with a short rate
    int32_t pol, m, state, bucket;
    double r;
};

// Tables the surrogate's kernels share (device pointers).
struct SurTables {
    const double2* tab;    // F64 decrement table entries (p, q), tab_pad per table
    int tab_pad;
    const double2* curve;  // per month t: (dA_t, dB_t), ln P((t+1)/12 | r) - ln P(t/12 | r) = dA_t - dB_t r
    const float2* comm;    // commutation columns D, N, M per (table, grid rate), sur_comm_len(tab_pad) entries
                           // each, as FP32 head + tail pairs of the FP64 values
    double a, b, sigma;    // the Vasicek model
    float af, k1, k2;      // a, (a^2 b - sigma^2/2)/a^2 and sigma^2/(4a) in FP32 for the base value's yield
};

// Flat reference rates of the commutation columns (continuous, per year).
constexpr double SUR_COMM_LO = -0.10, SUR_COMM_STEP = 0.0025;
constexpr float SUR_COMM_LO_F = -0.10f, SUR_COMM_STEP_F = 0.0025f, SUR_COMM_INV_STEP_F = 400.0f;
constexpr int SUR_COMM_N = 141;
__host__ __device__ constexpr int sur_comm_len(int tab_pad) { return tab_pad + 2; }

}  // namespace rsv

#include "rsv.h"
namespace rsv {
// Per-unit expected reserves (device, n values) of n device queries grouped
// in n_seg segments of one short rate each (device offsets seg[n_seg + 1]),
// each at most Lmax months long: the network, then flagged buckets by the
// recurrence.  *n_fallback receives the number valued by the recurrence.
rsv_status sur_value_queries(rsv_ctx* c, const rsv_query* dq, long long n, const long long* seg, int n_seg, int Lmax,
                             double* V, long long* n_fallback);
}  // namespace rsv
