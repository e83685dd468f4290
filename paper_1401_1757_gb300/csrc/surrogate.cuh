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

__global__ void sur_label_kernel(const PolSur* pols, const double2* tab, int tab_pad, const SurQuery* qs, long long n,
                                 double a, double b, double sigma, const unsigned char* flag, double* V);
__global__ void sur_features_kernel(const PolSur* pols, const SurQuery* qs, long long n, __nv_bfloat16* X);

__global__ void sur_to_reserve_kernel(const float* __restrict__ yhat, long long n, double mu, double sd,
                                      double* __restrict__ V);

}  // namespace rsv
