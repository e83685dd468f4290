// mlp.cuh -- the surrogate network (dimensions, buffers, passes).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mlp_gemm.cuh"

namespace rsv {

constexpr int MLP_IN = 32;   // feature width (padded)
constexpr int MLP_H = 256;   // hidden width, 4 hidden layers

inline int mlp_in_dim(int l) { return l == 1 ? MLP_IN : MLP_H; }
size_t mlp_w_off(int l);     // offset of W_l ([in][H], row-major) in the flat FP32 parameters, l = 1..5
size_t mlp_b_off(int l);     // offset of b_l [H]
size_t mlp_w5_off();         // head weights w5 [H], then b5 [1]
size_t mlp_n_params();

struct Mlp {
    float* params = nullptr;  // FP32 master weights (flat)
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    __nv_bfloat16* wbf = nullptr;   // BF16 W_1..W_4
    int cap = 0;                    // rows the activation buffers hold
    int step = 0;                   // Adam steps taken
    __nv_bfloat16* X = nullptr;     // batch features [cap][MLP_IN]
    float* Z[4] = {};               // pre-activations
    __nv_bfloat16* A[4] = {};       // activations
    float* dZf[4] = {};
    __nv_bfloat16* dZb[4] = {};
    float *y = nullptr, *t = nullptr, *dy = nullptr, *sq = nullptr, *loss = nullptr;

    cudaError_t ensure(int batch);
    void release();
    __nv_bfloat16* wb(int l) const;
    cudaError_t refresh_bf16(cudaStream_t st);
    cudaError_t forward(const __nv_bfloat16* X, int B, float* y, const float* target, cudaStream_t st);
    cudaError_t backward(const __nv_bfloat16* X, int B, cudaStream_t st);
    cudaError_t adam_step(float lr, cudaStream_t st);
};

}  // namespace rsv
