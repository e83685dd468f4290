// mlp.cuh -- the surrogate network (dimensions, buffers, passes).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "mlp_gemm.cuh"

namespace rsv {

constexpr int MLP_IN = 32;   // feature width (padded)
constexpr int MLP_XW = 64;   // stored input width: each feature as a hi + lo BF16 pair
constexpr int MLP_H = 256;   // hidden width, 4 hidden layers

inline int mlp_in_dim(int l) { return l == 1 ? MLP_IN : MLP_H; }
// GEMM inner dimension of layer l: the first layer reads the hi and lo halves
// of every feature against the same (tied) weights, [W1; W1].
inline int mlp_k_dim(int l) { return l == 1 ? MLP_XW : MLP_H; }
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
    __nv_bfloat16* X = nullptr;     // batch features [cap][MLP_XW] (hi halves, then lo halves)
    float* dW1 = nullptr;           // [MLP_XW][MLP_H] weight gradient of the tied first layer
    float* Z[4] = {};               // pre-activations
    __nv_bfloat16* A[4] = {};       // activations
    float* A4f = nullptr;           // last hidden activations in FP32 (the head's input)
    float* dZf[4] = {};
    __nv_bfloat16* dZb[4] = {};
    float *y = nullptr, *t = nullptr, *dy = nullptr, *sq = nullptr, *loss = nullptr;
    float* part = nullptr;          // column-sum partials [cap / 128 + 1][MLP_H]
    __nv_bfloat16* wt = nullptr;    // W_l^T (K-major) BF16 copies for the tcgen05 inference kernel
    bool wt_fresh = false;          // wt matches params (cleared whenever the BF16 weights are refreshed)
    bool use_tc = true;             // inference on tcgen05 (else the mma.sync kernels)
    __nv_bfloat16* Xi = nullptr;    // inference-only features [cap_i][MLP_XW] (tcgen05 path)
    float* yi = nullptr;            // and outputs [cap_i]
    int cap_i = 0;

    cudaError_t ensure(int batch);
    cudaError_t ensure_infer(int batch);   // Xi, yi only: the tcgen05 path needs no activation buffers
    void release();
    __nv_bfloat16* wb(int l) const;
    cudaError_t refresh_bf16(cudaStream_t st);
    cudaError_t forward(const __nv_bfloat16* X, int B, float* y, const float* target, cudaStream_t st);
    cudaError_t backward(const __nv_bfloat16* X, int B, cudaStream_t st);
    cudaError_t adam_step(float lr, cudaStream_t st);
    // inference only: X [n][MLP_XW], n a multiple of 128, all four layers and
    // the head in one tcgen05 kernel (mlp_tc.cu)
    // trace_z / trace_a (optional, device): every layer's pre-activations
    // [4][n][256] FP32 and the BF16 operands of the next layer [3][n][256]
    // (2 gelu(z): the next layer's weights are staged halved)
    cudaError_t forward_tc(const __nv_bfloat16* X, int n, float* y, int sm_count, int32_t* status, cudaStream_t st,
                           float* trace_z = nullptr, void* trace_a = nullptr);
};

}  // namespace rsv
