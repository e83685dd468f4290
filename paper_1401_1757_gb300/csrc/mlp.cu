// mlp.cu -- the reserve surrogate network on sm_103a: a 32 -> 256 -> 256 ->
// 256 -> 256 -> 1 perceptron with GELU (tanh form), BF16 weights and
// activations, FP32 accumulation, FP32 master weights and Adam.
//
// Forward per layer l = 1..4:  Z_l = A_{l-1} W_l + b_l,  A_l = gelu(Z_l)
// (A_0 = features), head y = A_4 w5 + b5.  Loss: mean squared error.
// The activations the tensor cores read are BF16; the head reads the last
// hidden layer in FP32, since BF16 rounding of its 256 inputs alone would put
// ~1e-3 of noise on the output, the size of the surrogate's error target.
// Backward: dZ_4 = (dy w5^T) * gelu'(Z_4); for l = 4..1: dW_l = A_{l-1}^T dZ_l,
// db_l = column sums of dZ_l, dZ_{l-1} = (dZ_l W_l^T) * gelu'(Z_{l-1}).
// Every product runs on the tensor cores (mlp_gemm.cuh); sums over the batch
// are in a fixed order, so a step is deterministic.
#include <cmath>
#include <cstdint>
#include <vector>

#include "mlp.cuh"

namespace rsv {

// parameter offsets in the flat FP32 vector
size_t mlp_w_off(int l) {   // l = 1..4
    size_t o = 0;
    for (int i = 1; i < l; ++i) o += (size_t)mlp_in_dim(i) * MLP_H + MLP_H;
    return o;
}
size_t mlp_b_off(int l) { return mlp_w_off(l) + (size_t)mlp_in_dim(l) * MLP_H; }
size_t mlp_w5_off() { return mlp_w_off(5); }
size_t mlp_n_params() { return mlp_w5_off() + MLP_H + 1; }

namespace {

template <bool AK, bool BK, int EPI>
cudaError_t gemm(const GemmArgs& g, cudaStream_t st) {
    dim3 grid((g.N + GBN - 1) / GBN, (g.M + GBM - 1) / GBM);
    gemm_bf16_kernel<AK, BK, EPI><<<grid, GTHREADS, 0, st>>>(g);
    return cudaGetLastError();
}

// y[r] = A4[r] . w5 + b5; with a target: dy[r] = 2 (y - t) / B and the
// per-block sums of squared errors (fixed order).
__global__ void head_fwd_kernel(const float* __restrict__ A4, const float* __restrict__ w5,
                                const float* __restrict__ b5, int B, float* __restrict__ y,
                                const float* __restrict__ target, float* __restrict__ dy,
                                float* __restrict__ sq_part) {
    __shared__ float red[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * 8 + warp;
    float se = 0.0f;
    if (r < B) {
        float s = 0.0f;
        for (int k = lane; k < MLP_H; k += 32) s += A4[(size_t)r * MLP_H + k] * w5[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        s += b5[0];
        if (lane == 0) {
            if (y) y[r] = s;
            if (target) {
                const float e = s - target[r];
                dy[r] = 2.0f * e / (float)B;
                se = e * e;
            }
        }
    }
    if (lane == 0) red[warp] = se;
    __syncthreads();
    if (threadIdx.x == 0 && sq_part) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += red[w];
        sq_part[blockIdx.x] = t;
    }
}

// dZ4[r][k] = dy[r] w5[k] gelu'(Z4[r][k])
__global__ void head_bwd_kernel(const float* __restrict__ dy, const float* __restrict__ w5,
                                const float* __restrict__ Z4, int B, float* __restrict__ dZf,
                                __nv_bfloat16* __restrict__ dZb) {
    const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= (size_t)B * MLP_H) return;
    const int r = (int)(i / MLP_H), k = (int)(i % MLP_H);
    const float g = dy[r] * w5[k] * gelu_grad_f(Z4[i]);
    dZf[i] = g;
    dZb[i] = __float2bfloat16_rn(g);
}

// out[c] = sum_r X[r][c] * (wr ? wr[r] : 1) in two fixed-order passes: sums
// over chunks of kColsumRows rows (one thread per column and chunk), then
// over the chunks.
constexpr int kColsumRows = 128;

__global__ void colsum_partial_kernel(const float* __restrict__ X, const float* __restrict__ wr, int R, int C,
                                      float* __restrict__ part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
    if (c >= C) return;
    const int r1 = min(R, (ch + 1) * kColsumRows);
    float s = 0.0f;
    for (int r = ch * kColsumRows; r < r1; ++r) {
        const float x = X[(size_t)r * C + c];
        s += wr ? x * wr[r] : x;
    }
    part[(size_t)ch * C + c] = s;
}

__global__ void colsum_final_kernel(const float* __restrict__ part, int n_chunks, int C, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float s = 0.0f;
    for (int ch = 0; ch < n_chunks; ++ch) s += part[(size_t)ch * C + c];
    out[c] = s;
}

cudaError_t colsum(const float* X, const float* wr, int R, int C, float* part, float* out, cudaStream_t st) {
    const int n_chunks = (R + kColsumRows - 1) / kColsumRows;
    colsum_partial_kernel<<<dim3((C + 127) / 128, n_chunks), 128, 0, st>>>(X, wr, R, C, part);
    colsum_final_kernel<<<(C + 127) / 128, 128, 0, st>>>(part, n_chunks, C, out);
    return cudaGetLastError();
}

__global__ void sum_kernel(const float* __restrict__ x, int n, float* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.0f;
        for (int i = 0; i < n; ++i) s += x[i];
        out[0] = s;
    }
}

// Adam on the FP32 master weights; refresh the BF16 working copies.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// [W1; W1] in BF16 from the FP32 W1 [MLP_IN][MLP_H]
__global__ void tied_w1_kernel(const float* __restrict__ w1, __nv_bfloat16* __restrict__ y) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_IN * MLP_H; i += gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(w1[i]);
        y[i] = b;
        y[MLP_IN * MLP_H + i] = b;
    }
}

// dW1 = dW1' (hi rows) + dW1' (lo rows): the gradient of tied weights
__global__ void fold_dw1_kernel(const float* __restrict__ dw, float* __restrict__ g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_IN * MLP_H; i += gridDim.x * blockDim.x)
        g[i] = dw[i] + dw[MLP_IN * MLP_H + i];
}

}  // namespace

cudaError_t Mlp::ensure(int batch) {
    if (batch <= cap) return cudaSuccess;
    const size_t B = (size_t)batch;
    const size_t P = mlp_n_params();
    cudaError_t e;
#define ALLOC(ptr, bytes)                                       \
    do {                                                        \
        if (ptr) cudaFree(ptr);                                 \
        e = cudaMalloc((void**)&ptr, (bytes));                  \
        if (e != cudaSuccess) return e;                         \
    } while (0)
    if (!params) {
        ALLOC(params, P * 4);
        ALLOC(grads, P * 4);
        ALLOC(adam_m, P * 4);
        ALLOC(adam_v, P * 4);
        ALLOC(wbf, (size_t)MLP_XW * MLP_H * 2 + 3 * (size_t)MLP_H * MLP_H * 2);
        ALLOC(dW1, (size_t)MLP_XW * MLP_H * 4);
        cudaMemset(adam_m, 0, P * 4);
        cudaMemset(adam_v, 0, P * 4);
    }
    ALLOC(X, B * MLP_XW * 2);
    for (int l = 0; l < 4; ++l) {
        ALLOC(Z[l], B * MLP_H * 4);
        ALLOC(A[l], B * MLP_H * 2);
        ALLOC(dZf[l], B * MLP_H * 4);
        ALLOC(dZb[l], B * MLP_H * 2);
    }
    ALLOC(A4f, B * MLP_H * 4);
    ALLOC(y, B * 4);
    ALLOC(t, B * 4);
    ALLOC(dy, B * 4);
    ALLOC(sq, (B / 8 + 1) * 4);
    ALLOC(part, (B / 128 + 1) * MLP_H * 4);
    ALLOC(loss, 4);
#undef ALLOC
    cap = batch;
    return cudaSuccess;
}

cudaError_t Mlp::ensure_infer(int batch) {
    if (batch <= cap_i) return cudaSuccess;
    if (Xi) cudaFree(Xi);
    if (yi) cudaFree(yi);
    Xi = nullptr;
    yi = nullptr;
    cap_i = 0;
    cudaError_t e = cudaMalloc((void**)&Xi, (size_t)batch * MLP_XW * 2);
    if (e != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&yi, (size_t)batch * 4)) != cudaSuccess) return e;
    cap_i = batch;
    return cudaSuccess;
}

void Mlp::release() {
    void* ps[] = {params, grads, adam_m, adam_v, wbf, dW1, A4f, X, y, t, dy, sq, loss, wt, part, Xi, yi};
    for (void* p : ps)
        if (p) cudaFree(p);
    for (int l = 0; l < 4; ++l) {
        if (Z[l]) cudaFree(Z[l]);
        if (A[l]) cudaFree(A[l]);
        if (dZf[l]) cudaFree(dZf[l]);
        if (dZb[l]) cudaFree(dZb[l]);
    }
    *this = Mlp();
}

__nv_bfloat16* Mlp::wb(int l) const {   // BF16 copy of W_l as the GEMM reads it, [k][H]
    size_t o = 0;
    for (int i = 1; i < l; ++i) o += (size_t)mlp_k_dim(i) * MLP_H;
    return wbf + o;
}

cudaError_t Mlp::refresh_bf16(cudaStream_t st) {
    wt_fresh = false;
    tied_w1_kernel<<<32, 256, 0, st>>>(params + mlp_w_off(1), wb(1));
    for (int l = 2; l <= 4; ++l) {
        const size_t n = (size_t)MLP_H * MLP_H;
        to_bf16_kernel<<<64, 256, 0, st>>>(params + mlp_w_off(l), wb(l), n);
    }
    return cudaGetLastError();
}

// X (BF16 [B][32], batch a multiple of 64) -> y; with `target`, also the loss
// (mean squared error) and dy.
cudaError_t Mlp::forward(const __nv_bfloat16* Xin, int B, float* yout, const float* target, cudaStream_t st) {
    cudaError_t e;
    const __nv_bfloat16* in = Xin;
    for (int l = 1; l <= 4; ++l) {
        GemmArgs g{};
        g.A = in;
        g.B = wb(l);
        g.M = B;
        g.N = MLP_H;
        g.K = mlp_k_dim(l);
        g.lda = g.K;
        g.ldb = MLP_H;
        g.Cf = Z[l - 1];
        g.Cb = A[l - 1];
        g.bias = params + mlp_b_off(l);
        g.Af = l == 4 ? A4f : nullptr;
        if ((e = gemm<true, false, EPI_BIAS_GELU>(g, st)) != cudaSuccess) return e;
        in = A[l - 1];
    }
    head_fwd_kernel<<<(B + 7) / 8, 256, 0, st>>>(A4f, params + mlp_w5_off(), params + mlp_w5_off() + MLP_H, B,
                                                  yout, target, dy, target ? sq : nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (target) {
        sum_kernel<<<1, 32, 0, st>>>(sq, (B + 7) / 8, loss);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Gradients of the mean squared error of the last forward(X, B, ., target).
cudaError_t Mlp::backward(const __nv_bfloat16* Xin, int B, cudaStream_t st) {
    cudaError_t e;
    const size_t w5 = mlp_w5_off();
    if ((e = colsum(A4f, dy, B, MLP_H, part, grads + w5, st)) != cudaSuccess) return e;
    if ((e = colsum(dy, nullptr, B, 1, part, grads + w5 + MLP_H, st)) != cudaSuccess) return e;
    head_bwd_kernel<<<(unsigned)(((size_t)B * MLP_H + 255) / 256), 256, 0, st>>>(dy, params + w5, Z[3], B, dZf[3],
                                                                                 dZb[3]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int l = 4; l >= 1; --l) {
        const int K = mlp_k_dim(l);
        // dW_l = A_{l-1}^T dZ_l : A operand stored [B][K] = [k][m]; B operand dZ_l stored [B][H] = [k][n]
        GemmArgs g{};
        g.A = l > 1 ? A[l - 2] : Xin;
        g.B = dZb[l - 1];
        g.M = K;
        g.N = MLP_H;
        g.K = B;
        g.lda = K;
        g.ldb = MLP_H;
        g.Cf = l > 1 ? grads + mlp_w_off(l) : dW1;
        if ((e = gemm<false, false, EPI_F32>(g, st)) != cudaSuccess) return e;
        if (l == 1) {
            fold_dw1_kernel<<<32, 256, 0, st>>>(dW1, grads + mlp_w_off(1));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if ((e = colsum(dZf[l - 1], nullptr, B, MLP_H, part, grads + mlp_b_off(l), st)) != cudaSuccess) return e;
        if (l > 1) {
            // dZ_{l-1} = (dZ_l W_l^T) * gelu'(Z_{l-1}) : B operand W_l stored [K][H] = [n][k]
            GemmArgs h{};
            h.A = dZb[l - 1];
            h.B = wb(l);
            h.M = B;
            h.N = K;
            h.K = MLP_H;
            h.lda = MLP_H;
            h.ldb = MLP_H;
            h.Cf = dZf[l - 2];
            h.Cb = dZb[l - 2];
            h.Zin = Z[l - 2];
            if ((e = gemm<true, true, EPI_GELU_BWD>(h, st)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

cudaError_t Mlp::adam_step(float lr, cudaStream_t st) {
    ++step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)step), c2 = 1.0f - std::pow(b2, (float)step);
    adam_kernel<<<256, 256, 0, st>>>(params, grads, adam_m, adam_v, mlp_n_params(), lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return refresh_bf16(st);
}

}  // namespace rsv
