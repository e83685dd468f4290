// mlp_gemm.cuh -- BF16 tensor-core GEMM with FP32 accumulation for the
// reserve surrogate MLP (sm_103a, mma.sync.m16n8k16).
//
//   C[M x N] = A[M x K] . B[K x N]
//
// A is stored row-major ("K-major", [M][K]) or column-major ([K][M]); B is
// stored [K][N] or [N][K].  Tiles are copied to shared memory as stored
// (cp.async, double-buffered) and the transposition, where needed, happens in
// ldmatrix(.trans), so the forward (X . W), input-gradient (dZ . W^T) and
// weight-gradient (X^T . dZ) products all run without a transposed copy.
// M, N and K must be multiples of 32; tiles past M or N are masked.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace rsv {

enum GemmEpi : int {
    EPI_F32 = 0,        // Cf = acc
    EPI_BIAS_GELU = 1,  // Z = acc + bias (FP32, optional), A = gelu(Z) (BF16)
    EPI_GELU_BWD = 2    // G = acc * gelu'(Zin) (FP32 and BF16)
};

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int M, N, K;
    int lda, ldb;            // leading dimensions as stored
    float* Cf;               // FP32 output [M][N] (EPI_F32, EPI_BIAS_GELU: Z, EPI_GELU_BWD: G)
    __nv_bfloat16* Cb;       // BF16 output [M][N] (activations or gradients)
    const float* bias;       // [N] (EPI_BIAS_GELU)
    float* Af;               // FP32 activations [M][N] (EPI_BIAS_GELU, optional)
    const float* Zin;        // [M][N] pre-activations (EPI_GELU_BWD)
};

// GELU in the tanh form of Hendrycks & Gimpel (2016),
//   gelu(z) = z (1 + tanh(u)) / 2,  u = sqrt(2/pi) (z + 0.044715 z^3),
// within 5e-4 of z Phi(z), and its derivative
//   (1 + t) / 2 + z (1 - t^2) u' / 2,  u' = sqrt(2/pi) (1 + 3 0.044715 z^2).
// tanh is the hardware approximation (one MUFU operation, relative error
// about 2^-11, below the BF16 rounding of the activations).  Training and
// inference share these two functions.
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kGeluC = 0.7978845608028654f;              // sqrt(2/pi)
constexpr float kGeluCK = 0.7978845608028654f * 0.044715f;  // sqrt(2/pi) 0.044715
__device__ __forceinline__ float gelu_f(float z) {
    const float z2 = z * z;
    const float t = tanh_hw(z * fmaf(kGeluCK, z2, kGeluC));
    const float h = 0.5f * z;
    return fmaf(h, t, h);
}
__device__ __forceinline__ float gelu_grad_f(float z) {
    const float z2 = z * z;
    const float t = tanh_hw(z * fmaf(kGeluCK, z2, kGeluC));
    const float du = fmaf(3.0f * kGeluCK, z2, kGeluC);
    return fmaf(0.5f * z * du, fmaf(-t, t, 1.0f), 0.5f * (1.0f + t));
}

__device__ __forceinline__ uint32_t cvta_smem(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool pred) {
    const int n = pred ? 16 : 0;   // zero-fill when the source is masked
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(cvta_smem(smem)), "l"(gmem), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(cvta_smem(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(cvta_smem(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 64 x 64 x 32 tiles, 4 warps (2 x 2), warp tile 32 x 32 (2 x 4 mma tiles).
constexpr int GBM = 64, GBN = 64, GBK = 32, GTHREADS = 128;
constexpr int PAD = 8;   // bf16 elements of row padding (16 B) against bank conflicts

template <bool A_KMAJOR, bool B_KMAJOR, int EPI>
__global__ void __launch_bounds__(GTHREADS) gemm_bf16_kernel(const GemmArgs g) {
    // shared tiles, as stored: A [GBM][GBK] or [GBK][GBM]; B [GBN][GBK] or [GBK][GBN]
    constexpr int A_ROWS = A_KMAJOR ? GBM : GBK, A_COLS = A_KMAJOR ? GBK : GBM;
    constexpr int B_ROWS = B_KMAJOR ? GBN : GBK, B_COLS = B_KMAJOR ? GBK : GBN;
    __shared__ __align__(16) __nv_bfloat16 As[2][A_ROWS][A_COLS + PAD];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][B_ROWS][B_COLS + PAD];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

    auto load_tile = [&](int buf, int k0) {
        // A: 64 x 32 elements = 256 chunks of 8
#pragma unroll
        for (int c = tid; c < (GBM * GBK) / 8; c += GTHREADS) {
            if constexpr (A_KMAJOR) {
                const int r = c / (GBK / 8), col = (c % (GBK / 8)) * 8;
                const bool ok = m0 + r < g.M;
                cp_async16(&As[buf][r][col], g.A + (size_t)(ok ? m0 + r : 0) * g.lda + k0 + col, ok);
            } else {
                const int r = c / (GBM / 8), col = (c % (GBM / 8)) * 8;
                const bool ok = m0 + col < g.M;
                cp_async16(&As[buf][r][col], g.A + (size_t)(k0 + r) * g.lda + (ok ? m0 + col : 0), ok);
            }
        }
#pragma unroll
        for (int c = tid; c < (GBN * GBK) / 8; c += GTHREADS) {
            if constexpr (B_KMAJOR) {
                const int r = c / (GBK / 8), col = (c % (GBK / 8)) * 8;
                const bool ok = n0 + r < g.N;
                cp_async16(&Bs[buf][r][col], g.B + (size_t)(ok ? n0 + r : 0) * g.ldb + k0 + col, ok);
            } else {
                const int r = c / (GBN / 8), col = (c % (GBN / 8)) * 8;
                const bool ok = n0 + col < g.N;
                cp_async16(&Bs[buf][r][col], g.B + (size_t)(k0 + r) * g.ldb + (ok ? n0 + col : 0), ok);
            }
        }
        cp_async_commit();
    };

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.0f;

    const int nk = g.K / GBK;
    load_tile(0, 0);
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            load_tile(buf ^ 1, (kt + 1) * GBK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[2][4], bf[2][4];
            const int r8 = lane & 7, j = lane >> 3;
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int mb = wm + mi * 16;
                if constexpr (A_KMAJOR) {
                    ldsm_x4(af[mi], &As[buf][mb + (lane & 15)][kk + (lane >> 4) * 8]);
                } else {   // stored [k][m]: matrices (k0,m0) (k0,m8) (k8,m0) (k8,m8), transposed
                    ldsm_x4_t(af[mi], &As[buf][kk + (j >> 1) * 8 + r8][mb + (j & 1) * 8]);
                }
            }
#pragma unroll
            for (int ni = 0; ni < 2; ++ni) {   // each x4 covers n16 x k16 (two n8 tiles)
                const int nb = wn + ni * 16;
                if constexpr (B_KMAJOR) {   // stored [n][k]: (n0,k0) (n0,k8) (n8,k0) (n8,k8)
                    ldsm_x4(bf[ni], &Bs[buf][nb + (j >> 1) * 8 + r8][kk + (j & 1) * 8]);
                } else {                    // stored [k][n]: (k0,n0) (k8,n0) (k0,n8) (k8,n8), transposed
                    ldsm_x4_t(bf[ni], &Bs[buf][kk + (j & 1) * 8 + r8][nb + (j >> 1) * 8]);
                }
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 2; ++ni) {
                    mma_bf16(acc[mi][ni * 2 + 0], af[mi], bf[ni][0], bf[ni][1]);
                    mma_bf16(acc[mi][ni * 2 + 1], af[mi], bf[ni][2], bf[ni][3]);
                }
        }
        __syncthreads();
    }

    // epilogue: accumulator (row = lane/4 (+8), col = 2*(lane%4) + {0,1})
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int row = m0 + wm + mi * 16 + (lane >> 2) + h * 8;
                const int col = n0 + wn + nj * 8 + (lane & 3) * 2;
                if (row >= g.M || col >= g.N) continue;
                float v0 = acc[mi][nj][h * 2 + 0], v1 = acc[mi][nj][h * 2 + 1];
                const size_t o = (size_t)row * g.N + col;
                if constexpr (EPI == EPI_F32) {
                    *reinterpret_cast<float2*>(g.Cf + o) = make_float2(v0, v1);
                } else if constexpr (EPI == EPI_BIAS_GELU) {
                    v0 += g.bias[col];
                    v1 += g.bias[col + 1];
                    if (g.Cf) *reinterpret_cast<float2*>(g.Cf + o) = make_float2(v0, v1);
                    const float a0 = gelu_f(v0), a1 = gelu_f(v1);
                    *reinterpret_cast<__nv_bfloat162*>(g.Cb + o) = __floats2bfloat162_rn(a0, a1);
                    if (g.Af) *reinterpret_cast<float2*>(g.Af + o) = make_float2(a0, a1);
                } else {
                    const float2 z = *reinterpret_cast<const float2*>(g.Zin + o);
                    v0 *= gelu_grad_f(z.x);
                    v1 *= gelu_grad_f(z.y);
                    if (g.Cf) *reinterpret_cast<float2*>(g.Cf + o) = make_float2(v0, v1);
                    *reinterpret_cast<__nv_bfloat162*>(g.Cb + o) = __floats2bfloat162_rn(v0, v1);
                }
            }
}

}  // namespace rsv
