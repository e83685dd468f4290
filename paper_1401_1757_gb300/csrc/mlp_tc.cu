// mlp_tc.cu -- surrogate inference on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in TMEM, operands staged by TMA).
//
// One CTA (16 warps) runs the whole network on 128-row tiles of queries:
//   for l = 1..4:  D = A_{l-1} . W_l  (tcgen05.mma m128 n256 k16, FP32 in TMEM)
//                  A_l = gelu(D + b_l) (BF16, written back into shared memory as
//                  the next layer's A operand)
//   y = gelu(D_4 + b_4) . w5 + b5     (FP32 head from the TMEM accumulator)
// A and W^T are K-major BF16 tiles in shared memory with the 128-byte swizzle
// (TMA writes them; the epilogue writes A_l with the same pattern).  A warp
// may only read its own quarter of the TMEM lanes, so warp w reads lanes
// 32 (w % 4) .. +31 (rows of the tile) and columns 64 (w / 4) .. +63: four
// warps per lane quarter share the epilogue.  Thread 0 issues the TMA copies
// and the MMAs.  Every mbarrier wait is bounded; on a timeout the kernel
// records it in the status word, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "mlp.cuh"
#include "rsv_device.cuh"

namespace rsv {
namespace {

constexpr int TM = 128;                         // rows per tile (MMA M)
constexpr int TN = MLP_H;                       // MMA N = 256
constexpr int SLAB_K = 64;                      // K elements per 128-byte swizzle row
constexpr int A_SLAB = TM * 128;                // 16 KiB
constexpr int W_SLAB = TN * 128;                // 32 KiB
constexpr int A_BYTES = 4 * A_SLAB;             // 64 KiB (K = 256)
constexpr int W_BYTES = 4 * W_SLAB;             // 128 KiB
constexpr uint32_t kPoll = 1u << 24;
constexpr int kThreads = 512;                   // 16 warps: 4 lane quarters x 4 column groups
constexpr int kColsPerWarp = TN / 4;            // 64

struct TcArgs {
    const float* bias[4];
    const float* w5;      // [256] then b5
    float* y;             // [n_rows]
    int n_tiles;
    int32_t* status;
};

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t sw128_desc(const void* smem) {
    const uint64_t addr = smem_u32(smem);
    uint64_t d = 0;
    d |= (addr >> 4) & 0x3FFFull;            // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                  // descriptor version (tcgen05)
    d |= (uint64_t)2 << 61;                  // layout: 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both
// K-major, M = 128, N = 256.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Byte offset of element (row, k) in a K-major, 128-byte-swizzled operand made
// of 64-column slabs of `rows` rows.
__device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
    const int slab = k >> 6, kc = k & 63;
    const int chunk = (kc >> 3) ^ (row & 7);
    return slab * rows * 128 + row * 128 + chunk * 16 + (kc & 7) * 2;
}

// ---- the kernel -------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1)
    mlp_fwd_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapW1,
                      const __grid_constant__ CUtensorMap mapW2, const __grid_constant__ CUtensorMap mapW3,
                      const __grid_constant__ CUtensorMap mapW4, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* Abuf = base;
    unsigned char* Wbuf = base + A_BYTES;
    __shared__ uint64_t bar_x, bar_w, bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ float head_part[4][TM];   // partial head sums per column group
    __shared__ float bias_s[4][TN];      // b_1..b_4
    __shared__ float w5_s[TN + 1];       // head weights and bias

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 4 * TN; i += kThreads) bias_s[i / TN][i % TN] = a.bias[i / TN][i % TN];
    for (int i = tid; i <= TN; i += kThreads) w5_s[i] = a.w5[i];
    if (tid == 0) {
        mbar_init(&bar_x, 1);
        mbar_init(&bar_w, 1);
        mbar_init(&bar_mma, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    const CUtensorMap* maps[4] = {&mapW1, &mapW2, &mapW3, &mapW4};
    uint32_t ph_x = 0, ph_w = 0, ph_m = 0;
    bool failed = false;

    auto wait = [&](uint64_t* bar, uint32_t& ph) {
        bool ok = mbar_wait_bounded(bar, ph, kPoll);
        ph ^= 1u;
        ok = __syncthreads_and(ok);
        return ok;
    };

    for (int tile = blockIdx.x; tile < a.n_tiles && !failed; tile += gridDim.x) {
        if (tid == 0) {
            mbar_arrive_expect_tx(&bar_x, TM * 128);
            tma_load_2d(Abuf, &mapX, 0, tile * TM, &bar_x);
            mbar_arrive_expect_tx(&bar_w, TN * 128);
            tma_load_2d(Wbuf, &mapW1, 0, 0, &bar_w);
        }
        if (!wait(&bar_x, ph_x)) { failed = true; break; }
        for (int l = 0; l < 4; ++l) {
            if (!wait(&bar_w, ph_w)) { failed = true; break; }
            const int kslabs = l == 0 ? 1 : 4;
            if (tid == 0) {
                fence_after();
                for (int s = 0; s < kslabs; ++s)
                    for (int kk = 0; kk < 4; ++kk)   // 4 x k16 per 64-wide slab: +32 bytes each
                        mma_f16(tmem, sw128_desc(Abuf + s * A_SLAB + kk * 32), sw128_desc(Wbuf + s * W_SLAB + kk * 32),
                                (s | kk) != 0);
                mma_commit(&bar_mma);
            }
            if (!wait(&bar_mma, ph_m)) { failed = true; break; }
            fence_after();
            if (tid == 0 && l < 3) {   // the MMAs are done with Wbuf: fetch the next layer's weights
                mbar_arrive_expect_tx(&bar_w, 4 * W_SLAB);
                for (int s = 0; s < 4; ++s) tma_load_2d(Wbuf + s * W_SLAB, maps[l + 1], s * SLAB_K, 0, &bar_w);
            }
            // epilogue: row = 32 (warp % 4) + lane, columns 64 (warp / 4) .. +63 in chunks of 32
            const int quarter = warp & 3, cgrp = warp >> 2;
            const int row = quarter * 32 + lane;
            const float* bias = bias_s[l];
            float ysum = 0.0f;
            for (int c0 = cgrp * kColsPerWarp; c0 < (cgrp + 1) * kColsPerWarp; c0 += 32) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + c0, v);
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = gelu_f(v[i] + bias[c0 + i]);
                if (l < 3) {
#pragma unroll
                    for (int i = 0; i < 32; i += 8) {
                        const uint4 pk = make_uint4(pack_bf16x2(v[i], v[i + 1]), pack_bf16x2(v[i + 2], v[i + 3]),
                                                    pack_bf16x2(v[i + 4], v[i + 5]), pack_bf16x2(v[i + 6], v[i + 7]));
                        *reinterpret_cast<uint4*>(Abuf + sw128_off(row, c0 + i, TM)) = pk;
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) ysum += v[i] * w5_s[c0 + i];
                }
            }
            if (l == 3) {   // uniform across the block
                head_part[cgrp][row] = ysum;
                __syncthreads();
                if (cgrp == 0)
                    a.y[tile * TM + row] =
                        ((head_part[0][row] + head_part[1][row]) + (head_part[2][row] + head_part[3][row])) + w5_s[TN];
            }
            fence_before();
            fence_async_smem();   // A_l written by the generic proxy, read next by the tensor cores
            __syncthreads();
            fence_after();
        }
    }
    if (failed) {
        // let copies and products still in flight land before the memory is released
        if (tid == 0) atomicExch(a.status, DEV_TIMEOUT);
        mbar_wait_bounded(&bar_x, ph_x, kPoll);
        mbar_wait_bounded(&bar_w, ph_w, kPoll);
        mbar_wait_bounded(&bar_mma, ph_m, kPoll);
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
}

// ---- host: tensor maps through the driver entry point ---------------------
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    static EncodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPoint("cuTensorMapEncodeTiled", &p, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// 2-D BF16 map over [rows][cols] (cols contiguous), box 64 columns x box_rows,
// 128-byte swizzle.
bool make_map(CUtensorMap* m, const void* ptr, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    EncodeTiled enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {SLAB_K, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// W_l^T (K-major, [256][K]) BF16 copies for the tensor cores
__global__ void transpose_w_kernel(const float* __restrict__ W, int K, __nv_bfloat16* __restrict__ Wt, bool tied) {
    // W [K_in][256] FP32 (K_in = 32 for the tied first layer) -> Wt [256][K]
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * MLP_H; i += gridDim.x * blockDim.x) {
        const int n = i / K, k = i % K;
        const int kin = tied ? (k % MLP_IN) : k;
        Wt[i] = __float2bfloat16_rn(W[(size_t)kin * MLP_H + n]);
    }
}

}  // namespace

// Inference of rows [0, n) of X (BF16 [n][MLP_XW], n a multiple of 128) into
// y (FP32 [n]) on the tensor cores.  Returns cudaErrorNotSupported when the
// tensor-map encoder is unavailable.
cudaError_t Mlp::forward_tc(const __nv_bfloat16* Xin, int n, float* yout, int sm_count, int32_t* status,
                            cudaStream_t st) {
    if (n % TM) return cudaErrorInvalidValue;
    cudaError_t e;
    if (!wt) {
        if ((e = cudaMalloc((void**)&wt, (size_t)(MLP_XW + 3 * MLP_H) * MLP_H * 2)) != cudaSuccess) return e;
    }
    // refresh the transposed weights (cheap: 200k elements)
    transpose_w_kernel<<<64, 256, 0, st>>>(params + mlp_w_off(1), MLP_XW, wt, true);
    for (int l = 2; l <= 4; ++l)
        transpose_w_kernel<<<128, 256, 0, st>>>(params + mlp_w_off(l), MLP_H,
                                                wt + (size_t)(MLP_XW + (l - 2) * MLP_H) * MLP_H, false);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap mx, mw[4];
    if (!make_map(&mx, Xin, MLP_XW, n, TM) || !make_map(&mw[0], wt, MLP_XW, MLP_H, MLP_H))
        return cudaErrorNotSupported;
    for (int l = 1; l < 4; ++l)
        if (!make_map(&mw[l], wt + (size_t)(MLP_XW + (l - 1) * MLP_H) * MLP_H, MLP_H, MLP_H, MLP_H))
            return cudaErrorNotSupported;
    TcArgs a;
    for (int l = 0; l < 4; ++l) a.bias[l] = params + mlp_b_off(l + 1);
    a.w5 = params + mlp_w5_off();
    a.y = yout;
    a.n_tiles = n / TM;
    a.status = status;
    const size_t smem = A_BYTES + W_BYTES + 1024;
    if ((e = cudaFuncSetAttribute(mlp_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const int grid = std::min(a.n_tiles, sm_count);
    mlp_fwd_tc_kernel<<<grid, kThreads, smem, st>>>(mx, mw[0], mw[1], mw[2], mw[3], a);
    return cudaGetLastError();
}

}  // namespace rsv
