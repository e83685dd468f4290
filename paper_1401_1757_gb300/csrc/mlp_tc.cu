// mlp_tc.cu -- surrogate inference on the 5th-generation tensor cores
// (tcgen05.mma, accumulators and activations in TMEM, operands staged by TMA).
//
// One CTA runs the whole network on 128-row tiles of queries, two tiles at a
// time.  Every layer is split into two N = 128 halves, h = 0, 1:
//   D = A_{l-1} . W_l[:, half h]   (tcgen05.mma m128 n128 k16, FP32 in TMEM)
//   A_l[:, half h] = 2 gelu(D + b_l) (BF16, written back into TMEM by tcgen05.st
//                                   as the next layer's A operand; the next
//                                   layer's weights are staged as W / 2)
//   y = 2 gelu(D_4 + b_4) . (w5 / 2) + b5  (FP32 head from the TMEM accumulators)
// The first layer reads its A operand (the query features X) from shared
// memory; the later ones read A from TMEM, two BF16 values per 32-bit column,
// the even K index in the low half.  Each of the two tiles in flight (slots)
// owns 128 accumulator columns and 128 activation columns of TMEM, so the
// tensor cores work on one slot while the epilogue drains the other (see the
// kernel).  Warp 16 (one thread) issues the products, warp 17 (one thread)
// the TMA copies; warps 0-15 run the epilogue: warp w may only touch TMEM lanes 32 (w % 4) ..
// +31 (the rows of the tile), and takes columns 32 (w / 4) .. +31 of each
// half.  Every mbarrier wait is bounded; on a timeout the kernel records it in
// the status word, skips the later waits, lets the copies and products in
// flight land, frees its TMEM and returns.
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
constexpr int TN = MLP_H;                       // layer width 256
constexpr int NH = TN / 2;                      // MMA N = 128 (one half of a layer)
constexpr int SLAB_K = 64;                      // K elements per 128-byte swizzle row
constexpr int X_BYTES = TM * 128;               // 16 KiB: the features, K = 64
constexpr int WH_SLAB = NH * 128;               // 16 KiB: one K slab of one half of W_l^T
constexpr int W_SLAB = 2 * WH_SLAB;             // 32 KiB: both halves of one K slab
constexpr int W_BYTES = 4 * W_SLAB;             // 128 KiB (K = 256)
constexpr uint32_t kPoll = 1u << 24;
constexpr int kEpiWarps = 16;                   // 4 lane quarters x 4 column groups
constexpr int kThreads = 32 * (kEpiWarps + 2);  // + the issuing warp and the staging warp
constexpr uint32_t kTmemCols = 512;
// TMEM columns of slot s: its accumulator at 256 s, its activation buffer at 256 s + 128
__device__ __forceinline__ uint32_t dcol_of(int s) { return 256u * (uint32_t)s; }
__device__ __forceinline__ uint32_t acol_of(int s) { return 256u * (uint32_t)s + 128u; }

struct TcArgs {
    const float* bias[4];
    const float* w5;      // [256] then b5
    float* y;             // [n_rows]
    int n_tiles;
    int32_t* status;
    // layer-by-layer test output, or null: pre-activations z = D + b of every
    // layer [4][n_rows][256] and the BF16 operands written to TMEM for the next
    // layer, 2 gelu(z), [3][n_rows][256]
    float* trace_z;
    uint32_t* trace_a;    // BF16 pairs
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
// K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NH >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

// D (TMEM) [+]= A . B with A from shared memory
__device__ __forceinline__ void mma_ss(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accum)
        : "memory");
}
// D (TMEM) [+]= A . B with A from tensor memory
__device__ __forceinline__ void mma_ts(uint32_t tmem, uint32_t a_tmem, uint64_t b, uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem),
        "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 columns of this warp's 32 lanes from TMEM, without waiting: the values
// may be used only after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// Wait for this thread's TMEM loads; the registers pass through an empty asm
// after the wait, so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) asm volatile("" : "+r"(r[i]));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// 2 gelu(z) in the tanh form, z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))), of
// z = acc + bias for two columns at once.  The factor 1/2 of gelu is carried
// by the next layer's weights (and the head's), which saves a multiply per
// element; powers of two scale BF16 and FP32 exactly.  The arithmetic runs in
// packed FP32 pairs (each half rounded as the scalar instruction rounds, in
// half the issue slots); tanh.approx stays scalar.
__device__ __forceinline__ void bias_gelu2_x2(float& z0, float& z1, float b0, float b1, f32x2 cK, f32x2 cC) {
    const f32x2 z = x2_add(x2_pack(z0, z1), x2_pack(b0, b1));
    float u0, u1;
    x2_unpack(x2_mul(z, x2_fma(cK, x2_mul(z, z), cC)), u0, u1);
    x2_unpack(x2_fma(z, x2_pack(tanh_hw(u0), tanh_hw(u1)), z), z0, z1);
}

// 8 columns of this warp's 32 lanes from registers into TMEM; with WAIT, waits for completion
template <bool WAIT = true>
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
    if (WAIT) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- the kernel -------------------------------------------------------------
// Two tiles in flight per CTA (slots s = 0, 1): slot s has one accumulator of
// 128 TMEM columns (dcol_of(s)) and one activation buffer of 128 columns
// (acol_of(s): K = 256 BF16).  The products run step by step in the order
// (s, h) = (0, 0), (1, 0), (0, 1), (1, 1) of every layer, so that the epilogue
// of one slot runs while the other slot's products run:
//   products (s, l, 0): D_s = A_s(l-1) . W_l[:, 0:128]
//   epilogue (s, l, 0): D_s into registers as the BF16 of 2 gelu(z + b), held;
//                       D_s is released
//   products (s, l, 1): D_s = A_s(l-1) . W_l[:, 128:256]
//   epilogue (s, l, 1): D_s into registers; A_s(l-1) is read no more, so both
//                       halves of A_s(l) are written into TMEM; the slot is
//                       released for layer l + 1
// Layer 4's epilogue feeds the head.  W_l is staged per half (K-major,
// 128-byte swizzle); half h is refilled with the next layer's once both
// slots' products on it are done, which the issuing thread checks only after
// it has queued the next step's products.  A pair's second tile may lie past
// the last one: its features load as zeros and it writes nothing.
// TRACE: also write the traced layer values (a.trace_z, a.trace_a).
template <bool TRACE>
__global__ void __launch_bounds__(kThreads, 1)
    mlp_fwd_tc_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapW1,
                      const __grid_constant__ CUtensorMap mapW2, const __grid_constant__ CUtensorMap mapW3,
                      const __grid_constant__ CUtensorMap mapW4, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzle atoms
    unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* Xbuf = base;                  // slot s at s * X_BYTES
    unsigned char* Wbuf = base + 2 * X_BYTES;    // K slab k, half h at k * W_SLAB + h * WH_SLAB
    // bar_m0: the products of one step of slot 0 are done; bar_m1[h]: those of
    // slot 1 on weight half h (and every product issued before them); bar_dfree[s]:
    // the epilogue (s, l, 0) has read D_s; bar_act[s]: the epilogue (s, l, 1) is done
    __shared__ uint64_t bar_x[2], bar_w[2], bar_m0, bar_m1[2], bar_dfree[2], bar_act[2];
    __shared__ uint32_t tmem_slot;
    __shared__ float head_part[2][4][TM];              // partial head sums per slot and column group
    __shared__ __align__(16) float bias_s[4][TN];      // b_1..b_4
    __shared__ __align__(16) float w5_s[TN + 4];       // head weights and bias

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 4 * TN; i += kThreads) bias_s[i / TN][i % TN] = a.bias[i / TN][i % TN];
    for (int i = tid; i <= TN; i += kThreads) w5_s[i] = i < TN ? 0.5f * a.w5[i] : a.w5[i];   // w5 / 2, then b5
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bar_x[i], 1);
            mbar_init(&bar_w[i], 1);
            mbar_init(&bar_m1[i], 1);
            mbar_init(&bar_dfree[i], kEpiWarps);   // one arrival per epilogue warp
            mbar_init(&bar_act[i], kEpiWarps);
        }
        mbar_init(&bar_m0, 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;
    // pairs of tiles: this CTA takes pairs blockIdx.x + p gridDim.x, pair P holding
    // tiles 2P and 2P + 1; step g = 4 p + l - 1 (every barrier below completes a
    // fixed number of times per step, so phase parities follow g)
    const int n_pairs = (a.n_tiles + 1) / 2;
    const int n_my = (int)blockIdx.x < n_pairs ? (n_pairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    bool failed = false;

    auto wait_on = [&](uint64_t* bar, uint32_t parity) {   // a bounded wait; a timeout is recorded
        if (failed) return;
        if (!mbar_wait_bounded(bar, parity, kPoll)) {
            failed = true;
            atomicExch(a.status, DEV_TIMEOUT);
        }
    };
    if (warp == kEpiWarps) {
        // ---- the products (one thread).  Step (g, h), g = 4 p + l - 1: slot 0's
        // products of layer l, half h, then slot 1's.
        if (lane == 0) {
            // shared-memory descriptors of the operand buffers, built once: the
            // issuing thread runs alone, so every instruction of its address
            // arithmetic would sit on the products' issue path
            const uint64_t wdesc0 = sw128_desc(Wbuf), xdesc0 = sw128_desc(Xbuf);
            bool pend0 = false, pend1[2] = {false, false};   // commits in flight
            uint32_t par0 = 0, par1[2] = {0, 0};
            for (int p = 0; p < n_my && !failed; ++p) {
                for (int l = 1; l <= 4 && !failed; ++l) {
                    const int g = p * 4 + l - 1;
                    for (int h = 0; h < 2 && !failed; ++h) {
                        wait_on(&bar_w[h], (uint32_t)(g & 1));
                        for (int sl = 0; sl < 2 && !failed; ++sl) {
                            if (h == 0) {
                                // A_s(l-1) written and D_s free
                                if (g > 0) wait_on(&bar_act[sl], (uint32_t)((g - 1) & 1));
                                if (l == 1) wait_on(&bar_x[sl], (uint32_t)(p & 1));
                            } else {
                                wait_on(&bar_dfree[sl], (uint32_t)(g & 1));   // the epilogue (s, l, 0) has read D_s
                            }
                            if (failed) break;
                            fence_after();
                            const uint32_t d = tmem + dcol_of(sl);
                            // descriptors advance by the byte offset / 16 in their start
                            // address field (shared addresses stay below 2^18, so the
                            // field cannot carry); every offset is a constant
                            const uint64_t wd = wdesc0 + (uint64_t)((h * WH_SLAB) >> 4);
                            if (l == 1) {
                                const uint64_t xd = xdesc0 + (uint64_t)((sl * X_BYTES) >> 4);
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk)   // 4 x k16 per 64-wide slab: +32 bytes each
                                    mma_ss(d, xd + (uint64_t)((kk * 32) >> 4), wd + (uint64_t)((kk * 32) >> 4), kk != 0);
                            } else {
                                const uint32_t ac = tmem + acol_of(sl);   // A column 8 j holds K = 16 j .. 16 j + 15
#pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    mma_ts(d, ac + 8 * j, wd + (uint64_t)(((j >> 2) * W_SLAB + (j & 3) * 32) >> 4), j != 0);
                            }
                            if (sl == 0) {
                                mma_commit(&bar_m0);
                                pend0 = true;
                                par0 = (uint32_t)h;
                            } else {
                                mma_commit(&bar_m1[h]);
                                pend1[h] = true;
                                par1[h] = (uint32_t)(g & 1);
                            }
                        }
                    }
                }
            }
            if (failed) {   // let the products in flight land before the memory is released
                if (pend0) mbar_wait_bounded(&bar_m0, par0, kPoll);
                for (int h = 0; h < 2; ++h)
                    if (pend1[h]) mbar_wait_bounded(&bar_m1[h], par1[h], kPoll);
            }
        }
        __syncwarp();
    } else if (warp == kEpiWarps + 1) {
        // ---- staging (one thread): the features and the weights by TMA.  Weight
        // half h of the next layer (or of the next pair's layer 1) is copied as
        // soon as slot 1's products on it are done (bar_m1[h], which also covers
        // slot 0's, issued before them), and the next pair's features once
        // layer 1's second half is done, so that no copy waits for the issuing
        // thread.  bar_w[h] and bar_x[s] complete once per layer and per pair.
        if (lane == 0) {
            const CUtensorMap* maps[4] = {&mapW1, &mapW2, &mapW3, &mapW4};
            bool pend_x = false, pend_w[2] = {false, false};
            uint32_t par_x = 0, par_w[2] = {0, 0};
            auto load_w = [&](int h, int layer, uint32_t parity) {   // half h of W_layer
                const int ns = layer == 1 ? 1 : 4;
                mbar_arrive_expect_tx(&bar_w[h], ns * WH_SLAB);
                for (int k = 0; k < ns; ++k)
                    tma_load_2d(Wbuf + k * W_SLAB + h * WH_SLAB, maps[layer - 1], k * SLAB_K, h * NH, &bar_w[h]);
                pend_w[h] = true;
                par_w[h] = parity;
            };
            auto load_x = [&](int p) {   // both slots' features of this CTA's pair p
                const int pair = (int)blockIdx.x + p * (int)gridDim.x;
                for (int sl = 0; sl < 2; ++sl) {
                    mbar_arrive_expect_tx(&bar_x[sl], X_BYTES);
                    tma_load_2d(Xbuf + sl * X_BYTES, &mapX, 0, (2 * pair + sl) * TM, &bar_x[sl]);
                }
                pend_x = true;
                par_x = (uint32_t)(p & 1);
            };
            if (n_my > 0) {
                load_x(0);
                load_w(0, 1, 0);
                load_w(1, 1, 0);
            }
            for (int p = 0; p < n_my && !failed; ++p) {
                for (int l = 1; l <= 4 && !failed; ++l) {
                    const int g = p * 4 + l - 1;
                    const int next = l < 4 ? l + 1 : (p + 1 < n_my ? 1 : 0);
                    for (int h = 0; h < 2 && !failed; ++h) {
                        const bool x_next = l == 1 && h == 1 && p + 1 < n_my;
                        if (!next && !x_next) continue;
                        wait_on(&bar_m1[h], (uint32_t)(g & 1));
                        if (failed) break;
                        if (next) load_w(h, next, (uint32_t)((g + 1) & 1));
                        if (x_next) load_x(p + 1);
                    }
                }
            }
            if (failed) {   // let the copies in flight land before the memory is released
                for (int i = 0; i < 2; ++i) {
                    if (pend_x) mbar_wait_bounded(&bar_x[i], par_x, kPoll);
                    if (pend_w[i]) mbar_wait_bounded(&bar_w[i], par_w[i], kPoll);
                }
            }
        }
        __syncwarp();
    } else {
        // epilogue: row = 32 (warp % 4) + lane; columns 32 (warp / 4) .. +31 of
        // each half, in two sub-chunks of 16
        const int quarter = warp & 3, cgrp = warp >> 2, row = quarter * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
        const f32x2 cK = x2_pack(kGeluCK, kGeluCK), cC = x2_pack(kGeluC, kGeluC);
        for (int p = 0; p < n_my; ++p) {
            const int pair = (int)blockIdx.x + p * (int)gridDim.x;
            f32x2 ysum[2] = {0ull, 0ull};   // the head's dot products: even and odd columns
            uint32_t hold[2][16];           // the BF16 pairs of half 0 of each slot, until half 1 is done
            for (int l = 1; l <= 4; ++l) {
                const int g = p * 4 + l - 1;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
#pragma unroll
                    for (int sl = 0; sl < 2; ++sl) {
                        const int tile = 2 * pair + sl;
                        // a timeout is recorded and the later waits skipped, so that
                        // every warp still reaches the block-wide barriers below
                        bool ok = true;
                        if (lane == 0 && !failed)
                            ok = sl == 0 ? mbar_wait_bounded(&bar_m0, (uint32_t)h, kPoll)
                                         : mbar_wait_bounded(&bar_m1[h], (uint32_t)(g & 1), kPoll);
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                        if (!ok && !failed) {
                            failed = true;
                            if (lane == 0) atomicExch(a.status, DEV_TIMEOUT);
                        }
                        fence_after();
                        const size_t trow = (size_t)tile * TM + row;   // the row in the traced outputs
                        const bool traced = TRACE && tile < a.n_tiles;
                        // both column chunks into registers first; after half 0 the
                        // accumulator is released before the arithmetic, so that the
                        // products of half 1 need not wait for it
                        uint32_t r2[2][16];
                        tmem_ld16_async(tmem + lane_base + dcol_of(sl) + cgrp * 32, r2[0]);
                        tmem_ld16_async(tmem + lane_base + dcol_of(sl) + cgrp * 32 + 16, r2[1]);
                        tmem_wait_ld(r2[0]);
#pragma unroll
                        for (int i = 0; i < 16; ++i) asm volatile("" : "+r"(r2[1][i]));
                        if (h == 0) {
                            fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&bar_dfree[sl]);
                        }
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const int col = h * NH + cgrp * 32 + c * 16;   // column of the layer
                            float v[16];
#pragma unroll
                            for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r2[c][i]);
                            const float4* b4 = reinterpret_cast<const float4*>(&bias_s[l - 1][col]);
                            if constexpr (TRACE) {
                                if (traced) {
                                    float* tz = a.trace_z + (((size_t)(l - 1) * a.n_tiles * TM + trow) * TN + col);
#pragma unroll
                                    for (int i = 0; i < 4; ++i) {
                                        const float4 b = b4[i];
                                        tz[4 * i] = v[4 * i] + b.x;
                                        tz[4 * i + 1] = v[4 * i + 1] + b.y;
                                        tz[4 * i + 2] = v[4 * i + 2] + b.z;
                                        tz[4 * i + 3] = v[4 * i + 3] + b.w;
                                    }
                                }
                            }
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                const float4 b = b4[i];
                                bias_gelu2_x2(v[4 * i], v[4 * i + 1], b.x, b.y, cK, cC);
                                bias_gelu2_x2(v[4 * i + 2], v[4 * i + 3], b.z, b.w, cK, cC);
                            }
                            if (l < 4) {
                                uint32_t q[8];
#pragma unroll
                                for (int m = 0; m < 8; ++m) q[m] = pack_bf16x2(v[2 * m], v[2 * m + 1]);
                                if (h == 0) {
#pragma unroll
                                    for (int m = 0; m < 8; ++m) hold[sl][c * 8 + m] = q[m];
                                } else {
                                    // both halves of A_s(l) for these 16 + 16 columns
                                    const uint32_t ac = tmem + lane_base + acol_of(sl);
                                    uint32_t q0[8];
#pragma unroll
                                    for (int m = 0; m < 8; ++m) q0[m] = hold[sl][c * 8 + m];
                                    tmem_st8<false>(ac + (cgrp * 32 + c * 16) / 2, q0);
                                    tmem_st8<false>(ac + (NH + cgrp * 32 + c * 16) / 2, q);
                                    if constexpr (TRACE) {
                                        if (traced) {
                                            uint32_t* ta = a.trace_a + ((size_t)(l - 1) * a.n_tiles * TM + trow) * TN / 2;
#pragma unroll
                                            for (int m = 0; m < 8; ++m) {
                                                ta[(cgrp * 32 + c * 16) / 2 + m] = q0[m];
                                                ta[(NH + cgrp * 32 + c * 16) / 2 + m] = q[m];
                                            }
                                        }
                                    }
                                }
                            } else {
#pragma unroll
                                for (int i = 0; i < 16; i += 2)
                                    ysum[sl] = x2_fma(x2_pack(v[i], v[i + 1]),
                                                      x2_pack(w5_s[col + i], w5_s[col + i + 1]), ysum[sl]);
                            }
                        }
                        if (h == 1) {
                            if (l < 4) tmem_wait_st();
                            fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&bar_act[sl]);
                        }
                    }
                }
            }
#pragma unroll
            for (int sl = 0; sl < 2; ++sl) {
                float y_even, y_odd;
                x2_unpack(ysum[sl], y_even, y_odd);
                head_part[sl][cgrp][row] = y_even + y_odd;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
            if (cgrp < 2) {   // column groups 0 and 1 finish slots 0 and 1
                const int sl = cgrp, tile = 2 * pair + sl;
                if (tile < a.n_tiles)
                    a.y[(size_t)tile * TM + row] = ((head_part[sl][0][row] + head_part[sl][1][row]) +
                                                    (head_part[sl][2][row] + head_part[sl][3][row])) +
                                                   w5_s[TN];
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---- host: tensor maps through the driver entry point ---------------------
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
    // looked up once (thread-safe static initialisation), as the driver
    // version that introduced it (12.0) defines it
    static const EncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiled>(p);
        return static_cast<EncodeTiled>(nullptr);
    }();
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

// W_l^T (K-major, [256][K]) BF16 copies for the tensor cores, times `scale`
// (a power of two, so the BF16 value is the scaled BF16 of the weight)
__global__ void transpose_w_kernel(const float* __restrict__ W, int K, __nv_bfloat16* __restrict__ Wt, bool tied,
                                   float scale) {
    // W [K_in][256] FP32 (K_in = 32 for the tied first layer) -> Wt [256][K]
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < K * MLP_H; i += gridDim.x * blockDim.x) {
        const int n = i / K, k = i % K;
        const int kin = tied ? (k % MLP_IN) : k;
        Wt[i] = __float2bfloat16_rn(W[(size_t)kin * MLP_H + n] * scale);
    }
}

}  // namespace

// Inference of rows [0, n) of X (BF16 [n][MLP_XW], n a multiple of 128) into
// y (FP32 [n]) on the tensor cores.  Returns cudaErrorNotSupported when the
// tensor-map encoder is unavailable.
cudaError_t Mlp::forward_tc(const __nv_bfloat16* Xin, int n, float* yout, int sm_count, int32_t* status,
                            cudaStream_t st, float* trace_z, void* trace_a) {
    if (n % TM) return cudaErrorInvalidValue;
    cudaError_t e;
    if (!wt) {
        if ((e = cudaMalloc((void**)&wt, (size_t)(MLP_XW + 3 * MLP_H) * MLP_H * 2)) != cudaSuccess) return e;
        wt_fresh = false;
    }
    if (!wt_fresh) {   // the transposed weights, once per change of the parameters (200k elements)
        // layers 2-4 read 2 gelu(z) (see the epilogue): their weights carry the 1/2
        transpose_w_kernel<<<64, 256, 0, st>>>(params + mlp_w_off(1), MLP_XW, wt, true, 1.0f);
        for (int l = 2; l <= 4; ++l)
            transpose_w_kernel<<<128, 256, 0, st>>>(params + mlp_w_off(l), MLP_H,
                                                    wt + (size_t)(MLP_XW + (l - 2) * MLP_H) * MLP_H, false, 0.5f);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        wt_fresh = true;
    }
    CUtensorMap mx, mw[4];   // weight boxes are one N half (128 rows of W_l^T)
    if (!make_map(&mx, Xin, MLP_XW, n, TM) || !make_map(&mw[0], wt, MLP_XW, MLP_H, NH))
        return cudaErrorNotSupported;
    for (int l = 1; l < 4; ++l)
        if (!make_map(&mw[l], wt + (size_t)(MLP_XW + (l - 1) * MLP_H) * MLP_H, MLP_H, MLP_H, NH))
            return cudaErrorNotSupported;
    TcArgs a;
    for (int l = 0; l < 4; ++l) a.bias[l] = params + mlp_b_off(l + 1);
    a.w5 = params + mlp_w5_off();
    a.y = yout;
    a.n_tiles = n / TM;
    a.status = status;
    a.trace_z = trace_z;
    a.trace_a = static_cast<uint32_t*>(trace_a);
    const size_t smem = 2 * X_BYTES + W_BYTES + 1024;
    auto kern = trace_z || trace_a ? mlp_fwd_tc_kernel<true> : mlp_fwd_tc_kernel<false>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    const int grid = std::min((a.n_tiles + 1) / 2, sm_count);
    kern<<<grid, kThreads, smem, st>>>(mx, mw[0], mw[1], mw[2], mw[3], a);
    return cudaGetLastError();
}

}  // namespace rsv
