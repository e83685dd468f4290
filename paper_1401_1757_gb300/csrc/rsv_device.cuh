// rsv_device.cuh -- device-side building blocks of the reserve recurrence kernels
// (sm_103a): work records, double-float arithmetic, TMA bulk staging with a
// bounded mbarrier wait.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rsv {

// Reduced model of a policy tile (zero-reserve states removed, Section 3.6.4).
enum Kind : int32_t {
    K_ANN = 0,  // 1 state, r = v p (c + r')            (Section 4.1.1)
    K_ASS = 1,  // 1 state, r = v (q c + p r')          (Section 4.1.3, reduced)
    K_JL = 2,   // 3 states 00, 01, 10 of the two-life model (Section 4.2)
    K_ANN2 = 3, // 1 state, r = v px py (c + r')       (joint-life annuity)
    K_ASS2 = 4, // 1 state, r = v ((1 - px py) c + px py r')  (joint-status assurance)
    K_LS2 = 5   // 3 states 00, x only, y only of the nine-state two-life assurance
                // model with the benefit on the second death (Section 4.2.3)
};

// F_DEFL: the recurrence in deflated units, compensated FP32 (defl_kernel.cuh)
enum Form : int32_t { F_F64 = 0, F_F32 = 1, F_COMP = 2, F_DEFL = 3 };

// Device status word values.
enum : int32_t { DEV_OK = 0, DEV_TIMEOUT = 1 };

// One policy slot of a tile.  All lanes of a warp read the same slot, so the
// loads are broadcasts.  Padding slots repeat the previous slot with pol = -1.
struct SlotRec {
    int32_t idx1;    // staged-table index of life 1 at t = 0 (table * tab_pad + age)
    int32_t idx2;    // life 2 (JL only)
    int32_t S;       // number of steps
    int32_t pol;     // index in the caller's portfolio, -1 = padding
    float rho_h;     // reversion rho as a hi/lo pair (JL only)
    float rho_l;
    int32_t state0;  // reduced state reported at t = 0
    float bnd;       // boundary r_S per unit amount (1: endowment at maturity)
};
static_assert(sizeof(SlotRec) == 32, "SlotRec layout");

struct RecurArgs {
    const void* tab;          // staged decrement tables, form-specific entries, n_tab * tab_pad
    int32_t tab_bytes;        // bytes staged into shared memory (multiple of 16)
    const void* v;            // scenario plane [n_steps][s_pad], form-specific element
    int32_t s_pad;            // row stride (elements), multiple of 128
    int32_t n_scen;
    int32_t n_steps;          // T
    const SlotRec* slots;     // [n_tiles * P], tiles in decreasing cost order
    const int32_t* tile_kind; // [n_tiles]
    const double* amount;     // [n_pol]
    int32_t n_tiles;
    int32_t n_chunks;         // scenario chunks of 32*M per tile
    int32_t n_items;          // n_tiles * n_chunks
    int32_t* counter;         // work-queue head, zero before the launch
    int32_t* status;          // DEV_* error word
    float* V0f;               // [n_pol][n_scen] or null
    double* V0d;              // [n_pol][n_scen] or null
    double* partial;          // [n_tiles][s_pad] per-tile scenario sums or null
    double* pt_sum;           // [n_pol][T+1] sums over scenarios or null
    double* traj;             // [n_pol][T+1][n_scen] or null
    int32_t v0_ld;            // row stride of V0 (= n_scen unless a column block is computed)
    const void* vf;           // fractional discount plane v_t^f, same layout as v (fractional payments)
    int32_t tabf_off;         // entries from the staged tables to the fractional-survival tables
    const void* cf;           // cash-flow multipliers c_t, [n_pol][cf_ld] (double for FP64, else float), or null
    int32_t cf_ld;            // row length of cf (steps from valuation)
};

// When an annuity's cash flow is paid within each step (the fraction f of
// Eq. generalForm); assurance benefits are always paid at the step's end.
// PAY_END_GENERAL is f = 1 on unshifted states, for cash flows that vary
// from step to step (c_t = cf_t c, Section 4.1.1 and 4.6).  The variants
// other than PAY_END all take the multipliers cf_t when they are given.
enum Pay : int32_t { PAY_END = 0, PAY_START = 1, PAY_FRACTION = 2, PAY_END_GENERAL = 3 };

// ------------------------------------------------------------------------
// double-float ("df") numbers: value = h + l with |l| about ulp(h) or less.
// All products use explicit fused multiply-adds; the kernels are compiled
// with contraction off, so nothing else is fused behind our back.
struct df {
    float h, l;
};

__device__ __forceinline__ df df_make(float h, float l) { return df{h, l}; }

// (a.h + a.l)(b.h + b.l): exact product of the heads (TwoProd via FMA)
// plus the two cross terms; the lo*lo term (about 2^-48 relative) is dropped.
// The result is not renormalised; its tail stays within a few ulps of the head.
__device__ __forceinline__ df df_mul(df a, df b) {
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return df{p, e};
}

// Sum of two non-negative df numbers.  The heads are ordered by value (both
// >= 0, so by magnitude) and added with Fast2Sum, whose error term is exact;
// the tails are added to it.
__device__ __forceinline__ df df_add_pos(df a, df b) {
    float hi = fmaxf(a.h, b.h), lo = fminf(a.h, b.h);
    float s = __fadd_rn(hi, lo);
    float e = __fsub_rn(lo, __fsub_rn(s, hi));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return df{s, e};
}

// 1 + a for df a >= 0 (a.l may be any sign but |a.l| << a.h or a == 0).
__device__ __forceinline__ df df_add_one(df a) {
    float hi = fmaxf(1.0f, a.h), lo = fminf(1.0f, a.h);
    float s = __fadd_rn(hi, lo);
    float e = __fsub_rn(lo, __fsub_rn(s, hi));
    e = __fadd_rn(e, a.l);
    return df{s, e};
}

// a + b for df a >= 0 and float b >= 0 (b carries no tail).
__device__ __forceinline__ df df_add_float_pos(df a, float b) {
    float hi = fmaxf(a.h, b), lo = fminf(a.h, b);
    float s = __fadd_rn(hi, lo);
    float e = __fsub_rn(lo, __fsub_rn(s, hi));
    e = __fadd_rn(e, a.l);
    return df{s, e};
}

// 1 + g R for df g >= 0 and R >= 1 (a shifted reserve R = 1 + r).  The head
// h = fl(1 + g.h R.h) is one FMA; h - 1 is exact for 1 <= h < 2^24, so a
// second FMA recovers the rounding error of h to within 2^-24 of itself, and
// the cross terms add the tails.  Five operations, no ordering needed.
__device__ __forceinline__ df df_one_plus_mul(df g, df R) {
    const float h = __fmaf_rn(g.h, R.h, 1.0f);
    const float d = __fsub_rn(h, 1.0f);
    float e = __fmaf_rn(g.h, R.h, -d);
    e = __fmaf_rn(g.h, R.l, e);
    e = __fmaf_rn(g.l, R.h, e);
    return df{h, e};
}

// c + g R for float c >= 0 and df g, R >= 0: the product as in df_mul, then
// the head sum ordered by magnitude (Fast2Sum) and the tails added.
__device__ __forceinline__ df df_float_plus_mul(float c, df g, df R) {
    const float p = __fmul_rn(g.h, R.h);
    float e = __fmaf_rn(g.h, R.h, -p);
    e = __fmaf_rn(g.h, R.l, e);
    e = __fmaf_rn(g.l, R.h, e);
    const float hi = fmaxf(p, c), lo = fminf(p, c);
    const float s = __fadd_rn(hi, lo);
    const float err = __fsub_rn(lo, __fsub_rn(s, hi));
    return df{s, __fadd_rn(err, e)};
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.h + (double)a.l; }

// ------------------------------------------------------------------------
// TMA (bulk async copy) staging of a contiguous global block into shared
// memory, completed on an mbarrier; the wait is bounded.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// 1-D bulk copy global -> shared; size and both addresses multiples of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Poll an mbarrier phase at most `limit` times.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

constexpr uint32_t kBulkChunk = 32768;      // bytes per bulk copy instruction
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait polls before giving up

// Stage `bytes` (multiple of 16, <= 1 MiB) from global `src` into shared `dst`
// with TMA.  Block-wide; returns false (and sets *status) if the copy did not
// complete within the poll limit, after a second bounded wait for the copies
// still in flight.
__device__ __forceinline__ bool stage_to_smem(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, int32_t* status) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, bytes);
        for (uint32_t off = 0; off < bytes; off += kBulkChunk) {
            uint32_t n = bytes - off < kBulkChunk ? bytes - off : kBulkChunk;
            bulk_g2s(static_cast<char*>(dst) + off, static_cast<const char*>(src) + off, n, bar);
        }
    }
    bool ok = mbar_wait_bounded(bar, 0, kWaitLimit);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(status, DEV_TIMEOUT);
        mbar_wait_bounded(bar, 0, kWaitLimit);   // let copies in flight land before exit
    }
    return ok;
}

// ---- packed FP32 pairs (sm_100 and later): fma/mul/add/sub .f32x2 apply the
// scalar IEEE single-precision operation, rounded to nearest, to each half of
// a 64-bit register pair in one issue slot; x is the low half, y the high half.
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 x2_pack(float x, float y) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void x2_unpack(f32x2 r, float& x, float& y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(r));
}
__device__ __forceinline__ f32x2 x2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 x2_mul(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_add(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 x2_sub(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

}  // namespace rsv
