// defl_kernel.cuh -- the backward recurrence in deflated units (compensated FP32).
//
// Multiply the reserve of Eq. (generalForm) at step t by the deflator
// G_t = D_t l_{x+t} / l_x, the product of the discount factors of the steps
// before t (D_t = v_0 ... v_{t-1}) and the survival to t.  For the reduced
// one-state models (Section 3.6.4, Section 4.1) r_t = v_t p_t (c + r_{t+1})
// becomes
//     U_t = U_{t+1} + c G_{t+1},        U = G r,  U_S = G_S r_S,
// the same backward substitution (Section 3.8.2) with the multiplicative
// factor of every step equal to 1.  The reserve at valuation is r_0 = U_0.
// G splits into a scenario part and a policy part: D_{t+1} is one FP64
// running product per scenario (the discount-factor products over long
// terms, computed once per scenario by defl_plane_kernel) and l_{x+t+1} /
// l_x comes from the life table {l_k} (Section 5 computes it per policy; here
// it is one table, built once in FP64).  A chain-step is one FP32 fused
// multiply-add of the two; no rounding compounds along the chain, because no
// rounded value is ever multiplied by the next step's factor.
//
// The weights w_t = D_{t+1} E_t, with E_t the policy's expected cash flow at
// the end of step t per unit amount:
//   K_ANN   l_{x+t+1}                                     (Section 4.1.1)
//   K_ASS   l_{x+t} q_{x+t}  (deaths in the step),  U_S = D_S l_{x+S} bnd
//                                                          (Sections 4.1.2-4.1.3)
//   K_ANN2  P^x P^y, P^x = l^x_{x+t+1}/l^x_x, P^y = l^y_{y+t+1}/l^y_y  (joint life, Section 4.2)
//   K_JL    P^x + P^y (1 - P^x) with P^x = l^x_{x+t+1}/l^x_x, P^y = rho l^y_{y+t+1}/l^y_y
//           in state 00; P^y = 0 in state 01 and P^x = 0 in state 10
//           (c = (1, 1, rho) of the reversionary annuity, Section 4.2.1:
//           r00 = a_x + rho (a_y - a_xy) is the sum of these weights).
// K_ANN and K_ASS carry the factor 1 / l_x in the per-policy scale applied at
// the end.  The tables are normalised to l_0 = 2^100, so that every ratio
// down to 2^-220 stays in FP32's normal range.
//
// Accumulation.  Terms are added in FP32 by fused multiply-adds into two
// accumulators (alternate steps), each taking 8 terms; every 16 steps their
// sum is folded into a double-float (h, l) by an ordered Fast2Sum, whose
// error term is exact.  An FP32 sum of 8 positive terms is within 8 u of its
// value (u = 2^-24), the two-accumulator add adds u, the inputs D and E are
// rounded once each (and E of the JL product up to 3 u), so every reserve is
// within about 14 u = 8.3e-7 of the value the exact arithmetic gives on the
// FP64 inputs, whatever the projection length; the errors are independent
// roundings, so typical errors are far smaller.  The two-level variants fold
// once per 32-step block: the two spans' partial sums are first added in
// FP32 (one more rounding, about 15 u = 8.9e-7 in all).
//
// Mapping.  A work item is a super-tile of NW tiles of P policies (the tiles
// of one reduced model, consecutive in decreasing-length order) times one
// chunk of 32 M scenarios; a CTA of NW warps takes one item, warp w the
// policies [w P, (w+1) P) of the super-tile, lane l the scenarios
// chunk + m 32 + l (m < M).  The deflator plane is read in blocks of 32
// steps: each block of the chunk is staged into shared memory by TMA bulk
// copies, NBUF blocks in flight, completing on one mbarrier per buffer
// (bounded waits, agreed on by the whole CTA).  The life tables are staged
// once per CTA, as four copies shifted by one entry, so that four
// consecutive steps of any policy are one aligned 16-byte shared-memory load.
// Items come from an atomic queue in decreasing-cost order; thread 0 claims
// them ahead of use, so the staging of the next item overlaps this one.
//
// Packed pairs (X2 variants).  sm_100 and later issue fma/mul/add/sub on two
// FP32 values held in one 64-bit register pair (.f32x2), each half rounded
// exactly as the scalar instruction rounds.  The two accumulators of a chain
// are one pair {even steps, odd steps}, and four consecutive steps of a
// deflator row and of a weight row are two pairs, so a pair instruction does
// the work of two chain-steps.  The fold of a span into (h, l) runs on pairs
// of chains (scenarios m and m + 1): the ordering by max and min per chain (the
// terms are non-negative), then the ordered Fast2Sum on the pair, so the X2
// variants give the same bits as the scalar ones.
//
// Sums in tensor memory (TM variants).  A chain's double-float sum is touched
// once per fold, so the packed variants can keep it in the warp's columns of
// tensor memory (tcgen05.ld/st) instead of registers: 128 registers a thread,
// 16 warps a CTA instead of 12, the same bits.  The two-level variant (TM2)
// also parks the first span's accumulators of each 32-step block there and
// folds once per block.
#pragma once

#include <type_traits>

#include "rsv_device.cuh"

namespace rsv {

constexpr int DEFL_KB = 32;        // steps per staged block of the deflator plane
constexpr uint32_t kDeflTmemCols = 128;   // the TMEM lanes: four warps per lane quarter x 32 columns
constexpr int DEFL_G = DEFL_KB / 4; // float4 rows (groups of four steps) per block

// One policy slot of a deflated super-tile (64 bytes).  All lanes of a warp
// read the same slot.
struct DeflSlot {
    int32_t off1;    // float4 index of life 1's run in the staged main array (A or deaths)
    int32_t off2;    // float4 index of life 2's run in A (K_JL, K_ANN2)
    int32_t S;       // steps; padding slots repeat a shape with pol = -1
    int32_t pol;     // portfolio index, -1 = padding
    float ix, iy;    // K_JL: 1/l_x and rho/l_y of the valuation state (0 where a life is dead);
                     // K_ANN2: 1/l_x and 1/l_y
    float mat;       // deflated boundary weight bnd * l_{x+S} (endowments), else 0
    int32_t kind;
    double scale;    // V0 = scale * U: amount / l_x (K_ANN, K_ASS) or amount (K_JL, K_ANN2)
    float sc_h, sc_l;// scale as an FP32 head and tail
    int32_t gz1, gz2;// first group of four steps whose table entries are all zero (past the
                     // table's end), life 1 and life 2: reads of later groups read that one
    int32_t pad[2];
};
static_assert(sizeof(DeflSlot) == 64, "DeflSlot layout");

struct DeflArgs {
    const float* tab;        // staged tables: [2 arrays (A, deaths)][n_tab][4 shifted copies][dpad]
    int32_t tab_bytes;       // bytes to stage (multiple of 16)
    const float4* D;         // deflator plane [n_groups][s_pad]: D_{t+1} for t = 4g .. 4g+3
    int32_t s_pad;           // row length of the plane (scenarios, multiple of 128)
    int32_t n_scen;          // valid scenario columns from the plane's first column
    int32_t n_groups;        // rows of the plane (a multiple of DEFL_G)
    const DeflSlot* slots;   // [n_st][W] (W = NW * P), super-tiles in decreasing cost order
    const int32_t* st_kind;  // [n_st]
    int32_t n_st;
    int32_t n_chunks;        // scenario chunks of 32 M
    int32_t n_items;         // n_st * n_chunks
    int32_t* counter;        // work-queue head, zero before the launch
    int32_t* status;         // DEV_* error word
    float* V0f;              // [n_pol][v0_ld] or null
    double* V0d;             // [n_pol][v0_ld] or null
    int32_t v0_ld;
    double* partial;         // [n_st][part_ld] per-super-tile scenario sums or null
    int32_t part_ld;
};

// Sum b >= 0 into the double-float (h, l), h >= 0: Fast2Sum on the heads
// ordered by size (exact error term), the tail accumulates it.
__device__ __forceinline__ void defl_fold(float& h, float& l, float b) {
    const float hi = fmaxf(h, b), lo = fminf(h, b);
    const float s = __fadd_rn(hi, lo);
    const float e = __fsub_rn(lo, __fsub_rn(s, hi));
    h = s;
    l = __fadd_rn(l, e);
}

// Header of a staged block: which item and block it holds.
struct DeflBlock {
    int32_t item;   // -1: no more work
    int32_t j;      // block index (steps j*32 .. j*32+31)
    int32_t first;  // first block of the item (its longest block)
    int32_t q;      // the item's number in this CTA's sequence (its partial-sum slot is q & 1);
                    // bit 30 set: block 0, the item's epilogue follows
};

template <int P, int M, int NW, int NBUF>
struct DeflSmem {
    static constexpr int CH = 32 * M;                      // scenarios per chunk
    static constexpr size_t ring = (size_t)NBUF * DEFL_G * CH * sizeof(float4);
    static constexpr size_t red = (size_t)2 * NW * CH * sizeof(float2);
    static constexpr size_t slots = (size_t)2 * NW * P * sizeof(DeflSlot);   // two items' slot records
    static constexpr size_t hdr = (size_t)NBUF * sizeof(DeflBlock);
    static constexpr size_t bars = (size_t)2 * NBUF * sizeof(uint64_t);
    // layout after the tables (tab_bytes, a multiple of 16): ring | red | slots | hdr | bars
    static size_t bytes(size_t tab_bytes) { return tab_bytes + ring + red + slots + hdr + bars; }
};

__device__ __forceinline__ void defl_mbar_arrive(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

// Per-lane state of one item: P policies x M scenarios.
template <int P, int M>
struct DeflLane {
    static constexpr bool packed = false, two_level = false;
    float a0[P][M], a1[P][M];   // the current 16 steps' two FP32 accumulators
    float h[P][M], l[P][M];     // double-float sums of the folded spans
    __device__ __forceinline__ void start(int i, const float (&h0)[M]) {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            h[i][m] = h0[m];
            l[i][m] = 0.0f;
        }
    }
    __device__ __forceinline__ void sum(int i, float (&H)[M], float (&L)[M]) const {
#pragma unroll
        for (int m = 0; m < M; ++m) {
            H[m] = h[i][m];
            L[m] = l[i][m];
        }
    }
    __device__ __forceinline__ void clear_acc() {   // a span that opens mid-way starts from zero
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) a0[i][m] = a1[i][m] = 0.0f;
    }
};

// The same state in packed pairs (M even): acc = {a0, a1} of each chain,
// (h, l) of scenarios 2k (x) and 2k + 1 (y).
template <int P, int M>
struct DeflLaneX2 {
    static constexpr bool packed = true, two_level = false;
    static_assert(M % 2 == 0, "pairs of scenarios");
    f32x2 acc[P][M];
    f32x2 h[P][M / 2], l[P][M / 2];
    __device__ __forceinline__ void start(int i, const float (&h0)[M]) {
#pragma unroll
        for (int k = 0; k < M / 2; ++k) {
            h[i][k] = x2_pack(h0[2 * k], h0[2 * k + 1]);
            l[i][k] = 0ull;
        }
    }
    __device__ __forceinline__ void sum(int i, float (&H)[M], float (&L)[M]) const {
#pragma unroll
        for (int k = 0; k < M / 2; ++k) {
            x2_unpack(h[i][k], H[2 * k], H[2 * k + 1]);
            x2_unpack(l[i][k], L[2 * k], L[2 * k + 1]);
        }
    }
    __device__ __forceinline__ void clear_acc() {   // a span that opens mid-way starts from zero
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) acc[i][m] = 0ull;
    }
};

// Tensor-memory access of one warp: 32 consecutive columns of its 32 lanes
// (lane quarter warp % 4), one register a column.
__device__ __forceinline__ void defl_tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}
// Store 32 columns and wait for the stores (the next access to them is a
// span later, so the wait costs nothing and every later load sees them).
__device__ __forceinline__ void defl_tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]),
        "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]),
        "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// Packed pairs with the double-float sums in tensor memory: (h, l) of a
// chain are touched once per 16 steps, so the warp keeps them in its 32 TMEM
// columns (h of chain j = i M + m in column j, l in column 16 + j) and only
// the accumulators stay in registers.  At 128 registers a thread the CTA
// holds 16 warps instead of 12.  The arithmetic is DeflLaneX2's: same bits.
template <int P, int M>
struct DeflLaneTM {
    static constexpr bool packed = true, two_level = false;
    static_assert(M % 2 == 0 && P * M == 16, "h and l of 16 chains in 32 columns");
    f32x2 acc[P][M];
    uint32_t taddr = 0;
    __device__ __forceinline__ void start_all(const float (&h0)[P][M]) const {
        uint32_t r[32];
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) {
                r[i * M + m] = __float_as_uint(h0[i][m]);
                r[16 + i * M + m] = 0u;
            }
        defl_tmem_st32(taddr, r);
    }
    __device__ __forceinline__ void sum_all(float (&H)[P][M], float (&L)[P][M]) const {
        uint32_t r[32];
        defl_tmem_ld32(taddr, r);
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) {
                H[i][m] = __uint_as_float(r[i * M + m]);
                L[i][m] = __uint_as_float(r[16 + i * M + m]);
            }
    }
};

// The sums in tensor memory, folded once per block: the first span of a
// block parks its accumulators in 32 more columns (mid), and after the
// second span mid is added to the accumulators (one FP32 rounding) before
// the one fold of the block.  Each FP32 partial sum then carries 8 terms and
// one addition (9 u instead of 8 u), for half the folds.
template <int P, int M>
struct DeflLaneTM2 : DeflLaneTM<P, M> {
    static constexpr bool two_level = true;
};

// What a block needs of a warp's P slots.
template <int P>
struct DeflPol {
    int off1[P], off2[P], S[P], gz1[P], gz2[P];
    float ix[P], iy[P];
};

// The fields of a warp's P slot records that product kind KIND reads, loaded
// from shared memory at each staged block, so that no other kind's fields
// stay live in registers across the block loop.
template <int KIND, int P>
__device__ __forceinline__ DeflPol<P> defl_pol(const DeflSlot* __restrict__ rec) {
    DeflPol<P> pp;
#pragma unroll
    for (int i = 0; i < P; ++i) {
        const int4 q4 = *reinterpret_cast<const int4*>(&rec[i].off1);   // off1, off2, S, pol
        pp.off1[i] = q4.x;
        pp.S[i] = q4.w < 0 ? 0 : q4.z;
        if constexpr (KIND != K_ANN) {
            const int2 z2 = *reinterpret_cast<const int2*>(&rec[i].gz1);
            pp.gz1[i] = z2.x;
            pp.gz2[i] = z2.y;
        }
        if constexpr (KIND == K_JL || KIND == K_ANN2) {
            const float2 f2 = *reinterpret_cast<const float2*>(&rec[i].ix);
            pp.off2[i] = q4.y;
            pp.ix[i] = f2.x;
            pp.iy[i] = f2.y;
        }
    }
    return pp;
}

// The expected cash flows E of four steps t = 4g .. 4g+3 of policy i
// (per unit amount; for K_ANN and K_ASS unscaled), zero past its end.
template <int KIND, int P>
__device__ __forceinline__ float4 defl_weights(const DeflPol<P>& pp, int i, const float4* __restrict__ tab, int g,
                                               bool check) {
    // A policy's steps run past its table's end where a term assurance outlives
    // the limiting age or where the other life of a two-life product lives
    // longer; those entries are zero, and the staged tables hold one zero group
    // past each table's end, which the reads of later groups are clamped to.
    float4 e;
    if constexpr (KIND == K_ANN) {   // S never runs past the table's end
        e = tab[pp.off1[i] + g];
    } else if constexpr (KIND == K_ASS) {
        e = tab[pp.off1[i] + min(g, pp.gz1[i])];
    } else if constexpr (KIND == K_ANN2) {   // E = P^x P^y
        const float4 x = tab[pp.off1[i] + min(g, pp.gz1[i])], y = tab[pp.off2[i] + min(g, pp.gz2[i])];
        const float ix = pp.ix[i], iy = pp.iy[i];
        e.x = __fmul_rn(__fmul_rn(x.x, ix), __fmul_rn(y.x, iy));
        e.y = __fmul_rn(__fmul_rn(x.y, ix), __fmul_rn(y.y, iy));
        e.z = __fmul_rn(__fmul_rn(x.z, ix), __fmul_rn(y.z, iy));
        e.w = __fmul_rn(__fmul_rn(x.w, ix), __fmul_rn(y.w, iy));
    } else {   // K_JL: E = P^x (1 - P^y) + P^y
        const float4 x = tab[pp.off1[i] + min(g, pp.gz1[i])], y = tab[pp.off2[i] + min(g, pp.gz2[i])];
        const float ix = pp.ix[i], iy = pp.iy[i];
        float px = __fmul_rn(x.x, ix), py = __fmul_rn(y.x, iy);
        e.x = __fmaf_rn(px, __fsub_rn(1.0f, py), py);
        px = __fmul_rn(x.y, ix); py = __fmul_rn(y.y, iy);
        e.y = __fmaf_rn(px, __fsub_rn(1.0f, py), py);
        px = __fmul_rn(x.z, ix); py = __fmul_rn(y.z, iy);
        e.z = __fmaf_rn(px, __fsub_rn(1.0f, py), py);
        px = __fmul_rn(x.w, ix); py = __fmul_rn(y.w, iy);
        e.w = __fmaf_rn(px, __fsub_rn(1.0f, py), py);
    }
    if (check) {   // steps at or past the end contribute nothing
        const int t0 = 4 * g, S = pp.S[i];
        if (t0 >= S) e.x = 0.0f;
        if (t0 + 1 >= S) e.y = 0.0f;
        if (t0 + 2 >= S) e.z = 0.0f;
        if (t0 + 3 >= S) e.w = 0.0f;
    }
    return e;
}

// One group of four steps (descending t) of the warp's P x M chains: the
// weights of every policy first, then the fused multiply-adds step by step
// across all chains (the two accumulators take alternate steps).  FIRST: the
// group opens a 16-step span, whose products start the accumulators.
template <int KIND, int P, int M, bool FIRST, class Lane>
__device__ __forceinline__ void defl_group(Lane& st, const DeflPol<P>& pp, const float4* __restrict__ tab,
                                           const float4 (&d)[M], int g, bool check) {
    float4 e[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        // a group wholly past the policy's end reads nothing (its table entries
        // may lie beyond what was staged for it)
        if (check && 4 * g >= pp.S[i]) e[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        else e[i] = defl_weights<KIND, P>(pp, i, tab, g, check);
    }
    if constexpr (Lane::packed) {   // steps {4g+2, 4g+3}, then {4g, 4g+1}
        f32x2 dl[M], dh[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            dl[m] = x2_pack(d[m].x, d[m].y);
            dh[m] = x2_pack(d[m].z, d[m].w);
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const f32x2 eh = x2_pack(e[i].z, e[i].w);
#pragma unroll
            for (int m = 0; m < M; ++m) st.acc[i][m] = FIRST ? x2_mul(dh[m], eh) : x2_fma(dh[m], eh, st.acc[i][m]);
        }
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const f32x2 el = x2_pack(e[i].x, e[i].y);
#pragma unroll
            for (int m = 0; m < M; ++m) st.acc[i][m] = x2_fma(dl[m], el, st.acc[i][m]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m)
                st.a1[i][m] = FIRST ? __fmul_rn(d[m].w, e[i].w) : __fmaf_rn(d[m].w, e[i].w, st.a1[i][m]);
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m)
                st.a0[i][m] = FIRST ? __fmul_rn(d[m].z, e[i].z) : __fmaf_rn(d[m].z, e[i].z, st.a0[i][m]);
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) st.a1[i][m] = __fmaf_rn(d[m].y, e[i].y, st.a1[i][m]);
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m) st.a0[i][m] = __fmaf_rn(d[m].x, e[i].x, st.a0[i][m]);
    }
}

// After the steps of one 16-step span: fold the two accumulators into (h, l).
template <int P, int M>
__device__ __forceinline__ void defl_fold_all(DeflLane<P, M>& st) {
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int m = 0; m < M; ++m) defl_fold(st.h[i][m], st.l[i][m], __fadd_rn(st.a0[i][m], st.a1[i][m]));
}
// Packed: b = a0 + a1 of two chains, ordered against h by max and min per
// chain (both non-negative), then the ordered Fast2Sum on the pair and l += e:
// the scalar fold's operations, so the same bits.
template <int P, int M>
__device__ __forceinline__ void defl_fold_all(DeflLaneX2<P, M>& st) {
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int k = 0; k < M / 2; ++k) {
            float x0, y0, x1, y1, h0, h1;
            x2_unpack(st.acc[i][2 * k], x0, y0);
            x2_unpack(st.acc[i][2 * k + 1], x1, y1);
            x2_unpack(st.h[i][k], h0, h1);
            const float b0 = __fadd_rn(x0, y0), b1 = __fadd_rn(x1, y1);
            const f32x2 hi = x2_pack(fmaxf(h0, b0), fmaxf(h1, b1));
            const f32x2 lo = x2_pack(fminf(h0, b0), fminf(h1, b1));
            const f32x2 s = x2_add(hi, lo);
            st.h[i][k] = s;
            st.l[i][k] = x2_add(st.l[i][k], x2_sub(lo, x2_sub(s, hi)));
        }
}

template <int P, int M>
__device__ __forceinline__ void defl_fold_all(DeflLaneTM<P, M>& st) {
    uint32_t r[32];
    defl_tmem_ld32(st.taddr, r);
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int k = 0; k < M / 2; ++k) {
            const int j0 = i * M + 2 * k, j1 = j0 + 1;
            float x0, y0, x1, y1;
            x2_unpack(st.acc[i][2 * k], x0, y0);
            x2_unpack(st.acc[i][2 * k + 1], x1, y1);
            const float h0 = __uint_as_float(r[j0]), h1 = __uint_as_float(r[j1]);
            const float b0 = __fadd_rn(x0, y0), b1 = __fadd_rn(x1, y1);
            const f32x2 hi = x2_pack(fmaxf(h0, b0), fmaxf(h1, b1));
            const f32x2 lo = x2_pack(fminf(h0, b0), fminf(h1, b1));
            const f32x2 s = x2_add(hi, lo);
            const f32x2 l = x2_add(x2_pack(__uint_as_float(r[16 + j0]), __uint_as_float(r[16 + j1])),
                                   x2_sub(lo, x2_sub(s, hi)));
            float s0, s1, l0, l1;
            x2_unpack(s, s0, s1);
            x2_unpack(l, l0, l1);
            r[j0] = __float_as_uint(s0);
            r[j1] = __float_as_uint(s1);
            r[16 + j0] = __float_as_uint(l0);
            r[16 + j1] = __float_as_uint(l1);
        }
    defl_tmem_st32(st.taddr, r);
}

template <int P, int M>
__device__ __forceinline__ void defl_stash(DeflLaneTM2<P, M>& st) {   // mid = the accumulators
    uint32_t r[32];
#pragma unroll
    for (int i = 0; i < P; ++i)
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float x, y;
            x2_unpack(st.acc[i][m], x, y);
            r[2 * (i * M + m)] = __float_as_uint(x);
            r[2 * (i * M + m) + 1] = __float_as_uint(y);
        }
    defl_tmem_st32(st.taddr + 32u, r);
}
template <int P, int M>
__device__ __forceinline__ void defl_fold_all(DeflLaneTM2<P, M>& st) {
    {
        uint32_t r[32];
        defl_tmem_ld32(st.taddr + 32u, r);
#pragma unroll
        for (int i = 0; i < P; ++i)
#pragma unroll
            for (int m = 0; m < M; ++m)
                st.acc[i][m] = x2_add(x2_pack(__uint_as_float(r[2 * (i * M + m)]), __uint_as_float(r[2 * (i * M + m) + 1])),
                                      st.acc[i][m]);
    }
    defl_fold_all(static_cast<DeflLaneTM<P, M>&>(st));
}

// One 16-step span (four groups, descending) from the staged rows r0+3 .. r0.
// STAGE (two-level lanes): 1 parks the span's accumulators, 2 folds both spans.
template <int KIND, int P, int M, int STAGE = 0, class Lane>
__device__ __forceinline__ void defl_span(Lane& st, const DeflPol<P>& pp, const float4* __restrict__ tab,
                                          const float4* __restrict__ ring_b, int g0, int lane, bool check) {
#pragma unroll
    for (int u = 3; u >= 0; --u) {
        float4 d[M];
#pragma unroll
        for (int m = 0; m < M; ++m) d[m] = ring_b[u * (32 * M) + m * 32 + lane];
        if (u == 3) defl_group<KIND, P, M, true>(st, pp, tab, d, g0 + u, check);
        else defl_group<KIND, P, M, false>(st, pp, tab, d, g0 + u, check);
    }
    if constexpr (STAGE == 1) defl_stash(st);
    else defl_fold_all(st);
}

// One staged block (two spans, descending) of one item.  The packed lanes
// unroll the two spans of a block that no policy ends in, so that the
// scheduler can overlap the first span's fold with the second span's loads.
template <int KIND, int P, int M, class Lane>
__device__ __forceinline__ void defl_block(Lane& st, const DeflPol<P>& pp, const float4* __restrict__ tab,
                                           const float4* __restrict__ ring_b, int j, int lane, int smin, int smax) {
    const int t_lo = j * DEFL_KB;
    if (t_lo >= smax) return;                       // every policy of this warp has ended before the block
    const int g_lo = j * DEFL_G;
    if (t_lo + DEFL_KB > smin) {                    // some policy ends within or before the block
        if constexpr (Lane::two_level) {
            defl_span<KIND, P, M, 1>(st, pp, tab, ring_b + 4 * (32 * M), g_lo + 4, lane, true);
            defl_span<KIND, P, M, 2>(st, pp, tab, ring_b, g_lo, lane, true);
        } else {
#pragma unroll 1
            for (int h = 1; h >= 0; --h)
                defl_span<KIND, P, M>(st, pp, tab, ring_b + h * 4 * (32 * M), g_lo + 4 * h, lane, true);
        }
    } else if constexpr (Lane::packed) {
        defl_span<KIND, P, M, Lane::two_level ? 1 : 0>(st, pp, tab, ring_b + 4 * (32 * M), g_lo + 4, lane, false);
        defl_span<KIND, P, M, Lane::two_level ? 2 : 0>(st, pp, tab, ring_b, g_lo, lane, false);
    } else {
#pragma unroll 1
        for (int h = 1; h >= 0; --h) defl_span<KIND, P, M>(st, pp, tab, ring_b + h * 4 * (32 * M), g_lo + 4 * h, lane, false);
    }
}

// Roles: warps 0 .. NW-1 value chains; warp NW stages the deflator blocks.
// The warps are not synchronised with each other after the table staging:
// each consumes the staged blocks in order, releasing each buffer with an
// mbarrier arrival; the producer refills a buffer once all NW warps have
// released it.  The per-scenario sums of an item are joined by the warp that
// finishes the item last (a shared-memory counter), in warp order.
template <int P, int M, int NW, int NBUF, int MINB, int X2>
__global__ void __launch_bounds__((NW + 1) * 32, MINB) defl_kernel(const DeflArgs a) {
    using SM = DeflSmem<P, M, NW, NBUF>;
    constexpr int CH = SM::CH, W = NW * P;
    constexpr int kLast = 1 << 30;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t tbar;
    __shared__ int red_cnt[2];
    __shared__ volatile int done_items, abort_flag;
    __shared__ uint32_t tmem_slot;
    unsigned char* base = smem_raw + a.tab_bytes;
    float4* ring = reinterpret_cast<float4*>(base);
    float2* red = reinterpret_cast<float2*>(base + SM::ring);
    DeflSlot* sslot = reinterpret_cast<DeflSlot*>(base + SM::ring + SM::red);
    DeflBlock* hdr = reinterpret_cast<DeflBlock*>(base + SM::ring + SM::red + SM::slots);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + SM::ring + SM::red + SM::slots + SM::hdr);
    uint64_t* empty = full + NBUF;

    if (!stage_to_smem(smem_raw, a.tab, (uint32_t)a.tab_bytes, &tbar, a.status)) return;
    const float4* tab = reinterpret_cast<const float4*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr uint32_t row_bytes = CH * sizeof(float4), blk_bytes = DEFL_G * row_bytes;

    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], NW);
        }
        fence_barrier_init();
        red_cnt[0] = red_cnt[1] = 0;
        done_items = 0;
        abort_flag = 0;
    }
    constexpr uint32_t kCols = X2 == 3 ? 2 * kDeflTmemCols : kDeflTmemCols;
    if constexpr (X2 >= 2) {   // 32 (64) TMEM columns for each valuing warp of a lane quarter
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tmem_slot)),
                         "r"(kCols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if constexpr (X2 >= 2) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (warp == NW) {
        // ---------------- producer: lane 0 claims items and stages their blocks
        if (lane != 0) return;
        int k = 0;
        for (int q = 0;; ++q) {
            const int it = atomicAdd(a.counter, 1);
            const bool more = it < a.n_items;
            int jmax = 0, chunk = 0;
            if (more) {
                const int stt = it / a.n_chunks;
                chunk = it - stt * a.n_chunks;
                const int Smax = a.slots[(size_t)stt * W].S;
                jmax = Smax > 0 ? (Smax - 1) / DEFL_KB : 0;
                // item q writes partial-sum slot q & 1, last used by item q - 2
                if (q >= 2) {
                    uint32_t n = 0;
                    while (done_items < q - 1 && !abort_flag && ++n < kWaitLimit) __nanosleep(64);
                    if (done_items < q - 1) abort_flag = 1;
                    __threadfence_block();   // the slot's reset is seen before its reuse is released
                }
            }
            for (int j = jmax; j >= 0 && !abort_flag; --j, ++k) {
                const int b = k % NBUF;
                if (k >= NBUF && !mbar_wait_bounded(&empty[b], (uint32_t)(((k / NBUF) - 1) & 1), kWaitLimit)) {
                    abort_flag = 1;
                    break;
                }
                if (!more) {   // no more work: a closing header, no copy
                    hdr[b] = DeflBlock{-1, 0, 0, 0};
                    defl_mbar_arrive(&full[b]);
                    break;
                }
                hdr[b] = DeflBlock{it, j, j == jmax ? 1 : 0, q | (j == 0 ? kLast : 0)};
                constexpr uint32_t slot_bytes = (uint32_t)(W * sizeof(DeflSlot));
                mbar_arrive_expect_tx(&full[b], blk_bytes + (j == jmax ? slot_bytes : 0u));
                if (j == jmax)   // the item's slot records, with its first block, into area q & 1
                    bulk_g2s(sslot + (size_t)(q & 1) * W, a.slots + (size_t)(it / a.n_chunks) * W, slot_bytes,
                             &full[b]);
                const float4* src = a.D + (size_t)j * DEFL_G * a.s_pad + (size_t)chunk * CH;
                for (int r = 0; r < DEFL_G; ++r)
                    bulk_g2s(ring + ((size_t)b * DEFL_G + r) * CH, src + (size_t)r * a.s_pad, row_bytes, &full[b]);
            }
            if (!more || abort_flag) break;
        }
        if (abort_flag) {
            atomicExch(a.status, DEV_TIMEOUT);
            // let the copies still in flight land before the CTA exits
            for (int q = 1; q <= NBUF && k - q >= 0; ++q)
                mbar_wait_bounded(&full[(k - q) % NBUF], (uint32_t)(((k - q) / NBUF) & 1), kWaitLimit);
        }
        return;
    }

    // -------------------- consumers
    using Lane = typename std::conditional<
        X2 == 3, DeflLaneTM2<P, M>,
        typename std::conditional<X2 == 2, DeflLaneTM<P, M>,
                                  typename std::conditional<X2 == 1, DeflLaneX2<P, M>, DeflLane<P, M>>::type>::type>::type;
    constexpr bool kTm = X2 >= 2;
    Lane st;
    if constexpr (kTm)
        st.taddr = tmem_slot + (((uint32_t)(warp & 3) * 32u) << 16) + (uint32_t)(warp >> 2) * (kCols / 4);
    int smin = 0, smax = 0, kind = K_ANN, stt = 0, chunk = 0;
    for (int k = 0;; ++k) {
        const int b = k % NBUF;
        if (!mbar_wait_bounded(&full[b], (uint32_t)((k / NBUF) & 1), kWaitLimit)) {
            abort_flag = 1;
            if (lane == 0) atomicExch(a.status, DEV_TIMEOUT);
            break;
        }
        const DeflBlock hb = hdr[b];
        if (hb.item < 0) break;
        // this warp's P slot records of the item, staged with its first block
        const DeflSlot* rec = sslot + (size_t)(hb.q & 1) * W + warp * P;
        if (hb.first) {   // a new item: this warp's P policies
            stt = hb.item / a.n_chunks;
            chunk = hb.item - stt * a.n_chunks;
            kind = rec[0].kind;
            smin = 1 << 30;
            smax = 0;
            float h0all[P][M];
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int4 q4 = *reinterpret_cast<const int4*>(&rec[i].off1);   // off1, off2, S, pol
                const int S = q4.w < 0 ? 0 : q4.z;
                const float mat = rec[i].mat;
                smin = min(smin, S);
                smax = max(smax, S);
                float h0s[M];
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    float h0 = 0.0f;
                    if (mat != 0.0f && q4.w >= 0) {   // U_S = D_S l_{x+S} bnd
                        float dS = 1.0f;
                        if (S > 0) {
                            const int t = S - 1, s = chunk * CH + m * 32 + lane;
                            dS = reinterpret_cast<const float*>(a.D + (size_t)(t >> 2) * a.s_pad + s)[t & 3];
                        }
                        h0 = __fmul_rn(dS, mat);
                    }
                    h0s[m] = h0;
                    h0all[i][m] = h0;
                }
                if constexpr (!kTm) st.start(i, h0s);
            }
            if constexpr (kTm) st.start_all(h0all);
        }
        const float4* ring_b = ring + (size_t)b * DEFL_G * CH;
        if (kind == K_ANN) defl_block<K_ANN, P, M>(st, defl_pol<K_ANN, P>(rec), tab, ring_b, hb.j, lane, smin, smax);
        else if (kind == K_ASS) defl_block<K_ASS, P, M>(st, defl_pol<K_ASS, P>(rec), tab, ring_b, hb.j, lane, smin, smax);
        else if (kind == K_JL) defl_block<K_JL, P, M>(st, defl_pol<K_JL, P>(rec), tab, ring_b, hb.j, lane, smin, smax);
        else defl_block<K_ANN2, P, M>(st, defl_pol<K_ANN2, P>(rec), tab, ring_b, hb.j, lane, smin, smax);
        __syncwarp();
        if (lane == 0) defl_mbar_arrive(&empty[b]);   // this warp is done with buffer b

        if (hb.q & kLast) {   // epilogue: scale, write V0, join the per-scenario sums
            float ph[M], pl[M];
#pragma unroll
            for (int m = 0; m < M; ++m) ph[m] = pl[m] = 0.0f;
            float Hall[P][M], Lall[P][M];
            if constexpr (kTm) st.sum_all(Hall, Lall);
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int pol = rec[i].pol;
                if (pol < 0) continue;
                const float sh = rec[i].sc_h, sl = rec[i].sc_l;
                float Hs[M], Ls[M];
                if constexpr (kTm) {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        Hs[m] = Hall[i][m];
                        Ls[m] = Lall[i][m];
                    }
                } else {
                    st.sum(i, Hs, Ls);
                }
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const int s = chunk * CH + m * 32 + lane;
                    if (s >= a.n_scen) continue;
                    const float H = Hs[m], L = Ls[m];
                    const size_t o = (size_t)pol * a.v0_ld + s;
                    // (H + L)(sh + sl) as a double-float, for V0 and the sums
                    const float p = __fmul_rn(H, sh);
                    float e = __fmaf_rn(H, sh, -p);
                    e = __fmaf_rn(H, sl, e);
                    e = __fmaf_rn(L, sh, e);
                    if (a.V0f) a.V0f[o] = __fadd_rn(p, e);
                    if (a.V0d) a.V0d[o] = ((double)H + (double)L) * rec[i].scale;
                    defl_fold(ph[m], pl[m], p);
                    pl[m] = __fadd_rn(pl[m], e);
                }
            }
            // every warp reports; the last one joins the sums and releases the
            // item's areas (partial sums and slot records) for item q + 2
            const int slot = hb.q & 1;
            float2* rs = red + (size_t)slot * NW * CH;
            if (a.partial) {
#pragma unroll
                for (int m = 0; m < M; ++m) rs[warp * CH + m * 32 + lane] = make_float2(ph[m], pl[m]);
            }
            __threadfence_block();
            __syncwarp();
            int old = 0;
            if (lane == 0) old = atomicAdd(&red_cnt[slot], 1);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == NW - 1) {
                if (a.partial) {
                    // the last warp of this item joins the NW double-floats in a
                    // fixed order (warp 0 first) with an exact TwoSum on the heads,
                    // in FP32: GB300's narrow FP64 pipe took a warp-instruction per
                    // 64 cycles here; only the result is widened to FP64
                    __threadfence_block();
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int c = m * 32 + lane;
                        float h = 0.0f, l = 0.0f;
                        for (int w = 0; w < NW; ++w) {
                            const float2 v = rs[w * CH + c];
                            const float s = __fadd_rn(h, v.x);
                            const float bb = __fsub_rn(s, h);
                            const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(v.x, bb));
                            h = s;
                            l = __fadd_rn(l, __fadd_rn(e, v.y));
                        }
                        a.partial[(size_t)stt * a.part_ld + chunk * CH + c] = (double)h + (double)l;
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    red_cnt[slot] = 0;
                    __threadfence_block();
                    atomicAdd((int*)&done_items, 1);
                }
            }
        }
        if (abort_flag) break;
    }
    if constexpr (kTm) {   // every valuing warp is done with its columns
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        asm volatile("bar.sync 1, %0;" ::"n"(NW * 32) : "memory");
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"(kCols)
                         : "memory");
    }
}

// ------------------------------------------------------ variant registry ----
struct DeflVariant {
    int P, M, NW, NBUF;
    const char* name;
    cudaError_t (*launch)(const DeflArgs&, int grid, size_t smem, cudaStream_t st);
    cudaError_t (*occupancy)(int* blocks_per_sm, size_t smem);
};

template <int P, int M, int NW, int NBUF, int MINB, int X2>
cudaError_t set_defl_attributes(size_t smem) {
    auto k = defl_kernel<P, M, NW, NBUF, MINB, X2>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

template <int P, int M, int NW, int NBUF, int MINB, int X2>
cudaError_t launch_defl(const DeflArgs& a, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = set_defl_attributes<P, M, NW, NBUF, MINB, X2>(smem);
    if (e != cudaSuccess) return e;
    defl_kernel<P, M, NW, NBUF, MINB, X2><<<grid, (NW + 1) * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int P, int M, int NW, int NBUF, int MINB, int X2>
cudaError_t occupancy_defl(int* blocks, size_t smem) {
    cudaError_t e = set_defl_attributes<P, M, NW, NBUF, MINB, X2>(smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, defl_kernel<P, M, NW, NBUF, MINB, X2>,
                                                         (NW + 1) * 32, smem);
}

#define RSV_DEFL_VARIANT(P, M, NW, NBUF, MINB, X2, NAME)                                              \
    DeflVariant {                                                                                         \
        P, M, NW, NBUF, NAME, &launch_defl<P, M, NW, NBUF, MINB, X2>, &occupancy_defl<P, M, NW, NBUF, MINB, X2> \
    }

const DeflVariant* variants_defl(int* n);
// smem bytes of a variant beyond its staged tables
size_t defl_smem_extra(const DeflVariant& v);

}  // namespace rsv
