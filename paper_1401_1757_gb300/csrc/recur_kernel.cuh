// recur_kernel.cuh -- the backward vector reserve recurrence on sm_103a.
//
// Eq. (generalForm) of Tucker & Bull with f = 1 and zero-reserve states
// removed (Section 3.6.4) becomes, per policy and scenario, per unit amount:
//   K_ANN  r_t = v_t p_t (1 + r_{t+1})                          (Section 4.1.1)
//   K_ASS  r_t = v_t (q_t + p_t r_{t+1})                        (Section 4.1.3)
//   K_JL   three states of the two-life model (Section 4.2), c = (1, 1, rho):
//            r01 = v px (1 + r01')          r10 = v py (rho + r10')
//            r00 = v [px py (1 + r00') + px qy (1 + r01') + qx py (rho + r10')].
//          With independent lives the reduced vector is, at every step, a
//          combination of three single-state annuities (the reversionary
//          annuity a_{x|y} = a_y - a_xy of Section 4.2.1):
//            r00 = a_x + rho (a_y - a_xy),  r01 = a_x,  r10 = rho a_y,
//            a_x = v px (1 + a_x'),  a_y = v py (1 + a_y'),  a_xy = v px py (1 + a_xy'),
//          which is the recurrence above regrouped (substitute and use
//          px + qx = 1), for any payment time within the step and any
//          cash-flow sequence.  The kernel runs the three annuity chains.
//   K_LS2  the nine-state two-life assurance model (Section 4.2.3) with the
//          benefit on the second death, reduced to the states 00, x only,
//          y only (the "died in the step" and "dead" states of the other
//          life share a reserve; both-dead states are zero-reserve states):
//            rx = v (qx + px rx')           ry = v (qy + py ry')
//            r00 = v [qx qy + px qy rx' + qx py ry' + px py r00']
// run backward from the boundary r_S (Section 3.8.2).
//
// Mapping.  A work item is one tile of P policies (same kind, similar S) times
// one chunk of 32*M scenarios, owned by one warp: lane l holds scenarios
// s0 .. s0+M-1 of all P policies (P*M chains in registers).  Per step a lane
// makes one vector load of its M discount factors (coalesced across the
// warp, step-major plane) and, per policy, one shared-memory broadcast of the
// decrement-table entry.  The table is staged once per CTA by TMA.  Warps
// claim items from an atomic queue in decreasing-cost order (persistent grid,
// no inter-warp synchronisation after staging).
#pragma once

#include <type_traits>

#include "rsv_device.cuh"

namespace rsv {

// ---------------------------------------------------------------- traits ----
template <int FORM>
struct Tr;

template <>
struct Tr<F_F64> {
    using Val = double;
    using TabE = double2;  // (p, q)
    using VE = double;
    __device__ static Val p(const TabE& e) { return e.x; }
    __device__ static Val q(const TabE& e) { return e.y; }
    __device__ static Val v(const VE& e) { return e; }
    __device__ static Val pair(float h, float l) { return (double)h + (double)l; }
    __device__ static Val cst(float x) { return (double)x; }
    __device__ static double dbl(Val x) { return x; }
};

template <>
struct Tr<F_F32> {
    using Val = float;
    using TabE = float2;   // (p, q)
    using VE = float;
    __device__ static Val p(const TabE& e) { return e.x; }
    __device__ static Val q(const TabE& e) { return e.y; }
    __device__ static Val v(const VE& e) { return e; }
    __device__ static Val pair(float h, float) { return h; }
    __device__ static Val cst(float x) { return x; }
    __device__ static double dbl(Val x) { return (double)x; }
};

template <>
struct Tr<F_COMP> {
    using Val = df;
    using TabE = float4;   // (p_hi, p_lo, q_hi, q_lo)
    using VE = float2;     // (v_hi, v_lo)
    __device__ static Val p(const TabE& e) { return df{e.x, e.y}; }
    __device__ static Val q(const TabE& e) { return df{e.z, e.w}; }
    __device__ static Val v(const VE& e) { return df{e.x, e.y}; }
    __device__ static Val pair(float h, float l) { return df{h, l}; }
    __device__ static Val cst(float x) { return df{x, 0.0f}; }
    __device__ static double dbl(Val x) { return df_to_double(x); }
};

// ------------------------------------------------------- step arithmetic ----
// Plain forms (double or float): explicit roundings and fused multiply-adds.
__device__ __forceinline__ float p_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double p_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float p_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double p_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float p_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double p_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class R>
__device__ __forceinline__ R step_ann(R v, R p, R V) {       // v p (1 + V)
    R g = p_mul(v, p);
    return p_fma(g, V, g);
}
template <class R>
__device__ __forceinline__ R step_ass(R v, R p, R q, R V) {  // v (q + p V)
    return p_mul(v, p_fma(p, V, q));
}
// Joint status "both alive" of two independent lives: p = px py and
// q = 1 - px py = qx + px qy (the latter without cancellation).
template <class R>
__device__ __forceinline__ void joint_pq(R px, R qx, R py, R qy, R& p, R& q) {
    p = p_mul(px, py);
    q = p_fma(px, qy, qx);
}
// The reversionary annuity's three annuity chains: Vxy = a_xy, Vx = a_x, Vy = a_y.
template <class R>
__device__ __forceinline__ void step_jl(R v, R px, R py, R& Vxy, R& Vx, R& Vy) {
    const R gx = p_mul(v, px), gy = p_mul(v, py), gxy = p_mul(gx, py);
    Vx = p_fma(gx, Vx, gx);                     // v px (1 + a_x')
    Vy = p_fma(gy, Vy, gy);                     // v py (1 + a_y')
    Vxy = p_fma(gxy, Vxy, gxy);                 // v px py (1 + a_xy')
}
// Second-death assurance, benefit c per unit amount in this step.
template <class R>
__device__ __forceinline__ void step_ls2(R v, R px, R qx, R py, R qy, R c, R& V00, R& Vx, R& Vy) {
    R t = p_mul(p_mul(qx, py), Vy);             // qx py ry'
    t = p_fma(p_mul(px, qy), Vx, t);            //   + px qy rx'
    t = p_fma(p_mul(qx, qy), c, t);             //   + qx qy c
    V00 = p_mul(v, p_fma(p_mul(px, py), V00, t));
    Vx = p_mul(v, p_fma(px, Vx, p_mul(qx, c)));
    Vy = p_mul(v, p_fma(py, Vy, p_mul(qy, c)));
}

// Compensated form.  Quantities that multiply along the chain (the discount
// x survival factors and the running reserve) are double-floats built from
// hi/lo inputs, so their per-step error stays near 2^-44 and cannot compound.
// Terms injected additively at one step (the assurance's death probability
// q, the reversion rho, and the JL one-step death transitions qy r01 + qx r10)
// enter the reserve once, weighted by their own share of it, so their FP32
// rounding bounds the relative error of every r_t by a few 2^-24 (~2e-7)
// however long the projection.  The double-floats are never renormalised:
// their tails carry the accumulated compensation and grow to ~1e-5 of the
// head over a thousand steps, so a computed value enters an FP32 term as
// head + tail, not as its head alone.
//
// Annuity-type states are carried shifted, R = 1 + r (boundary R_S = 1):
// r_t = g_t (1 + r_{t+1}) becomes R_t = 1 + g_t R_{t+1}, one df_one_plus_mul;
// the JL product's three annuity chains likewise.
__device__ __forceinline__ df step_ann(df v, df p, df R) {
    return df_one_plus_mul(df_mul(v, p), R);
}
__device__ __forceinline__ df step_ass(df v, df p, df q, df V) {
    return df_mul(v, df_add_float_pos(df_mul(p, V), q.h));
}
// the joint survival as a double-float product; q enters one step additively (FP32 head)
__device__ __forceinline__ void joint_pq(df px, df qx, df py, df qy, df& p, df& q) {
    p = df_mul(px, py);
    q = df{__fmaf_rn(px.h, qy.h, qx.h), 0.0f};
}
// The reversionary annuity's three annuity chains, shifted: Vxy = 1 + a_xy,
// Vx = 1 + a_x, Vy = 1 + a_y.
__device__ __forceinline__ void step_jl(df v, df px, df py, df& Vxy, df& Vx, df& Vy) {
    const df gx = df_mul(v, px), gy = df_mul(v, py);
    const df gxy = df_mul(gx, py);
    Vx = df_one_plus_mul(gx, Vx);
    Vy = df_one_plus_mul(gy, Vy);
    Vxy = df_one_plus_mul(gxy, Vxy);
}
// Second-death assurance: the survival chain px py r00' in double-float; the
// one-step terms qx qy c + px qy rx' + qx py ry' (non-negative) in FP32.
__device__ __forceinline__ void step_ls2(df v, df px, df qx, df py, df qy, float c, df& V00, df& Vx, df& Vy) {
    const float rx = __fadd_rn(Vx.h, Vx.l), ry = __fadd_rn(Vy.h, Vy.l);
    float t = __fmul_rn(__fmul_rn(qx.h, py.h), ry);
    t = __fmaf_rn(__fmul_rn(px.h, qy.h), rx, t);
    t = __fmaf_rn(__fmul_rn(qx.h, qy.h), c, t);
    V00 = df_mul(v, df_add_float_pos(df_mul(df_mul(px, py), V00), t));
    Vx = df_mul(v, df_add_float_pos(df_mul(px, Vx), __fmul_rn(qx.h, c)));
    Vy = df_mul(v, df_add_float_pos(df_mul(py, Vy), __fmul_rn(qy.h, c)));
}

// Annuity-type steps with the payment at the start of the step (f = 0, a = 1),
// at the fraction f (a = v^f p^f, the fractional cash-flow term of
// Eq. generalForm) or with a varying cash flow, on unshifted states:
// r = a + v p r'.  The JL product runs its three annuity chains this way too.
template <class R>
__device__ __forceinline__ R step_ann_a(R a, R g, R V) { return p_fma(g, V, a); }
// Compensated: the one-step cash-flow term in FP32 (it enters once, weighted
// by its share), the products along the chain in double-float.
__device__ __forceinline__ df step_ann_a(float a, df g, df V) { return df_float_plus_mul(a, g, V); }

// M consecutive scenario-plane elements of one lane, one vector load.
template <class E, int M>
struct alignas(sizeof(E) * M) Pack {
    E e[M];
};

// ------------------------------------------------------------- one item ----
// Where a tile reads its discount factors and writes its side outputs.
struct TileEnv {
    const SlotRec* slots;
    const void* v;       // scenario plane, rows = steps from the valuation point, [rows][s_pad]
    int s_pad;
    int n_valid;         // valid scenario columns
    int n_steps;         // side-output row length - 1
    const double* amount;
    double* traj;
    double* pt_sum;
    int v0_ld;           // row stride of V0 (the caller's scenario count)
    const void* vf;      // fractional discount plane (PAY_FRACTION), layout of v
    int tabf_off;        // entries from the staged tables to the fractional ones (PAY_FRACTION)
    const void* cf;      // cash-flow multipliers [n_pol][cf_ld] or null (variants other than PAY_END)
    int cf_ld;
};

template <int FORM, int P, int M, int KIND, bool EXTRA, int PAY = PAY_END>
struct Tile {
    using T = Tr<FORM>;
    using Val = typename T::Val;
    using TabE = typename T::TabE;
    using VE = typename T::VE;
    using VP = Pack<VE, M>;
    static constexpr int NS = (KIND == K_JL || KIND == K_LS2) ? 3 : 1;

    const TileEnv& e;
    const TabE* __restrict__ tab;
    const VE* __restrict__ vplane;
    int s0;
    int idx1[P], idx2[P], Sp[P], st0[P], pol[P];
    Val rho[P];
    double amt[P];
    Val V[NS][P][M];

    // t_off > 0 starts every policy of the tile t_off steps after valuation (a
    // valuation node of the nested run): ages advance by t_off, the remaining
    // projection is S - t_off, and row 0 of the plane is the node's first step.
    // Policies already past their end (S < t_off) become padding.
    __device__ __forceinline__ Tile(const TileEnv& env, const TabE* t, int tile, int chunk, int lane,
                                    int t_off = 0)
        : e(env), tab(t), vplane(static_cast<const VE*>(env.v)) {
        s0 = (chunk * 32 + lane) * M;
        const SlotRec* rec = e.slots + (size_t)tile * P;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const SlotRec r = rec[i];
            idx1[i] = r.idx1 + t_off;
            idx2[i] = r.idx2 + t_off;
            Sp[i] = r.S - t_off;
            st0[i] = r.state0;
            pol[i] = Sp[i] < 0 ? -1 : r.pol;
            rho[i] = T::pair(r.rho_h, r.rho_l);
            amt[i] = (EXTRA && pol[i] >= 0) ? e.amount[pol[i]] : 0.0;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                V[0][i][m] = T::cst(SHIFTED ? 1.0f + r.bnd : r.bnd);
#pragma unroll
                for (int k = 1; k < NS; ++k)   // the second-death endowment pays if either is alive
                    V[k][i][m] = T::cst(SHIFTED ? 1.0f : (KIND == K_LS2 ? r.bnd : 0.0f));
            }
        }
    }

    __device__ __forceinline__ VP load(int t) const {
        return *reinterpret_cast<const VP*>(vplane + (size_t)t * e.s_pad + s0);
    }

    // The compensated form carries annuity-type states shifted (see step_ann):
    // the ANN state and the JL product's three annuity chains as 1 + a.
    static constexpr bool ANNUITY = KIND == K_ANN || KIND == K_ANN2 || KIND == K_JL;
    static constexpr bool SHIFTED = FORM == F_COMP && ANNUITY && PAY == PAY_END;
    // payment within the step, or general cash flows: unshifted states
    static constexpr bool PAYF = ANNUITY && PAY != PAY_END;
    // the JL product as the annuity chains (a_xy, a_x, a_y)
    static constexpr bool JLDEC = KIND == K_JL;

    // the one-step terms: FP32 heads in the compensated form
    using A = typename std::conditional<FORM == F_COMP, float, Val>::type;
    using CfE = typename std::conditional<FORM == F_F64, double, float>::type;
    // c_t / c of policy i (1 for a level cash flow; warp-uniform load)
    __device__ __forceinline__ A cfac(int i, int t) const {
        if (PAY == PAY_END || e.cf == nullptr || pol[i] < 0) return A(1);
        return (A) static_cast<const CfE*>(e.cf)[(size_t)pol[i] * e.cf_ld + t];
    }

    // r of state k of policy i, scenario m, in FP64
    __device__ __forceinline__ double dval(int k, int i, int m) const {
        if constexpr (JLDEC) {   // r00 = a_x + rho (a_y - a_xy), r01 = a_x, r10 = rho a_y
            const double off = SHIFTED ? 1.0 : 0.0, r = T::dbl(rho[i]);
            if (k == 1) return T::dbl(V[1][i][m]) - off;
            if (k == 2) return r * (T::dbl(V[2][i][m]) - off);
            return (T::dbl(V[1][i][m]) - off) + r * (T::dbl(V[2][i][m]) - T::dbl(V[0][i][m]));
        }
        const double x = T::dbl(V[k][i][m]);
        if constexpr (SHIFTED) return x - 1.0;
        return x;
    }

    // (the state is selected among compile-time indices: a runtime index into
    // V would move the whole register array to local memory)
    __device__ __forceinline__ double out_state(int i, int m) const {
        if constexpr (NS == 1) {
            return dval(0, i, m);
        } else {
            const double x0 = dval(0, i, m), x1 = dval(1, i, m), x2 = dval(2, i, m);
            return st0[i] == 0 ? x0 : (st0[i] == 1 ? x1 : x2);
        }
    }

    // traj / pt_mean side outputs of r_t for policy i (diagnostic runs only)
    __device__ __forceinline__ void record(int t, int i) {
        if (pol[i] < 0) return;
        double sum = 0.0;
        const size_t row = (size_t)pol[i] * (e.n_steps + 1) + t;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int s = s0 + m;
            if (s < e.n_valid) {
                const double x = amt[i] * out_state(i, m);
                if (e.traj) e.traj[row * e.n_valid + s] = x;
                sum += x;
            }
        }
        if (e.pt_sum) {
            // a fixed order: a butterfly over the lanes, then the tile's warp
            // adds its scenario chunks one after the other (recur_kernel gives
            // every chunk of a tile to one warp when side outputs are on)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if ((threadIdx.x & 31) == 0) e.pt_sum[row] += sum;
        }
    }

    // the fractional cash-flow terms need v^f of this step (PAY_FRACTION)
    __device__ __forceinline__ VP loadf(int t) const {
        return *reinterpret_cast<const VP*>(static_cast<const VE*>(e.vf) + (size_t)t * e.s_pad + s0);
    }

    template <bool CHECK>
    __device__ __forceinline__ void step(int t, const VP& vv) {
        if constexpr (PAYF) {
            step_pay<CHECK>(t, vv);
        } else {
            step_end<CHECK>(t, vv);
        }
    }

    // payment at the end of the step
    template <bool CHECK>
    __device__ __forceinline__ void step_end(int t, const VP& vv) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (CHECK && t >= Sp[i]) continue;
            const TabE e1 = tab[idx1[i] + t];
            const Val px = T::p(e1), qx = T::q(e1);
            if constexpr (KIND == K_JL) {
                const Val py = T::p(tab[idx2[i] + t]);
#pragma unroll
                for (int m = 0; m < M; ++m) step_jl(T::v(vv.e[m]), px, py, V[0][i][m], V[1][i][m], V[2][i][m]);
            } else if constexpr (KIND == K_LS2) {
                const TabE e2 = tab[idx2[i] + t];
                const Val py = T::p(e2), qy = T::q(e2);
                const A c = cfac(i, t);
#pragma unroll
                for (int m = 0; m < M; ++m)
                    step_ls2(T::v(vv.e[m]), px, qx, py, qy, c, V[0][i][m], V[1][i][m], V[2][i][m]);
            } else if constexpr (KIND == K_ANN2 || KIND == K_ASS2) {
                const TabE e2 = tab[idx2[i] + t];
                Val p, q;
                joint_pq(px, qx, T::p(e2), T::q(e2), p, q);
                if constexpr (KIND == K_ASS2 && PAY != PAY_END) q = scale_q(q, cfac(i, t));
#pragma unroll
                for (int m = 0; m < M; ++m)
                    V[0][i][m] = KIND == K_ANN2 ? step_ann(T::v(vv.e[m]), p, V[0][i][m])
                                                : step_ass(T::v(vv.e[m]), p, q, V[0][i][m]);
            } else if constexpr (KIND == K_ANN) {
#pragma unroll
                for (int m = 0; m < M; ++m) V[0][i][m] = step_ann(T::v(vv.e[m]), px, V[0][i][m]);
            } else {
                Val q = qx;   // the death benefit of this step, c_t / c times the level one
                if constexpr (PAY != PAY_END) q = scale_q(q, cfac(i, t));
#pragma unroll
                for (int m = 0; m < M; ++m) V[0][i][m] = step_ass(T::v(vv.e[m]), px, q, V[0][i][m]);
            }
            if constexpr (EXTRA) record(t, i);
        }
    }

    // q c_t / c: the compensated assurance step takes the death term as an FP32 head
    __device__ static __forceinline__ df scale_q(df q, float c) { return df{__fmul_rn(q.h, c), 0.0f}; }
    __device__ static __forceinline__ float scale_q(float q, float c) { return p_mul(q, c); }
    __device__ static __forceinline__ double scale_q(double q, double c) { return p_mul(q, c); }

    // Annuity-type step with the payment at the start of the step, at the
    // fraction f, or at the end with a varying cash flow: r = a + v W r' with
    // the cash-flow term a = v^f W_f c_t.
    template <bool CHECK>
    __device__ __forceinline__ void step_pay(int t, const VP& vv) {
        VP vf{};
        if constexpr (PAY == PAY_FRACTION) vf = loadf(t);
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (CHECK && t >= Sp[i]) continue;
            const TabE e1 = tab[idx1[i] + t];
            const Val px = T::p(e1), qx = T::q(e1);
            TabE e2{}, f1{}, f2{};
            if constexpr (KIND != K_ANN) e2 = tab[idx2[i] + t];
            if constexpr (PAY == PAY_FRACTION) {
                f1 = tab[e.tabf_off + idx1[i] + t];
                if constexpr (KIND != K_ANN) f2 = tab[e.tabf_off + idx2[i] + t];
            } else if constexpr (PAY == PAY_END_GENERAL) {   // W_f = W_1
                f1 = e1;
                f2 = e2;
            }
            const A c = cfac(i, t);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const Val v = T::v(vv.e[m]);
                A vfm = c, pxf = A(1), pyf = A(1);
                if constexpr (PAY == PAY_FRACTION || PAY == PAY_END_GENERAL) {
                    vfm = (PAY == PAY_FRACTION ? head(T::v(vf.e[m])) : head(v)) * c;
                    pxf = head(T::p(f1));
                    if constexpr (KIND != K_ANN) pyf = head(T::p(f2));
                }
                if constexpr (KIND == K_JL) {   // the chains a_x, a_y, a_xy
                    const Val py = T::p(e2);
                    const A ax = vfm * pxf, ay = vfm * pyf, axy = ax * pyf;
                    if constexpr (FORM == F_COMP) {
                        const df gx = df_mul(v, px);
                        V[1][i][m] = step_ann_a(ax, gx, V[1][i][m]);
                        V[2][i][m] = step_ann_a(ay, df_mul(v, py), V[2][i][m]);
                        V[0][i][m] = step_ann_a(axy, df_mul(gx, py), V[0][i][m]);
                    } else {
                        const Val gx = p_mul(v, px);
                        V[1][i][m] = step_ann_a(ax, gx, V[1][i][m]);
                        V[2][i][m] = step_ann_a(ay, p_mul(v, py), V[2][i][m]);
                        V[0][i][m] = step_ann_a(axy, p_mul(gx, py), V[0][i][m]);
                    }
                } else {
                    Val p = px;
                    A a = vfm * pxf;
                    if constexpr (KIND == K_ANN2) {
                        Val q;
                        joint_pq(px, qx, T::p(e2), T::q(e2), p, q);
                        a = a * pyf;
                    }
                    if constexpr (FORM == F_COMP) {
                        V[0][i][m] = step_ann_a(a, df_mul(v, p), V[0][i][m]);
                    } else {
                        V[0][i][m] = step_ann_a(a, p_mul(v, p), V[0][i][m]);
                    }
                }
            }
        }
    }
    // the leading part of a value (the head of a double-float), for one-step terms
    __device__ static __forceinline__ float head(df x) { return x.h; }
    __device__ static __forceinline__ float head(float x) { return x; }
    __device__ static __forceinline__ double head(double x) { return x; }

    static constexpr int U = 4;   // steps per prefetch group

    __device__ __forceinline__ void load_group(VP (&g)[U], int t) const {
#pragma unroll
        for (int u = 0; u < U; ++u) g[u] = load(t - u);
    }
    __device__ __forceinline__ void run_group(const VP (&g)[U], int t) {
#pragma unroll
        for (int u = 0; u < U; ++u) step<false>(t - u, g[u]);
    }

    // Backward substitution from each policy's boundary down to t = 0.
    __device__ __forceinline__ void run_steps() {
        const int Smax = Sp[0];
        const int Smin = Sp[P - 1] > 0 ? Sp[P - 1] : 0;
        if constexpr (EXTRA) {
            // r at t = S_i (the boundary) for the side outputs
#pragma unroll
            for (int i = 0; i < P; ++i)
                if (Sp[i] >= 0 && Sp[i] <= e.n_steps) record(Sp[i], i);
        }
        int t = Smax - 1;
        for (; t >= Smin; --t) step<true>(t, load(t));      // ragged head: some policies idle
        if (t + 1 >= 2 * U) {                                 // bulk: double-buffered groups
            VP A[U], B[U];
            load_group(A, t);
            for (;;) {
                bool more = (t - U + 1) >= U;
                if (more) load_group(B, t - U);
                run_group(A, t);
                t -= U;
                if (!more) break;
                more = (t - U + 1) >= U;
                if (more) load_group(A, t - U);
                run_group(B, t);
                t -= U;
                if (!more) break;
            }
        }
        for (; t >= 0; --t) step<false>(t, load(t));
    }

    // Epilogue of a valuation run: scale by the amount, write V0, per-tile
    // scenario sums.
    __device__ __forceinline__ void epilogue_v0(int tile, float* V0f, double* V0d, double* partial) {
        double part[M];
#pragma unroll
        for (int m = 0; m < M; ++m) part[m] = 0.0;
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (pol[i] < 0) continue;
            const double A = e.amount[pol[i]];
#pragma unroll
            for (int m = 0; m < M; ++m) {
                const int s = s0 + m;
                if (s < e.n_valid) {
                    const double x = A * out_state(i, m);
                    const size_t o = (size_t)pol[i] * e.v0_ld + s;
                    if (V0f) V0f[o] = (float)x;
                    if (V0d) V0d[o] = x;
                    part[m] += x;
                }
            }
        }
        if (partial) {
#pragma unroll
            for (int m = 0; m < M; ++m) partial[(size_t)tile * e.s_pad + s0 + m] = part[m];
        }
    }

    // Epilogue of a nested valuation: add sum_j w_j r_j of every policy to acc,
    // with w = amount x in-force probability of each reduced state at the node
    // (wts[pol * stride + j]).
    __device__ __forceinline__ void epilogue_weighted(double (&acc)[M], const double* __restrict__ wts,
                                                      size_t stride) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (pol[i] < 0) continue;
            const double* w = wts + (size_t)pol[i] * stride;
            const double w0 = w[0];
            double w1 = 0.0, w2 = 0.0;
            if constexpr (NS == 3) {
                w1 = w[1];
                w2 = w[2];
            }
#pragma unroll
            for (int m = 0; m < M; ++m) {
                double x = w0 * dval(0, i, m);
                if constexpr (NS == 3) x += w1 * dval(1, i, m) + w2 * dval(2, i, m);
                acc[m] += x;
            }
        }
    }
};

// One work item of one reduced model.
template <int FORM, int P, int M, int KIND, bool EXTRA, int PAY, class TabE>
__device__ __forceinline__ void run_item(const TileEnv& env, const TabE* tab, int tile, int chunk, int lane,
                                         const RecurArgs& a) {
    Tile<FORM, P, M, KIND, EXTRA, PAY> w(env, tab, tile, chunk, lane);
    w.run_steps();
    w.epilogue_v0(tile, a.V0f, a.V0d, a.partial);
}

// TWO: the portfolio has tiles of the other two-life models (K_ANN2, K_ASS2,
// K_LS2).  The kernel is compiled with and without them: the three hot
// models alone keep their register allocation free of spills.
template <int FORM, int P, int M, int NT, int MINB, bool EXTRA, bool TWO, int PAY>
__global__ void __launch_bounds__(NT, MINB) recur_kernel(const RecurArgs a) {
    using TabE = typename Tr<FORM>::TabE;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    TabE* tab = reinterpret_cast<TabE*>(smem_raw);
    if (!stage_to_smem(tab, a.tab, (uint32_t)a.tab_bytes, &bar, a.status)) return;

    const TileEnv env{a.slots, a.v, a.s_pad, a.n_scen, a.n_steps, a.amount, a.traj, a.pt_sum, a.v0_ld, a.vf,
                      a.tabf_off, a.cf, a.cf_ld};
    const int lane = threadIdx.x & 31;
    // With side outputs a work item is a whole tile, its scenario chunks run
    // in order by one warp, so that the per-step sums over scenarios are added
    // in a fixed order; otherwise an item is one (tile, chunk).
    const int n_work = EXTRA ? a.n_tiles : a.n_items;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_work) break;
        if constexpr (EXTRA) {
            const int kind = a.tile_kind[item];
            for (int chunk = 0; chunk < a.n_chunks; ++chunk) {
                if (kind == K_JL) run_item<FORM, P, M, K_JL, EXTRA, PAY>(env, tab, item, chunk, lane, a);
                else if (kind == K_ANN) run_item<FORM, P, M, K_ANN, EXTRA, PAY>(env, tab, item, chunk, lane, a);
                else if (!TWO || kind == K_ASS) run_item<FORM, P, M, K_ASS, EXTRA, PAY>(env, tab, item, chunk, lane, a);
                else if constexpr (TWO) {
                    if (kind == K_ANN2) run_item<FORM, P, M, K_ANN2, EXTRA, PAY>(env, tab, item, chunk, lane, a);
                    else if (kind == K_ASS2) run_item<FORM, P, M, K_ASS2, EXTRA, PAY>(env, tab, item, chunk, lane, a);
                    else run_item<FORM, P, M, K_LS2, EXTRA, PAY>(env, tab, item, chunk, lane, a);
                }
            }
            continue;
        }
        const int tile = item / a.n_chunks;
        const int chunk = item - tile * a.n_chunks;
        const int kind = a.tile_kind[tile];
        if (kind == K_JL) run_item<FORM, P, M, K_JL, EXTRA, PAY>(env, tab, tile, chunk, lane, a);
        else if (kind == K_ANN) run_item<FORM, P, M, K_ANN, EXTRA, PAY>(env, tab, tile, chunk, lane, a);
        else if (!TWO || kind == K_ASS) run_item<FORM, P, M, K_ASS, EXTRA, PAY>(env, tab, tile, chunk, lane, a);
        else if constexpr (TWO) {
            if (kind == K_ANN2) run_item<FORM, P, M, K_ANN2, EXTRA, PAY>(env, tab, tile, chunk, lane, a);
            else if (kind == K_ASS2) run_item<FORM, P, M, K_ASS2, EXTRA, PAY>(env, tab, tile, chunk, lane, a);
            else run_item<FORM, P, M, K_LS2, EXTRA, PAY>(env, tab, tile, chunk, lane, a);
        }
    }
}

// ------------------------------------------------------ variant registry ----
struct Variant {
    int form, P, M, NT;
    bool extra;
    int pay;   // PAY_END, or the variant that pays annuities within the step
    const char* name;
    // [0]: the three single-table/JL models; [1]: also the two-life single-state ones
    cudaError_t (*launch[2])(const RecurArgs&, int grid, size_t smem, cudaStream_t st);
    cudaError_t (*occupancy[2])(int* blocks_per_sm, size_t smem);
};

// Every CTA stages its own copy of the decrement tables: the largest
// shared-memory carveout lets the register-bound number of small CTAs fit.
template <int FORM, int P, int M, int NT, int MINB, bool EXTRA, bool TWO, int PAY>
cudaError_t set_recur_attributes(size_t smem) {
    auto k = recur_kernel<FORM, P, M, NT, MINB, EXTRA, TWO, PAY>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

template <int FORM, int P, int M, int NT, int MINB, bool EXTRA, bool TWO, int PAY>
cudaError_t launch_recur(const RecurArgs& a, int grid, size_t smem, cudaStream_t st) {
    auto k = recur_kernel<FORM, P, M, NT, MINB, EXTRA, TWO, PAY>;
    cudaError_t e = set_recur_attributes<FORM, P, M, NT, MINB, EXTRA, TWO, PAY>(smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

template <int FORM, int P, int M, int NT, int MINB, bool EXTRA, bool TWO, int PAY>
cudaError_t occupancy_recur(int* blocks, size_t smem) {
    auto k = recur_kernel<FORM, P, M, NT, MINB, EXTRA, TWO, PAY>;
    cudaError_t e = set_recur_attributes<FORM, P, M, NT, MINB, EXTRA, TWO, PAY>(smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k, NT, smem);
}

#define RSV_VARIANT_PAY(FORM, P, M, NT, MINB, EXTRA, PAY, NAME)                                              \
    Variant {                                                                                                 \
        FORM, P, M, NT, EXTRA, PAY, NAME,                                                                     \
            {&launch_recur<FORM, P, M, NT, MINB, EXTRA, false, PAY>, &launch_recur<FORM, P, M, NT, MINB, EXTRA, true, PAY>}, \
        {                                                                                                     \
            &occupancy_recur<FORM, P, M, NT, MINB, EXTRA, false, PAY>,                                         \
                &occupancy_recur<FORM, P, M, NT, MINB, EXTRA, true, PAY>                                       \
        }                                                                                                     \
    }
#define RSV_VARIANT(FORM, P, M, NT, MINB, EXTRA, NAME) RSV_VARIANT_PAY(FORM, P, M, NT, MINB, EXTRA, PAY_END, NAME)

// Each form's translation unit defines these.
const Variant* variants_f64(int* n);
const Variant* variants_f32(int* n);
const Variant* variants_comp(int* n);

}  // namespace rsv
