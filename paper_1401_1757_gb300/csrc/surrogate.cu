// surrogate.cu -- the reserve surrogate of the nested valuation's inner loop.
//
// The inner Monte Carlo loop of the nested valuation estimates, for a policy
// in reduced state j at a node with short rate r, E[r_j | r].  Under the
// Vasicek model with deterministic mortality that expectation is exactly the
// recurrence (Eq. generalForm) run on the forward curve P(t+1|r)/P(t|r) (the
// recurrence is linear in the discount products, Eq. basicReserveSummation).
// Labels are that recurrence, in FP64, for sampled (policy, node, state,
// rate) queries of the loaded portfolio; the network learns
// ln(reserve per unit amount) from 16 features.  Held-out queries are scored
// against the same recurrence; buckets (product and state x age x remaining
// term x rate) whose error exceeds the tolerance fall back to the recurrence.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>

#include "ctx.cuh"
#include "abi_guard.cuh"
#include "philox.cuh"
#include "surrogate.cuh"
#include "fp64_series.cuh"

namespace rsv {

// z-score of a node rate under the Vasicek model at month m from r0 (the
// rate at month 0 is r0 itself: anything else is out of the model's range).
// FP32: it only picks a bucket, and calibration and use share this function.
__device__ __forceinline__ float sur_rate_z(int m, double r, double a, double b, double sigma, double r0) {
    const float t = m / 12.0f, af = (float)a, bf = (float)b;
    const float mean = bf + ((float)r0 - bf) * expf(-af * t);
    const float sd = (float)sigma * sqrtf(-expm1f(-2.0f * af * t) / (2.0f * af));
    const float rf = (float)r;
    if (sd > 0.0f) return (rf - mean) / sd;
    return rf == mean ? 0.0f : 1e30f;
}

// Gate bucket of a query: product and state, 10-year age band of the life the
// value depends on (from age 20), 10-year band of the remaining term, and the
// node rate's z-score in half standard deviations (beyond 4 in the last band).
__device__ __forceinline__ int sur_bucket(const PolSur& P, int m, int state, double r, double a, double b,
                                          double sigma, double r0) {
    const int ps = P.product == RSV_SL_ANNUITY ? 0
                   : P.product == RSV_JL_REVERSIONARY ? 1 + state
                   : P.product == RSV_TERM_ASSURANCE ? 4 : 5;
    int age = P.age1;   // the life (or for state 00 the older life) the value depends on
    if (P.product == RSV_JL_REVERSIONARY) age = state == 2 ? P.age2 : (state == 1 ? P.age1 : max(P.age1, P.age2));
    const int ab = min(SUR_NB_AGE - 1, max(0, (age + m - 240) / 120));   // months; truncation as the clamp wants
    const int tb = min(SUR_NB_TERM - 1, max(0, (P.S - m) / 120));
    const float z = sur_rate_z(m, r, a, b, sigma, r0);
    const int rb = fabsf(z) < 4.0f ? min(SUR_NB_R - 2, max(0, (int)floorf(2.0f * z + 8.0f))) : SUR_NB_R - 1;
    return ((ps * SUR_NB_AGE + ab) * SUR_NB_TERM + tb) * SUR_NB_R + rb;
}

namespace {

// Queries: policy uniform, an annual node before the policy's end (at most
// max_node_m), a reduced state its lives can be in, and a short rate from the
// model's distribution at that month widened by `widen` standard deviations.
__global__ void sample_queries_kernel(const PolSur* __restrict__ pols, int n_pol, uint64_t seed, uint32_t stream,
                                      long long n, double a, double b, double sigma, double r0, double widen,
                                      int max_node_m, SurQuery* __restrict__ out) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double inv32 = 2.3283064365386963e-10;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        uint32_t w[4], g[4];
        philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), 0u, stream << 24, k0, k1, w);
        philox4x32_10((uint32_t)q, (uint32_t)(q >> 32), 1u, stream << 24, k0, k1, g);
        SurQuery Q;
        Q.pol = (int)(w[0] % (uint32_t)n_pol);
        const PolSur P = pols[Q.pol];
        if (P.S < 1) {
            Q.m = 0;
            Q.state = -1;
            Q.r = r0;
            Q.bucket = 0;
            out[q] = Q;
            continue;
        }
        const int maxk = min((P.S - 1) / 12, max_node_m / 12);
        Q.m = 12 * (int)(w[1] % (uint32_t)(maxk + 1));
        Q.state = 0;
        if (P.product == RSV_JL_REVERSIONARY) {
            const bool x = P.age1 + Q.m < P.lim1, y = P.age2 + Q.m < P.lim2;
            int cand[3], nc = 0;
            if (x && y) cand[nc++] = 0;
            if (x) cand[nc++] = 1;
            if (y) cand[nc++] = 2;
            Q.state = nc ? cand[w[2] % (uint32_t)nc] : -1;
        }
        const double t = Q.m / 12.0;
        const double mean = b + (r0 - b) * exp(-a * t);
        const double sd = sigma * sqrt(-expm1(-2.0 * a * t) / (2.0 * a));
        const double u1 = ((double)g[0] + 0.5) * inv32, u2 = ((double)g[1] + 0.5) * inv32;
        const double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
        Q.r = mean + widen * sd * z;
        Q.bucket = sur_bucket(P, Q.m, Q.state, Q.r, a, b, sigma, r0);
        out[q] = Q;
    }
}

}  // namespace

// Forward-curve increments of the Vasicek zero-coupon price at monthly points:
// ln P(T_{t+1} | r) - ln P(T_t | r) = dA_t - dB_t r with T_t = t/12 and
// B(T) = (1 - e^{-aT})/a, ln P = (B - T)(a^2 b - sigma^2/2)/a^2 - sigma^2 B^2/(4a) - B r
// (Vasicek 1977).  dB is formed without cancellation.
__global__ void sur_curve_kernel(double a, double b, double sigma, int n, double2* __restrict__ curve) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double T0 = t / 12.0, T1 = (t + 1) / 12.0;
    const double B0 = -expm1(-a * T0) / a, B1 = -expm1(-a * T1) / a;
    const double dB = exp(-a * T0) * (-expm1(-a / 12.0)) / a;
    const double K1 = (a * a * b - 0.5 * sigma * sigma) / (a * a), K2 = sigma * sigma / (4.0 * a);
    curve[t] = make_double2((dB - 1.0 / 12.0) * K1 - K2 * dB * (B0 + B1), dB);
}

// Commutation columns of each decrement table at each flat reference rate
// delta (one thread per (table, rate)): l_k = prod_{j<k} p_j from month 0,
// D_k = v^k l_k, N_k = sum_{j>=k} D_j, C_k = v^{k+1} l_k q_k, M_k = sum_{j>=k} C_j,
// v = exp(-delta/12); survival is zero past the table's end.  Computed in FP64
// and stored as FP32 head + tail pairs (about 48 bits), so that the
// differences N_a - N_b of the base values keep their precision in FP32.
__device__ __forceinline__ float2 sur_split(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double sur_join(float2 x) { return (double)x.x + (double)x.y; }

__global__ void sur_comm_kernel(const double2* __restrict__ tab, int tab_pad, int n_tab, float2* __restrict__ comm) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n_tab * SUR_COMM_N) return;
    const int t = id / SUR_COMM_N, g = id % SUR_COMM_N;
    const int CL = sur_comm_len(tab_pad);
    float2* D = comm + (size_t)id * 3 * CL;
    float2* N = D + CL;
    float2* M = N + CL;
    const double v = exp(-(SUR_COMM_LO + g * SUR_COMM_STEP) / 12.0);
    double l = 1.0, vk = 1.0;
    for (int k = 0; k <= tab_pad; ++k) {
        const double p = k < tab_pad ? tab[(size_t)t * tab_pad + k].x : 0.0;
        D[k] = sur_split(vk * l);
        M[k] = sur_split(vk * v * l * (1.0 - p));   // C_k, summed below
        l *= p;
        vk *= v;
    }
    D[tab_pad + 1] = make_float2(0.0f, 0.0f);
    double sn = 0.0, sm = 0.0;
    N[tab_pad + 1] = make_float2(0.0f, 0.0f);
    M[tab_pad + 1] = make_float2(0.0f, 0.0f);
    for (int k = tab_pad; k >= 0; --k) {
        sn += sur_join(D[k]);
        sm += sur_join(M[k]);
        N[k] = sur_split(sn);
        M[k] = sur_split(sm);
    }
}

// Reserve per unit amount in the query's state: the FP64 recurrence on the
// Vasicek forward curve from the policy's end back to the node; vt(t) is the
// one-month discount factor t months after the node.
template <class VT>
__device__ __forceinline__ double sur_recurrence(const PolSur& P, const SurTables& T, const SurQuery& Q, VT vt) {
    const int Sn = P.S - Q.m;
    const double2* tx = T.tab + (size_t)P.tab1 * T.tab_pad + P.age1 + Q.m;
    const double2* ty = T.tab + (size_t)P.tab2 * T.tab_pad + P.age2 + Q.m;
    double V00 = P.product == RSV_ENDOWMENT ? 1.0 : 0.0, V01 = 0.0, V10 = 0.0;
    for (int t = Sn - 1; t >= 0; --t) {
        const double v = vt(t);
        const double2 ex = tx[t];
        if (P.product == RSV_SL_ANNUITY) {
            V00 = v * ex.x * (1.0 + V00);
        } else if (P.product == RSV_JL_REVERSIONARY) {
            const double2 ey = ty[t];
            const double n01 = v * ex.x * (1.0 + V01);
            const double n10 = v * ey.x * (P.rho + V10);
            V00 = v * ex.x * ey.x * (1.0 + V00) + ey.y * n01 + ex.y * n10;
            V01 = n01;
            V10 = n10;
        } else {
            V00 = v * (ex.y + ex.x * V00);
        }
    }
    return Q.state == 0 ? V00 : (Q.state == 1 ? V01 : V10);
}

// The recurrence for n independent queries (one thread each).  With `flag`,
// only queries whose bucket is flagged are valued (the fallback).
__global__ void sur_label_kernel(const PolSur* __restrict__ pols, const SurTables T, const SurQuery* __restrict__ qs,
                                 long long n, const unsigned char* __restrict__ flag, double* __restrict__ V) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const SurQuery Q = qs[i];
        if (flag && (Q.state < 0 || !flag[Q.bucket])) continue;
        if (Q.state < 0) {
            V[i] = 0.0;
            continue;
        }
        const double r = Q.r;
        V[i] = sur_recurrence(pols[Q.pol], T, Q, [&](int t) {
            const double2 dc = T.curve[t];   // month t after the node
            return exp(dc.x - dc.y * r);
        });
    }
}

// The same reserve in the compensated form of the valuation kernels
// (double-float chains, shifted annuity states, the reversionary annuity as
// three annuity chains): the FP32 pipes instead of the FP64 one, to about
// 1e-8, far inside the surrogate's tolerance.  vc: the discount factors as
// hi/lo pairs; tab: the compensated decrement entries (p_hi, p_lo, q_hi, q_lo).
__device__ __forceinline__ double sur_recurrence_df(const PolSur& P, const float4* __restrict__ tab, int tab_pad,
                                                    const SurQuery& Q, const float2* vc) {
    const int Sn = P.S - Q.m;
    const float4* tx = tab + (size_t)P.tab1 * tab_pad + P.age1 + Q.m;
    if (P.product == RSV_SL_ANNUITY) {
        df R{1.0f, 0.0f};
        for (int t = Sn - 1; t >= 0; --t) R = step_ann(df{vc[t].x, vc[t].y}, df{tx[t].x, tx[t].y}, R);
        return df_to_double(R) - 1.0;
    }
    if (P.product == RSV_JL_REVERSIONARY) {
        const float4* ty = tab + (size_t)P.tab2 * tab_pad + P.age2 + Q.m;
        df Rxy{1.0f, 0.0f}, Rx{1.0f, 0.0f}, Ry{1.0f, 0.0f};
        for (int t = Sn - 1; t >= 0; --t)
            step_jl(df{vc[t].x, vc[t].y}, df{tx[t].x, tx[t].y}, df{ty[t].x, ty[t].y}, Rxy, Rx, Ry);
        const double ax = df_to_double(Rx) - 1.0;
        if (Q.state == 1) return ax;
        if (Q.state == 2) return P.rho * (df_to_double(Ry) - 1.0);
        return ax + P.rho * (df_to_double(Ry) - df_to_double(Rxy));
    }
    df V{P.product == RSV_ENDOWMENT ? 1.0f : 0.0f, 0.0f};   // term assurance or endowment
    for (int t = Sn - 1; t >= 0; --t)
        V = step_ass(df{vc[t].x, vc[t].y}, df{tx[t].x, tx[t].y}, df{tx[t].z, tx[t].w}, V);
    return df_to_double(V);
}

constexpr int kFallbackChunk = 4096;   // queries compacted per pass of the fallback kernel

// The fallback of the nested valuation: the queries of one (outer path, node)
// share its short rate, so each block builds that curve once in shared memory
// (Lmax months, FP64 then split hi/lo) and values the segment's flagged
// queries from it in the compensated form.
__global__ void sur_fallback_nodes_kernel(const PolSur* __restrict__ pols, const float4* __restrict__ tab,
                                          int tab_pad, const double2* __restrict__ curve,
                                          const SurQuery* __restrict__ qs, const long long* __restrict__ seg, int Lmax,
                                          const unsigned char* __restrict__ flag, double* __restrict__ V) {
    extern __shared__ float2 fb_smem[];
    float2* vcur = fb_smem;                                     // the segment's curve, Lmax months
    int* list = reinterpret_cast<int*>(fb_smem + Lmax);         // flagged queries of a chunk
    __shared__ int n_list, warp_off[32];
    const long long b = seg[blockIdx.x], e = seg[blockIdx.x + 1];
    if (b == e) return;
    const double r = qs[b].r;
    for (int t = threadIdx.x; t < Lmax; t += blockDim.x) {
        const double2 dc = curve[t];
        const double x = exp_small(dc.x - dc.y * r);
        const float h = __double2float_rn(x);
        vcur[t] = make_float2(h, __double2float_rn(x - (double)h));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // Only the flagged queries (a fifth or so) run a recurrence: compact them
    // first (in query order, kFallbackChunk at a time), so that every lane has one.
    for (long long c0 = b; c0 < e; c0 += kFallbackChunk) {
        const long long c1 = c0 + kFallbackChunk < e ? c0 + kFallbackChunk : e;
        if (threadIdx.x == 0) n_list = 0;
        __syncthreads();
        for (long long base = c0; base < c1; base += blockDim.x) {
            const long long i = base + threadIdx.x;
            bool f = false;
            if (i < c1) {
                const SurQuery Q = qs[i];
                f = Q.state >= 0 && flag[Q.bucket];
            }
            const unsigned m = __ballot_sync(0xffffffffu, f);
            if (lane == 0) warp_off[wid] = __popc(m);
            __syncthreads();
            if (threadIdx.x == 0) {
                int acc = n_list;
                for (int w = 0; w < nw; ++w) {
                    const int c = warp_off[w];
                    warp_off[w] = acc;
                    acc += c;
                }
                n_list = acc;
            }
            __syncthreads();
            if (f) list[warp_off[wid] + __popc(m & ((1u << lane) - 1u))] = (int)(i - c0);
            __syncthreads();
        }
        for (int k = threadIdx.x; k < n_list; k += blockDim.x) {
            const long long i = c0 + list[k];
            V[i] = sur_recurrence_df(pols[qs[i].pol], tab, tab_pad, qs[i], vcur);
        }
        __syncthreads();
    }
}

// Base value per unit amount from the commutation columns at flat rate
// grid point g: the classical actuarial values (annuity (N_{x+1} - N_{x+n+1})/D_x,
// term assurance (M_x - M_{x+n})/D_x, pure endowment D_{x+n}/D_x) for n
// months from attained month x.  The joint-life state 00 is the reversionary
// a_x + rho (a_y - a_xy), with the joint-life annuity a_xy estimated from the
// two single-life values: for constant monthly forces a monthly annuity in
// arrears satisfies ln(1 + 1/a) = (delta + mu)/12, and the joint life's force
// is the sum of the two, so ln(1 + 1/a_xy) = ln(1 + 1/a_x) + ln(1 + 1/a_y) - delta/12.
__device__ float sur_base_value(const PolSur& P, const SurTables& T, int g, int m, int state) {
    const int CL = sur_comm_len(T.tab_pad), n = P.S - m;
    auto col = [&](int tab) { return T.comm + ((size_t)tab * SUR_COMM_N + g) * 3 * CL; };
    // a - b of two head + tail pairs: the heads first (exact when they are close), then the tails
    auto diff = [](float2 a, float2 b) { return (a.x - b.x) + (a.y - b.y); };
    auto ann = [&](int tab, int x) {
        const float2* D = col(tab);
        const int e = min(x + n, T.tab_pad);
        return D[x].x > 0.0f ? diff(D[CL + x + 1], D[CL + e + 1]) / D[x].x : 0.0f;
    };
    const int x = P.age1 + m;
    if (P.product == RSV_SL_ANNUITY) return ann(P.tab1, x);
    if (P.product == RSV_JL_REVERSIONARY) {
        const int y = P.age2 + m;
        const float rho = (float)P.rho;
        if (state == 1) return ann(P.tab1, x);
        if (state == 2) return rho * ann(P.tab2, y);
        const float ax = ann(P.tab1, x), ay = ann(P.tab2, y);
        if (!(ax > 0.0f) || !(ay > 0.0f)) return ax + rho * ay;
        const float e = log1pf(1.0f / ax) + log1pf(1.0f / ay) - (SUR_COMM_LO_F + g * SUR_COMM_STEP_F) / 12.0f;
        const float axy = e > 0.0f ? fminf(1.0f / expm1f(e), fminf(ax, ay)) : fminf(ax, ay);
        return ax + rho * (ay - axy);
    }
    const float2* D = col(P.tab1);
    if (!(D[x].x > 0.0f)) return 1.0f;   // past the table: death in the first month
    const int e = min(x + n, T.tab_pad + 1);
    const float A1 = diff(D[2 * CL + x], D[2 * CL + e]) / D[x].x;
    return P.product == RSV_TERM_ASSURANCE ? A1 : A1 + D[e].x / D[x].x;
}

// ln of the base value at the query's own flat rate: the Vasicek yield to
// half the remaining term (between one month and 15 years), interpolated
// linearly in ln(base value) between the two nearest grid rates.  FP32
// throughout (GB300's FP64 pipe is narrow, and the value is only an offset
// that training and inference share).
__device__ float sur_ln_base(const PolSur& P, const SurTables& T, const SurQuery& Q, float* delta) {
    const int n = P.S - Q.m;
    const float h = min(max(n / 2, 1), 180) / 12.0f;
    const float B = -expm1f(-T.af * h) / T.af;
    const float lnP = (B - h) * T.k1 - T.k2 * B * B - B * (float)Q.r;
    const float d = -lnP / h;
    *delta = d;
    const float u = fminf(fmaxf((d - SUR_COMM_LO_F) * SUR_COMM_INV_STEP_F, 0.0f), (float)(SUR_COMM_N - 1));
    const int g0 = min((int)u, SUR_COMM_N - 2);
    const float f = u - g0;
    const float b0 = sur_base_value(P, T, g0, Q.m, Q.state), b1 = sur_base_value(P, T, g0 + 1, Q.m, Q.state);
    if (!(b0 > 0.0f) || !(b1 > 0.0f)) return 0.0f;
    return (1.0f - f) * logf(b0) + f * logf(b1);
}

// A feature row as exact hi + lo BF16 halves (the first layer's weights are
// tied across the halves, so it sees each feature to ~16 bits).
// The row is written as eight 16-byte stores (rows are 128-byte aligned).
__device__ __forceinline__ void sur_store_features(const float (&f)[MLP_IN], __nv_bfloat16* row) {
    uint32_t hi[MLP_IN / 2], lo[MLP_IN / 2];
#pragma unroll
    for (int k = 0; k < MLP_IN; k += 2) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(f[k], f[k + 1]);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(f[k] - hf.x, f[k + 1] - hf.y);
        hi[k / 2] = *reinterpret_cast<const uint32_t*>(&h);
        lo[k / 2] = *reinterpret_cast<const uint32_t*>(&l);
    }
    uint4* dst = reinterpret_cast<uint4*>(row);
#pragma unroll
    for (int q = 0; q < MLP_IN / 8; ++q) {
        dst[q] = make_uint4(hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
        dst[MLP_IN / 8 + q] = make_uint4(lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
    }
}

// Features of a query (zero-padded to MLP_IN, hi + lo BF16) and the ln base
// value the network's output is added to.
__global__ void sur_features_kernel(const PolSur* __restrict__ pols, const SurTables T, const SurQuery* __restrict__ qs,
                                    long long n, __nv_bfloat16* __restrict__ X, float* __restrict__ lnb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const SurQuery Q = qs[i];
        const PolSur P = pols[Q.pol];
        float f[MLP_IN];
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) f[k] = 0.0f;
        float base = 0.0f, delta = 0.0f;
        if (Q.state >= 0) base = sur_ln_base(P, T, Q, &delta);
        f[P.product] = 1.0f;
        f[4 + max(0, Q.state)] = 1.0f;
        const bool jl = P.product == RSV_JL_REVERSIONARY;
        const float age1 = ((P.age1 + Q.m) / 12.0f - 60.0f) / 25.0f;
        const float rem = (P.S - Q.m) / 12.0f / 40.0f;
        const float rr = ((float)Q.r - 0.04f) * 50.0f;
        f[7] = age1;
        f[8] = jl ? ((P.age2 + Q.m) / 12.0f - 60.0f) / 25.0f : 0.0f;
        f[9] = jl ? (float)P.rho : 0.0f;
        f[10] = rem;
        f[11] = rr;
        f[12] = (logf(fmaxf((float)P.amount, 1e-30f)) - 9.0f) / 2.0f;
        f[13] = age1 * age1;
        f[14] = rem * rem;
        f[15] = rr * rem;
        f[16] = log1pf((float)(P.S - Q.m)) / 7.0f;
        f[17] = base * 0.25f;
        f[18] = (delta - 0.04f) * 50.0f;
        sur_store_features(f, X + i * MLP_XW);
        lnb[i] = base;
    }
}

// reserve per unit = exp(network output, denormalised, + ln base value), in
// FP32 (about 3e-7 relative for arguments below 8 in magnitude)
__global__ void sur_to_reserve_kernel(const float* __restrict__ yhat, const float* __restrict__ lnb, long long n,
                                      float mu, float sd, double* __restrict__ V) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        V[i] = (double)expf(fmaf(yhat[i], sd, mu) + lnb[i]);
}

namespace {

__global__ void targets_kernel(const double* __restrict__ V, const float* __restrict__ lnb, long long n, double mu,
                               double sd, float* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (float)((log(V[i]) - lnb[i] - mu) / sd);
}

__global__ void gather_kernel(const __nv_bfloat16* __restrict__ X, const float* __restrict__ y, long long n,
                              uint64_t seed, uint32_t step, int B, __nv_bfloat16* __restrict__ Xb,
                              float* __restrict__ yb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B) return;
    uint32_t w[4];
    philox4x32_10((uint32_t)i, step, 0u, 5u << 24, (uint32_t)seed, (uint32_t)(seed >> 32), w);
    const long long j = (long long)((((uint64_t)w[0] << 32) | w[1]) % (uint64_t)n);
    const uint4* src = reinterpret_cast<const uint4*>(X + j * MLP_XW);
    uint4* dst = reinterpret_cast<uint4*>(Xb + (size_t)i * MLP_XW);
#pragma unroll
    for (int k = 0; k < MLP_XW * 2 / 16; ++k) dst[k] = src[k];
    yb[i] = y[j];
}

// relative error of the surrogate's reserve against the label
__global__ void rel_err_kernel(const double* __restrict__ pred, const double* __restrict__ V, long long n,
                               double* __restrict__ err) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        err[i] = V[i] > 0.0 ? pred[i] / V[i] - 1.0 : 0.0;
}

// moments of ln(label / base value) (FP64, fixed order per block, then on the host)
__global__ void log_moments_kernel(const double* __restrict__ V, const float* __restrict__ lnb, long long n,
                                   double* __restrict__ part) {
    __shared__ double s1[256], s2[256];
    double a = 0.0, b2 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double l = log(V[i]) - lnb[i];
        a += l;
        b2 += l * l;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1[0];
        part[2 * blockIdx.x + 1] = s2[0];
    }
}

}  // namespace

// ------------------------------------------------------------------ host ----
// The F64 decrement table, the forward-curve increments of the surrogate's
// Vasicek model and the commutation columns, rebuilt when their inputs change.
rsv_status sur_tables(rsv_ctx* c, SurTables& T) {
    SurrogateState& s = c->sur;
    size_t smem;
    rsv_status st = build_tables(c, F_F64, smem);
    if (st != RSV_OK) return st;
    const int pad = c->tab_pad_of[F_F64], n_tab = c->n_tab_of[F_F64];
    if (s.curve_key[0] != s.a || s.curve_key[1] != s.b || s.curve_key[2] != s.sigma) {
        CU(s.d_curve.ensure((size_t)(kMaxAgeSteps + 1) * sizeof(double2)));
        sur_curve_kernel<<<(kMaxAgeSteps + 1 + 127) / 128, 128, 0, c->stream>>>(s.a, s.b, s.sigma, kMaxAgeSteps + 1,
                                                                               s.d_curve.as<double2>());
        CU(cudaGetLastError());
        s.curve_key[0] = s.a;
        s.curve_key[1] = s.b;
        s.curve_key[2] = s.sigma;
    }
    if (s.comm_pad != pad || s.comm_ntab != n_tab || s.comm_gen != c->tab_gen) {
        const int jobs = n_tab * SUR_COMM_N;
        CU(s.d_comm.ensure((size_t)jobs * 3 * sur_comm_len(pad) * sizeof(float2)));
        sur_comm_kernel<<<(jobs + 63) / 64, 64, 0, c->stream>>>(c->d_tab[F_F64].as<double2>(), pad, n_tab,
                                                               s.d_comm.as<float2>());
        CU(cudaGetLastError());
        s.comm_pad = pad;
        s.comm_ntab = n_tab;
        s.comm_gen = c->tab_gen;
    }
    T.tab = c->d_tab[F_F64].as<double2>();
    T.tab_pad = pad;
    T.curve = s.d_curve.as<double2>();
    T.comm = s.d_comm.as<float2>();
    T.a = s.a;
    T.b = s.b;
    T.sigma = s.sigma;
    T.af = (float)s.a;
    T.k1 = (float)((s.a * s.a * s.b - 0.5 * s.sigma * s.sigma) / (s.a * s.a));
    T.k2 = (float)(s.sigma * s.sigma / (4.0 * s.a));
    return RSV_OK;
}

rsv_status sur_upload_policies(rsv_ctx* c, std::vector<PolSur>& host) {
    for (size_t i = 0; i < c->pols.size(); ++i)
        if (c->pols[i].product > RSV_ENDOWMENT)
            return fail(c, RSV_E_ARG, "policy %zu: the surrogate covers products 0-3 (SL, JL, term, endowment)", i);
    host.resize(c->pols.size());
    for (size_t i = 0; i < host.size(); ++i) {
        const rsv_policy& r = c->pols[i];
        PolSur& p = host[i];
        const bool jl = r.product == RSV_JL_REVERSIONARY;
        p.product = r.product;
        p.age1 = r.age1_m;
        p.age2 = jl ? r.age2_m : 0;
        p.tab1 = r.table1;
        p.tab2 = jl ? r.table2 : r.table1;
        p.lim1 = (int)c->tab[r.table1].size();
        p.lim2 = (int)c->tab[p.tab2].size();
        int S;
        if (r.product == RSV_SL_ANNUITY) {
            S = std::max(0, p.lim1 - r.age1_m);
            if (r.term_m > 0) S = std::min(S, r.term_m);
        } else if (jl) {
            S = std::max(0, std::max(p.lim1 - r.age1_m, p.lim2 - r.age2_m));
            if (r.term_m > 0) S = std::min(S, r.term_m);
        } else {
            S = r.term_m;
        }
        p.S = S;
        p.amount = r.amount;
        p.rho = jl ? r.reversion : 0.0;
    }
    CU(c->d_pols.ensure(std::max<size_t>(1, host.size()) * sizeof(PolSur)));
    CU(cudaMemcpyAsync(c->d_pols.p, host.data(), host.size() * sizeof(PolSur), cudaMemcpyHostToDevice, c->stream));
    c->pols_dev_gen = c->pol_gen;
    return RSV_OK;
}

// Reserves per unit amount of n queries (device) by the network; with
// `fallback`, queries in flagged buckets are then valued by the recurrence.
rsv_status sur_predict(rsv_ctx* c, const SurQuery* q, long long n, double* V, bool fallback, int batch) {
    SurrogateState& s = c->sur;
    SurTables T;
    rsv_status st = sur_tables(c, T);
    if (st != RSV_OK) return st;
    // the tcgen05 path needs only features and outputs: large batches keep
    // the feature kernel's dependent loads in flight
    const bool tc = c->mlp.use_tc;
    if (tc) {
        batch = std::max(batch, 1 << 19);
        CU(c->mlp.ensure_infer(batch));
    } else {
        CU(c->mlp.ensure(batch));
    }
    __nv_bfloat16* X = tc ? c->mlp.Xi : c->mlp.X;
    float* y = tc ? c->mlp.yi : c->mlp.y;
    batch = batch / 128 * 128;
    CU(s.d_lnb.ensure((size_t)batch * sizeof(float)));
    for (long long o = 0; o < n; o += batch) {
        const int nb = (int)std::min<long long>(batch, n - o);
        const int nb_pad = (nb + 127) / 128 * 128;
        if (nb_pad != nb) CU(cudaMemsetAsync(X, 0, (size_t)nb_pad * MLP_XW * 2, c->stream));
        const int grid = (int)std::min<long long>((nb + 255) / 256, (long long)c->sm_count * 16);
        sur_features_kernel<<<grid, 256, 0, c->stream>>>(c->d_pols.as<PolSur>(), T, q + o, nb, X,
                                                         s.d_lnb.as<float>());
        CU(cudaGetLastError());
        if (tc) {
            CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
            CU(c->mlp.forward_tc(X, nb_pad, y, c->sm_count, c->d_ctl.as<int32_t>() + 1, c->stream));
        } else {
            CU(c->mlp.forward(X, nb_pad, y, nullptr, c->stream));
        }
        sur_to_reserve_kernel<<<grid, 256, 0, c->stream>>>(y, s.d_lnb.as<float>(), nb, (float)s.y_mean, (float)s.y_std,
                                                           V + o);
        CU(cudaGetLastError());
    }
    if (fallback) {
        sur_label_kernel<<<c->sm_count * 8, 128, 0, c->stream>>>(c->d_pols.as<PolSur>(), T, q, n,
                                                                 s.d_flag.as<unsigned char>(), V);
        CU(cudaGetLastError());
    }
    return RSV_OK;
}

}  // namespace rsv

// ------------------------------------------------------------------ ABI ----
namespace rsv {
namespace {

// He-normal weights, zero biases, a small head (SplitMix64 + Box-Muller).
void he_init(std::vector<float>& p, uint64_t seed) {
    uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto gauss = [&]() {
        const double u1 = ((next() >> 11) + 0.5) * 0x1.0p-53, u2 = ((next() >> 11) + 0.5) * 0x1.0p-53;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    };
    p.assign(mlp_n_params(), 0.0f);
    for (int l = 1; l <= 4; ++l) {
        const double sd = std::sqrt(2.0 / mlp_in_dim(l));
        for (size_t i = 0; i < (size_t)mlp_in_dim(l) * MLP_H; ++i) p[mlp_w_off(l) + i] = (float)(sd * gauss());
    }
    for (int k = 0; k < MLP_H; ++k) p[mlp_w5_off() + k] = (float)(gauss() / std::sqrt((double)MLP_H));
}

rsv_status mlp_upload(rsv_ctx* c, const float* host) {
    CU(c->mlp.ensure(64));
    CU(cudaMemcpyAsync(c->mlp.params, host, mlp_n_params() * 4, cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->mlp.adam_m, 0, mlp_n_params() * 4, c->stream));
    CU(cudaMemsetAsync(c->mlp.adam_v, 0, mlp_n_params() * 4, c->stream));
    c->mlp.step = 0;
    CU(c->mlp.refresh_bf16(c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->mlp_ready = true;
    return RSV_OK;
}

// FP32 feature rows [n][MLP_IN] -> hi + lo BF16 rows [n][MLP_XW]
__global__ void f32_to_bf16_rows(const float* __restrict__ x, long long rows, __nv_bfloat16* __restrict__ y) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x) {
        float f[MLP_IN];
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) f[k] = x[r * MLP_IN + k];
        sur_store_features(f, y + r * MLP_XW);
    }
}

rsv_status mlp_stage_inputs(rsv_ctx* c, const float* X, long long n, long long n_pad) {
    CU(c->mlp.ensure((int)n_pad));
    CU(c->sur.d_aux.ensure((size_t)n_pad * MLP_IN * 4));
    CU(cudaMemsetAsync(c->sur.d_aux.p, 0, (size_t)n_pad * MLP_IN * 4, c->stream));
    CU(cudaMemcpyAsync(c->sur.d_aux.p, X, (size_t)n * MLP_IN * 4, cudaMemcpyHostToDevice, c->stream));
    f32_to_bf16_rows<<<c->sm_count * 4, 256, 0, c->stream>>>(c->sur.d_aux.as<float>(), n_pad, c->mlp.X);
    CU(cudaGetLastError());
    return RSV_OK;
}

__global__ void query_prep_kernel(const PolSur* __restrict__ pols, int n_pol, const rsv_query* __restrict__ in,
                                  long long n, double a, double b, double sigma, double r0,
                                  SurQuery* __restrict__ out, int* __restrict__ bad,
                                  const unsigned char* __restrict__ flag, unsigned long long* __restrict__ n_flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const rsv_query r = in[i];
        SurQuery Q;
        Q.pol = r.pol;
        Q.m = r.m;
        Q.state = r.state;
        Q.r = r.r;
        Q.bucket = 0;
        const bool ok = r.pol >= 0 && r.pol < n_pol && r.m >= 0 && isfinite(r.r) && r.state >= 0 &&
                        r.state <= (pols[r.pol >= 0 && r.pol < n_pol ? r.pol : 0].product == RSV_JL_REVERSIONARY ? 2 : 0) &&
                        r.m < pols[r.pol >= 0 && r.pol < n_pol ? r.pol : 0].S;
        bool flagged = false;
        if (!ok) {
            atomicAdd(bad, 1);
            Q.pol = 0;
            Q.state = -1;
        } else {
            Q.bucket = sur_bucket(pols[r.pol], r.m, r.state, r.r, a, b, sigma, r0);
            flagged = flag && flag[Q.bucket];
        }
        // one atomic per warp for the flagged count
        const unsigned active = __activemask();
        const unsigned fm = __ballot_sync(active, flagged);
        if (fm && (threadIdx.x & 31) == __ffs(active) - 1) atomicAdd(n_flag, (unsigned long long)__popc(fm));
        out[i] = Q;
    }
}

__global__ void scale_by_amount_kernel(const PolSur* __restrict__ pols, const SurQuery* __restrict__ q, long long n,
                                       double* __restrict__ V) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        V[i] = q[i].state < 0 ? 0.0 : V[i] * pols[q[i].pol].amount;
}

// Compaction of the queries the network serves (valid and in an unflagged
// bucket), in query order: per-block counts, one block's exclusive scan of
// the counts, then each block writes its served queries at its offset plus
// their rank within the block.
constexpr int kCompactBlock = 1024;

__device__ __forceinline__ bool sur_served(const SurQuery& Q, const unsigned char* __restrict__ flag) {
    return Q.state >= 0 && !flag[Q.bucket];
}

__global__ void __launch_bounds__(kCompactBlock) served_count_kernel(const SurQuery* __restrict__ q, long long n,
                                                                     const unsigned char* __restrict__ flag,
                                                                     int* __restrict__ counts) {
    const long long i = blockIdx.x * (long long)kCompactBlock + threadIdx.x;
    const bool on = i < n && sur_served(q[i], flag);
    const int c = __syncthreads_count(on);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// Exclusive scan of counts[0 .. nb) in place (one block); total -> counts[nb].
__global__ void __launch_bounds__(1024) exclusive_scan_kernel(int* __restrict__ counts, int nb) {
    __shared__ long long part[1024];
    const int per = (nb + 1023) / 1024, lo = threadIdx.x * per, hi = min(nb, lo + per);
    long long sum = 0;
    for (int k = lo; k < hi; ++k) sum += counts[k];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {   // inclusive scan of the thread sums
        const long long y = threadIdx.x >= d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += y;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;   // exclusive start of this thread's range
    for (int k = lo; k < hi; ++k) {
        const int c = counts[k];
        counts[k] = (int)run;
        run += c;
    }
    if (threadIdx.x == 1023) counts[nb] = (int)part[1023];
}

__global__ void __launch_bounds__(kCompactBlock) served_gather_kernel(const SurQuery* __restrict__ q, long long n,
                                                                      const unsigned char* __restrict__ flag,
                                                                      const int* __restrict__ offsets,
                                                                      SurQuery* __restrict__ q2, int* __restrict__ idx) {
    __shared__ int wsum[kCompactBlock / 32];
    const long long i = blockIdx.x * (long long)kCompactBlock + threadIdx.x;
    SurQuery Q{};
    const bool on = i < n && sur_served(Q = q[i], flag);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, on);
    if (lane == 0) wsum[warp] = __popc(m);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    if (on) {
        const int pos = offsets[blockIdx.x] + before + __popc(m & ((1u << lane) - 1u));
        q2[pos] = Q;
        idx[pos] = (int)i;
    }
}

__global__ void scatter_served_kernel(const double* __restrict__ v2, const int* __restrict__ idx, long long n2,
                                      double* __restrict__ V) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n2; k += (long long)gridDim.x * blockDim.x)
        V[idx[k]] = v2[k];
}

}  // namespace

// Per-unit expected reserves (device, n values) of device queries by the
// network with fallback; *n_fallback receives the number valued by the
// recurrence.  Used by the nested valuation's surrogate mode.
rsv_status sur_value_queries(rsv_ctx* c, const rsv_query* dq, long long n, const long long* seg, int n_seg, int Lmax,
                             double* V, long long* n_fallback) {
    SurrogateState& s = c->sur;
    if (c->pols_dev_gen != c->pol_gen) {
        std::vector<PolSur> hp;
        rsv_status st = sur_upload_policies(c, hp);
        if (st != RSV_OK) return st;
    }
    CU(s.d_q.ensure((size_t)n * sizeof(SurQuery)));
    CU(s.d_err.ensure(16));
    CU(cudaMemsetAsync(s.d_err.p, 0, 16, c->stream));
    SurQuery* q = s.d_q.as<SurQuery>();
    query_prep_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(
        c->d_pols.as<PolSur>(), (int)c->pols.size(), dq, n, s.a, s.b, s.sigma, s.r0, q,
        s.d_err.as<int>(), s.d_flag.as<unsigned char>(), reinterpret_cast<unsigned long long*>(s.d_err.as<char>() + 8));
    CU(cudaGetLastError());
    // only the served queries go through features and the network
    if (n > 0x7fffffffLL) return fail(c, RSV_E_ARG, "too many nested surrogate queries (%lld)", n);
    const int nb = (int)((n + kCompactBlock - 1) / kCompactBlock);
    CU(s.d_cnt.ensure(((size_t)nb + 1) * sizeof(int)));
    CU(s.d_q2.ensure((size_t)std::max(1LL, n) * sizeof(SurQuery)));
    CU(s.d_idx.ensure((size_t)std::max(1LL, n) * sizeof(int)));
    CU(s.d_v2.ensure((size_t)std::max(1LL, n) * sizeof(double)));
    int n_served = 0;
    if (nb > 0) {
        served_count_kernel<<<nb, kCompactBlock, 0, c->stream>>>(q, n, s.d_flag.as<unsigned char>(), s.d_cnt.as<int>());
        exclusive_scan_kernel<<<1, 1024, 0, c->stream>>>(s.d_cnt.as<int>(), nb);
        served_gather_kernel<<<nb, kCompactBlock, 0, c->stream>>>(q, n, s.d_flag.as<unsigned char>(), s.d_cnt.as<int>(),
                                                                  s.d_q2.as<SurQuery>(), s.d_idx.as<int>());
        CU(cudaGetLastError());
        CU(cudaMemcpyAsync(&n_served, s.d_cnt.as<int>() + nb, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    rsv_status st = RSV_OK;
    if (n_served > 0) {
        if ((st = sur_predict(c, s.d_q2.as<SurQuery>(), n_served, s.d_v2.as<double>(), false, 65536)) != RSV_OK)
            return st;
        scatter_served_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(s.d_v2.as<double>(), s.d_idx.as<int>(), n_served,
                                                                      V);
        CU(cudaGetLastError());
    }
    SurTables T;
    if ((st = sur_tables(c, T)) != RSV_OK) return st;
    size_t smem_c;
    if ((st = build_tables(c, F_COMP, smem_c)) != RSV_OK) return st;   // the compensated entries, same padding
    sur_fallback_nodes_kernel<<<n_seg, 256, (size_t)Lmax * sizeof(float2) + kFallbackChunk * sizeof(int), c->stream>>>(
        c->d_pols.as<PolSur>(), c->d_tab[F_COMP].as<float4>(), c->tab_pad_of[F_COMP], T.curve, q, seg, Lmax,
        s.d_flag.as<unsigned char>(), V);
    CU(cudaGetLastError());
    long long cnt[2] = {0, 0};
    CU(cudaMemcpyAsync(cnt, s.d_err.p, 16, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if ((int)cnt[0]) return fail(c, RSV_E_ARG, "a nested surrogate query is invalid");
    if (n_fallback) *n_fallback = cnt[1];
    return RSV_OK;
}

}  // namespace rsv

using namespace rsv;

extern "C" {

rsv_status rsv_surrogate_query(rsv_ctx* c, const rsv_query* queries, int64_t n, int32_t how, double* reserve) try {
    if (!c) return RSV_E_ARG;
    if (!queries || !reserve || n < 1 || n > (int64_t(1) << 31) || how < RSV_QUERY_NETWORK || how > RSV_QUERY_FALLBACK)
        return fail(c, RSV_E_ARG, "bad query arguments");
    if (c->pols.empty()) return fail(c, RSV_E_STATE, "no portfolio loaded");
    if (how != RSV_QUERY_RECURRENCE && !c->sur.trained) return fail(c, RSV_E_STATE, "surrogate not trained");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    rsv_status st = build_layout(c, 2, 0, kMaxAgeSteps);
    if (st != RSV_OK) return st;
    size_t smem;
    if ((st = build_tables(c, F_F64, smem)) != RSV_OK) return st;
    if (c->pols_dev_gen != c->pol_gen) {
        std::vector<PolSur> hp;
        if ((st = sur_upload_policies(c, hp)) != RSV_OK) return st;
    }
    SurrogateState& s = c->sur;
    CU(s.d_aux.ensure((size_t)n * sizeof(rsv_query) + 16));
    CU(s.d_q.ensure((size_t)n * sizeof(SurQuery)));
    CU(s.d_pred.ensure((size_t)n * 8));
    CU(s.d_err.ensure(16));
    CU(cudaMemsetAsync(s.d_err.p, 0, 16, c->stream));
    CU(cudaMemcpyAsync(s.d_aux.p, queries, (size_t)n * sizeof(rsv_query), cudaMemcpyHostToDevice, c->stream));
    SurQuery* q = s.d_q.as<SurQuery>();
    const int grid = c->sm_count * 8;
    query_prep_kernel<<<grid, 256, 0, c->stream>>>(c->d_pols.as<PolSur>(), (int)c->pols.size(),
                                                   s.d_aux.as<rsv_query>(), n, s.a, s.b, s.sigma, s.r0, q,
                                                   s.d_err.as<int>(), nullptr, nullptr);
    CU(cudaGetLastError());
    double* V = s.d_pred.as<double>();
    CU(cudaEventRecord(c->ev0, c->stream));
    if (how == RSV_QUERY_RECURRENCE) {
        SurTables T;
        if ((st = sur_tables(c, T)) != RSV_OK) return st;
        sur_label_kernel<<<grid, 128, 0, c->stream>>>(c->d_pols.as<PolSur>(), T, q, n, nullptr, V);
        CU(cudaGetLastError());
    } else if ((st = sur_predict(c, q, n, V, how == RSV_QUERY_FALLBACK, 65536)) != RSV_OK) {
        return st;
    }
    CU(cudaEventRecord(c->ev1, c->stream));
    c->ev_recorded = true;
    scale_by_amount_kernel<<<grid, 256, 0, c->stream>>>(c->d_pols.as<PolSur>(), q, n, V);
    CU(cudaGetLastError());
    int bad = 0;
    CU(cudaMemcpyAsync(&bad, s.d_err.p, 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(reserve, V, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, RSV_E_ARG, "%d queries name a bad policy, state or month", bad);
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

int64_t rsv_mlp_param_count(void) { return (int64_t)mlp_n_params(); }

rsv_status rsv_mlp_init(rsv_ctx* c, uint64_t seed) try {
    if (!c) return RSV_E_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    std::vector<float> p;
    he_init(p, seed);
    c->sur.trained = false;
    return mlp_upload(c, p.data());
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_mlp_set_params(rsv_ctx* c, const float* params, int64_t n) try {
    if (!c) return RSV_E_ARG;
    if (!params || n != (int64_t)mlp_n_params()) return fail(c, RSV_E_ARG, "expected %zu parameters", mlp_n_params());
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    c->sur.trained = false;
    return mlp_upload(c, params);
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_mlp_get_params(rsv_ctx* c, float* params, int64_t n) try {
    if (!c) return RSV_E_ARG;
    if (!params || n != (int64_t)mlp_n_params()) return fail(c, RSV_E_ARG, "expected %zu parameters", mlp_n_params());
    if (!c->mlp_ready) return fail(c, RSV_E_STATE, "network not initialised");
    CU(cudaMemcpyAsync(params, c->mlp.params, mlp_n_params() * 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_mlp_set_backend(rsv_ctx* c, int32_t backend) try {
    if (!c) return RSV_E_ARG;
    if (backend != RSV_MLP_MMA_SYNC && backend != RSV_MLP_TCGEN05) return fail(c, RSV_E_ARG, "bad backend");
    c->mlp.use_tc = backend == RSV_MLP_TCGEN05;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_mlp_forward(rsv_ctx* c, const float* X, int64_t n, float* y) try {
    if (!c) return RSV_E_ARG;
    if (!X || !y || n < 1 || n > (1 << 20)) return fail(c, RSV_E_ARG, "bad forward arguments");
    if (!c->mlp_ready) return fail(c, RSV_E_STATE, "network not initialised");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    const long long n_pad = (n + 127) / 128 * 128;
    rsv_status st = mlp_stage_inputs(c, X, n, n_pad);
    if (st != RSV_OK) return st;
    if (c->mlp.use_tc) {
        CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
        CU(cudaMemsetAsync(c->d_ctl.p, 0, 2 * sizeof(int32_t), c->stream));
        if (!c->mlp.wt_fresh)   // the transposed weights first, outside the timed region
            CU(c->mlp.forward_tc(c->mlp.X, 128, c->mlp.y, c->sm_count, c->d_ctl.as<int32_t>() + 1, c->stream));
        CU(cudaEventRecord(c->ev0, c->stream));
        CU(c->mlp.forward_tc(c->mlp.X, (int)n_pad, c->mlp.y, c->sm_count, c->d_ctl.as<int32_t>() + 1, c->stream));
    } else {
        CU(cudaEventRecord(c->ev0, c->stream));
        CU(c->mlp.forward(c->mlp.X, (int)n_pad, c->mlp.y, nullptr, c->stream));
    }
    CU(cudaEventRecord(c->ev1, c->stream));
    c->ev_recorded = true;
    CU(cudaMemcpyAsync(y, c->mlp.y, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_mlp_gradient(rsv_ctx* c, const float* X, const float* target, int64_t n, float* grads, float* loss) try {
    if (!c) return RSV_E_ARG;
    if (!X || !target || !grads || n < 64 || n % 64 || n > (1 << 20))
        return fail(c, RSV_E_ARG, "bad gradient arguments (n a multiple of 64)");
    if (!c->mlp_ready) return fail(c, RSV_E_STATE, "network not initialised");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    rsv_status st = mlp_stage_inputs(c, X, n, n);
    if (st != RSV_OK) return st;
    CU(cudaMemcpyAsync(c->mlp.t, target, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
    CU(c->mlp.forward(c->mlp.X, (int)n, c->mlp.y, c->mlp.t, c->stream));
    CU(c->mlp.backward(c->mlp.X, (int)n, c->stream));
    CU(cudaMemcpyAsync(grads, c->mlp.grads, mlp_n_params() * 4, cudaMemcpyDeviceToHost, c->stream));
    float l = 0.0f;
    CU(cudaMemcpyAsync(&l, c->mlp.loss, 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (loss) *loss = l / (float)n;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_mlp_trace(rsv_ctx* c, int32_t backend, const float* X, const float* target, int64_t n, uint16_t* Xb,
                         float* Z, uint16_t* A, float* y, float* dZ, uint16_t* dZb, float* grads) try {
    if (!c) return RSV_E_ARG;
    const bool tc = backend == RSV_MLP_TCGEN05;
    if ((backend != RSV_MLP_MMA_SYNC && !tc) || !X || !Z || !A || !y || n < 128 || n % 128 || n > 4096)
        return fail(c, RSV_E_ARG, "bad trace arguments (n a multiple of 128, at most 4096)");
    if (tc && (target || dZ || dZb || grads)) return fail(c, RSV_E_ARG, "the tcgen05 path traces the forward pass only");
    if (!tc && (target != nullptr) != (dZ != nullptr && dZb != nullptr && grads != nullptr))
        return fail(c, RSV_E_ARG, "a target needs dZ, dZb and grads (and they need a target)");
    if (!c->mlp_ready) return fail(c, RSV_E_STATE, "network not initialised");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    rsv_status st = mlp_stage_inputs(c, X, n, n);
    if (st != RSV_OK) return st;
    const size_t L = (size_t)n * MLP_H;   // one layer's values
    if (tc) {
        CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
        CU(cudaMemsetAsync(c->d_ctl.p, 0, 2 * sizeof(int32_t), c->stream));
        CU(c->d_mlp_trace.ensure(4 * L * 4 + 3 * L * 2));
        float* tz = c->d_mlp_trace.as<float>();
        uint16_t* ta = reinterpret_cast<uint16_t*>(tz + 4 * L);
        CU(c->mlp.forward_tc(c->mlp.X, (int)n, c->mlp.y, c->sm_count, c->d_ctl.as<int32_t>() + 1, c->stream, tz, ta));
        CU(cudaMemcpyAsync(Z, tz, 4 * L * 4, cudaMemcpyDeviceToHost, c->stream));
        CU(cudaMemcpyAsync(A, ta, 3 * L * 2, cudaMemcpyDeviceToHost, c->stream));
    } else {
        if (target) CU(cudaMemcpyAsync(c->mlp.t, target, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
        CU(c->mlp.forward(c->mlp.X, (int)n, c->mlp.y, target ? c->mlp.t : nullptr, c->stream));
        if (target) CU(c->mlp.backward(c->mlp.X, (int)n, c->stream));
        for (int l = 0; l < 4; ++l) {
            CU(cudaMemcpyAsync(Z + l * L, c->mlp.Z[l], L * 4, cudaMemcpyDeviceToHost, c->stream));
            CU(cudaMemcpyAsync(A + l * L, c->mlp.A[l], L * 2, cudaMemcpyDeviceToHost, c->stream));
            if (target) {
                CU(cudaMemcpyAsync(dZ + l * L, c->mlp.dZf[l], L * 4, cudaMemcpyDeviceToHost, c->stream));
                CU(cudaMemcpyAsync(dZb + l * L, c->mlp.dZb[l], L * 2, cudaMemcpyDeviceToHost, c->stream));
            }
        }
        if (target) CU(cudaMemcpyAsync(grads, c->mlp.grads, mlp_n_params() * 4, cudaMemcpyDeviceToHost, c->stream));
    }
    if (Xb) CU(cudaMemcpyAsync(Xb, c->mlp.X, (size_t)n * MLP_XW * 2, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(y, c->mlp.y, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    if (tc) {
        int32_t ctl[2] = {0, 0};
        CU(cudaMemcpy(ctl, c->d_ctl.p, sizeof ctl, cudaMemcpyDeviceToHost));
        if (ctl[1] == DEV_TIMEOUT) return fail(c, RSV_E_TIMEOUT, "a bounded device wait ran out (tcgen05 inference)");
    }
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

}  // extern "C"

namespace {
// FNV-1a, 64 bit, over a byte range (the file's integrity check)
uint64_t fnv1a(const unsigned char* p, size_t n, uint64_t h = 1469598103934665603ull) {
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}
const char kSurMagic[8] = {'R', 'S', 'V', 'S', 'U', 'R', '0', '1'};
constexpr int kSurDoubles = 7;   // y_mean, y_std, tol, a, b, sigma, r0
}  // namespace

extern "C" {

rsv_status rsv_surrogate_save(rsv_ctx* c, const char* path) try {
    if (!c) return RSV_E_ARG;
    if (!path) return fail(c, RSV_E_ARG, "path must not be NULL");
    if (!c->sur.trained || !c->mlp_ready) return fail(c, RSV_E_STATE, "surrogate not trained");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    const SurrogateState& s = c->sur;
    const int64_t np = (int64_t)mlp_n_params(), nb = SUR_NBUCKETS;
    std::vector<unsigned char> buf;
    auto put = [&](const void* x, size_t n) {
        const unsigned char* b = static_cast<const unsigned char*>(x);
        buf.insert(buf.end(), b, b + n);
    };
    put(kSurMagic, 8);
    put(&np, 8);
    put(&nb, 8);
    const double d[kSurDoubles] = {s.y_mean, s.y_std, s.tol, s.a, s.b, s.sigma, s.r0};
    put(d, sizeof d);
    put(s.flag.data(), (size_t)nb);
    std::vector<float> w((size_t)np);
    CU(cudaMemcpyAsync(w.data(), c->mlp.params, (size_t)np * 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    put(w.data(), w.size() * 4);
    const uint64_t h = fnv1a(buf.data(), buf.size());
    put(&h, 8);
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c, RSV_E_ARG, "cannot open %s for writing", path);
    const size_t wr = std::fwrite(buf.data(), 1, buf.size(), f);
    const int cl = std::fclose(f);
    if (wr != buf.size() || cl != 0) return fail(c, RSV_E_ARG, "writing %s failed", path);
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_surrogate_load(rsv_ctx* c, const char* path) try {
    if (!c) return RSV_E_ARG;
    if (!path) return fail(c, RSV_E_ARG, "path must not be NULL");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, RSV_E_ARG, "cannot open %s", path);
    std::vector<unsigned char> buf;
    unsigned char tmp[65536];
    size_t got;
    while ((got = std::fread(tmp, 1, sizeof tmp, f)) > 0) buf.insert(buf.end(), tmp, tmp + got);
    std::fclose(f);
    const int64_t np = (int64_t)mlp_n_params(), nb = SUR_NBUCKETS;
    const size_t want = 8 + 16 + kSurDoubles * 8 + (size_t)nb + (size_t)np * 4 + 8;
    if (buf.size() != want || std::memcmp(buf.data(), kSurMagic, 8) != 0)
        return fail(c, RSV_E_ARG, "%s is not a surrogate file of this library (%zu bytes)", path, buf.size());
    int64_t fnp, fnb;
    std::memcpy(&fnp, buf.data() + 8, 8);
    std::memcpy(&fnb, buf.data() + 16, 8);
    uint64_t h;
    std::memcpy(&h, buf.data() + want - 8, 8);
    if (fnp != np || fnb != nb || h != fnv1a(buf.data(), want - 8))
        return fail(c, RSV_E_ARG, "%s: shape or checksum mismatch", path);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    size_t off = 24;
    double d[kSurDoubles];
    std::memcpy(d, buf.data() + off, sizeof d);
    off += sizeof d;
    SurrogateState& s = c->sur;
    s.flag.assign(buf.data() + off, buf.data() + off + nb);
    off += (size_t)nb;
    std::vector<float> w((size_t)np);
    std::memcpy(w.data(), buf.data() + off, (size_t)np * 4);
    rsv_status st = mlp_upload(c, w.data());
    if (st != RSV_OK) return st;
    CU(s.d_flag.ensure((size_t)nb));
    CU(cudaMemcpyAsync(s.d_flag.p, s.flag.data(), (size_t)nb, cudaMemcpyHostToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    s.y_mean = d[0];
    s.y_std = d[1];
    s.tol = d[2];
    s.a = d[3];
    s.b = d[4];
    s.sigma = d[5];
    s.r0 = d[6];
    s.trained = true;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_surrogate_train(rsv_ctx* c, const rsv_surrogate_cfg* cfg, rsv_surrogate_report* rep) try {
    if (!c) return RSV_E_ARG;
    if (!cfg || !rep) return fail(c, RSV_E_ARG, "cfg and report must not be NULL");
    if (cfg->n_train < 1024 || cfg->n_val < 1024 || cfg->epochs < 0 || cfg->batch < 64 || cfg->batch % 64 ||
        cfg->batch > 65536 || !(cfg->lr > 0) || !(cfg->a > 0) || !(cfg->sigma >= 0) || !(cfg->tol > 0) ||
        cfg->max_node_m < 0 || !(cfg->widen >= 0) || !(cfg->margin > 0) || !(cfg->margin <= 1))
        return fail(c, RSV_E_ARG, "bad surrogate configuration");
    if (c->pols.empty()) return fail(c, RSV_E_STATE, "no portfolio loaded");
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice failed");
    rsv_status st = build_layout(c, 2, 0, kMaxAgeSteps);   // validates the records
    if (st != RSV_OK) return st;
    size_t smem;
    if ((st = build_tables(c, F_F64, smem)) != RSV_OK) return st;
    std::vector<PolSur> hp;
    if ((st = sur_upload_policies(c, hp)) != RSV_OK) return st;
    SurrogateState& s = c->sur;
    s.a = cfg->a;
    s.b = cfg->b;
    s.sigma = cfg->sigma;
    s.r0 = cfg->r0;
    s.tol = cfg->tol;
    const long long nt = cfg->n_train, nv = cfg->n_val, n = nt + nv;
    CU(s.d_q.ensure((size_t)n * sizeof(SurQuery)));
    CU(s.d_lab.ensure((size_t)n * 8));
    CU(s.d_y.ensure((size_t)n * 4));
    CU(s.d_X.ensure((size_t)n * MLP_XW * 2));
    CU(s.d_err.ensure((size_t)nv * 8));
    SurQuery* q = s.d_q.as<SurQuery>();
    cudaEvent_t e0, e1, e2, e3;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    cudaEventCreate(&e3);

    // queries (train: stream 6, held out: stream 7) and their labels
    const int grid = c->sm_count * 8;
    sample_queries_kernel<<<grid, 128, 0, c->stream>>>(c->d_pols.as<PolSur>(), (int)hp.size(), cfg->seed, 6u, nt,
                                                       cfg->a, cfg->b, cfg->sigma, cfg->r0, cfg->widen,
                                                       cfg->max_node_m, q);
    sample_queries_kernel<<<grid, 128, 0, c->stream>>>(c->d_pols.as<PolSur>(), (int)hp.size(), cfg->seed, 7u, nv,
                                                       cfg->a, cfg->b, cfg->sigma, cfg->r0, cfg->widen,
                                                       cfg->max_node_m, q + nt);
    CU(cudaGetLastError());
    SurTables T;
    if ((st = sur_tables(c, T)) != RSV_OK) return st;
    CU(s.d_lnb.ensure((size_t)n * sizeof(float)));
    CU(cudaEventRecord(e0, c->stream));
    sur_label_kernel<<<grid, 128, 0, c->stream>>>(c->d_pols.as<PolSur>(), T, q, n, nullptr, s.d_lab.as<double>());
    CU(cudaGetLastError());
    CU(cudaEventRecord(e1, c->stream));
    sur_features_kernel<<<grid, 256, 0, c->stream>>>(c->d_pols.as<PolSur>(), T, q, n, s.d_X.as<__nv_bfloat16>(),
                                                     s.d_lnb.as<float>());
    CU(cudaGetLastError());
    // target normalisation from the training labels
    const int mb = 256;
    DevBuf part;
    CU(part.ensure(mb * 2 * 8));
    log_moments_kernel<<<mb, 256, 0, c->stream>>>(s.d_lab.as<double>(), s.d_lnb.as<float>(), nt, part.as<double>());
    std::vector<double> hpart(mb * 2);
    CU(cudaMemcpyAsync(hpart.data(), part.p, mb * 2 * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    part.release();
    double s1 = 0, s2 = 0;
    for (int i = 0; i < mb; ++i) {
        s1 += hpart[2 * i];
        s2 += hpart[2 * i + 1];
    }
    s.y_mean = s1 / nt;
    s.y_std = std::sqrt(std::max(s2 / nt - s.y_mean * s.y_mean, 1e-12));
    if (!std::isfinite(s.y_mean)) return fail(c, RSV_E_ASSUMPTION, "a training label is not positive");
    targets_kernel<<<grid, 256, 0, c->stream>>>(s.d_lab.as<double>(), s.d_lnb.as<float>(), n, s.y_mean, s.y_std,
                                                s.d_y.as<float>());
    CU(cudaGetLastError());

    // training: Adam on random batches, cosine learning rate
    if (!c->mlp_ready) {
        std::vector<float> p;
        he_init(p, cfg->seed);
        if ((st = mlp_upload(c, p.data())) != RSV_OK) return st;
    }
    const int B = cfg->batch;
    CU(c->mlp.ensure(std::max(B, 65536)));
    const long long steps = (long long)cfg->epochs * (nt / B);
    CU(cudaEventRecord(e2, c->stream));
    for (long long k = 0; k < steps; ++k) {
        const float lr = (float)(cfg->lr * (0.02 + 0.98 * 0.5 * (1.0 + std::cos(3.141592653589793 * k / steps))));
        gather_kernel<<<(B + 255) / 256, 256, 0, c->stream>>>(s.d_X.as<__nv_bfloat16>(), s.d_y.as<float>(), nt,
                                                              cfg->seed, (uint32_t)k, B, c->mlp.X, c->mlp.t);
        CU(cudaGetLastError());
        CU(c->mlp.forward(c->mlp.X, B, nullptr, c->mlp.t, c->stream));
        CU(c->mlp.backward(c->mlp.X, B, c->stream));
        CU(c->mlp.adam_step(lr, c->stream));
    }
    CU(cudaEventRecord(e3, c->stream));
    float last = 0.0f;
    if (steps > 0) CU(cudaMemcpyAsync(&last, c->mlp.loss, 4, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    float label_ms = 0, train_ms = 0;
    cudaEventElapsedTime(&label_ms, e0, e1);
    cudaEventElapsedTime(&train_ms, e2, e3);

    // held-out scoring against the recurrence (buffers allocated before the timed region)
    CU(s.d_pred.ensure((size_t)nv * 8));
    if (c->mlp.use_tc) CU(c->mlp.ensure_infer(1 << 19));
    CU(cudaEventRecord(e0, c->stream));
    if ((st = sur_predict(c, q + nt, nv, s.d_pred.as<double>(), false, 65536)) != RSV_OK) return st;
    CU(cudaEventRecord(e1, c->stream));
    rel_err_kernel<<<grid, 256, 0, c->stream>>>(s.d_pred.as<double>(), s.d_lab.as<double>() + nt, nv,
                                                s.d_err.as<double>());
    CU(cudaGetLastError());
    std::vector<double> err(nv);
    std::vector<SurQuery> hq(nv);
    CU(cudaMemcpyAsync(err.data(), s.d_err.p, (size_t)nv * 8, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(hq.data(), q + nt, (size_t)nv * sizeof(SurQuery), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    float infer_ms = 0;
    cudaEventElapsedTime(&infer_ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);

    // statistics; fallback map calibrated on the first half, scored on the second
    std::vector<double> ae;
    ae.reserve(nv);
    for (long long i = 0; i < nv; ++i)
        if (hq[i].state >= 0) ae.push_back(std::fabs(err[i]));
    std::vector<double> srt = ae;
    std::sort(srt.begin(), srt.end());
    auto quant = [&](const std::vector<double>& v, double f) { return v.empty() ? 0.0 : v[(size_t)(f * (v.size() - 1))]; };
    double rms = 0;
    for (double x : ae) rms += x * x;
    rms = ae.empty() ? 0 : std::sqrt(rms / ae.size());
    std::vector<double> bmax(SUR_NBUCKETS, 0.0);
    std::vector<long long> bcnt(SUR_NBUCKETS, 0);
    const long long half = nv / 2;
    for (long long i = 0; i < half; ++i) {
        if (hq[i].state < 0) continue;
        bmax[hq[i].bucket] = std::max(bmax[hq[i].bucket], std::fabs(err[i]));
        ++bcnt[hq[i].bucket];
    }
    s.flag.assign(SUR_NBUCKETS, 0);
    long long n_flag = 0;
    for (int k = 0; k < SUR_NBUCKETS; ++k) {
        // unseen, thinly seen, not clearly inside the tolerance, or a rate
        // beyond 4 sd of the model: recurrence
        s.flag[k] = (bcnt[k] < 32 || bmax[k] > cfg->margin * cfg->tol || k % SUR_NB_R == SUR_NB_R - 1) ? 1 : 0;
        n_flag += s.flag[k];
    }
    CU(s.d_flag.ensure(SUR_NBUCKETS));
    CU(cudaMemcpyAsync(s.d_flag.p, s.flag.data(), SUR_NBUCKETS, cudaMemcpyHostToDevice, c->stream));
    double comb = 0;
    long long fb = 0, m2 = 0;
    for (long long i = half; i < nv; ++i) {
        if (hq[i].state < 0) continue;
        ++m2;
        if (s.flag[hq[i].bucket]) ++fb;
        else comb = std::max(comb, std::fabs(err[i]));
    }
    CU(cudaStreamSynchronize(c->stream));
    s.trained = true;
    rep->train_loss = last / B;
    rep->val_max_rel = srt.empty() ? 0 : srt.back();
    rep->val_p99_rel = quant(srt, 0.99);
    rep->val_median_rel = quant(srt, 0.5);
    rep->val_rms_rel = rms;
    rep->frac_fallback = m2 ? (double)fb / m2 : 0.0;
    rep->combined_max_rel = comb;
    rep->label_ms = label_ms;
    rep->train_ms = train_ms;
    rep->infer_ms = infer_ms;
    rep->n_label = n;
    rep->n_infer = nv;
    rep->n_buckets = SUR_NBUCKETS;
    rep->n_flagged = n_flag;
    rep->y_mean = s.y_mean;
    rep->y_std = s.y_std;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

}  // extern "C"
