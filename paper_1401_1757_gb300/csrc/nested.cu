// nested.cu -- the nested ("brute force") Solvency II valuation on sm_103a.
//
// Tucker & Bull (Section 2) value every policy under 1000 Monte Carlo
// scenarios at each future valuation node and take the 5th largest of the
// 1000 liabilities as the 99.5% value.  Here, for outer Vasicek paths o,
// nodes n at months m_n = n * node_step and inner paths i started from the
// outer path's short rate at the node:
//
//   L_{o,n,i} = sum_p amount_p sum_j pi_{p,n,j} r_{p,j}(node; inner path i)
//
// where pi_{p,n,j} is the probability that policy p is in reduced state j at
// the node (deterministic mortality, FP64 on the host) and r_{p,j} is the
// reserve at the node by the backward recurrence (Eq. generalForm) on the
// inner path's discount factors -- the same tile kernels as the valuation
// run, started t_off = m_n steps later.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11), counter (k, c1, c2,
// c3), key (seed lo, seed hi); step 2k takes words 0,1 and step 2k+1 words
// 2,3 as uniforms (w + 1/2) 2^-32, Box-Muller in FP64 (the inner paths
// with table-driven logarithm, sine and cosine, and a series for the
// month's discount factor: below.  Outer path o:
// (k, o, 0, 2 << 24); inner path (o, n, i): (k, i, n, (3 << 24) | o).
// Vasicek exact monthly step of (r, integral of r) (Glasserman 2004 3.3.1);
// v = exp(-integral), FP64, stored in the form's plane format.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fp64_series.cuh"
#include "nested.cuh"
#include "defl_kernel.cuh"
#include "philox.cuh"
#include "rsv.h"
#include "abi_guard.cuh"

namespace rsv {

// ------------------------------------------------------------ generator ----
VasStep vasicek_step_constants(double a, double b, double sigma, double dt) {
    VasStep s;
    const double one_m_e = -std::expm1(-a * dt), one_m_e2 = -std::expm1(-2.0 * a * dt);
    const double var_r = sigma * sigma * one_m_e2 / (2.0 * a);
    const double var_i = sigma * sigma / (a * a) * (dt - 2.0 * one_m_e / a + one_m_e2 / (2.0 * a));
    const double cov = sigma * sigma / (2.0 * a * a) * one_m_e * one_m_e;
    s.e = std::exp(-a * dt);
    s.k1 = one_m_e / a;
    s.l11 = std::sqrt(var_r);
    s.l21 = s.l11 > 0 ? cov / s.l11 : 0.0;
    s.l22 = std::sqrt(std::max(var_i - s.l21 * s.l21, 0.0));
    s.b = b;
    s.dt = dt;
    return s;
}

// Host tables of the Box-Muller step (see nested.cuh).
const double2* bm_tables_host() {
    static const std::vector<double2> t = [] {
        std::vector<double2> v(BM_SC + BM_LG);
        const long double two_pi = 6.283185307179586476925286766559005768L;
        for (int j = 0; j < BM_SC; ++j) {
            const long double x = two_pi * j / BM_SC;
            v[j] = make_double2((double)std::sin(x), (double)std::cos(x));
        }
        for (int j = 0; j < BM_LG; ++j) {
            const double c = 1.0 + (j + 0.5) / BM_LG;
            const double inv = std::ldexp(std::nearbyint(std::ldexp(1.0 / c, 18)), -18);
            const int k = j >= BM_LG_K0 ? 1 : 0;
            v[BM_SC + j] = make_double2(inv, (double)(-std::log(std::ldexp((long double)inv, k))));
        }
        return v;
    }();
    return t.data();
}

constexpr double kLn2 = 0.6931471805599453094;
constexpr double kTwoPi32 = 6.283185307179586477 / 4294967296.0;   // 2 pi 2^-32 (a power-of-two scaling of 2 pi)

// ln u for the uniform u = (w + 1/2) 2^-32 by Tang's table-driven method in
// FP64: w + 1/2 = 2^e y with y in [1, 2); interval j = the top 7 bits of y's
// mantissa; r = y inv_j - 1 is exact (inv_j has 18 significant bits, y at
// most 33) and |r| < 2^-8; ln u = (e + k_j - 32) ln 2 + L_j + log1p(r) with
// L_j = -ln(2^k_j inv_j), k_j = 1 above sqrt 2, and log1p by its Taylor
// series to r^7 (remainder below 2^-60 r).  For u >= 1 - 2^-8, where L_j and
// log1p(r) would cancel, r = u - 1 (exact) and ln u = log1p(r).
__device__ __forceinline__ double bm_log_u(uint32_t w, const double2* __restrict__ lg) {
    const double m = (double)w + 0.5;
    const int e = w ? 31 - __clz((int)w) : -1;
    const double y = m * __longlong_as_double((long long)(1023 - e) << 52);
    const int j = (int)((__double_as_longlong(y) >> 45) & (BM_LG - 1));
    const double2 t = lg[j];
    const bool near1 = w >= 0xFF000000u;
    const double r = near1 ? __dmul_rn(__dadd_rn(m, -4294967296.0), 0x1.0p-32) : __fma_rn(y, t.x, -1.0);
    double q = __fma_rn(r, 1.0 / 7.0, -1.0 / 6.0);
    q = __fma_rn(r, q, 1.0 / 5.0);
    q = __fma_rn(r, q, -0.25);
    q = __fma_rn(r, q, 1.0 / 3.0);
    q = __fma_rn(r, q, -0.5);
    const double p = __fma_rn(__dmul_rn(r, r), q, r);
    const int k = j >= BM_LG_K0 ? 1 : 0;
    return near1 ? p : __fma_rn((double)(e + k - 32), kLn2, __dadd_rn(t.y, p));
}

// (sin, cos)(2 pi u) for u = (w + 1/2) 2^-32: the top 10 bits of w pick
// alpha = 2 pi j / 1024 from the table, the rest give beta = 2 pi f with
// 0 <= beta < 2 pi / 1024; sin beta and cos beta - 1 by their Taylor series
// (to beta^5 and beta^6: remainders below 1e-19), then the addition theorems.
__device__ __forceinline__ void bm_sincos_2pi_u(uint32_t w, const double2* __restrict__ sc, double& sn, double& cs) {
    const double2 t = sc[w >> 22];
    const double b = __dmul_rn(__dadd_rn((double)(w & 0x3FFFFFu), 0.5), kTwoPi32);
    const double b2 = __dmul_rn(b, b);
    const double sb = __fma_rn(__dmul_rn(b2, b), __fma_rn(b2, 1.0 / 120.0, -1.0 / 6.0), b);
    const double cm1 = __dmul_rn(b2, __fma_rn(b2, __fma_rn(b2, -1.0 / 720.0, 1.0 / 24.0), -0.5));
    sn = __fma_rn(t.y, sb, __fma_rn(t.x, cm1, t.x));
    cs = __fma_rn(-t.x, sb, __fma_rn(t.y, cm1, t.y));
}

// One path: n_steps monthly steps from rate r; calls `emit(t, v_t)`.  `bm`
// holds the Box-Muller tables (BM_SC sine/cosine entries, then BM_LG
// logarithm entries).
template <class Emit>
__device__ __forceinline__ double vasicek_path(const VasStep& s, uint64_t seed, uint32_t c1, uint32_t c2,
                                               uint32_t c3, double r, int n_steps, const double2* __restrict__ bm,
                                               Emit emit) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double bdt = s.b * s.dt;
    for (int t = 0; t < n_steps; t += 2) {
        uint32_t w[4];
        philox4x32_10((uint32_t)(t >> 1), c1, c2, c3, k0, k1, w);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (t + h >= n_steps) break;
            const double R = sqrt(-2.0 * bm_log_u(w[2 * h], bm + BM_SC));
            double sn, cs;
            bm_sincos_2pi_u(w[2 * h + 1], bm, sn, cs);
            const double z1 = R * cs, z2 = R * sn;
            const double dr = r - s.b;
            const double I = __fma_rn(s.l22, z2, __fma_rn(s.l21, z1, __fma_rn(dr, s.k1, bdt)));
            r = __fma_rn(s.l11, z1, __fma_rn(dr, s.e, s.b));
            emit(t + h, exp_small(-I), r);
        }
    }
    return r;
}

// Outer paths, one warp each.  The draws of a step depend only on its
// counter, so the lanes take 32 consecutive steps at once; the rate update
// r_{t+1} = e r_t + c_t (c_t = b (1 - e) + l11 z1_t) is affine with a common
// multiplier, so a warp scan of the maps gives every lane the rate at the
// start of its step, and a product scan the discount to its end.  The same
// path as the serial recursion up to the order of rounding.
__global__ void outer_paths_kernel(VasStep s, uint64_t seed, int o_first, int n_outer, int n_nodes, int node_step,
                                   double r0, double* __restrict__ r_node, double* __restrict__ d0) {
    const int lane = threadIdx.x & 31;
    const int o = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (o >= n_outer) return;   // whole warps leave together
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const double inv32 = 2.3283064365386963e-10;   // 2^-32
    const int n_steps = (n_nodes - 1) * node_step;
    if (lane == 0) {
        r_node[(size_t)o * n_nodes] = r0;
        d0[(size_t)o * n_nodes] = 1.0;
    }
    double r = r0, D = 1.0;   // at the start of the block of 32 steps
    for (int t0 = 0; t0 < n_steps; t0 += 32) {
        const int t = t0 + lane;
        const bool live = t < n_steps;
        double z1 = 0.0, z2 = 0.0;
        if (live) {   // the serial generator's draw for step t
            uint32_t w[4];
            philox4x32_10((uint32_t)(t >> 1), (uint32_t)(o_first + o), 0u, 2u << 24, k0, k1, w);
            const int h = t & 1;
            const double u1 = ((double)w[2 * h] + 0.5) * inv32;
            const double u2 = ((double)w[2 * h + 1] + 0.5) * inv32;
            const double R = sqrt(-2.0 * log(u1));
            double sn, cs;
            sincospi(2.0 * u2, &sn, &cs);
            z1 = R * cs;
            z2 = R * sn;
        }
        // inclusive scan of the maps x -> A x + B over the lanes: A = e^(lane+1)
        double A = s.e, B = live ? s.b * (1.0 - s.e) + s.l11 * z1 : 0.0;
        if (!live) A = 1.0;   // identity past the end
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double Au = __shfl_up_sync(0xffffffffu, A, d), Bu = __shfl_up_sync(0xffffffffu, B, d);
            if (lane >= d) {   // this map after the lower lanes' composition
                B = A * Bu + B;
                A = A * Au;
            }
        }
        // the rate at the start of step t: the exclusive prefix applied to r
        double Ae = __shfl_up_sync(0xffffffffu, A, 1), Be = __shfl_up_sync(0xffffffffu, B, 1);
        if (lane == 0) {
            Ae = 1.0;
            Be = 0.0;
        }
        const double rt = Ae * r + Be;
        const double I = s.b * s.dt + (rt - s.b) * s.k1 + s.l21 * z1 + s.l22 * z2;
        double v = live ? exp(-I) : 1.0;
        // inclusive product scan of the discount factors
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const double vu = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v *= vu;
        }
        const double r_after = A * r + B, D_after = D * v;
        if (live && (t + 1) % node_step == 0) {
            const int nd = (t + 1) / node_step;
            r_node[(size_t)o * n_nodes + nd] = r_after;
            d0[(size_t)o * n_nodes + nd] = D_after;
        }
        r = __shfl_sync(0xffffffffu, r_after, 31);
        D = __shfl_sync(0xffffffffu, D_after, 31);
    }
}

template <class VE>
__device__ __forceinline__ VE to_plane(double x);
template <>
__device__ __forceinline__ double to_plane<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_plane<float>(double x) { return __double2float_rn(x); }
template <>
__device__ __forceinline__ float2 to_plane<float2>(double x) {
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(x - (double)h));
}

// Inner paths of outer paths [o0, o0 + B), every node: one thread per path.
// Plane layout [B][n_nodes][Lmax][i_pad]; node n fills rows 0 .. Ln[n]-1.
template <class VE>
__global__ void inner_paths_kernel(VasStep s, uint64_t seed, int o_first, int o0, int B, int n_nodes, int n_inner, int i_pad,
                                   int Lmax, const int* __restrict__ Ln, const double* __restrict__ r_node,
                                   const double2* __restrict__ bm_g, VE* __restrict__ plane) {
    __shared__ double2 bm[BM_SC + BM_LG];   // 18 KiB: the Box-Muller tables
    for (int k = threadIdx.x; k < BM_SC + BM_LG; k += blockDim.x) bm[k] = bm_g[k];
    __syncthreads();
    const size_t total = (size_t)B * n_nodes * i_pad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % i_pad);
        const int n = (int)((idx / i_pad) % n_nodes);
        const int ol = (int)(idx / ((size_t)i_pad * n_nodes));
        const int o = o0 + ol;
        VE* base = plane + ((size_t)ol * n_nodes + n) * Lmax * i_pad + i;
        const int L = Ln[n];
        if (i >= n_inner) {   // padding lanes read finite factors
            for (int t = 0; t < L; ++t) base[(size_t)t * i_pad] = to_plane<VE>(1.0);
            continue;
        }
        vasicek_path(s, seed, (uint32_t)i, (uint32_t)n, (3u << 24) | (uint32_t)(o_first + o),
                     r_node[(size_t)o * n_nodes + n], L, bm,
                     [&](int t, double v, double) { base[(size_t)t * i_pad] = to_plane<VE>(v); });
    }
}

// The curve mode with the outer paths on the lanes: every outer path's node
// rate gives one curve, and all outer paths share the in-force weights, so
// plane[n][t][o] holds outer path o's curve at node n (one virtual outer
// path whose "inner paths" are the real outer paths).  Padding lanes get 1.
template <class VE>
__global__ void curve_planes_lanes_kernel(double a, double b, double sigma, double dt, int n_outer, int n_nodes,
                                          int o_pad, int Lmax, const int* __restrict__ Ln,
                                          const double* __restrict__ r_node, VE* __restrict__ plane) {
    const size_t total = (size_t)n_nodes * Lmax * o_pad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int o = (int)(idx % o_pad);
        const int t = (int)((idx / o_pad) % Lmax);
        const int n = (int)(idx / ((size_t)o_pad * Lmax));
        double v = 1.0;
        if (o < n_outer && t < Ln[n]) {
            const double r = r_node[(size_t)o * n_nodes + n];
            v = exp(vasicek_lnP((t + 1) * dt, r, a, b, sigma) - vasicek_lnP(t * dt, r, a, b, sigma));
        }
        plane[idx] = to_plane<VE>(v);
    }
}

// L[o][n] = Lt[n][o] (the curve mode's node liabilities back to outer-major)
__global__ void transpose_on_kernel(const double* __restrict__ Lt, int n_outer, int n_nodes, double* __restrict__ L) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_outer * n_nodes) return;
    const int o = i / n_nodes, n = i - o * n_nodes;
    L[i] = Lt[(size_t)n * n_outer + o];
}

// ------------------------------------------------------- nested recurrence ----
// One CTA per item (o, n, chunk of 32 inner paths); its warps share the
// policy tiles, each lane accumulates the pi-weighted reserves of its path,
// and the CTA adds the warps' sums in a fixed order (deterministic).
template <int FORM, int P, int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 3 : 1) nested_kernel(const NestedArgs a) {
    using TabE = typename Tr<FORM>::TabE;
    using VE = typename Tr<FORM>::VE;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ int s_item;
    __shared__ double red[NW][32];
    TabE* tab = reinterpret_cast<TabE*>(smem_raw);
    if (!stage_to_smem(tab, a.tab, (uint32_t)a.tab_bytes, &bar, a.status)) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        // items run node-major: early nodes (longest projections) first
        const int chunk = item % a.n_chunks;
        const int ol = (item / a.n_chunks) % a.B;
        const int n = item / (a.n_chunks * a.B);
        const int m = n * a.node_step;
        const VE* plane = static_cast<const VE*>(a.v) + ((size_t)ol * a.n_nodes + n) * a.Lmax * a.i_pad;
        const TileEnv env{a.slots, plane, a.i_pad, a.n_inner, 0, nullptr, nullptr, nullptr, a.n_inner};
        const double* wts = a.wts + (size_t)n * 3;
        const size_t wstride = (size_t)a.n_nodes * 3;
        double acc[1] = {0.0};
        for (int tile = warp; tile < a.n_tiles; tile += NW) {
            if (a.slots[(size_t)tile * P].S < m) continue;   // whole tile ended before the node
            const int kind = a.tile_kind[tile];
            if (kind == K_JL) {
                Tile<FORM, P, 1, K_JL, false> w(env, tab, tile, chunk, lane, m);
                w.run_steps();
                w.epilogue_weighted(acc, wts, wstride);
            } else if (kind == K_ANN) {
                Tile<FORM, P, 1, K_ANN, false> w(env, tab, tile, chunk, lane, m);
                w.run_steps();
                w.epilogue_weighted(acc, wts, wstride);
            } else if (kind == K_ANN2) {
                Tile<FORM, P, 1, K_ANN2, false> w(env, tab, tile, chunk, lane, m);
                w.run_steps();
                w.epilogue_weighted(acc, wts, wstride);
            } else if (kind == K_ASS2) {
                Tile<FORM, P, 1, K_ASS2, false> w(env, tab, tile, chunk, lane, m);
                w.run_steps();
                w.epilogue_weighted(acc, wts, wstride);
            } else if (kind == K_LS2) {
                Tile<FORM, P, 1, K_LS2, false> w(env, tab, tile, chunk, lane, m);
                w.run_steps();
                w.epilogue_weighted(acc, wts, wstride);
            } else {
                Tile<FORM, P, 1, K_ASS, false> w(env, tab, tile, chunk, lane, m);
                w.run_steps();
                w.epilogue_weighted(acc, wts, wstride);
            }
        }
        red[warp][lane] = acc[0];
        __syncthreads();
        if (warp == 0) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) sum += red[w][lane];
            const int i = chunk * 32 + lane;
            if (i < a.n_inner)
                a.L_all[((size_t)(a.o0 + ol) * a.n_nodes + n) * a.n_inner + i] = sum;
        }
        __syncthreads();
    }
}

// Mean and k-th largest over the inner paths of each (o, n), one CTA each.
// The k-th largest is found by descending thresholds: the largest value
// below the current threshold and its multiplicity, until k values are
// covered, so ties need no special care.
__global__ void node_stats_kernel(const double* __restrict__ L_all, int n_inner, int k, double* __restrict__ mean,
                                  double* __restrict__ kth) {
    __shared__ double sd[256];
    __shared__ int si[256];
    const size_t on = blockIdx.x;
    const double* x = L_all + on * n_inner;
    double s = 0.0;
    for (int i = threadIdx.x; i < n_inner; i += blockDim.x) s += x[i];
    sd[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sd[threadIdx.x] += sd[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mean[on] = sd[0] / n_inner;
    __syncthreads();
    double thr = INFINITY;
    int left = k;
    for (int round = 0; round < k; ++round) {
        double mx = -INFINITY;
        for (int i = threadIdx.x; i < n_inner; i += blockDim.x)
            if (x[i] < thr) mx = fmax(mx, x[i]);
        sd[threadIdx.x] = mx;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + w]);
            __syncthreads();
        }
        const double m = sd[0];
        __syncthreads();
        int c = 0;
        for (int i = threadIdx.x; i < n_inner; i += blockDim.x) c += (x[i] == m);
        si[threadIdx.x] = c;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) si[threadIdx.x] += si[threadIdx.x + w];
            __syncthreads();
        }
        const int cnt = si[0];
        __syncthreads();
        if (cnt >= left || m == -INFINITY) {
            if (threadIdx.x == 0) kth[on] = m;
            break;
        }
        left -= cnt;
        thr = m;
    }
}

// ------------------------------------------- deflated brute-force mode ----
// Inner paths as deflator planes: D_i(m, m+tau+1), the FP64 running product
// of the path's monthly discount factors from the node, rounded to FP32, in
// rows of four steps [B][n_nodes][G4][i_pad]; zeros from the node's remaining
// length to the end of its last group of four.  One thread per path.
__global__ void inner_paths_defl_kernel(VasStep s, uint64_t seed, int o_first, int o0, int B, int n_nodes, int n_inner, int i_pad,
                                        int G4, const int* __restrict__ Ln, const double* __restrict__ r_node,
                                        const double2* __restrict__ bm_g, float* __restrict__ plane) {
    __shared__ double2 bm[BM_SC + BM_LG];   // 18 KiB: the Box-Muller tables
    for (int k = threadIdx.x; k < BM_SC + BM_LG; k += blockDim.x) bm[k] = bm_g[k];
    __syncthreads();
    const size_t total = (size_t)B * n_nodes * i_pad;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % i_pad);
        const int n = (int)((idx / i_pad) % n_nodes);
        const int ol = (int)(idx / ((size_t)i_pad * n_nodes));
        const int o = o0 + ol;
        // element (tau, i) at ((ol n_nodes + n) G4 + tau / 4) i_pad 4 + 4 i + tau % 4
        float* base = plane + ((size_t)ol * n_nodes + n) * G4 * i_pad * 4 + 4 * (size_t)i;
        const int L = Ln[n], Lr = (L + 3) / 4 * 4;
        auto at = [&](int tau) -> float& { return base[(size_t)(tau >> 2) * i_pad * 4 + (tau & 3)]; };
        if (i >= n_inner) {   // padding lanes: finite factors, never written out
            for (int tau = 0; tau < Lr; ++tau) at(tau) = 1.0f;
            continue;
        }
        double D = 1.0;
        vasicek_path(s, seed, (uint32_t)i, (uint32_t)n, (3u << 24) | (uint32_t)(o_first + o),
                     r_node[(size_t)o * n_nodes + n], L, bm, [&](int t, double v, double) {
                         D = __dmul_rn(D, v);
                         at(t) = __double2float_rn(D);
                     });
        for (int tau = L; tau < Lr; ++tau) at(tau) = 0.0f;
    }
}

// Node liabilities by the deflated recurrence.  One CTA per item (node n,
// outer path of the batch, chunk of 32 M inner paths); its NW warps share the
// policy tiles, lane l holds inner paths chunk + m 32 + l of every policy of
// its tile (P x M chains).  Per chain-step one FP32 fused multiply-add of the
// path's deflator and the policy's expected cash flow (two accumulators on
// alternate steps, folded into a double-float every 16 steps); per tile the
// scaled sums are added into each path's double-float liability, and the
// CTA adds its warps' liabilities in a fixed order in FP64.
// One whole 16-step span from the node, groups g0 .. g0 - 3 (g0 = 3 mod 4),
// the inner paths' deflator rows read from the plane (row stride i_pad).
template <int KIND, int P, int M, bool CHECK, class Lane>
__device__ __forceinline__ void nest_span(Lane& st, const DeflPol<P>& pp, const float4* __restrict__ tab,
                                          const float4* __restrict__ plane, int i_pad, int g0) {
    const float4* row = plane + (size_t)g0 * i_pad;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        float4 d[M];
#pragma unroll
        for (int q = 0; q < M; ++q) d[q] = row[q * 32];
        row -= i_pad;
        if (u == 0) defl_group<KIND, P, M, true>(st, pp, tab, d, g0 - u, CHECK);
        else defl_group<KIND, P, M, false>(st, pp, tab, d, g0 - u, CHECK);
    }
    defl_fold_all(st);
}

template <int P, int M, int NW>
__global__ void __launch_bounds__(NW * 32, 2) nested_defl_kernel(const NestDeflArgs a) {
    using Lane = DeflLaneX2<P, M>;   // packed pairs, as the valuation kernel
    constexpr int CH = 32 * M;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    __shared__ int s_item;
    __shared__ float2 red[NW][CH];
    if (!stage_to_smem(smem_raw, a.tab, (uint32_t)a.tab_bytes, &bar, a.status)) return;
    const float4* tab = reinterpret_cast<const float4*>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int dpad4 = a.dpad / 4;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= a.n_items) break;
        // node-major: the early nodes (longest projections) first
        const int chunk = item % a.n_chunks;
        const int ol = (item / a.n_chunks) % a.B;
        const int n = item / (a.n_chunks * a.B);
        const int m = n * a.node_step;
        const float4* plane = a.D + ((size_t)ol * a.n_nodes + n) * a.G4 * a.i_pad + (size_t)chunk * CH + lane;
        float acc_h[M], acc_l[M];
#pragma unroll
        for (int q = 0; q < M; ++q) acc_h[q] = acc_l[q] = 0.0f;
        for (int tile = warp; tile < a.n_tiles; tile += NW) {
            const NestSlot* rec = a.slots + (size_t)tile * P;
            if (rec[0].S < m) continue;   // the tile's longest policy ended before the node
            const int kind = a.tile_kind[tile];
            // the runs of the tile's policies from the node
            DeflPol<P> pp;
            int smin = 1 << 30, smax = 0;
            Lane st;
            float h0s[P][M];
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const NestSlot r = rec[i];
                int S = r.S - m;
                const bool live = r.pol >= 0 && S >= 0 && !(r.unit && m > 0);
                if (!live) S = 0;
                pp.S[i] = S;
                smin = min(smin, S);
                smax = max(smax, S);
                pp.ix[i] = r.ix;
                pp.iy[i] = r.iy;
                // life 1: aligned run at age + m, or a zero group; the unit group at node 0
                const int a1 = r.age1 + m;
                if (r.unit) {
                    pp.off1[i] = r.base1 + (a.dpad - 8) / 4;
                    pp.gz1[i] = 1;
                } else if (a1 >= r.z1) {
                    pp.off1[i] = r.base1 + (r.z1 + 3) / 4;
                    pp.gz1[i] = 0;
                } else {
                    pp.off1[i] = r.base1 + (a1 & 3) * dpad4 + (a1 >> 2);
                    pp.gz1[i] = (r.z1 - a1 + 3) / 4;
                }
                const int a2 = r.age2 + m;
                if (a2 >= r.z2) {
                    pp.off2[i] = r.base2 + (r.z2 + 3) / 4;
                    pp.gz2[i] = 0;
                } else {
                    pp.off2[i] = r.base2 + (a2 & 3) * dpad4 + (a2 >> 2);
                    pp.gz2[i] = (r.z2 - a2 + 3) / 4;
                }
#pragma unroll
                for (int q = 0; q < M; ++q) {   // the boundary D(m, S) mat
                    float h0 = 0.0f;
                    if (live && r.mat != 0.0f) {
                        float dS = 1.0f;
                        if (S > 0) dS = reinterpret_cast<const float*>(plane + (size_t)((S - 1) >> 2) * a.i_pad + q * 32)[(S - 1) & 3];
                        h0 = __fmul_rn(dS, r.mat);
                    }
                    h0s[i][q] = h0;
                }
            }
#pragma unroll
            for (int i = 0; i < P; ++i) st.start(i, h0s[i]);
            st.clear_acc();
            if (smax > 0) {
                // groups of four steps from the node, descending; 16-step spans
                // aligned at the node (a span opens at g = 3 mod 4 and is folded at
                // g = 0 mod 4; the top span may be partial and starts from zero)
                const int g_top = (smax - 1) >> 2;
                auto run = [&](auto kind_c) {
                    constexpr int KIND = decltype(kind_c)::value;
                    int g = g_top;
#pragma unroll 1
                    for (; g >= 0 && (g & 3) != 3; --g) {   // the partial top span
                        float4 d[M];
#pragma unroll
                        for (int q = 0; q < M; ++q) d[q] = plane[(size_t)g * a.i_pad + q * 32];
                        defl_group<KIND, P, M, false>(st, pp, tab, d, g, true);
                        if ((g & 3) == 0) defl_fold_all(st);
                    }
                    // whole spans g .. g - 3; only those reaching a policy's end check
#pragma unroll 1
                    for (; g >= 3; g -= 4) {
                        if (4 * g + 3 >= smin) nest_span<KIND, P, M, true>(st, pp, tab, plane, a.i_pad, g);
                        else nest_span<KIND, P, M, false>(st, pp, tab, plane, a.i_pad, g);
                    }
                };
                if (kind == K_ANN) run(std::integral_constant<int, K_ANN>{});
                else if (kind == K_ASS) run(std::integral_constant<int, K_ASS>{});
                else if (kind == K_JL) run(std::integral_constant<int, K_JL>{});
                else run(std::integral_constant<int, K_ANN2>{});
            }
            // this tile's scaled sums into the paths' liabilities
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const float sh = rec[i].sc_h, sl = rec[i].sc_l;
                float Hs[M], Ls[M];
                st.sum(i, Hs, Ls);
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const float H = Hs[q], L = Ls[q];
                    const float p = __fmul_rn(H, sh);
                    float e = __fmaf_rn(H, sh, -p);
                    e = __fmaf_rn(H, sl, e);
                    e = __fmaf_rn(L, sh, e);
                    defl_fold(acc_h[q], acc_l[q], p);
                    acc_l[q] = __fadd_rn(acc_l[q], e);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < M; ++q) red[warp][q * 32 + lane] = make_float2(acc_h[q], acc_l[q]);
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < M; ++q) {
                double x = 0.0;
                for (int w = 0; w < NW; ++w) {
                    const float2 v = red[w][q * 32 + lane];
                    x += (double)v.x + (double)v.y;
                }
                const int i = chunk * CH + q * 32 + lane;
                if (i < a.n_inner) a.L_all[((size_t)(a.o0 + ol) * a.n_nodes + n) * a.n_inner + i] = x;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- launchers ----
cudaError_t launch_inner_paths_defl(const VasStep& s, uint64_t seed, int o_first, int o0, int B, int n_nodes, int n_inner,
                                    int i_pad, int G4, const int* Ln, const double* r_node, const double2* bm,
                                    float4* plane, int sm_count, int ctas_per_sm, cudaStream_t st) {
    inner_paths_defl_kernel<<<sm_count * ctas_per_sm, 128, 0, st>>>(s, seed, o_first, o0, B, n_nodes, n_inner, i_pad, G4, Ln, r_node, bm,
                                                          reinterpret_cast<float*>(plane));
    return cudaGetLastError();
}

cudaError_t launch_nested_defl(const NestDeflArgs& a, int sm_count, int max_per_sm, cudaStream_t st) {
    constexpr int P = kNestDeflP, M = 2, NW = 8;
    auto k = nested_defl_kernel<P, M, NW>;
    const size_t smem = (size_t)a.tab_bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, NW * 32, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>((long long)sm_count * std::min(bps, max_per_sm), std::max(1, a.n_items));
    k<<<(int)grid, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int FORM, int P, int NT>
cudaError_t launch_nested_t(const NestedArgs& a, int sm_count, size_t smem, cudaStream_t st) {
    auto k = nested_kernel<FORM, P, NT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, NT, smem);
    if (e != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const long long grid = std::min<long long>((long long)sm_count * bps, std::max(1, a.n_items));
    k<<<(int)grid, NT, smem, st>>>(a);
    return cudaGetLastError();
}

int nested_tile_width(int form) { return form == F_F32 ? 4 : (form == F_COMP ? 6 : 2); }

cudaError_t launch_nested(int form, const NestedArgs& a, int sm_count, size_t smem, cudaStream_t st) {
    switch (form) {
    case F_F64: return launch_nested_t<F_F64, 2, 256>(a, sm_count, smem, st);
    case F_F32: return launch_nested_t<F_F32, 4, 256>(a, sm_count, smem, st);
    default: return launch_nested_t<F_COMP, 6, 128>(a, sm_count, smem, st);
    }
}

cudaError_t launch_outer_paths(const VasStep& s, uint64_t seed, int o_first, int n_outer, int n_nodes, int node_step, double r0,
                               double* r_node, double* d0, cudaStream_t st) {
    outer_paths_kernel<<<(n_outer + 3) / 4, 128, 0, st>>>(s, seed, o_first, n_outer, n_nodes, node_step, r0, r_node, d0);
    return cudaGetLastError();
}

cudaError_t launch_inner_paths(int form, const VasStep& s, uint64_t seed, int o_first, int o0, int B, int n_nodes, int n_inner,
                               int i_pad, int Lmax, const int* Ln, const double* r_node, const double2* bm,
                               void* plane, int sm_count, cudaStream_t st) {
    const int grid = sm_count * 8;
    if (form == F_F64)
        inner_paths_kernel<double><<<grid, 128, 0, st>>>(s, seed, o_first, o0, B, n_nodes, n_inner, i_pad, Lmax, Ln, r_node,
                                                          bm, static_cast<double*>(plane));
    else if (form == F_F32)
        inner_paths_kernel<float><<<grid, 128, 0, st>>>(s, seed, o_first, o0, B, n_nodes, n_inner, i_pad, Lmax, Ln, r_node,
                                                         bm, static_cast<float*>(plane));
    else
        inner_paths_kernel<float2><<<grid, 128, 0, st>>>(s, seed, o_first, o0, B, n_nodes, n_inner, i_pad, Lmax, Ln, r_node,
                                                          bm, static_cast<float2*>(plane));
    return cudaGetLastError();
}

// The generator's functions on given draws (a test entry point).
__global__ void generator_math_kernel(const uint32_t* __restrict__ w, const double* __restrict__ x, long long n,
                                      const double2* __restrict__ bm_g, double* __restrict__ out) {
    __shared__ double2 bm[BM_SC + BM_LG];
    for (int k = threadIdx.x; k < BM_SC + BM_LG; k += blockDim.x) bm[k] = bm_g[k];
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double sn, cs;
        bm_sincos_2pi_u(w[i], bm, sn, cs);
        out[4 * i] = bm_log_u(w[i], bm + BM_SC);
        out[4 * i + 1] = sn;
        out[4 * i + 2] = cs;
        out[4 * i + 3] = exp_small(x[i]);
    }
}

cudaError_t launch_curve_planes_lanes(int form, double a, double b, double sigma, int n_outer, int n_nodes, int o_pad,
                                      int Lmax, const int* Ln, const double* r_node, void* plane, int sm_count,
                                      cudaStream_t st) {
    const int grid = sm_count * 8;
    const double dt = 1.0 / 12.0;
    if (form == F_F64)
        curve_planes_lanes_kernel<double><<<grid, 128, 0, st>>>(a, b, sigma, dt, n_outer, n_nodes, o_pad, Lmax, Ln,
                                                                 r_node, static_cast<double*>(plane));
    else if (form == F_F32)
        curve_planes_lanes_kernel<float><<<grid, 128, 0, st>>>(a, b, sigma, dt, n_outer, n_nodes, o_pad, Lmax, Ln,
                                                                r_node, static_cast<float*>(plane));
    else
        curve_planes_lanes_kernel<float2><<<grid, 128, 0, st>>>(a, b, sigma, dt, n_outer, n_nodes, o_pad, Lmax, Ln,
                                                                 r_node, static_cast<float2*>(plane));
    return cudaGetLastError();
}

cudaError_t launch_transpose_on(const double* Lt, int n_outer, int n_nodes, double* L, cudaStream_t st) {
    const int n = n_outer * n_nodes;
    if (n <= 0) return cudaSuccess;
    transpose_on_kernel<<<(n + 255) / 256, 256, 0, st>>>(Lt, n_outer, n_nodes, L);
    return cudaGetLastError();
}

cudaError_t launch_node_stats(const double* L_all, int n_on, int n_inner, int k, double* mean, double* kth,
                              cudaStream_t st) {
    if (n_on <= 0) return cudaSuccess;
    node_stats_kernel<<<n_on, 256, 0, st>>>(L_all, n_inner, k, mean, kth);
    return cudaGetLastError();
}

}  // namespace rsv

extern "C" rsv_status rsv_selftest_generator_math(int32_t device, void* cuda_stream, const uint32_t* w, const double* x,
                                                  int64_t n, double* out) try {
    if (n < 0 || (n > 0 && (!w || !x || !out))) return RSV_E_ARG;
    if (n == 0) return RSV_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaSetDevice(device) != cudaSuccess) return RSV_E_CUDA;
    uint32_t* dw = nullptr;
    double *dx = nullptr, *dout = nullptr;
    double2* dbm = nullptr;
    const size_t nb = (size_t)(rsv::BM_SC + rsv::BM_LG) * sizeof(double2);
    rsv_status rc = RSV_OK;
    if (cudaMalloc(&dw, (size_t)n * 4) != cudaSuccess || cudaMalloc(&dx, (size_t)n * 8) != cudaSuccess ||
        cudaMalloc(&dout, (size_t)n * 32) != cudaSuccess || cudaMalloc(&dbm, nb) != cudaSuccess) {
        rc = RSV_E_NOMEM;
    } else if (cudaMemcpyAsync(dw, w, (size_t)n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
               cudaMemcpyAsync(dx, x, (size_t)n * 8, cudaMemcpyHostToDevice, st) != cudaSuccess ||
               cudaMemcpyAsync(dbm, rsv::bm_tables_host(), nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = RSV_E_CUDA;
    } else {
        const int grid = (int)std::min<long long>((n + 127) / 128, 1024);
        rsv::generator_math_kernel<<<grid, 128, 0, st>>>(dw, dx, n, dbm, dout);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(out, dout, (size_t)n * 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = RSV_E_CUDA;
    }
    cudaFree(dw);
    cudaFree(dx);
    cudaFree(dout);
    cudaFree(dbm);
    return rc;
} catch (...) {
    return rsv::host_error(nullptr);
}
