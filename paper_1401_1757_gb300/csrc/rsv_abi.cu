// rsv_abi.cu -- host side of the C ABI declared in include/rsv.h.
//
// Loads copy the caller's host data; compute builds (and caches) the device
// work layout: the decrement tables in the form's entry format, the policy
// tiles grouped by reduced model and sorted by decreasing projection length
// (so the persistent kernel's queue hands out the longest work first; the
// paper spreads policies over OpenMP threads, Section 6.2), and the scratch of
// the per-scenario totals.
#include <algorithm>
#include <thread>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rsv.h"
#include "abi_guard.cuh"
#include "ctx.cuh"
#include "nested.cuh"
#include "scan.cuh"
#include "summation.cuh"
#include "defl_kernel.cuh"

using namespace rsv;

namespace {

// The tunable variants come first; then the side-output one and those that
// pay annuities within the step.
int tunable_count(const Variant* vl, int n) {
    int k = 0;
    while (k < n && !vl[k].extra && vl[k].pay == PAY_END) ++k;
    return k;
}
int special_variant(const Variant* vl, int n, bool extra, int pay) {
    for (int k = 0; k < n; ++k)
        if (vl[k].extra == extra && vl[k].pay == pay) return k;
    return 0;
}

// FP32 copy of the FP64 cash-flow multipliers
__global__ void cf_to_f32_kernel(const double* __restrict__ a, float* __restrict__ b, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        b[i] = __double2float_rn(a[i]);
}

// Cash-flow multipliers of one payment schedule per policy (FP64), rows of
// n_steps: cf_t = [t >= first, (t - first) mod every = 0] (1 + increase n_t)
// (1 + escalation)^n_t with n_t = floor((t + since) / steps_per_year).
__global__ void schedule_kernel(const rsv_schedule* __restrict__ sch, int64_t n_pol, int n_steps,
                                double* __restrict__ cf64, float* __restrict__ cf32) {
    const size_t total = (size_t)n_pol * n_steps;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const rsv_schedule s = sch[i / n_steps];
        const int t = (int)(i % n_steps);
        double x = 0.0;
        if (t >= s.first && (t - s.first) % s.every == 0) {
            const int n = (t + s.since) / s.steps_per_year;
            x = (1.0 + s.increase * n) * pow(1.0 + s.escalation, (double)n);
        }
        cf64[i] = x;
        cf32[i] = __double2float_rn(x);
    }
}

// Per policy: 1 if its cash-flow row is all ones (level), one warp per row.
__global__ void cf_level_kernel(const double* __restrict__ cf, int64_t n_pol, int n_steps,
                                unsigned char* __restrict__ level) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; p < n_pol; p += warps) {
        bool one = true;
        for (int t = lane; t < n_steps; t += 32) one &= cf[(size_t)p * n_steps + t] == 1.0;
        one = __all_sync(0xffffffffu, one);
        if (lane == 0) level[p] = one ? 1 : 0;
    }
}

const Variant* variant_list(int form, int* n) {
    switch (form) {
    case F_F64: return variants_f64(n);
    case F_F32: return variants_f32(n);
    case F_COMP: return variants_comp(n);
    default: *n = 0; return nullptr;
    }
}

__global__ void split_planes_kernel(const double* __restrict__ v, int layout, int n_scen, int n_steps,
                                    int s_pad, double* __restrict__ p64, float* __restrict__ p32,
                                    float2* __restrict__ p2) {
    const size_t total = (size_t)n_steps * s_pad;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int t = (int)(i / s_pad), s = (int)(i % s_pad);
        double x = 1.0;   // padding scenarios: any finite factor, never written out
        if (s < n_scen) x = layout == 0 ? v[(size_t)s * n_steps + t] : v[(size_t)t * n_scen + s];
        const float h = __double2float_rn(x);
        p64[i] = x;
        p32[i] = h;
        p2[i] = make_float2(h, __double2float_rn(x - (double)h));
    }
}

// Fixed-order two-level sum of the per-tile scenario sums (deterministic).
__global__ void reduce_tiles_kernel(const double* __restrict__ partial, int n_tiles, int s_pad, int G,
                                    double* __restrict__ part2) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= s_pad) return;
    const int t0 = blockIdx.y * G, t1 = min(n_tiles, t0 + G);
    double acc = 0.0;
    for (int t = t0; t < t1; ++t) acc += partial[(size_t)t * s_pad + s];
    part2[(size_t)blockIdx.y * s_pad + s] = acc;
}

__global__ void reduce_groups_kernel(const double* __restrict__ part2, int n_groups, int s_pad, int n_scen,
                                     double* __restrict__ total) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scen) return;
    double acc = 0.0;
    for (int g = 0; g < n_groups; ++g) acc += part2[(size_t)g * s_pad + s];
    total[s] = acc;
}

// L[k] = base[k] + sum over q in [seg[k], seg[k+1]) of w[q] V[q], one block per
// (outer path, node), fixed order.
__global__ void segment_wsum_kernel(const long long* __restrict__ seg, const double* __restrict__ w,
                                    const double* __restrict__ V, const double* __restrict__ base,
                                    double* __restrict__ L) {
    __shared__ double sd[256];
    const long long a = seg[blockIdx.x], b = seg[blockIdx.x + 1];
    double s = 0.0;
    for (long long q = a + threadIdx.x; q < b; q += blockDim.x) s += w[q] * V[q];
    sd[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) sd[threadIdx.x] += sd[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) L[blockIdx.x] = base[blockIdx.x] + sd[0];
}

// The surrogate mode's queries: node n's list of in-force (policy, state)
// queries (offsets noff[n], weights nw) repeated for every outer path o, at
// that path's node rate.  Segment k = o NN + n spans
// [o Qn + noff[n], o Qn + noff[n+1]) and starts from base[n].
__global__ void expand_node_queries_kernel(const rsv_query* __restrict__ nq, const double* __restrict__ nw,
                                           long long Qn, int NO, int NN, int step, const double* __restrict__ rn,
                                           rsv_query* __restrict__ q, double* __restrict__ w) {
    const long long n_all = Qn * NO;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_all; i += (long long)gridDim.x * blockDim.x) {
        const long long o = i / Qn, j = i - o * Qn;
        rsv_query x = nq[j];
        x.r = rn[o * NN + x.m / step];
        q[i] = x;
        w[i] = nw[j];
    }
}

__global__ void node_segments_kernel(const long long* __restrict__ noff, const double* __restrict__ nbase,
                                     long long Qn, int NO, int NN, long long* __restrict__ seg,
                                     double* __restrict__ base) {
    const long long on_n = (long long)NO * NN;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k <= on_n; k += (long long)gridDim.x * blockDim.x) {
        const long long o = k / NN, n = k - o * NN;
        seg[k] = k == on_n ? Qn * NO : o * Qn + noff[n];
        if (k < on_n) base[k] = nbase[n];
    }
}

__global__ void scale_kernel(double* __restrict__ x, size_t n, double f) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

}  // namespace

namespace {

int table_len(const rsv_ctx* c, int id) { return (int)c->tab[id].size(); }


// One record against the tables and the scenario length: its reduced model
// (Section 3.6.4), steps and boundary; on failure the message goes to msg.
rsv_status prep_one(const rsv_ctx* c, int64_t i, int horizon, int max_steps, PolPrep& q, int& need, int& n_tab,
                    char (&msg)[160]) {
    const rsv_policy& r = c->pols[i];
    ProductModel pm;
    if (!product_model(r.product, pm) || r.reserved != 0) {
        snprintf(msg, sizeof msg, "policy %lld: bad product %d", (long long)i, r.product);
        return RSV_E_ARG;
    }
    const bool two = pm.two_life;
    if (r.table1 < 0 || r.table1 >= kMaxTables || c->tab[r.table1].empty() ||
        (two && (r.table2 < 0 || r.table2 >= kMaxTables || c->tab[r.table2].empty()))) {
        snprintf(msg, sizeof msg, "policy %lld: decrement table not loaded", (long long)i);
        return RSV_E_ARG;
    }
    if (r.age1_m < 0 || (two && r.age2_m < 0) || r.term_m < 0) {
        snprintf(msg, sizeof msg, "policy %lld: negative age or term", (long long)i);
        return RSV_E_ARG;
    }
    if (r.state0 < 0 || r.state0 > (pm.multi_state ? 2 : 0)) {
        snprintf(msg, sizeof msg, "policy %lld: bad state0 %d", (long long)i, r.state0);
        return RSV_E_ARG;
    }
    if (!std::isfinite(r.amount)) {
        snprintf(msg, sizeof msg, "policy %lld: amount not finite", (long long)i);
        return RSV_E_ASSUMPTION;
    }
    if (r.product == RSV_JL_REVERSIONARY && !(r.reversion >= 0.0 && r.reversion <= 1.0)) {
        snprintf(msg, sizeof msg, "policy %lld: reversion outside [0,1]", (long long)i);
        return RSV_E_ASSUMPTION;
    }
    int S = product_steps(r, table_len(c, r.table1), two ? table_len(c, r.table2) : 0);
    float bnd = pm.bnd;
    if (horizon > 0 && horizon < S) {
        S = horizon;
        bnd = 0.0f;   // truncated projection: r_horizon = 0
    }
    if (S > max_steps) {
        snprintf(msg, sizeof msg, "policy %lld: %d steps but scenarios have %d", (long long)i, S, max_steps);
        return RSV_E_ASSUMPTION;
    }
    const int top = std::max(r.age1_m + S, two ? r.age2_m + S : 0);
    if (top > kMaxAgeSteps) {
        snprintf(msg, sizeof msg, "policy %lld: age + steps %d exceeds %d", (long long)i, top, kMaxAgeSteps);
        return RSV_E_ARG;
    }
    need = std::max(need, top);
    n_tab = std::max(n_tab, std::max(r.table1, two ? r.table2 : 0) + 1);
    q.kind = pm.kind;
    q.S = S;
    q.idx_age1 = r.age1_m;
    q.idx_age2 = two ? r.age2_m : 0;
    q.table1 = r.table1;
    q.table2 = two ? r.table2 : 0;
    q.state0 = r.state0;
    q.pol = (int)i;
    q.bnd = bnd;
    q.rho = r.product == RSV_JL_REVERSIONARY ? r.reversion : (r.product == RSV_LAST_SURVIVOR ? 1.0 : 0.0);
    return RSV_OK;
}

// Validate every record and derive its reduced model, steps and boundary,
// on several host threads for large portfolios.  The error reported is the
// first bad record in portfolio order.
rsv_status prep_policies(rsv_ctx* c, int horizon, int max_steps, std::vector<PolPrep>& out, int& tab_pad,
                         int& n_tab, double& chain_steps) {
    const int64_t n = (int64_t)c->pols.size();
    out.resize(n);
    struct Part {
        int need = 1, n_tab = 1;
        double steps = 0.0;
        int64_t bad = -1;
        rsv_status st = RSV_OK;
        char msg[160] = {0};
    };
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(hw, 16), n / 16384));
    std::vector<Part> part(T);
    auto run = [&](int k) {
        Part& pr = part[k];
        const int64_t lo = n * k / T, hi = n * (k + 1) / T;
        for (int64_t i = lo; i < hi; ++i) {
            const rsv_status st = prep_one(c, i, horizon, max_steps, out[i], pr.need, pr.n_tab, pr.msg);
            if (st != RSV_OK) {
                pr.st = st;
                pr.bad = i;
                return;
            }
            pr.steps += out[i].S;
        }
    };
    run_parts(T, run);
    int need = 1;
    n_tab = 1;
    chain_steps = 0;
    for (const Part& pr : part) {   // parts in portfolio order: the first failure is the earliest record
        if (pr.st != RSV_OK) return fail(c, pr.st, "%s", pr.msg);
        need = std::max(need, pr.need);
        n_tab = std::max(n_tab, pr.n_tab);
        chain_steps += pr.steps;
    }
    for (int t = 0; t < n_tab; ++t) need = std::max(need, table_len(c, t));
    tab_pad = (need + 31) / 32 * 32;
    return RSV_OK;
}

}  // namespace

rsv_status rsv::build_layout(rsv_ctx* c, int P, int horizon, int max_steps, int P_general) {
    Layout& L = c->lay;
    // the general group exists only while cash flows are loaded for this portfolio
    const bool split = P_general > 0 && c->cf_pol > 0 && c->cf_pol == (int64_t)c->pols.size();
    if (!split) P_general = 0;
    const unsigned long long gen = c->pol_gen * 1000003ull + c->tab_gen * 7919ull + (unsigned)max_steps +
                                   (split ? c->cf_gen * 104729ull : 0ull);
    if (L.P == P && L.P_general == P_general && L.horizon == horizon && L.gen == gen) return RSV_OK;
    // host scratch kept across rebuilds: no allocation or first-touch cost per call
    std::vector<PolPrep>& pp = L.h_pp;
    int tab_pad, n_tab;
    double cs;
    rsv_status st = prep_policies(c, horizon, max_steps, pp, tab_pad, n_tab, cs);
    if (st != RSV_OK) return st;
    auto group = [&](const PolPrep& q) { return split && !c->cf_level[q.pol] ? 1 : 0; };

    // group by (cash-flow group, reduced model), longest projection first:
    // three-state tiles, then joint and single-life annuities, then assurances
    static const int kind_rank[6] = {3, 5, 0, 2, 4, 1};   // by kind
    static const int rank_kind[6] = {K_JL, K_LS2, K_ANN2, K_ANN, K_ASS2, K_ASS};
    // stable counting sort on the key: S <= kMaxAgeSteps
    const int span = kMaxAgeSteps + 1, per_group = 6 * span;
    const int nb = 2 * per_group;
    std::vector<int>& bucket_start = L.h_bucket;
    std::vector<int>& order = L.h_order;
    bucket_start.assign(nb + 1, 0);
    order.resize(pp.size());
    auto key = [&](const PolPrep& q) {
        return group(q) * per_group + kind_rank[q.kind] * span + (kMaxAgeSteps - q.S);
    };
    // in parallel for large portfolios: each part counts its contiguous range,
    // the parts' starts per bucket follow part order, and each part scatters
    // its range in order, so the sort stays stable
    const int64_t n_pp = (int64_t)pp.size();
    const int hw_s = (int)std::max(1u, std::thread::hardware_concurrency());
    const int TS = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(hw_s, 16), n_pp / 65536));
    std::vector<int>& cnt = L.h_cnt;
    cnt.assign((size_t)TS * nb, 0);
    run_parts(TS, [&](int k) {
        int* h = cnt.data() + (size_t)k * nb;
        for (int64_t i = n_pp * k / TS, e = n_pp * (k + 1) / TS; i < e; ++i) ++h[key(pp[i])];
    });
    for (int b = 0, run = 0; b < nb; ++b) {
        bucket_start[b] = run;
        for (int k = 0; k < TS; ++k) {
            const int v = cnt[(size_t)k * nb + b];
            cnt[(size_t)k * nb + b] = run;
            run += v;
        }
        bucket_start[b + 1] = run;
    }
    int run_lo[12], run_hi[12];   // sorted ranges of the (group, kind rank) runs
    for (int r = 0; r < 12; ++r) {
        run_lo[r] = bucket_start[r * span];
        run_hi[r] = bucket_start[(r + 1) * span];
    }
    run_parts(TS, [&](int k) {
        int* h = cnt.data() + (size_t)k * nb;
        for (int64_t i = n_pp * k / TS, e = n_pp * (k + 1) / TS; i < e; ++i) order[h[key(pp[i])]++] = (int)i;
    });

    // Tiles: each run is cut into tiles of Pg policies (the last one padded).
    // A tile's cost is its model's weight times the S of its first, longest
    // policy.
    std::vector<int>& t_start = L.h_first;
    std::vector<int>& kinds = L.h_kinds;
    std::vector<int>& grps = L.h_grps;
    std::vector<double>& cost = L.h_cost;
    t_start.clear();
    kinds.clear();
    grps.clear();
    cost.clear();
    int run_t0[13];               // first tile of each run
    for (int r = 0; r < 12; ++r) {
        run_t0[r] = (int)kinds.size();
        const int g = r / 6, kind = rank_kind[r % 6], Pg = g ? P_general : P;
        if (run_hi[r] > run_lo[r] && Pg <= 0) return fail(c, RSV_E_ARG, "internal: empty tile width");
        const double w = kind == K_JL ? 3.0 : (kind == K_LS2 ? 4.0 : (kind == K_ANN2 || kind == K_ASS2 ? 1.4 : 1.0));
        for (int st0 = run_lo[r]; st0 < run_hi[r]; st0 += Pg) {
            t_start.push_back(st0);
            kinds.push_back(kind);
            grps.push_back(g);
            cost.push_back(w * pp[order[st0]].S);
        }
    }
    run_t0[12] = (int)kinds.size();
    const int n_tiles = (int)kinds.size();

    // tiles in decreasing cost order within each group (longest-processing-time
    // first): the tiles of each run are already in decreasing cost, so merge
    // the runs (ties keep creation order)
    std::vector<int>& to = L.h_to;
    to.clear();
    to.reserve(n_tiles);
    int grp_tiles[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
        int head[6], end[6];
        for (int r = 0; r < 6; ++r) {
            head[r] = run_t0[g * 6 + r];
            end[r] = run_t0[g * 6 + r + 1];
        }
        const int cnt = run_t0[g * 6 + 6] - run_t0[g * 6];
        for (int out = 0; out < cnt; ++out) {
            int best = -1;
            for (int r = 0; r < 6; ++r)
                if (head[r] < end[r] && (best < 0 || cost[head[r]] > cost[head[best]])) best = r;
            to.push_back(head[best]++);
        }
        grp_tiles[g] = cnt;
    }

    // the slots, written in their final places (several host threads for
    // large portfolios): policy records gathered in sorted order, padding
    // slots repeating the last policy of their tile with pol = -1
    std::vector<SlotRec>& s2 = L.h_s2;
    std::vector<int>& k2 = L.h_k2;
    const size_t n_slots = (size_t)grp_tiles[0] * P + (size_t)grp_tiles[1] * (P_general > 0 ? P_general : 0);
    s2.resize(n_slots);
    k2.resize(n_tiles);
    auto fill = [&](int f0, int f1) {
        for (int f = f0; f < f1; ++f) {
            const int src = to[f], g = grps[src], Pg = g ? P_general : P;
            const size_t o = f < grp_tiles[0] ? (size_t)f * P
                                                : (size_t)grp_tiles[0] * P + (size_t)(f - grp_tiles[0]) * P_general;
            const int r = (g ? 6 : 0) + kind_rank[kinds[src]];
            const int st0 = t_start[src], len = std::min(Pg, run_hi[r] - st0);
            k2[f] = kinds[src];
            for (int k = 0; k < Pg; ++k) {
                SlotRec sl;
                if (k < len) {
                    const PolPrep& q = pp[order[st0 + k]];
                    sl.idx1 = q.table1 * tab_pad + q.idx_age1;
                    sl.idx2 = q.table2 * tab_pad + q.idx_age2;
                    sl.S = q.S;
                    sl.pol = q.pol;
                    sl.rho_h = (float)q.rho;
                    sl.rho_l = (float)(q.rho - (double)sl.rho_h);
                    sl.state0 = q.state0;
                    sl.bnd = q.bnd;
                } else {
                    sl = s2[o + k - 1];   // padding: same shape, never written out
                    sl.pol = -1;
                }
                s2[o + k] = sl;
            }
        }
    };
    {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        // by slots, not tiles: wide tiles (the deflated form's 60 policies) are few
        const int T = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::min(hw, 16), n_slots / 16384));
        run_parts(T, [&](int k) {
            fill((int)((long long)n_tiles * k / T), (int)((long long)n_tiles * (k + 1) / T));
        });
    }
    L.dev_ok = false;
    L.P = P;
    L.P_general = P_general;
    L.horizon = horizon;
    L.gen = gen;
    L.n_tiles = n_tiles;
    L.grp_tiles[0] = grp_tiles[0];
    L.grp_tiles[1] = grp_tiles[1];
    L.grp_slot0[0] = 0;
    L.grp_slot0[1] = (size_t)grp_tiles[0] * P;
    L.tab_pad = tab_pad;
    L.n_tab = n_tab;
    L.chain_steps = cs;
    L.max_S = 0;
    L.has_two = false;
    L.grp_two[0] = L.grp_two[1] = false;
    {
        struct Scan {
            int max_S = 0;
            bool two[2] = {false, false};
        };
        std::vector<Scan> sc(TS);
        run_parts(TS, [&](int k) {
            Scan& r = sc[k];
            for (int64_t i = n_pp * k / TS, e = n_pp * (k + 1) / TS; i < e; ++i) {
                const PolPrep& q = pp[i];
                r.max_S = std::max(r.max_S, q.S);
                if (q.kind == K_ANN2 || q.kind == K_ASS2 || q.kind == K_LS2) r.two[group(q)] = true;
            }
        });
        for (const Scan& r : sc) {
            L.max_S = std::max(L.max_S, r.max_S);
            L.grp_two[0] |= r.two[0];
            L.grp_two[1] |= r.two[1];
        }
        L.has_two = L.grp_two[0] || L.grp_two[1];
    }
    return RSV_OK;
}

rsv_status rsv::layout_to_device(rsv_ctx* c) {
    Layout& L = c->lay;
    if (L.dev_ok) return RSV_OK;
    CU(L.slots.ensure(std::max<size_t>(1, L.h_s2.size()) * sizeof(SlotRec)));
    CU(L.kinds.ensure(std::max<size_t>(1, L.h_k2.size()) * sizeof(int)));
    if (L.n_tiles) {
        // pageable sources: each copy is staged before the call returns
        CU(cudaMemcpyAsync(L.slots.p, L.h_s2.data(), L.h_s2.size() * sizeof(SlotRec), cudaMemcpyHostToDevice,
                           c->stream));
        CU(cudaMemcpyAsync(L.kinds.p, L.h_k2.data(), L.h_k2.size() * sizeof(int), cudaMemcpyHostToDevice,
                           c->stream));
    }
    L.dev_ok = true;
    return RSV_OK;
}

namespace {
// Entries (p, q) of tables src[0..n_tab) in the format of `form`, pad entries
// per table, zero survival past each table's end.
void write_entries(int form, const std::vector<double>* src, int n_tab, int pad, unsigned char* h) {
    for (int t = 0; t < n_tab; ++t) {
        for (int k = 0; k < pad; ++k) {
            const double p = k < (int)src[t].size() ? src[t][k] : 0.0;
            const double q = 1.0 - p;
            const size_t i = (size_t)t * pad + k;
            if (form == F_F64) {
                reinterpret_cast<double2*>(h)[i] = make_double2(p, q);
            } else if (form == F_F32) {
                reinterpret_cast<float2*>(h)[i] = make_float2((float)p, (float)q);
            } else {
                const float ph = (float)p, qh = (float)q;
                reinterpret_cast<float4*>(h)[i] = make_float4(ph, (float)(p - (double)ph), qh, (float)(q - (double)qh));
            }
        }
    }
}
}  // namespace

// Decrement tables in the entry format of `form`, zero survival past each
// table's end, staged per CTA.
rsv_status rsv::fail_msg(rsv_ctx* c, rsv_status st, const char* msg) noexcept { return fail(c, st, "%s", msg); }

rsv_status rsv::build_tables(rsv_ctx* c, int form, size_t& smem) {
    return stage_tables(c, form, c->lay.tab_pad, c->lay.n_tab, smem);
}

rsv_status rsv::stage_tables(rsv_ctx* c, int form, int pad, int n_tab, size_t& smem) {
    const size_t esz = form == F_F32 ? sizeof(float2) : 16;
    smem = (size_t)n_tab * pad * esz;
    if (smem > kMaxSmem)
        return fail(c, RSV_E_ARG, "decrement tables need %zu bytes of shared memory (max %zu)", smem, kMaxSmem);
    if (c->tab_pad_of[form] == pad && c->n_tab_of[form] == n_tab && c->tab_gen_of[form] == c->tab_gen)
        return RSV_OK;
    std::vector<unsigned char> h(smem);
    write_entries(form, c->tab, n_tab, pad, h.data());
    CU(c->d_tab[form].ensure(smem));
    CU(cudaMemcpyAsync(c->d_tab[form].p, h.data(), smem, cudaMemcpyHostToDevice, c->stream));   // staged
    c->tab_pad_of[form] = pad;
    c->n_tab_of[form] = n_tab;
    c->tab_gen_of[form] = c->tab_gen;
    return RSV_OK;
}

rsv_status rsv::scenario_totals(rsv_ctx* c, const double* partial, int n_rows, int s_pad, int n_scen, double* tot) {
    const int G = 256, groups = (n_rows + G - 1) / G;
    CU(c->d_part2.ensure((size_t)groups * s_pad * sizeof(double)));
    dim3 g1((s_pad + 127) / 128, groups);
    reduce_tiles_kernel<<<g1, 128, 0, c->stream>>>(partial, n_rows, s_pad, G, c->d_part2.as<double>());
    CU(cudaGetLastError());
    reduce_groups_kernel<<<(n_scen + 127) / 128, 128, 0, c->stream>>>(c->d_part2.as<double>(), groups, s_pad, n_scen,
                                                                     tot);
    CU(cudaGetLastError());
    return RSV_OK;
}

// The tables followed by the fractional-survival tables (RSV_PAY_FRACTION),
// staged together; *tabf_off receives the offset in entries.
rsv_status build_tables_frac(rsv_ctx* c, int form, size_t& smem, int& tabf_off) {
    const int pad = c->lay.tab_pad, n_tab = c->lay.n_tab;
    for (int t = 0; t < n_tab; ++t)
        if (!c->tab[t].empty() && c->tabf[t].size() != c->tab[t].size())
            return fail(c, RSV_E_STATE, "table %d has no fractional-survival table of its length", t);
    const size_t esz = form == F_F32 ? sizeof(float2) : 16, half = (size_t)n_tab * pad * esz;
    smem = 2 * half;
    tabf_off = n_tab * pad;
    if (smem > kMaxSmem)
        return fail(c, RSV_E_ARG, "tables and fractional tables need %zu bytes of shared memory (max %zu)", smem,
                    kMaxSmem);
    const unsigned long long key = c->tab_gen * 1000003ull + c->tabf_gen * 7919ull + (unsigned)pad * 31u + n_tab;
    if (c->tabf_key[form] == key) return RSV_OK;
    std::vector<unsigned char> h(smem);
    write_entries(form, c->tab, n_tab, pad, h.data());
    write_entries(form, c->tabf, n_tab, pad, h.data() + half);
    CU(c->d_tabf[form].ensure(smem));
    CU(cudaMemcpyAsync(c->d_tabf[form].p, h.data(), smem, cudaMemcpyHostToDevice, c->stream));   // staged
    c->tabf_key[form] = key;
    return RSV_OK;
}

namespace {

rsv_status upload_amounts(rsv_ctx* c) {
    if (!c->amount_dirty) return RSV_OK;
    std::vector<double> a(c->pols.size());
    for (size_t i = 0; i < a.size(); ++i) a[i] = c->pols[i].amount;
    CU(c->d_amount.ensure(std::max<size_t>(1, a.size()) * sizeof(double)));
    if (!a.empty()) {
        CU(cudaMemcpyAsync(c->d_amount.p, a.data(), a.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    c->amount_dirty = false;
    return RSV_OK;
}

rsv_status compute(rsv_ctx* c, const rsv_opts* o, rsv_out* out) {
    if (!c) return RSV_E_ARG;
    if (!o || !out) return fail(c, RSV_E_ARG, "opts and out must not be NULL");
    if (o->form < F_F64 || o->form > F_DEFL) return fail(c, RSV_E_ARG, "bad form %d", o->form);
    if (o->horizon < 0 || (o->on_device != 0 && o->on_device != 1))
        return fail(c, RSV_E_ARG, "bad horizon or on_device");
    if (c->pols.empty() && c->n_scen == 0) return fail(c, RSV_E_STATE, "no portfolio and no scenarios loaded");
    if (c->n_scen == 0) return fail(c, RSV_E_STATE, "no scenarios loaded");
    bool any_tab = false;
    for (auto& t : c->tab) any_tab |= !t.empty();
    if (!any_tab) return fail(c, RSV_E_STATE, "no decrement table loaded");
    const int outs = o->outputs;
    if (outs & ~15) return fail(c, RSV_E_ARG, "bad outputs bits 0x%x", outs);
    if ((outs & RSV_OUT_V0) && !out->V0 && !out->V0d) return fail(c, RSV_E_ARG, "V0 requested but NULL");
    if ((outs & RSV_OUT_SCEN_TOTAL) && !out->scen_total) return fail(c, RSV_E_ARG, "scen_total NULL");
    if ((outs & RSV_OUT_PT_MEAN) && !out->pt_mean) return fail(c, RSV_E_ARG, "pt_mean NULL");
    if ((outs & RSV_OUT_TRAJ) && !out->traj) return fail(c, RSV_E_ARG, "traj NULL");
    if (o->form == F_DEFL) return compute_deflated(c, o, out);

    const int64_t n_pol = (int64_t)c->pols.size();
    const int T = c->n_steps, NSc = c->n_scen;
    const size_t n_v0 = (size_t)n_pol * NSc;
    const size_t n_pt = (size_t)n_pol * (T + 1);
    const size_t n_traj = n_pt * NSc;
    if ((outs & RSV_OUT_TRAJ) && n_traj * sizeof(double) > kMaxTraj)
        return fail(c, RSV_E_ARG, "trajectory output of %zu bytes exceeds 1 GiB", n_traj * sizeof(double));

    int nv = 0;
    const Variant* vl = variant_list(o->form, &nv);
    const bool extra = (outs & (RSV_OUT_PT_MEAN | RSV_OUT_TRAJ)) != 0;
    const bool scan = o->variant == RSV_VARIANT_TIME_SCAN, summ = o->variant == RSV_VARIANT_SUMMATION;
    if ((scan || summ) && o->form != F_F64) return fail(c, RSV_E_ARG, "the %s variant runs the FP64 form",
                                                        scan ? "time-scan" : "summation");
    if ((scan || summ) && (outs & RSV_OUT_PT_MEAN))
        return fail(c, RSV_E_ARG, "the %s variant has no per-step means", scan ? "time-scan" : "summation");
    const int pay = o->payment;
    if (pay < PAY_END || pay > PAY_FRACTION) return fail(c, RSV_E_ARG, "bad payment %d", pay);
    if (pay != PAY_END && (extra || scan || summ))
        return fail(c, RSV_E_ARG, "payment within the step: V0 and totals of the scenario-parallel kernels only");
    const bool cfl = c->cf_pol > 0;   // varying cash flows loaded
    if (cfl && c->cf_pol != n_pol)
        return fail(c, RSV_E_STATE, "cash flows loaded for %lld policies, portfolio has %lld", (long long)c->cf_pol,
                    (long long)n_pol);
    if (cfl && extra && !scan && !summ)
        return fail(c, RSV_E_ARG, "per-step outputs with varying cash flows: use the time-scan or summation variant");
    const int nt = tunable_count(vl, nv);
    // With cash flows loaded and f = 1, the policies whose sequence is level
    // keep the fast kernel (tile group 0) and the others take the
    // general-cash-flow kernel (group 1).
    const bool split = cfl && pay == PAY_END && !extra && !scan && !summ;
    int vi, vg = -1;
    if (extra || scan || summ) {
        vi = special_variant(vl, nv, true, PAY_END);
    } else if (pay != PAY_END) {
        vi = special_variant(vl, nv, false, pay);
    } else if (o->variant >= 0) {
        if (o->variant >= nt) return fail(c, RSV_E_ARG, "variant %d out of range", o->variant);
        vi = o->variant;
    } else if (o->variant == -1) {
        vi = c->tuned[o->form] >= 0 ? c->tuned[o->form] : 0;
    } else {
        return fail(c, RSV_E_ARG, "variant %d out of range", o->variant);
    }
    if (split) vg = special_variant(vl, nv, false, PAY_END_GENERAL);
    const Variant& V = vl[vi];

    rsv_status st = build_layout(c, (scan || summ) ? 1 : V.P, o->horizon, c->n_steps, split ? vl[vg].P : 0);
    if (st == RSV_OK) st = layout_to_device(c);
    if (st != RSV_OK) return st;
    if (cfl && c->lay.max_S > c->cf_steps)
        return fail(c, RSV_E_STATE, "a projection of %d steps is longer than the cash-flow rows (%d)", c->lay.max_S,
                    c->cf_steps);
    size_t smem = 0;
    int tabf_off = 0;
    if (pay == PAY_FRACTION) {
        if (c->vf_scen != c->n_scen || c->vf_steps != c->n_steps)
            return fail(c, RSV_E_STATE, "fractional discount factors not loaded for the scenario set's shape");
        if ((st = build_tables_frac(c, o->form, smem, tabf_off)) != RSV_OK) return st;
    } else if ((st = build_tables(c, o->form, smem)) != RSV_OK) {
        return st;
    }
    if ((st = upload_amounts(c)) != RSV_OK) return st;

    const Layout& L = c->lay;
    float* V0f = (outs & RSV_OUT_V0) ? out->V0 : nullptr;
    double* V0d = (outs & RSV_OUT_V0) ? out->V0d : nullptr;
    double* tot = (outs & RSV_OUT_SCEN_TOTAL) ? out->scen_total : nullptr;
    double* pt = (outs & RSV_OUT_PT_MEAN) ? out->pt_mean : nullptr;
    double* traj = (outs & RSV_OUT_TRAJ) ? out->traj : nullptr;
    float* hV0f = V0f;
    double *hV0d = V0d, *htot = tot, *hpt = pt, *htraj = traj;
    if (!o->on_device) {   // device staging of host outputs
        if (V0f) { CU(c->d_o_v0f.ensure(n_v0 * sizeof(float))); V0f = c->d_o_v0f.as<float>(); }
        if (V0d) { CU(c->d_o_v0d.ensure(n_v0 * sizeof(double))); V0d = c->d_o_v0d.as<double>(); }
        if (tot) { CU(c->d_o_tot.ensure(NSc * sizeof(double))); tot = c->d_o_tot.as<double>(); }
        if (pt) { CU(c->d_o_pt.ensure(n_pt * sizeof(double))); pt = c->d_o_pt.as<double>(); }
        if (traj) { CU(c->d_o_traj.ensure(n_traj * sizeof(double))); traj = c->d_o_traj.as<double>(); }
    }
    CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
    CU(cudaMemsetAsync(c->d_ctl.p, 0, 2 * sizeof(int32_t), c->stream));
    if (pt) CU(cudaMemsetAsync(pt, 0, n_pt * sizeof(double), c->stream));
    if (traj) CU(cudaMemsetAsync(traj, 0, n_traj * sizeof(double), c->stream));
    if (tot) CU(c->d_partial.ensure((size_t)std::max(1, L.n_tiles) * c->s_pad * sizeof(double)));
    if (tot && L.n_tiles == 0) CU(cudaMemsetAsync(tot, 0, NSc * sizeof(double), c->stream));

    RecurArgs a{};
    a.tab = pay == PAY_FRACTION ? c->d_tabf[o->form].p : c->d_tab[o->form].p;
    a.tabf_off = tabf_off;
    a.vf = pay != PAY_FRACTION ? nullptr
                               : (o->form == F_F64 ? c->d_vf64.p : (o->form == F_F32 ? c->d_vf32.p : c->d_vf2.p));
    a.tab_bytes = (int32_t)smem;
    a.v = o->form == F_F64 ? c->d_v64.p : (o->form == F_F32 ? c->d_v32.p : c->d_v2.p);
    a.s_pad = c->s_pad;
    a.n_scen = NSc;
    a.n_steps = T;
    a.slots = L.slots.as<SlotRec>();
    a.tile_kind = L.kinds.as<int32_t>();
    a.amount = c->d_amount.as<double>();
    a.n_tiles = L.n_tiles;
    // the scan: one chain per item; the summation: one block of 32 steps of a chain per item
    const int wpc = summ ? ((outs & RSV_OUT_TRAJ) ? (L.max_S + 1 + 31) / 32 : 1) : 1;
    a.n_chunks = (scan || summ) ? NSc : (NSc + 32 * V.M - 1) / (32 * V.M);
    const long long items = (long long)L.n_tiles * a.n_chunks * wpc;
    if (items > 0x7fffffffLL) return fail(c, RSV_E_ARG, "too many work items (%lld)", items);
    a.n_items = (int32_t)items;
    a.counter = c->d_ctl.as<int32_t>();
    a.status = c->d_ctl.as<int32_t>() + 1;
    a.V0f = V0f;
    a.V0d = V0d;
    a.partial = tot ? c->d_partial.as<double>() : nullptr;
    a.pt_sum = pt;
    a.traj = traj;
    a.v0_ld = NSc;
    a.cf = !cfl ? nullptr : (o->form == F_F64 ? c->d_cf64.p : c->d_cf32.p);
    a.cf_ld = c->cf_steps;
    // One launch per non-empty tile group on the scenario columns of `base`:
    // group 0 by V (with the cash flows unless they are split off), group 1
    // by the general-cash-flow variant; each with its own zeroed queue head.
    auto launch_groups = [&](const RecurArgs& base) -> rsv_status {
        for (int g = 0; g < 2; ++g) {
            const int n_t = L.grp_tiles[g];
            if (n_t == 0) continue;
            const Variant& VV = g ? vl[vg] : V;
            const int two = L.grp_two[g] ? 1 : 0;   // kernels compiled with the other two-life models
            RecurArgs b = base;
            b.slots = L.slots.as<SlotRec>() + L.grp_slot0[g];
            b.tile_kind = L.kinds.as<int32_t>() + (g ? L.grp_tiles[0] : 0);
            b.n_tiles = n_t;
            b.n_chunks = (b.n_scen + 32 * VV.M - 1) / (32 * VV.M);
            b.n_items = n_t * b.n_chunks;
            b.partial = base.partial ? base.partial + (size_t)(g ? L.grp_tiles[0] : 0) * c->s_pad : nullptr;
            b.cf = (split && g == 0) ? nullptr : base.cf;
            int bps = 0;
            CU(VV.occupancy[two](&bps, smem));
            if (bps < 1) return fail(c, RSV_E_CUDA, "variant %s cannot be resident with %zu B smem", VV.name, smem);
            long long grid = (long long)c->sm_count * bps;
            grid = std::max(1LL, std::min(grid, ((long long)b.n_items * 32 + VV.NT - 1) / VV.NT));
            CU(cudaMemsetAsync(c->d_ctl.p, 0, sizeof(int32_t), c->stream));
            CU(VV.launch[two](b, (int)grid, smem, c->stream));
        }
        return RSV_OK;
    };

    // Host V0 of the scenario-parallel kernels: computed in column blocks of
    // scenarios, each block's V0 copied to the host on a second stream while
    // the next block computes (the copy of the last block alone stays exposed).
    const bool pipelined = !o->on_device && ((hV0f != nullptr) != (hV0d != nullptr)) && !extra && !scan && !summ &&
                           L.n_tiles > 0 && NSc >= 256;
    bool copied_v0 = false;
    if (pipelined) {
        const int blocks = std::min(4, NSc / 128);
        const int width = ((NSc + blocks - 1) / blocks + 127) / 128 * 128;   // multiple of 128 scenario columns
        if (!c->copy_stream) CU(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->ev_block) CU(cudaEventCreateWithFlags(&c->ev_block, cudaEventDisableTiming));
        const size_t esz_v = o->form == F_F64 ? sizeof(double) : (o->form == F_F32 ? sizeof(float) : sizeof(float2));
        const size_t esz_o = hV0f ? sizeof(float) : sizeof(double);
        char* dV0 = hV0f ? reinterpret_cast<char*>(V0f) : reinterpret_cast<char*>(V0d);
        char* hV0 = hV0f ? reinterpret_cast<char*>(hV0f) : reinterpret_cast<char*>(hV0d);
        CU(cudaEventRecord(c->ev0, c->stream));
        for (int s0 = 0; s0 < NSc; s0 += width) {
            const int w = std::min(width, NSc - s0);
            RecurArgs b = a;
            b.v = static_cast<const char*>(a.v) + (size_t)s0 * esz_v;
            b.vf = a.vf ? static_cast<const char*>(a.vf) + (size_t)s0 * esz_v : nullptr;
            b.n_scen = w;
            b.V0f = a.V0f ? a.V0f + s0 : nullptr;
            b.V0d = a.V0d ? a.V0d + s0 : nullptr;
            b.partial = a.partial ? a.partial + s0 : nullptr;
            if ((st = launch_groups(b)) != RSV_OK) return st;
            CU(cudaEventRecord(c->ev_block, c->stream));
            CU(cudaStreamWaitEvent(c->copy_stream, c->ev_block, 0));
            CU(cudaMemcpy2DAsync(hV0 + (size_t)s0 * esz_o, (size_t)NSc * esz_o, dV0 + (size_t)s0 * esz_o,
                                 (size_t)NSc * esz_o, (size_t)w * esz_o, (size_t)n_pol, cudaMemcpyDeviceToHost,
                                 c->copy_stream));
        }
        CU(cudaEventRecord(c->ev1, c->stream));
        CU(cudaEventRecord(c->ev_block, c->copy_stream));
        CU(cudaStreamWaitEvent(c->stream, c->ev_block, 0));   // the call's stream sees the copies done
        copied_v0 = true;
        c->ev_recorded = true;
    }

    if (L.n_tiles > 0 && !pipelined) {
        if (scan || summ) {
            CU(cudaEventRecord(c->ev0, c->stream));
            if (scan) CU(launch_scan(a, c->sm_count, smem, c->stream));
            else CU(launch_summation(a, wpc, c->sm_count, smem, c->stream));
            CU(cudaEventRecord(c->ev1, c->stream));
        } else {
            CU(cudaEventRecord(c->ev0, c->stream));
            if ((st = launch_groups(a)) != RSV_OK) return st;
            CU(cudaEventRecord(c->ev1, c->stream));
        }
        c->ev_recorded = true;
    }
    if (L.n_tiles > 0) {
        if (tot && (st = scenario_totals(c, a.partial, L.n_tiles, c->s_pad, NSc, tot)) != RSV_OK) return st;
        if (pt) {
            scale_kernel<<<c->sm_count * 4, 256, 0, c->stream>>>(pt, n_pt, 1.0 / NSc);
            CU(cudaGetLastError());
        }
    }
    if (!o->on_device) {
        if (hV0f && !copied_v0) CU(cudaMemcpyAsync(hV0f, V0f, n_v0 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (hV0d && !copied_v0) CU(cudaMemcpyAsync(hV0d, V0d, n_v0 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (htot) CU(cudaMemcpyAsync(htot, tot, NSc * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (hpt) CU(cudaMemcpyAsync(hpt, pt, n_pt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (htraj) CU(cudaMemcpyAsync(htraj, traj, n_traj * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        return rsv_synchronize(c);
    }
    return RSV_OK;
}

// In-force weights amount x Pr[reduced state j at node n] (FP64), the
// remaining projection length per node, and the nested launch sequence.
rsv_status compute_nested(rsv_ctx* c, const rsv_opts* o, const rsv_nested_spec* sp, rsv_nested_out* out) {
    if (!o || !sp || !out) return fail(c, RSV_E_ARG, "opts, spec and out must not be NULL");
    if (o->form < F_F64 || o->form > F_DEFL) return fail(c, RSV_E_ARG, "bad form %d", o->form);
    if (o->outputs != 0 || o->horizon != 0 || o->payment != 0 || (o->on_device != 0 && o->on_device != 1))
        return fail(c, RSV_E_ARG, "nested runs take outputs = 0, horizon = 0, payment 0, on_device 0/1");
    if (c->cf_pol > 0) return fail(c, RSV_E_STATE, "nested runs value level cash flows: clear the loaded sequence");
    if (sp->n_outer < 1 || sp->n_nodes < 1 || sp->node_step_m < 1 || sp->n_inner < 1 || sp->n_inner > (1 << 20))
        return fail(c, RSV_E_ARG, "bad nested sizes");
    if ((long long)(sp->n_nodes - 1) * sp->node_step_m > kMaxAgeSteps)
        return fail(c, RSV_E_ARG, "last node beyond %d months", kMaxAgeSteps);
    if (sp->mode != RSV_NESTED_MC && sp->mode != RSV_NESTED_CURVE && sp->mode != RSV_NESTED_SURROGATE)
        return fail(c, RSV_E_ARG, "bad mode %d", sp->mode);
    if (sp->mode == RSV_NESTED_SURROGATE) {
        if (!c->sur.trained) return fail(c, RSV_E_STATE, "surrogate not trained");
        if (c->sur.a != sp->a || c->sur.b != sp->b || c->sur.sigma != sp->sigma)
            return fail(c, RSV_E_ARG, "the surrogate was trained for other Vasicek parameters");
    }
    if (!(sp->a > 0.0) || !(sp->sigma >= 0.0) || !std::isfinite(sp->a) || !std::isfinite(sp->b) ||
        !std::isfinite(sp->sigma) || !std::isfinite(sp->r0) || sp->batch_outer < 0)
        return fail(c, RSV_E_ARG, "bad Vasicek parameters");
    // the outer index keys 24 bits of the random streams' counters
    if (sp->outer_first < 0 || (long long)sp->outer_first + sp->n_outer > (1LL << 24))
        return fail(c, RSV_E_ARG, "outer paths outer_first .. outer_first + n_outer - 1 must lie in [0, 2^24)");
    if (!out->L_mean || !out->L_q995) return fail(c, RSV_E_ARG, "L_mean and L_q995 are required");
    bool any_tab = false;
    for (auto& t : c->tab) any_tab |= !t.empty();
    if (!any_tab) return fail(c, RSV_E_STATE, "no decrement table loaded");

    // The deflated form values the brute-force mode in deflated units; the
    // curve and surrogate modes run it compensated.
    const bool mc = sp->mode == RSV_NESTED_MC;
    const bool defl = o->form == F_DEFL && mc;
    const int form = o->form == F_DEFL && !mc ? F_COMP : o->form;
    const int P = defl ? kNestDeflP : nested_tile_width(form);
    rsv_status st = build_layout(c, P, 0, kMaxAgeSteps);
    if (st == RSV_OK) st = layout_to_device(c);
    if (st != RSV_OK) return st;
    size_t smem = 0;
    DeflTabs T;
    if (defl) {
        if ((st = defl_table_shape(c, c->lay, T)) != RSV_OK) return st;
        if ((st = defl_table_stage(c, T)) != RSV_OK) return st;
        smem = T.bytes;
    } else if ((st = build_tables(c, form, smem)) != RSV_OK) {
        return st;
    }
    const Layout& L = c->lay;
    const int n_pol = (int)c->pols.size(), NN = sp->n_nodes, NO = sp->n_outer, step = sp->node_step_m;
    const bool sur = sp->mode == RSV_NESTED_SURROGATE;
    const int n_inner = mc ? sp->n_inner : 1;
    const int i_pad = defl ? (n_inner + 63) / 64 * 64 : (n_inner + 31) / 32 * 32;

    // weights and remaining lengths
    std::vector<double> w((size_t)std::max(1, n_pol) * NN * 3, 0.0);
    std::vector<int> Ln(NN, 0), Sp(std::max(1, n_pol), 0);
    for (int p = 0; p < n_pol; ++p) {
        const rsv_policy& r = c->pols[p];
        ProductModel pm;
        product_model(r.product, pm);   // validated by build_layout
        const bool jl = pm.multi_state, two = pm.two_life, ann = pm.annuity;
        const int S = product_steps(r, table_len(c, r.table1), two ? table_len(c, r.table2) : 0);
        Sp[p] = S;
        const std::vector<double>& tx = c->tab[r.table1];
        const std::vector<double>& ty = c->tab[two ? r.table2 : r.table1];
        double Px = 1.0, Py = 1.0;
        int u = 0;
        for (int n = 0; n < NN; ++n) {
            const int m = n * step;
            for (; u < m; ++u) {
                Px *= (r.age1_m + u < (int)tx.size()) ? tx[r.age1_m + u] : 0.0;
                if (two) Py *= (r.age2_m + u < (int)ty.size()) ? ty[r.age2_m + u] : 0.0;
            }
            if (S < m || (ann && r.term_m > 0 && r.term_m <= m)) continue;   // ended before the node
            Ln[n] = std::max(Ln[n], S - m);
            double* wp = &w[((size_t)p * NN + n) * 3];
            if (!jl) {
                wp[0] = two ? r.amount * Px * Py : r.amount * Px;   // joint products: both alive
            } else if (r.state0 == 0) {
                wp[0] = r.amount * Px * Py;
                wp[1] = r.amount * Px * (1.0 - Py);
                wp[2] = r.amount * (1.0 - Px) * Py;
            } else if (r.state0 == 1) {
                wp[1] = r.amount * Px;
            } else {
                wp[2] = r.amount * Py;
            }
        }
    }
    const int Lmax = std::max(1, *std::max_element(Ln.begin(), Ln.end()));
    const int G4 = (Lmax + 3) / 4;   // the deflated planes' rows of four steps
    const size_t esz = form == F_F32 ? sizeof(float) : 8;
    const size_t per_outer = defl ? (size_t)NN * G4 * i_pad * sizeof(float4) : (size_t)NN * Lmax * i_pad * esz;
    int B = sp->batch_outer > 0 ? sp->batch_outer : (int)std::max<size_t>(1, (size_t(4) << 30) / per_outer);
    // the deflated brute force pipelines the generator of batch i + 1 with the
    // valuation of batch i: two plane buffers, and at least eight batches so
    // that the first and last stages are short
    if (defl && sp->batch_outer <= 0) B = std::max(1, std::min(B / 2, (NO + 7) / 8));
    B = std::min(B, NO);

    CU(c->d_nest_w.ensure(w.size() * sizeof(double)));
    CU(c->d_nest_ln.ensure(NN * sizeof(int)));
    CU(c->d_nest_rn.ensure((size_t)NO * NN * sizeof(double)));
    CU(c->d_nest_d0.ensure((size_t)NO * NN * sizeof(double)));
    const bool curve = sp->mode == RSV_NESTED_CURVE;
    const int o_pad = (NO + 31) / 32 * 32;   // the curve mode: outer paths on the lanes
    const size_t curve_plane = (size_t)NN * Lmax * o_pad * esz;
    if (curve) CU(c->d_nest_plane.ensure(curve_plane + (size_t)NN * NO * sizeof(double)));
    else if (!sur) CU(c->d_nest_plane.ensure((size_t)(defl ? 2 : 1) * B * per_outer));
    CU(c->d_nest_mean.ensure((size_t)NO * NN * sizeof(double)));
    CU(c->d_nest_kth.ensure((size_t)NO * NN * sizeof(double)));
    double* Lall = (o->on_device && out->L_all) ? out->L_all : nullptr;
    if (!Lall) {
        CU(c->d_nest_all.ensure((size_t)NO * NN * n_inner * sizeof(double)));
        Lall = c->d_nest_all.as<double>();
    }
    CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
    CU(cudaMemcpyAsync(c->d_nest_w.p, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_nest_ln.p, Ln.data(), NN * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemsetAsync(c->d_ctl.p, 0, 2 * sizeof(int32_t), c->stream));

    const VasStep vs = vasicek_step_constants(sp->a, sp->b, sp->sigma, 1.0 / 12.0);
    CU(cudaEventRecord(c->ev0, c->stream));
    CU(launch_outer_paths(vs, sp->seed, sp->outer_first, NO, NN, step, sp->r0, c->d_nest_rn.as<double>(), c->d_nest_d0.as<double>(),
                          c->stream));
    NestedArgs a{};
    a.tab = c->d_tab[form].p;
    a.tab_bytes = (int32_t)smem;
    a.v = c->d_nest_plane.p;
    a.i_pad = i_pad;
    a.n_inner = n_inner;
    a.Lmax = Lmax;
    a.n_nodes = NN;
    a.node_step = step;
    a.slots = L.slots.as<SlotRec>();
    a.tile_kind = L.kinds.as<int32_t>();
    a.n_tiles = L.n_tiles;
    a.wts = c->d_nest_w.as<double>();
    a.n_chunks = i_pad / 32;
    a.counter = c->d_ctl.as<int32_t>();
    a.status = c->d_ctl.as<int32_t>() + 1;
    a.L_all = Lall;
    if (sur) {
        // one query per in-force (policy, state) and (outer path, node), at the
        // node's rate; the lists depend on the node only and are expanded over
        // the outer paths on the device
        const size_t on_n = (size_t)NO * NN;
        std::vector<rsv_query> nq;
        std::vector<double> nw, nbase(NN, 0.0);
        std::vector<long long> noff(NN + 1, 0);
        for (int n = 0; n < NN; ++n) {
            noff[n] = (long long)nq.size();
            const int m = n * step;
            for (int p = 0; p < n_pol; ++p)
                for (int j = 0; j < 3; ++j) {
                    const double wj = w[((size_t)p * NN + n) * 3 + j];
                    if (wj == 0.0) continue;
                    if (Sp[p] == m) {   // matures at the node: its boundary value, no projection
                        ProductModel pm;
                        product_model(c->pols[p].product, pm);
                        nbase[n] += pm.bnd * wj;
                        continue;
                    }
                    nq.push_back(rsv_query{p, m, j, 0, 0.0});
                    nw.push_back(wj);
                }
        }
        noff[NN] = (long long)nq.size();
        const long long Qn = (long long)nq.size();
        // outer paths in batches of at most ~32M queries; device per batch:
        // [V | w | queries | seg | base], plus the node lists
        const int Bo = (int)std::max(1LL, std::min<long long>(NO, Qn > 0 ? (32LL << 20) / Qn : NO));
        const long long nq_b = Qn * Bo;
        const size_t on_b = (size_t)Bo * NN;
        const size_t bytes = (size_t)std::max<long long>(1, nq_b) * (16 + sizeof(rsv_query)) +
                             (size_t)std::max<long long>(1, Qn) * (sizeof(rsv_query) + 8) + (NN + 1) * 8 + NN * 8 +
                             (on_b + 1) * 8 + on_b * 8 + 64;
        CU(c->d_nest_plane.ensure(bytes));
        char* cur = static_cast<char*>(c->d_nest_plane.p);
        auto take = [&](size_t n) { char* r = cur; cur += (n + 7) / 8 * 8; return r; };
        double* dV = reinterpret_cast<double*>(take(std::max<long long>(1, nq_b) * 8));
        double* dw = reinterpret_cast<double*>(take(std::max<long long>(1, nq_b) * 8));
        rsv_query* dq = reinterpret_cast<rsv_query*>(take(std::max<long long>(1, nq_b) * sizeof(rsv_query)));
        rsv_query* dnq = reinterpret_cast<rsv_query*>(take(std::max<long long>(1, Qn) * sizeof(rsv_query)));
        double* dnw = reinterpret_cast<double*>(take(std::max<long long>(1, Qn) * 8));
        long long* dnoff = reinterpret_cast<long long*>(take((NN + 1) * 8));
        double* dnbase = reinterpret_cast<double*>(take(NN * 8));
        long long* dseg = reinterpret_cast<long long*>(take((on_b + 1) * 8));
        double* dbase = reinterpret_cast<double*>(take(on_b * 8));
        if (Qn > 0) {
            CU(cudaMemcpyAsync(dnq, nq.data(), Qn * sizeof(rsv_query), cudaMemcpyHostToDevice, c->stream));
            CU(cudaMemcpyAsync(dnw, nw.data(), Qn * 8, cudaMemcpyHostToDevice, c->stream));
        }
        CU(cudaMemcpyAsync(dnoff, noff.data(), (NN + 1) * 8, cudaMemcpyHostToDevice, c->stream));
        CU(cudaMemcpyAsync(dnbase, nbase.data(), NN * 8, cudaMemcpyHostToDevice, c->stream));
        long long nfb = 0;
        for (int o0 = 0; o0 < NO; o0 += Bo) {
            const int Bc = std::min(Bo, NO - o0);
            const size_t on_c = (size_t)Bc * NN;
            node_segments_kernel<<<(unsigned)((on_c + 256) / 256), 256, 0, c->stream>>>(dnoff, dnbase, Qn, Bc, NN,
                                                                                      dseg, dbase);
            CU(cudaGetLastError());
            if (Qn > 0) {
                expand_node_queries_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(
                    dnq, dnw, Qn, Bc, NN, step, c->d_nest_rn.as<double>() + (size_t)o0 * NN, dq, dw);
                CU(cudaGetLastError());
                long long nfb_c = 0;
                st = sur_value_queries(c, dq, Qn * Bc, dseg, (int)on_c, Lmax, dV, &nfb_c);
                if (st != RSV_OK) return st;
                nfb += nfb_c;
            }
            segment_wsum_kernel<<<(unsigned)on_c, 256, 0, c->stream>>>(dseg, dw, dV, dbase, Lall + (size_t)o0 * NN);
            CU(cudaGetLastError());
        }
        if (out->n_fallback) *out->n_fallback = nfb;
    }
    if (curve) {
        // one virtual outer path whose "inner paths" are the outer paths: every
        // lane carries a different outer path's curve, all sharing the weights
        double* Lt = reinterpret_cast<double*>(static_cast<char*>(c->d_nest_plane.p) + curve_plane);
        CU(launch_curve_planes_lanes(form, sp->a, sp->b, sp->sigma, NO, NN, o_pad, Lmax, c->d_nest_ln.as<int>(),
                                     c->d_nest_rn.as<double>(), c->d_nest_plane.p, c->sm_count, c->stream));
        NestedArgs ac = a;
        ac.i_pad = o_pad;
        ac.n_inner = NO;
        ac.n_chunks = o_pad / 32;
        ac.B = 1;
        ac.o0 = 0;
        ac.n_items = NN * ac.n_chunks;
        ac.L_all = Lt;
        CU(cudaMemsetAsync(c->d_ctl.p, 0, sizeof(int32_t), c->stream));
        if (L.n_tiles > 0) CU(launch_nested(form, ac, c->sm_count, smem, c->stream));
        else CU(cudaMemsetAsync(Lt, 0, (size_t)NN * NO * sizeof(double), c->stream));
        CU(launch_transpose_on(Lt, NO, NN, Lall, c->stream));
    }
    if (!sur && !curve && !c->nest_bm_ready) {   // the generator's tables: once per context (static host copy)
        CU(c->d_nest_bm.ensure((size_t)(BM_SC + BM_LG) * sizeof(double2)));
        CU(cudaMemcpyAsync(c->d_nest_bm.p, bm_tables_host(), (size_t)(BM_SC + BM_LG) * sizeof(double2),
                           cudaMemcpyHostToDevice, c->stream));
        c->nest_bm_ready = true;
    }
    NestDeflArgs da{};
    if (defl) {   // policy slots of the deflated tiles: runs, scales, boundary weights
        std::vector<NestSlot> ns(L.h_s2.size());
        for (int f = 0; f < L.n_tiles; ++f) {
            const int kind = L.h_k2[f];
            for (int k = 0; k < P; ++k) {
                const SlotRec& r = L.h_s2[(size_t)f * P + k];
                NestSlot d{};
                const int tb1 = r.idx1 / L.tab_pad, a1 = r.idx1 % L.tab_pad;
                const int tb2 = r.idx2 / L.tab_pad, a2 = r.idx2 % L.tab_pad;
                const int arr1 = kind == K_ASS ? T.arr_d : 0;
                d.base1 = (arr1 * T.n_tab + tb1) * T.dpad;   // float4 index of copy 0: 4 dpad floats per copy
                d.base2 = (0 * T.n_tab + tb2) * T.dpad;
                d.age1 = a1;
                d.age2 = a2;
                d.z1 = (int)c->tab[tb1].size() + (kind == K_ASS ? 1 : 0);
                d.z2 = (int)c->tab[tb2].size();
                d.S = r.S;
                d.pol = r.pol;
                d.kind = kind;
                auto ell_at = [&](int tb, int a) { return a < (int)T.ell[tb].size() ? T.ell[tb][a] : 0.0; };
                const double lx = ell_at(tb1, a1), ly = ell_at(tb2, a2);
                const double amount = r.pol >= 0 ? c->pols[r.pol].amount : 0.0;
                const double rho = (double)r.rho_h + (double)r.rho_l;
                double scale = 0.0;
                if (kind == K_ANN || kind == K_ASS) {
                    scale = lx > 0.0 ? amount / lx : 0.0;
                    if (kind == K_ASS && r.bnd != 0.0f) d.mat = (float)((double)r.bnd * ell_at(tb1, a1 + r.S));
                    if (kind == K_ASS && r.S == 0) {
                        scale = amount;
                        d.mat = r.bnd;
                    } else if (kind == K_ASS && !(lx > 0.0)) {
                        scale = amount;
                        d.mat = 0.0f;
                        d.unit = 1;
                    }
                } else {
                    scale = amount;
                    const double ix = lx > 0.0 ? 1.0 / lx : 0.0, iy = ly > 0.0 ? 1.0 / ly : 0.0;
                    if (kind == K_ANN2) {
                        d.ix = (float)ix;
                        d.iy = (float)iy;
                    } else {
                        d.ix = r.state0 == 2 ? 0.0f : (float)ix;
                        d.iy = r.state0 == 1 ? 0.0f : (float)(rho * iy);
                    }
                }
                d.sc_h = (float)scale;
                d.sc_l = (float)(scale - (double)d.sc_h);
                ns[(size_t)f * P + k] = d;
            }
        }
        CU(c->d_defl_slots.ensure(std::max<size_t>(1, ns.size()) * sizeof(NestSlot)));
        CU(c->d_defl_kinds.ensure(std::max<size_t>(1, L.h_k2.size()) * sizeof(int32_t)));
        if (!ns.empty()) {
            CU(cudaMemcpyAsync(c->d_defl_slots.p, ns.data(), ns.size() * sizeof(NestSlot), cudaMemcpyHostToDevice,
                               c->stream));
            CU(cudaMemcpyAsync(c->d_defl_kinds.p, L.h_k2.data(), L.h_k2.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
        }
        c->defl_lay_key = 0;   // the valuation's slot records were overwritten
        da.tab = c->d_defl_tab.as<float>();
        da.tab_bytes = (int32_t)T.bytes;
        da.dpad = T.dpad;
        da.D = c->d_nest_plane.as<float4>();
        da.i_pad = i_pad;
        da.n_inner = n_inner;
        da.G4 = G4;
        da.n_nodes = NN;
        da.node_step = step;
        da.slots = c->d_defl_slots.as<NestSlot>();
        da.tile_kind = c->d_defl_kinds.as<int32_t>();
        da.n_tiles = L.n_tiles;
        da.n_chunks = i_pad / 64;
        da.counter = c->d_ctl.as<int32_t>();
        da.status = c->d_ctl.as<int32_t>() + 1;
        da.L_all = Lall;
    }
    if (defl && !sur && !curve) {
        // generator (FP64 pipe) and valuation (FP32 pipes) of consecutive batches
        // run concurrently: the generator of batch i + 1 on a low-priority stream
        // into the other plane buffer, the valuation of batch i on a
        // high-priority stream at one CTA per SM, so that both fit on every SM
        if (!c->nest_val) {
            int lo = 0, hi = 0;
            CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CU(cudaStreamCreateWithPriority(&c->nest_val, cudaStreamNonBlocking, hi));
            CU(cudaStreamCreateWithPriority(&c->nest_gen, cudaStreamNonBlocking, lo));
            for (cudaEvent_t& e : c->nest_ev) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        cudaEvent_t ev_start = c->nest_ev[0], *ev_gen = c->nest_ev + 1, *ev_val = c->nest_ev + 3;
        CU(cudaEventRecord(ev_start, c->stream));   // the outer paths, weights and queue word are ready
        CU(cudaStreamWaitEvent(c->nest_gen, ev_start, 0));
        CU(cudaStreamWaitEvent(c->nest_val, ev_start, 0));
        const size_t buf4 = (size_t)B * per_outer / sizeof(float4);
        int i = 0;
        for (int o0 = 0; o0 < NO; o0 += B, ++i) {
            const int Bc = std::min(B, NO - o0), bi = i & 1;
            float4* plane = c->d_nest_plane.as<float4>() + bi * buf4;
            if (i >= 2) CU(cudaStreamWaitEvent(c->nest_gen, ev_val[bi], 0));   // the buffer's last reader
            CU(launch_inner_paths_defl(vs, sp->seed, sp->outer_first, o0, Bc, NN, n_inner, i_pad, G4, c->d_nest_ln.as<int>(),
                                       c->d_nest_rn.as<double>(), c->d_nest_bm.as<double2>(), plane, c->sm_count, 4,
                                       c->nest_gen));
            CU(cudaEventRecord(ev_gen[bi], c->nest_gen));
            CU(cudaStreamWaitEvent(c->nest_val, ev_gen[bi], 0));
            const long long items = (long long)NN * Bc * da.n_chunks;
            if (items > 0x7fffffffLL) return fail(c, RSV_E_ARG, "too many nested work items");
            da.D = plane;
            da.B = Bc;
            da.o0 = o0;
            da.n_items = (int32_t)items;
            CU(cudaMemsetAsync(c->d_ctl.p, 0, sizeof(int32_t), c->nest_val));
            if (L.n_tiles > 0) {
                CU(launch_nested_defl(da, c->sm_count, 1, c->nest_val));
            } else {
                CU(cudaMemsetAsync(Lall + (size_t)o0 * NN * n_inner, 0, (size_t)Bc * NN * n_inner * sizeof(double),
                                   c->nest_val));
            }
            CU(cudaEventRecord(ev_val[bi], c->nest_val));
        }
        // the call's stream continues once both pipelines are done
        CU(cudaEventRecord(ev_gen[0], c->nest_gen));
        CU(cudaStreamWaitEvent(c->stream, ev_gen[0], 0));
        CU(cudaEventRecord(ev_val[0], c->nest_val));
        CU(cudaStreamWaitEvent(c->stream, ev_val[0], 0));
    }
    for (int o0 = 0; o0 < NO && !sur && !curve && !defl; o0 += B) {
        const int Bc = std::min(B, NO - o0);
        CU(launch_inner_paths(form, vs, sp->seed, sp->outer_first, o0, Bc, NN, n_inner, i_pad, Lmax, c->d_nest_ln.as<int>(),
                              c->d_nest_rn.as<double>(), c->d_nest_bm.as<double2>(), c->d_nest_plane.p, c->sm_count,
                              c->stream));
        const long long items = (long long)NN * Bc * a.n_chunks;
        if (items > 0x7fffffffLL) return fail(c, RSV_E_ARG, "too many nested work items");
        a.B = Bc;
        a.o0 = o0;
        a.n_items = (int32_t)items;
        CU(cudaMemsetAsync(c->d_ctl.p, 0, sizeof(int32_t), c->stream));
        if (L.n_tiles > 0) {
            CU(launch_nested(form, a, c->sm_count, smem, c->stream));
        } else {
            CU(cudaMemsetAsync(Lall + (size_t)o0 * NN * n_inner, 0, (size_t)Bc * NN * n_inner * sizeof(double),
                               c->stream));
        }
    }
    const int k = mc ? std::max(1, (int)std::ceil(0.005 * n_inner - 1e-9)) : 1;
    CU(launch_node_stats(Lall, NO * NN, n_inner, k, c->d_nest_mean.as<double>(), c->d_nest_kth.as<double>(),
                         c->stream));
    CU(cudaEventRecord(c->ev1, c->stream));
    c->ev_recorded = true;

    const size_t on = (size_t)NO * NN;
    const cudaMemcpyKind kind = o->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CU(cudaMemcpyAsync(out->L_mean, c->d_nest_mean.p, on * sizeof(double), kind, c->stream));
    CU(cudaMemcpyAsync(out->L_q995, c->d_nest_kth.p, on * sizeof(double), kind, c->stream));
    if (out->r_node) CU(cudaMemcpyAsync(out->r_node, c->d_nest_rn.p, on * sizeof(double), kind, c->stream));
    if (out->D0) CU(cudaMemcpyAsync(out->D0, c->d_nest_d0.p, on * sizeof(double), kind, c->stream));
    if (out->L_all && Lall != out->L_all)
        CU(cudaMemcpyAsync(out->L_all, Lall, on * n_inner * sizeof(double), kind, c->stream));
    if (!o->on_device) return rsv_synchronize(c);
    return RSV_OK;
}

}  // namespace

extern "C" {

rsv_status rsv_create(rsv_ctx** out, int device, void* cuda_stream) try {
    if (!out) return RSV_E_ARG;
    *out = nullptr;
    rsv_ctx* c = new (std::nothrow) rsv_ctx();
    if (!c) return RSV_E_NOMEM;
    c->device = device;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) {
        delete c;
        return RSV_E_CUDA;
    }
    *out = c;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(nullptr);
}

rsv_status rsv_destroy(rsv_ctx* c) try {
    if (!c) return RSV_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (DevBuf* b : {&c->d_amount, &c->d_vstage, &c->d_v64, &c->d_v32, &c->d_v2, &c->d_tab[0], &c->d_tab[1],
                      &c->d_tab[2], &c->lay.slots, &c->lay.kinds, &c->d_ctl, &c->d_partial, &c->d_part2,
                      &c->d_o_v0f, &c->d_o_v0d, &c->d_o_tot, &c->d_o_pt, &c->d_o_traj, &c->d_nest_w,
                      &c->d_nest_ln, &c->d_nest_rn, &c->d_nest_d0, &c->d_nest_plane, &c->d_nest_mean,
                      &c->d_nest_kth, &c->d_nest_all, &c->d_pols, &c->sur.d_flag, &c->sur.d_q, &c->sur.d_lab,
                      &c->sur.d_y, &c->sur.d_X, &c->sur.d_pred, &c->sur.d_err, &c->sur.d_aux, &c->sur.d_curve,
                      &c->sur.d_comm, &c->sur.d_lnb, &c->d_tabf[0], &c->d_tabf[1], &c->d_tabf[2], &c->d_vf64,
                      &c->d_vf32, &c->d_vf2, &c->d_cf64, &c->d_cf32, &c->d_ml_rec,
                      &c->d_ml_amount, &c->sur.d_cnt, &c->sur.d_q2, &c->sur.d_idx, &c->sur.d_v2, &c->d_nest_bm,
                      &c->d_defl_slots, &c->d_defl_kinds, &c->d_defl_tab, &c->d_defl_plane, &c->d_mlp_trace})
        b->release();
    c->mlp.release();
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    c->h_defl_stage.release();
    for (cudaEvent_t& e : c->nest_ev)
        if (e) cudaEventDestroy(e);
    if (c->nest_val) cudaStreamDestroy(c->nest_val);
    if (c->nest_gen) cudaStreamDestroy(c->nest_gen);
    if (c->ev_block) cudaEventDestroy(c->ev_block);
    if (c->copy_stream) {
        cudaStreamSynchronize(c->copy_stream);
        cudaStreamDestroy(c->copy_stream);
    }
    delete c;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_set_stream(rsv_ctx* c, void* cuda_stream) try {
    if (!c) return RSV_E_ARG;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_load_decrements(rsv_ctx* c, int32_t table_id, const double* p, int32_t n) try {
    if (!c) return RSV_E_ARG;
    if (table_id < 0 || table_id >= kMaxTables) return fail(c, RSV_E_ARG, "table id %d outside [0,8)", table_id);
    if (!p || n < 1 || n > kMaxAgeSteps) return fail(c, RSV_E_ARG, "bad table pointer or length %d", n);
    for (int k = 0; k < n; ++k)
        if (!(p[k] >= 0.0 && p[k] <= 1.0))
            return fail(c, RSV_E_ASSUMPTION, "table %d entry %d = %g is not a probability", table_id, k, p[k]);
    c->tab[table_id].assign(p, p + n);
    ++c->tab_gen;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_load_decrements_fraction(rsv_ctx* c, int32_t table_id, const double* p, int32_t n) try {
    if (!c) return RSV_E_ARG;
    if (table_id < 0 || table_id >= kMaxTables) return fail(c, RSV_E_ARG, "table id %d outside [0,8)", table_id);
    if (!p || n < 1 || n > kMaxAgeSteps) return fail(c, RSV_E_ARG, "bad table pointer or length %d", n);
    for (int k = 0; k < n; ++k)
        if (!(p[k] >= 0.0 && p[k] <= 1.0))
            return fail(c, RSV_E_ASSUMPTION, "fractional table %d entry %d = %g is not a probability", table_id, k,
                        p[k]);
    c->tabf[table_id].assign(p, p + n);
    ++c->tabf_gen;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_load_scenarios_fraction(rsv_ctx* c, const double* v, int32_t n_scen, int32_t n_steps, int32_t layout) try {
    if (!c) return RSV_E_ARG;
    if (!v || n_scen < 1 || n_steps < 1 || (layout != 0 && layout != 1))
        return fail(c, RSV_E_ARG, "bad fractional scenario arguments");
    const size_t n = (size_t)n_scen * n_steps;
    for (size_t i = 0; i < n; ++i)
        if (!(std::isfinite(v[i]) && v[i] > 0.0))
            return fail(c, RSV_E_ASSUMPTION, "fractional discount factor %zu = %g is not finite and positive", i, v[i]);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    const int s_pad = (n_scen + 127) / 128 * 128;
    const size_t np = (size_t)n_steps * s_pad;
    CU(c->d_vstage.ensure(n * sizeof(double)));
    CU(c->d_vf64.ensure(np * sizeof(double)));
    CU(c->d_vf32.ensure(np * sizeof(float)));
    CU(c->d_vf2.ensure(np * sizeof(float2)));
    CU(cudaMemcpyAsync(c->d_vstage.p, v, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    split_planes_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->d_vstage.as<double>(), layout, n_scen, n_steps,
                                                                s_pad, c->d_vf64.as<double>(), c->d_vf32.as<float>(),
                                                                c->d_vf2.as<float2>());
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));
    c->vf_scen = n_scen;
    c->vf_steps = n_steps;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

// The level flags of freshly written rows (device FP64) and the new generation.
static rsv_status finish_cashflows(rsv_ctx* c, int64_t n_pol, int32_t n_steps) {
    CU(c->d_vstage.ensure((size_t)n_pol));
    cf_level_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->d_cf64.as<double>(), n_pol, n_steps,
                                                            c->d_vstage.as<unsigned char>());
    CU(cudaGetLastError());
    c->cf_level.resize((size_t)n_pol);
    CU(cudaMemcpyAsync(c->cf_level.data(), c->d_vstage.p, (size_t)n_pol, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    c->cf_pol = n_pol;
    c->cf_steps = n_steps;
    ++c->cf_gen;
    return RSV_OK;
}

rsv_status rsv_load_cashflows(rsv_ctx* c, const double* cf, int64_t n_pol, int32_t n_steps) try {
    if (!c) return RSV_E_ARG;
    if (!cf || n_pol < 1 || n_steps < 1 || n_pol * (int64_t)n_steps > 0x7fffffffLL)
        return fail(c, RSV_E_ARG, "bad cash-flow arguments");
    const size_t n = (size_t)n_pol * n_steps;
    for (size_t i = 0; i < n; ++i)
        if (!(std::isfinite(cf[i]) && cf[i] >= 0.0))
            return fail(c, RSV_E_ASSUMPTION, "cash-flow multiplier %zu = %g is not finite and non-negative", i, cf[i]);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    c->cf_pol = 0;
    CU(c->d_cf64.ensure(n * sizeof(double)));
    CU(c->d_cf32.ensure(n * sizeof(float)));
    CU(cudaMemcpyAsync(c->d_cf64.p, cf, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    cf_to_f32_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->d_cf64.as<double>(), c->d_cf32.as<float>(), n);
    CU(cudaGetLastError());
    return finish_cashflows(c, n_pol, n_steps);
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_load_schedules(rsv_ctx* c, const rsv_schedule* sch, int64_t n_pol, int32_t n_steps) try {
    if (!c) return RSV_E_ARG;
    if (!sch || n_pol < 1 || n_steps < 1 || n_pol * (int64_t)n_steps > 0x7fffffffLL)
        return fail(c, RSV_E_ARG, "bad schedule arguments");
    for (int64_t p = 0; p < n_pol; ++p) {
        const rsv_schedule& s = sch[p];
        if (s.every < 1 || s.first < 0 || s.steps_per_year < 1 || s.since < 0 || s.since >= s.steps_per_year ||
            !(std::isfinite(s.escalation) && s.escalation > -1.0) || !(std::isfinite(s.increase) && s.increase >= 0.0))
            return fail(c, RSV_E_ARG, "schedule %lld has a parameter out of range", (long long)p);
    }
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    const size_t n = (size_t)n_pol * n_steps;
    c->cf_pol = 0;
    CU(c->d_vstage.ensure((size_t)n_pol * sizeof(rsv_schedule)));
    CU(c->d_cf64.ensure(n * sizeof(double)));
    CU(c->d_cf32.ensure(n * sizeof(float)));
    CU(cudaMemcpyAsync(c->d_vstage.p, sch, (size_t)n_pol * sizeof(rsv_schedule), cudaMemcpyHostToDevice, c->stream));
    schedule_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->d_vstage.as<rsv_schedule>(), n_pol, n_steps,
                                                            c->d_cf64.as<double>(), c->d_cf32.as<float>());
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));   // the staged schedules are read before d_vstage is reused
    return finish_cashflows(c, n_pol, n_steps);
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_clear_cashflows(rsv_ctx* c) try {
    if (!c) return RSV_E_ARG;
    c->cf_pol = 0;
    c->cf_steps = 0;
    c->cf_level.clear();
    ++c->cf_gen;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_load_portfolio(rsv_ctx* c, const rsv_policy* pols, int64_t n) try {
    if (!c) return RSV_E_ARG;
    if (n < 0 || n > 0x7fffffffLL || (n > 0 && !pols)) return fail(c, RSV_E_ARG, "bad portfolio size %lld", (long long)n);
    // copied by several host threads for large portfolios (no zero fill first)
    c->pols.resize((size_t)n);
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(hw, 16), n / 65536));
    run_parts(T, [&](int k) {
        const int64_t lo = n * k / T, hi = n * (k + 1) / T;
        if (hi > lo) memcpy(c->pols.data() + lo, pols + lo, (size_t)(hi - lo) * sizeof(rsv_policy));
    });
    ++c->pol_gen;
    c->amount_dirty = true;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_load_scenarios(rsv_ctx* c, const double* v, int32_t n_scen, int32_t n_steps, int32_t layout) try {
    if (!c) return RSV_E_ARG;
    if (!v || n_scen < 1 || n_steps < 1 || (layout != 0 && layout != 1))
        return fail(c, RSV_E_ARG, "bad scenario arguments");
    const size_t n = (size_t)n_scen * n_steps;
    for (size_t i = 0; i < n; ++i)
        if (!(std::isfinite(v[i]) && v[i] > 0.0))
            return fail(c, RSV_E_ASSUMPTION, "discount factor %zu = %g is not finite and positive", i, v[i]);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    const int s_pad = (n_scen + 127) / 128 * 128;
    const size_t np = (size_t)n_steps * s_pad;
    CU(c->d_vstage.ensure(n * sizeof(double)));
    CU(c->d_v64.ensure(np * sizeof(double)));
    CU(c->d_v32.ensure(np * sizeof(float)));
    CU(c->d_v2.ensure(np * sizeof(float2)));
    CU(cudaMemcpyAsync(c->d_vstage.p, v, n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    split_planes_kernel<<<c->sm_count * 8, 256, 0, c->stream>>>(c->d_vstage.as<double>(), layout, n_scen, n_steps,
                                                                s_pad, c->d_v64.as<double>(), c->d_v32.as<float>(),
                                                                c->d_v2.as<float2>());
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));
    c->n_scen = n_scen;
    c->n_steps = n_steps;
    c->s_pad = s_pad;
    c->lay.gen = ~0ull;   // scenario length changes validation
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_compute_reserves(rsv_ctx* c, const rsv_opts* o, rsv_out* out) try {
    if (!c) return RSV_E_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return compute(c, o, out);
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_compute_nested(rsv_ctx* c, const rsv_opts* o, const rsv_nested_spec* sp, rsv_nested_out* out) try {
    if (!c) return RSV_E_ARG;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return compute_nested(c, o, sp, out);
} catch (...) {
    return rsv::host_error(c);
}

int32_t rsv_variant_count(int32_t form) {
    int n = 0;
    if (form == F_DEFL) return variants_defl(&n) ? n : 0;
    const Variant* vl = variant_list(form, &n);
    return vl ? tunable_count(vl, n) : 0;
}

const char* rsv_variant_name(int32_t form, int32_t variant) {
    int n = 0;
    if (form == F_DEFL) {
        const DeflVariant* dv = variants_defl(&n);
        return (variant < 0 || variant >= n) ? "" : dv[variant].name;
    }
    const Variant* v = variant_list(form, &n);
    if (!v || variant < 0 || variant >= n) return "";
    return v[variant].name;
}

rsv_status rsv_tune(rsv_ctx* c, const rsv_opts* opts, int32_t reps, int32_t* best, float* ms_out) try {
    if (!c) return RSV_E_ARG;
    if (!opts || reps < 1) return fail(c, RSV_E_ARG, "bad tune arguments");
    if (c->cf_pol > 0) return fail(c, RSV_E_STATE, "tuning ranks the level-cash-flow variants: clear the loaded sequence");
    const int nv = rsv_variant_count(opts->form);
    if (nv < 1) return fail(c, RSV_E_ARG, "bad form %d", opts->form);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    const size_t n_v0 = c->pols.size() * (size_t)c->n_scen;
    CU(c->d_o_v0f.ensure(std::max<size_t>(1, n_v0) * sizeof(float)));
    CU(c->d_o_tot.ensure(std::max(1, c->n_scen) * sizeof(double)));
    rsv_opts o = *opts;
    o.outputs = RSV_OUT_V0 | RSV_OUT_SCEN_TOTAL;
    o.on_device = 1;
    rsv_out out{};
    out.V0 = c->d_o_v0f.as<float>();
    out.scen_total = c->d_o_tot.as<double>();
    int arg = -1;
    float best_ms = 0.0f;
    rsv_status last = RSV_OK;
    for (int v = 0; v < nv; ++v) {
        o.variant = v;
        float vbest = -1.0f;
        bool skip = false;
        for (int r = 0; r <= reps && !skip; ++r) {
            rsv_status st = compute(c, &o, &out);
            // a deflated variant whose staging does not fit beside the loaded
            // tables is skipped (time -1); the others decide
            if (st == RSV_E_ARG && opts->form == F_DEFL) {
                last = st;
                skip = true;
                break;
            }
            if (st != RSV_OK) return st;
            if ((st = rsv_synchronize(c)) != RSV_OK) return st;
            const float ms = rsv_last_kernel_ms(c);
            if (r > 0 && (vbest < 0 || ms < vbest)) vbest = ms;
        }
        if (ms_out) ms_out[v] = vbest;
        if (skip) continue;
        if (arg < 0 || vbest < best_ms) {
            arg = v;
            best_ms = vbest;
        }
    }
    if (arg < 0) return last;
    c->tuned[opts->form] = arg;
    if (best) *best = arg;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

rsv_status rsv_synchronize(rsv_ctx* c) try {
    if (!c) return RSV_E_ARG;
    CU(cudaStreamSynchronize(c->stream));
    if (c->d_ctl.p) {
        int32_t ctl[2] = {0, 0};
        CU(cudaMemcpy(ctl, c->d_ctl.p, sizeof ctl, cudaMemcpyDeviceToHost));
        if (ctl[1] == DEV_TIMEOUT) return fail(c, RSV_E_TIMEOUT, "a bounded device wait ran out (table staging)");
    }
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}

const char* rsv_last_error(const rsv_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

float rsv_last_kernel_ms(rsv_ctx* c) {
    if (!c || !c->ev_recorded) return -1.0f;
    if (cudaEventSynchronize(c->ev1) != cudaSuccess) return -1.0f;
    float ms = -1.0f;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) != cudaSuccess) return -1.0f;
    return ms;
}

int32_t rsv_device_sm_count(const rsv_ctx* c) { return c ? c->sm_count : 0; }

}  // extern "C"
