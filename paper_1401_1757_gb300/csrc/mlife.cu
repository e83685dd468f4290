// mlife.cu -- contracts on m = 1..4 independent lives (Section 4.3).
//
// The paper's transition matrix of m lives is the Kronecker product of the
// single-life matrices, W^m = w_1 (x) ... (x) w_m.  The reserve depends only
// on which lives are dead at the start of a step, so a chain carries 2^m
// reduced states (bit i of the state = life i dead).  One step,
//   r_t = v_t W^m_t (c + r_{t+1}),
// applies W^m as m one-life passes: the factor [[p_i, q_i], [0, 1]] of life i
// mixes each pair of states that differ in bit i, x[S] <- p_i x[S] + q_i x[S | bit i]
// (the dead-life entry is unchanged), m 2^(m-1) multiply-add pairs in place of
// a dense (2^m)^2 product.
//   annuity paid while at least k lives are alive: c[S] = 1 on those states;
//   benefit on the k-th death: the three-state model's "died in the step"
//     states only carry the benefit, so the states with k or more deaths
//     hold the benefit 1 (paid at the end of the step in which they are
//     reached) and are never updated.
// One warp takes one policy and 32 scenarios (a lane per scenario); the
// states live in registers (template on m).  The decrement tables are
// staged in shared memory by the bulk copy of the scenario-parallel kernels.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ctx.cuh"
#include "abi_guard.cuh"

namespace rsv {
namespace {

struct MlRec {
    int32_t idx[4];  // staged-table index of each life at t = 0
    int32_t S;       // steps
    int32_t pol;     // index in the caller's records
    int32_t k;
    int32_t flags;   // bit 0: assurance; bits 8..11: dead lives at valuation
};
static_assert(sizeof(MlRec) == 32, "MlRec layout");

struct MlArgs {
    const void* tab;
    int32_t tab_bytes;
    const void* v;       // scenario plane [steps][s_pad] of the form
    int32_t s_pad, n_scen;
    const MlRec* recs;   // records of this m, in decreasing cost order
    const double* amount;
    int32_t n_rec, n_chunks, n_items;
    int32_t* counter;
    int32_t* status;
    double* V0d;         // [n_pol][n_scen]
    float* V0f;          // or null
};

// arithmetic of the chain: plain FP64 / FP32 or double-float
__device__ __forceinline__ double mix(double p, double a, double q, double b) { return __fma_rn(p, a, __dmul_rn(q, b)); }
__device__ __forceinline__ float mix(float p, float a, float q, float b) { return __fmaf_rn(p, a, __fmul_rn(q, b)); }
__device__ __forceinline__ df mix(df p, df a, df q, df b) { return df_add_pos(df_mul(p, a), df_mul(q, b)); }
__device__ __forceinline__ double scale(double v, double x) { return __dmul_rn(v, x); }
__device__ __forceinline__ float scale(float v, float x) { return __fmul_rn(v, x); }
__device__ __forceinline__ df scale(df v, df x) { return df_mul(v, x); }
__device__ __forceinline__ double plus_one(double x) { return __dadd_rn(x, 1.0); }
__device__ __forceinline__ float plus_one(float x) { return __fadd_rn(x, 1.0f); }
__device__ __forceinline__ df plus_one(df x) { return df_add_float_pos(x, 1.0f); }

template <int FORM, int ML>
__global__ void __launch_bounds__(256) mlife_kernel(const MlArgs a) {
    using T = Tr<FORM>;
    using Val = typename T::Val;
    using TabE = typename T::TabE;
    using VE = typename T::VE;
    constexpr int NST = 1 << ML;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const TabE* tab = reinterpret_cast<const TabE*>(smem_raw);
    if (!stage_to_smem(smem_raw, a.tab, (uint32_t)a.tab_bytes, &bar, a.status)) return;
    const int lane = threadIdx.x & 31;
    const VE* plane = static_cast<const VE*>(a.v);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        const int ri = item / a.n_chunks, chunk = item - ri * a.n_chunks;
        const MlRec rec = a.recs[ri];
        const int s = chunk * 32 + lane;   // < s_pad: padded columns hold finite factors
        const bool ass = rec.flags & 1;
        const int dead0 = (rec.flags >> 8) & 15;
        // states paid (assurance: k or more deaths) and paying (annuity: k or more alive)
        unsigned mark = 0;
#pragma unroll
        for (int S = 0; S < NST; ++S) {
            const int dead = __popc(S);
            if (ass ? dead >= rec.k : ML - dead >= rec.k) mark |= 1u << S;
        }
        Val r[NST];
#pragma unroll
        for (int S = 0; S < NST; ++S) r[S] = T::cst((ass && (mark >> S & 1)) ? 1.0f : 0.0f);
        for (int t = rec.S - 1; t >= 0; --t) {
            const Val v = T::v(plane[(size_t)t * a.s_pad + s]);
            Val x[NST];
#pragma unroll
            for (int S = 0; S < NST; ++S) x[S] = (!ass && (mark >> S & 1)) ? plus_one(r[S]) : r[S];
#pragma unroll
            for (int i = 0; i < ML; ++i) {
                const TabE e = tab[rec.idx[i] + t];
                const Val p = T::p(e), q = T::q(e);
#pragma unroll
                for (int S = 0; S < NST; ++S)
                    if (!(S >> i & 1)) x[S] = mix(p, x[S], q, x[S | (1 << i)]);
            }
#pragma unroll
            for (int S = 0; S < NST; ++S)
                if (!ass || !(mark >> S & 1)) r[S] = scale(v, x[S]);
        }
        // the reserve in the valuation state (selected among compile-time indices)
        double out = 0.0;
#pragma unroll
        for (int S = 0; S < NST; ++S)
            if (S == dead0) out = T::dbl(r[S]);
        if (ass && (mark >> dead0 & 1)) out = 0.0;   // benefit already paid
        if (s < a.n_scen) {
            const double x = a.amount[rec.pol] * out;
            const size_t o = (size_t)rec.pol * a.n_scen + s;
            a.V0d[o] = x;
            if (a.V0f) a.V0f[o] = (float)x;
        }
    }
}

// per-scenario totals over the policies, in policy order
__global__ void colsum_kernel(const double* __restrict__ V, int64_t n, int n_scen, double* __restrict__ tot) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scen) return;
    double acc = 0.0;
    for (int64_t p = 0; p < n; ++p) acc += V[(size_t)p * n_scen + s];
    tot[s] = acc;
}

template <int FORM, int ML>
cudaError_t launch_ml(const MlArgs& a, int sm_count, size_t smem, cudaStream_t st) {
    auto k = mlife_kernel<FORM, ML>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, 256, smem)) != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const long long need = ((long long)a.n_items + 7) / 8;
    const int grid = (int)std::max(1LL, std::min((long long)sm_count * bps, need));
    k<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_form(int m, const MlArgs& a, int sm_count, size_t smem, cudaStream_t st) {
    switch (m) {
    case 1: return launch_ml<FORM, 1>(a, sm_count, smem, st);
    case 2: return launch_ml<FORM, 2>(a, sm_count, smem, st);
    case 3: return launch_ml<FORM, 3>(a, sm_count, smem, st);
    default: return launch_ml<FORM, 4>(a, sm_count, smem, st);
    }
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_compute_mlife(rsv_ctx* c, const rsv_mlife_policy* pols, int64_t n, const rsv_opts* o,
                                        rsv_out* out) try {
    if (!c) return RSV_E_ARG;
    if (!o || !out || n < 0 || n > 0x7fffffffLL || (n > 0 && !pols)) return fail(c, RSV_E_ARG, "bad m-life arguments");
    if (o->form < F_F64 || o->form > F_COMP) return fail(c, RSV_E_ARG, "bad form %d", o->form);
    if ((o->outputs & ~(RSV_OUT_V0 | RSV_OUT_SCEN_TOTAL)) || o->horizon != 0 || o->payment != 0 ||
        (o->variant != 0 && o->variant != -1) || (o->on_device != 0 && o->on_device != 1))
        return fail(c, RSV_E_ARG, "m-life runs take outputs V0 / totals, horizon 0, payment 0, variant 0 or -1");
    const bool want_v0 = o->outputs & RSV_OUT_V0, want_tot = o->outputs & RSV_OUT_SCEN_TOTAL;
    if (want_v0 && !out->V0 && !out->V0d) return fail(c, RSV_E_ARG, "V0 requested but NULL");
    if (want_tot && !out->scen_total) return fail(c, RSV_E_ARG, "scen_total NULL");
    if (c->n_scen == 0) return fail(c, RSV_E_STATE, "no scenarios loaded");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, RSV_E_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));

    // validate; steps; table span
    std::vector<MlRec> recs((size_t)n);
    std::vector<int> ms((size_t)n);
    int need = 1, n_tab = 1;
    for (int64_t i = 0; i < n; ++i) {
        const rsv_mlife_policy& r = pols[i];
        if (r.m < 1 || r.m > 4 || (r.kind != RSV_MLIFE_ANNUITY && r.kind != RSV_MLIFE_ASSURANCE) || r.k < 1 ||
            r.k > r.m || r.term_m < 0 || r.reserved != 0 || r.dead0 < 0 || r.dead0 >= (1 << r.m))
            return fail(c, RSV_E_ARG, "m-life policy %lld: bad record", (long long)i);
        const int dead = __builtin_popcount((unsigned)r.dead0);
        if (r.kind == RSV_MLIFE_ASSURANCE ? (r.term_m < 1 || dead >= r.k) : (r.m - dead < r.k))
            return fail(c, RSV_E_ARG, "m-life policy %lld: term or valuation state out of range", (long long)i);
        if (!std::isfinite(r.amount)) return fail(c, RSV_E_ASSUMPTION, "m-life policy %lld: amount not finite", (long long)i);
        int rem[4];
        for (int j = 0; j < r.m; ++j) {
            if (r.table[j] < 0 || r.table[j] >= kMaxTables || c->tab[r.table[j]].empty() || r.age_m[j] < 0)
                return fail(c, RSV_E_ARG, "m-life policy %lld: life %d has a bad age or table", (long long)i, j + 1);
            rem[j] = std::max(0, (int)c->tab[r.table[j]].size() - r.age_m[j]);
            n_tab = std::max(n_tab, r.table[j] + 1);
        }
        int S;
        if (r.kind == RSV_MLIFE_ASSURANCE) {
            S = r.term_m;
        } else {   // while k lives can be alive: the k-th longest remaining table
            std::sort(rem, rem + r.m);
            S = rem[r.m - r.k];
            if (r.term_m > 0) S = std::min(S, r.term_m);
        }
        if (S > c->n_steps)
            return fail(c, RSV_E_ASSUMPTION, "m-life policy %lld: %d steps but scenarios have %d", (long long)i, S,
                        c->n_steps);
        MlRec& q = recs[(size_t)i];
        for (int j = 0; j < 4; ++j) q.idx[j] = 0;
        for (int j = 0; j < r.m; ++j) {
            if (r.age_m[j] + S > kMaxAgeSteps)
                return fail(c, RSV_E_ARG, "m-life policy %lld: age + steps exceeds %d", (long long)i, kMaxAgeSteps);
            need = std::max(need, r.age_m[j] + S);
        }
        q.S = S;
        q.pol = (int)i;
        q.k = r.k;
        q.flags = (r.kind == RSV_MLIFE_ASSURANCE ? 1 : 0) | (r.dead0 << 8);
        ms[(size_t)i] = r.m;
    }
    for (int t = 0; t < n_tab; ++t) need = std::max(need, (int)c->tab[t].size());
    const int pad = (need + 31) / 32 * 32;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < ms[(size_t)i]; ++j) recs[(size_t)i].idx[j] = pols[i].table[j] * pad + pols[i].age_m[j];
    size_t smem = 0;
    rsv_status st = stage_tables(c, o->form, pad, n_tab, smem);
    if (st != RSV_OK) return st;

    // group by m, longest projections first
    std::vector<int> order((size_t)n);
    for (int64_t i = 0; i < n; ++i) order[(size_t)i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return ms[x] != ms[y] ? ms[x] < ms[y] : recs[x].S > recs[y].S;
    });
    std::vector<MlRec> sorted((size_t)n);
    for (int64_t i = 0; i < n; ++i) sorted[(size_t)i] = recs[order[(size_t)i]];

    const int NSc = c->n_scen;
    const size_t n_v0 = (size_t)n * NSc;
    std::vector<double> amount((size_t)n);
    for (int64_t i = 0; i < n; ++i) amount[(size_t)i] = pols[i].amount;
    CU(c->d_ml_rec.ensure(std::max<size_t>(1, sorted.size()) * sizeof(MlRec)));
    CU(c->d_ml_amount.ensure(std::max<size_t>(1, amount.size()) * sizeof(double)));
    double* V0d = (o->on_device && want_v0 && out->V0d) ? out->V0d : nullptr;
    if (!V0d) {
        CU(c->d_o_v0d.ensure(std::max<size_t>(1, n_v0) * sizeof(double)));
        V0d = c->d_o_v0d.as<double>();
    }
    float* V0f = nullptr;
    if (want_v0 && out->V0) {
        if (o->on_device) {
            V0f = out->V0;
        } else {
            CU(c->d_o_v0f.ensure(std::max<size_t>(1, n_v0) * sizeof(float)));
            V0f = c->d_o_v0f.as<float>();
        }
    }
    double* tot = nullptr;
    if (want_tot) {
        if (o->on_device) {
            tot = out->scen_total;
        } else {
            CU(c->d_o_tot.ensure(NSc * sizeof(double)));
            tot = c->d_o_tot.as<double>();
        }
    }
    CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
    if (n > 0) {
        CU(cudaMemcpyAsync(c->d_ml_rec.p, sorted.data(), sorted.size() * sizeof(MlRec), cudaMemcpyHostToDevice,
                           c->stream));
        CU(cudaMemcpyAsync(c->d_ml_amount.p, amount.data(), amount.size() * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream));
    }
    MlArgs a{};
    a.tab = c->d_tab[o->form].p;
    a.tab_bytes = (int32_t)smem;
    a.v = o->form == F_F64 ? c->d_v64.p : (o->form == F_F32 ? c->d_v32.p : c->d_v2.p);
    a.s_pad = c->s_pad;
    a.n_scen = NSc;
    a.amount = c->d_ml_amount.as<double>();
    a.n_chunks = (NSc + 31) / 32;
    a.counter = c->d_ctl.as<int32_t>();
    a.status = c->d_ctl.as<int32_t>() + 1;
    a.V0d = V0d;
    a.V0f = V0f;
    CU(cudaMemsetAsync(c->d_ctl.p, 0, 2 * sizeof(int32_t), c->stream));
    CU(cudaEventRecord(c->ev0, c->stream));
    for (size_t b = 0; b < sorted.size();) {
        const int m = ms[order[b]];
        size_t e2 = b;
        while (e2 < sorted.size() && ms[order[e2]] == m) ++e2;
        const long long items = (long long)(e2 - b) * a.n_chunks;
        if (items > 0x7fffffffLL) return fail(c, RSV_E_ARG, "too many m-life work items (%lld)", items);
        MlArgs g = a;
        g.recs = c->d_ml_rec.as<MlRec>() + b;
        g.n_rec = (int32_t)(e2 - b);
        g.n_items = (int32_t)items;
        CU(cudaMemsetAsync(c->d_ctl.p, 0, sizeof(int32_t), c->stream));   // queue head
        cudaError_t le = o->form == F_F64 ? launch_form<F_F64>(m, g, c->sm_count, smem, c->stream)
                         : o->form == F_F32 ? launch_form<F_F32>(m, g, c->sm_count, smem, c->stream)
                                            : launch_form<F_COMP>(m, g, c->sm_count, smem, c->stream);
        CU(le);
        b = e2;
    }
    if (tot) {
        colsum_kernel<<<(NSc + 127) / 128, 128, 0, c->stream>>>(V0d, n, NSc, tot);
        CU(cudaGetLastError());
    }
    CU(cudaEventRecord(c->ev1, c->stream));
    c->ev_recorded = true;
    if (!o->on_device) {
        if (want_v0 && out->V0d) CU(cudaMemcpyAsync(out->V0d, V0d, n_v0 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (V0f) CU(cudaMemcpyAsync(out->V0, V0f, n_v0 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (tot) CU(cudaMemcpyAsync(out->scen_total, tot, NSc * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        return rsv_synchronize(c);
    }
    return RSV_OK;
} catch (...) {
    return rsv::host_error(c);
}
