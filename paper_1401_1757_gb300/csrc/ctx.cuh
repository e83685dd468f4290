// ctx.cuh -- the library context shared by the translation units of the C ABI.
#pragma once

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "host_parts.h"
#include "rsv.h"
#include "mlp.cuh"
#include "recur_kernel.cuh"
#include "surrogate.cuh"

namespace rsv {

constexpr int kMaxTables = 8;
constexpr int kMaxAgeSteps = 4096;       // age + steps bound of the staged tables
constexpr size_t kMaxSmem = 200 * 1024;  // staged tables per CTA
constexpr size_t kMaxTraj = size_t(1) << 30;

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
        if (e == cudaSuccess) n = bytes;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// Pinned host staging for uploads built on the host: written in place, copied
// with one asynchronous copy at full link speed.  `ready` is recorded after
// the copy; the next writer waits for it, so a buffer is never rewritten while
// a copy from it may still run.
struct HostStage {
    void* p = nullptr;
    size_t n = 0;
    cudaEvent_t ready = nullptr;
    cudaError_t acquire(size_t bytes) {
        cudaError_t e;
        if (ready && (e = cudaEventSynchronize(ready)) != cudaSuccess) return e;
        if (bytes <= n && p) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        if ((e = cudaHostAlloc(&p, bytes ? bytes : 16, cudaHostAllocDefault)) != cudaSuccess) return e;
        n = bytes;
        return cudaSuccess;
    }
    cudaError_t upload(void* dst, size_t bytes, cudaStream_t st) {
        cudaError_t e;
        if (!ready && (e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming)) != cudaSuccess) return e;
        if (bytes && (e = cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
        return cudaEventRecord(ready, st);
    }
    void release() {
        if (ready) cudaEventSynchronize(ready);
        if (p) cudaFreeHost(p);
        if (ready) cudaEventDestroy(ready);
        p = nullptr;
        n = 0;
        ready = nullptr;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

// How a product maps onto the reduced models (Section 3.6.4): its kernel
// kind, whether it reads a second life, and its number of projection steps
// from the tables' lengths (the limiting ages) and the term.
struct ProductModel {
    int kind;          // K_ANN, K_ASS, K_JL, K_ANN2, K_ASS2, K_LS2
    bool two_life;     // reads the second life's age and table
    bool multi_state;  // a 3-state model, JL or K_LS2 (state0 may be 1 or 2)
    bool annuity;      // paid while (some) life is alive; term_m 0 = to the limiting age
    float bnd;         // boundary r_S per unit amount at maturity (endowments: 1)
};

inline bool product_model(int product, ProductModel& m) {
    switch (product) {
    case RSV_SL_ANNUITY: m = {K_ANN, false, false, true, 0.0f}; return true;
    case RSV_JL_REVERSIONARY: m = {K_JL, true, true, true, 0.0f}; return true;
    case RSV_TERM_ASSURANCE: m = {K_ASS, false, false, false, 0.0f}; return true;
    case RSV_ENDOWMENT: m = {K_ASS, false, false, false, 1.0f}; return true;
    case RSV_JOINT_ANNUITY: m = {K_ANN2, true, false, true, 0.0f}; return true;
    case RSV_LAST_SURVIVOR: m = {K_JL, true, true, true, 0.0f}; return true;
    case RSV_JOINT_TERM: m = {K_ASS2, true, false, false, 0.0f}; return true;
    case RSV_JOINT_ENDOWMENT: m = {K_ASS2, true, false, false, 1.0f}; return true;
    case RSV_LS_TERM: m = {K_LS2, true, true, false, 0.0f}; return true;
    case RSV_LS_ENDOWMENT: m = {K_LS2, true, true, false, 1.0f}; return true;
    default: return false;
    }
}

// Steps of a policy (len1, len2: its tables' lengths).  Reversionary and
// last-survivor annuities run while either life can be alive, the joint-life
// annuity while both can; term_m > 0 limits an annuity; assurances run for
// their term.
inline int product_steps(const rsv_policy& r, int len1, int len2) {
    int S;
    switch (r.product) {
    case RSV_SL_ANNUITY: S = std::max(0, len1 - r.age1_m); break;
    case RSV_JL_REVERSIONARY:
    case RSV_LAST_SURVIVOR: S = std::max(0, std::max(len1 - r.age1_m, len2 - r.age2_m)); break;
    case RSV_JOINT_ANNUITY: S = std::max(0, std::min(len1 - r.age1_m, len2 - r.age2_m)); break;
    default: return r.term_m;
    }
    return r.term_m > 0 ? std::min(S, r.term_m) : S;
}

// One policy after validation: reduced model, steps, boundary.
struct PolPrep {
    int kind, S, idx_age1, idx_age2, table1, table2, state0, pol;
    float bnd;
    double rho;
};

// Cached tiling for one (P, P_general, horizon, data generation).  Tiles come
// in up to two groups, each in decreasing cost order: group 0 of P policies,
// then group 1 of P_general policies whose loaded cash flows are not level
// (only when P_general > 0), valued by the general-cash-flow kernel.
struct Layout {
    int P = -1, P_general = -1, horizon = -1;
    unsigned long long gen = ~0ull;
    int n_tiles = 0, tab_pad = 0, n_tab = 0;
    int grp_tiles[2] = {0, 0};       // tiles per group
    size_t grp_slot0[2] = {0, 0};    // first slot of each group
    bool grp_two[2] = {false, false};
    double chain_steps = 0;  // sum over policies of S (per scenario)
    int max_S = 0;           // longest projection
    bool has_two = false;    // tiles of K_ANN2, K_ASS2 or K_LS2 present
    DevBuf slots, kinds;
    bool dev_ok = false;   // slots and kinds uploaded for the current build
    // host scratch of the rebuild, kept between calls
    std::vector<PolPrep> h_pp;
    std::vector<int> h_order, h_bucket, h_cnt, h_first, h_kinds, h_grps, h_to, h_k2;
    std::vector<double> h_cost;
    std::vector<SlotRec> h_s2;
};

// The trained surrogate: target normalisation, the per-bucket fallback map
// and its work buffers.
// Fallback buckets: product and state x age of the life the state depends on
// (10-year bins from 20) x remaining term (10-year bins) x the node rate's
// z-score under the model at that month (half-sd bins on [-4, 4), then one
// bin beyond 4 sd that is always valued by the recurrence).
constexpr int SUR_NB_PS = 6, SUR_NB_AGE = 10, SUR_NB_TERM = 8, SUR_NB_R = 17;
constexpr int SUR_NBUCKETS = SUR_NB_PS * SUR_NB_AGE * SUR_NB_TERM * SUR_NB_R;

struct SurrogateState {
    bool trained = false;
    double y_mean = 0.0, y_std = 1.0;   // normalisation of ln(reserve per unit amount)
    double tol = 1e-3;                  // fallback threshold (relative)
    double a = 0.1, b = 0.04, sigma = 0.01, r0 = 0.03;   // Vasicek model of the labels
    std::vector<unsigned char> flag;    // per bucket: 1 = value by the recurrence
    DevBuf d_flag, d_q, d_lab, d_y, d_X, d_pred, d_err, d_aux;
    DevBuf d_curve, d_comm, d_lnb;      // forward-curve increments, commutation columns, ln base values
    DevBuf d_cnt, d_q2, d_idx, d_v2;    // compaction of the served queries (nested surrogate mode)
    double curve_key[3] = {0.0, 0.0, -1.0};
    int comm_pad = -1, comm_ntab = -1;
    unsigned long long comm_gen = 0;
};

}  // namespace rsv

using rsv::DevBuf;
using rsv::HostStage;

struct rsv_ctx {
    using Layout = rsv::Layout;
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err = "no error";

    std::vector<double> tab[rsv::kMaxTables];
    unsigned long long tab_gen = 1;
    std::vector<double> tabf[rsv::kMaxTables];   // survival over the first fraction of each month
    unsigned long long tabf_gen = 1;

    std::vector<rsv_policy, rsv::DefaultInit<rsv_policy>> pols;   // resize leaves new records unset
    unsigned long long pol_gen = 1;
    DevBuf d_amount;
    bool amount_dirty = true;

    int n_scen = 0, n_steps = 0, s_pad = 0;
    DevBuf d_vstage, d_v64, d_v32, d_v2;

    DevBuf d_tab[3];
    int tab_pad_of[3] = {-1, -1, -1};
    int n_tab_of[3] = {-1, -1, -1};
    unsigned long long tab_gen_of[3] = {0, 0, 0};
    DevBuf d_tabf[3];                               // [tables | fractional tables] per form
    unsigned long long tabf_key[3] = {0, 0, 0};
    int vf_scen = 0, vf_steps = 0;                  // fractional discount planes
    DevBuf d_vf64, d_vf32, d_vf2;
    int64_t cf_pol = 0;                             // cash-flow multipliers: rows (0 = level)
    int cf_steps = 0;                               //   and row length
    DevBuf d_cf64, d_cf32;                          //   FP64 rows and their FP32 copy
    std::vector<unsigned char> cf_level;            //   per policy: 1 = the row is all ones
    unsigned long long cf_gen = 1;
    DevBuf d_ml_rec, d_ml_amount;                   // m-life records of the last call

    Layout lay;
    DevBuf d_ctl;       // [0] queue head, [1] status
    DevBuf d_partial, d_part2;
    DevBuf d_o_v0f, d_o_v0d, d_o_tot, d_o_pt, d_o_traj;   // staging for host outputs
    DevBuf d_nest_w, d_nest_ln, d_nest_rn, d_nest_d0, d_nest_plane, d_nest_mean, d_nest_kth, d_nest_all;
    DevBuf d_nest_bm;            // Box-Muller tables of the inner-path generator (staged once)
    bool nest_bm_ready = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t copy_stream = nullptr;   // device-to-host copies of V0 column blocks
    // the deflated brute force's two pipelines: valuation (high priority) and the
    // FP64 inner-path generator (low priority), with their ordering events
    cudaStream_t nest_val = nullptr, nest_gen = nullptr;
    cudaEvent_t nest_ev[5] = {};   // start, generated[2], valued[2]
    cudaEvent_t ev_block = nullptr;
    bool ev_recorded = false;
    int tuned[4] = {-1, -1, -1, -1};
    // the deflated form: super-tile slots, life tables, deflator plane
    DevBuf d_defl_slots, d_defl_kinds, d_defl_tab, d_defl_plane;
    HostStage h_defl_stage;   // the deflated slot records, built here and uploaded
    unsigned long long defl_lay_key = 0, defl_tab_key = 0;
    int defl_W = -1, defl_n_st = 0, defl_dpad = 0, defl_n_tab = 0;
    // surrogate network and its data
    rsv::Mlp mlp;
    bool mlp_ready = false;
    DevBuf d_pols;                  // policy records on the device (surrogate queries)
    unsigned long long pols_dev_gen = 0;
    rsv::SurrogateState sur;
    DevBuf d_mlp_trace;             // layer-by-layer outputs of rsv_mlp_trace (tcgen05 path)
};


namespace rsv {

inline rsv_status fail(rsv_ctx* c, rsv_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        try {
            c->err = buf;
        } catch (...) {   // no room for the message: the status still reports the failure
        }
    }
    return st;
}

// Cached device work layout (policy tiles) and decrement tables in a form's
// entry format (rsv_abi.cu).
rsv_status build_layout(rsv_ctx* c, int P, int horizon, int max_steps, int P_general = 0);
// Upload the layout's slot records and tile kinds (the kernels that read them
// call this; the deflated form builds its own records from the host copy).
rsv_status layout_to_device(rsv_ctx* c);
rsv_status build_tables(rsv_ctx* c, int form, size_t& smem);
// The first n_tab loaded tables, pad entries each, in a form's entry format
// on the device (cached by shape and table generation); smem = their bytes.
rsv_status stage_tables(rsv_ctx* c, int form, int pad, int n_tab, size_t& smem);
// rsv_compute_reserves in the deflated form (defl_abi.cu); opts checked by the caller
rsv_status compute_deflated(rsv_ctx* c, const rsv_opts* o, rsv_out* out);
// The deflated kernels' staged life tables (defl_abi.cu): their shape from the
// layout's kinds (RSV_E_ARG for a product the form does not take), then the
// FP64 life tables {l_k} (l_0 = 2^100) and the staged FP32 arrays.
struct DeflTabs {
    int n_tab = 0, dpad = 0, arr_d = 0;
    bool use_a = false, use_d = false;
    size_t bytes = 0;
    std::vector<std::vector<double>> ell;
};
rsv_status defl_table_shape(rsv_ctx* c, const Layout& L, DeflTabs& T);
rsv_status defl_table_stage(rsv_ctx* c, DeflTabs& T);
// Per-scenario totals from per-tile (row) partial sums [n_rows][s_pad], in a
// fixed order (rsv_abi.cu).
rsv_status scenario_totals(rsv_ctx* c, const double* partial, int n_rows, int s_pad, int n_scen, double* tot);

#define CU(call)                                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return rsv::fail(c, e_ == cudaErrorMemoryAllocation ? RSV_E_NOMEM : RSV_E_CUDA, "%s: %s", \
                             #call, cudaGetErrorString(e_));                                    \
    } while (0)

}  // namespace rsv
