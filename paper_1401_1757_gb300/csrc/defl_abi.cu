// defl_abi.cu -- host side of rsv_compute_reserves in the deflated form
// (RSV_FORM_F32_DEFLATED): life tables, super-tile slot records, the
// deflator plane and the launches.
#include <algorithm>
#include <thread>
#include <cmath>
#include <vector>

#include "ctx.cuh"
#include "defl_kernel.cuh"

namespace rsv {

cudaError_t launch_defl_plane(const double* v64, int n_steps, int s_pad, int n_groups, float4* out, cudaStream_t st);

namespace {

// l_0 of every staged life table: ratios l_k / l_0 down to 2^-220 stay in
// FP32's normal range, with room for the discount factors.
constexpr double kEllScale = 1267650600228229401496703205376.0;   // 2^100
constexpr double kEllMinRatio = 5.94e-67;                          // about 2^-220

// Life table {l_k} of one decrement table (Section 5's {l_{x+t}}), FP64:
// l_0 = 2^100, l_{k+1} = l_k p_k, p_k = 0 from the table's length on.
std::vector<double> life_table(const std::vector<double>& p, int n) {
    std::vector<double> l(n + 1, 0.0);
    l[0] = kEllScale;
    for (int k = 0; k < n; ++k) l[k + 1] = l[k] * (k < (int)p.size() ? p[k] : 0.0);
    return l;
}

int defl_smem_limit(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return 0;
    return v;
}

}  // namespace

// The staged tables of the deflated kernels: the survivors array A
// (annuities) and the deaths array (assurances), each only if a product needs
// it, for the tables in use, as four copies shifted by one entry.  A copy
// holds every entry up to the end of the longest table used, then zeros (at
// least one whole group of four past each table's end), a unit group and a
// last zero group.
rsv_status defl_table_shape(rsv_ctx* c, const Layout& L, DeflTabs& T) {
    T.use_a = T.use_d = false;
    for (int k : L.h_k2) {
        if (k != K_ANN && k != K_ASS && k != K_JL && k != K_ANN2)
            return fail(c, RSV_E_ARG,
                        "the deflated form values products 0-5 (single-life, reversionary, joint and last-survivor "
                        "annuities, term and endowment assurances); use RSV_FORM_F32_COMP for the others");
        (k == K_ASS ? T.use_d : T.use_a) = true;
    }
    T.n_tab = L.n_tab;
    int max_len = 1;
    for (int t = 0; t < T.n_tab; ++t) max_len = std::max(max_len, (int)c->tab[t].size());
    T.dpad = (max_len + 8 + 3) / 4 * 4 + 8;   // the last two groups: a unit group, then zeros
    T.arr_d = T.use_a ? 1 : 0;                 // index of the deaths array among the staged ones
    T.bytes = (size_t)(T.use_a + T.use_d) * T.n_tab * 4 * T.dpad * sizeof(float);
    return RSV_OK;
}

rsv_status defl_table_stage(rsv_ctx* c, DeflTabs& T) {
    const int n_tab = T.n_tab, dpad = T.dpad, arr_d = T.arr_d;
    const bool use_a = T.use_a, use_d = T.use_d;
    // life tables: [A | deaths][table][4 copies shifted by c][dpad], A_k = l_{k+1}, deaths_k = l_k q_k
    T.ell.assign(n_tab, {});
    for (int t = 0; t < n_tab; ++t) {
        T.ell[t] = life_table(c->tab[t], dpad + 4);
        for (int k = 0; k < (int)c->tab[t].size(); ++k)
            if (T.ell[t][k + 1] > 0.0 && T.ell[t][k + 1] < kEllMinRatio * kEllScale)
                return fail(c, RSV_E_ARG, "table %d: survival to age %d months is below 2^-220, out of the "
                                          "deflated form's range", t, k + 1);
    }
    const unsigned long long tkey = c->tab_gen * 1000003ull + (unsigned)dpad * 131ull + (unsigned)n_tab * 7ull +
                                    (use_a ? 1ull : 0ull) + (use_d ? 2ull : 0ull);
    if (c->defl_tab_key != tkey) {
        std::vector<float> h((size_t)(use_a + use_d) * n_tab * 4 * dpad, 0.0f);
        for (int t = 0; t < n_tab; ++t) {
            const std::vector<double>& l = T.ell[t];
            const std::vector<double>& p = c->tab[t];
            for (int cpy = 0; cpy < 4; ++cpy)
                for (int q = 0; q < dpad; ++q) {
                    const int k = q + cpy;
                    const double pk = k < (int)p.size() ? p[k] : 0.0;
                    if (use_a) h[(((size_t)0 * n_tab + t) * 4 + cpy) * dpad + q] = (float)l[k + 1];
                    if (use_d) h[(((size_t)arr_d * n_tab + t) * 4 + cpy) * dpad + q] = (float)(l[k] * (1.0 - pk));
                }
            if (use_d) h[(((size_t)arr_d * n_tab + t) * 4 + 0) * dpad + dpad - 8] = 1.0f;   // the unit group
        }
        CU(c->d_defl_tab.ensure(h.size() * sizeof(float)));
        CU(cudaMemcpyAsync(c->d_defl_tab.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice,
                           c->stream));   // staged (pageable source)
        c->defl_tab_key = tkey;
    }
    return RSV_OK;
}

rsv_status compute_deflated(rsv_ctx* c, const rsv_opts* o, rsv_out* out) {
    const int outs = o->outputs;
    if (outs & (RSV_OUT_PT_MEAN | RSV_OUT_TRAJ))
        return fail(c, RSV_E_ARG, "the deflated form outputs V0 and the totals; per-step outputs need another form");
    if (o->payment != RSV_PAY_END) return fail(c, RSV_E_ARG, "the deflated form pays at the end of each step");
    if (c->cf_pol > 0)
        return fail(c, RSV_E_STATE, "the deflated form values level cash flows: clear the loaded sequence");
    int nv = 0;
    const DeflVariant* vl = variants_defl(&nv);
    int vi;
    if (o->variant >= 0) {
        if (o->variant >= nv) return fail(c, RSV_E_ARG, "variant %d out of range", o->variant);
        vi = o->variant;
    } else if (o->variant == -1) {
        vi = c->tuned[F_DEFL] >= 0 ? c->tuned[F_DEFL] : 0;
    } else {
        return fail(c, RSV_E_ARG, "variant %d out of range (the deflated form has no scan or summation)", o->variant);
    }
    // A variant whose staging ring does not fit beside the tables is replaced
    // by the first that does, unless it was asked for by index.
    int W = 0;
    rsv_status st = RSV_OK;
    DeflTabs T;
    size_t smem = 0;
    const long long smem_max = defl_smem_limit(c->device);
    for (int pass = 0;; ++pass) {
        const DeflVariant& V = vl[vi];
        W = V.NW * V.P;
        if ((st = build_layout(c, W, o->horizon, c->n_steps)) != RSV_OK) return st;
        if ((st = defl_table_shape(c, c->lay, T)) != RSV_OK) return st;
        smem = T.bytes + defl_smem_extra(V);
        if ((long long)smem <= smem_max) break;
        int alt = -1;
        for (int k = 0; k < nv && alt < 0; ++k)
            if ((long long)(T.bytes + defl_smem_extra(vl[k])) <= smem_max) alt = k;
        if (o->variant >= 0 || alt < 0 || pass > 0)
            return fail(c, RSV_E_ARG, "variant %s needs %zu bytes of shared memory for %d tables (%lld available)",
                        V.name, smem, T.n_tab, smem_max);
        vi = alt;
    }
    const DeflVariant& V = vl[vi];
    const int CH = 32 * V.M;
    const Layout& L = c->lay;
    if ((st = defl_table_stage(c, T)) != RSV_OK) return st;
    const int n_tab = T.n_tab, dpad = T.dpad, arr_d = T.arr_d;
    const size_t tab_bytes = T.bytes;
    const std::vector<std::vector<double>>& ell = T.ell;

    // slot records of the super-tiles
    const unsigned long long lkey = L.gen * 31ull + (unsigned long long)dpad * 7ull + (unsigned)L.horizon * 3ull +
                                    (unsigned long long)arr_d;
    if (c->defl_lay_key != lkey || c->defl_W != W || c->defl_dpad != dpad || c->defl_n_st != L.n_tiles) {
        // written in place into pinned memory by several host threads
        const size_t n_slots = (size_t)L.n_tiles * W;
        CU(c->h_defl_stage.acquire(std::max<size_t>(1, n_slots) * sizeof(DeflSlot)));
        DeflSlot* ds = c->h_defl_stage.as<DeflSlot>();
        auto off = [&](int arr, int tb, int age) {
            const int cp = age & 3;
            return (int)(((((size_t)arr * n_tab + tb) * 4 + cp) * dpad + (age - cp)) / 4);
        };
        // A life's float4 run and its first all-zero group: entries are zero
        // from z on (z = the table's length for survivors, one more for deaths).
        // A life already at or past z reads one zero group of copy 0 for every
        // step.  Every read then stays below z + 7 <= dpad.
        auto run = [&](int arr, int tb, int age, int z, int& o, int& gz) {
            if (age >= z) {
                o = off(arr, tb, (z + 3) / 4 * 4);
                gz = 0;
            } else {
                o = off(arr, tb, age);
                gz = (z - age + 3) / 4;
            }
        };
        auto fill = [&](int f0, int f1) {
        for (int f = f0; f < f1; ++f) {
            const int kind = L.h_k2[f];
            for (int k = 0; k < W; ++k) {
                const SlotRec& r = L.h_s2[(size_t)f * W + k];
                DeflSlot d{};
                // (table, age) of each life; no division for the first table
                const int tp = L.tab_pad;
                const int tb1 = r.idx1 < tp ? 0 : r.idx1 / tp, a1 = r.idx1 - tb1 * tp;
                const int tb2 = r.idx2 < tp ? 0 : r.idx2 / tp, a2 = r.idx2 - tb2 * tp;
                // survivors are zero from the table's length on, deaths one step
                // later (everyone left dies in the month at the limiting age)
                const int z1 = (int)c->tab[tb1].size() + (kind == K_ASS ? 1 : 0), z2 = (int)c->tab[tb2].size();
                run(kind == K_ASS ? arr_d : 0, tb1, a1, z1, d.off1, d.gz1);
                run(0, tb2, a2, z2, d.off2, d.gz2);
                d.S = r.S;
                d.pol = r.pol;
                d.kind = kind;
                auto ell_at = [&](int tb, int k) { return k < (int)ell[tb].size() ? ell[tb][k] : 0.0; };
                const double lx = ell_at(tb1, a1), ly = ell_at(tb2, a2);
                const double amount = r.pol >= 0 ? c->pols[r.pol].amount : 0.0;
                const double rho = (double)r.rho_h + (double)r.rho_l;
                double scale = 0.0;
                if (kind == K_ANN || kind == K_ASS) {
                    scale = lx > 0.0 ? amount / lx : 0.0;
                    if (kind == K_ASS && r.bnd != 0.0f) d.mat = (float)((double)r.bnd * ell_at(tb1, a1 + r.S));
                    if (kind == K_ASS && r.S == 0) {   // at maturity: r_0 = bnd, whatever the survival
                        scale = amount;
                        d.mat = r.bnd;
                    } else if (kind == K_ASS && !(lx > 0.0)) {
                        // alive at an age the table gives no survival to: death in
                        // the first month is certain; the run is the unit group
                        // (1, 0, 0, 0) followed by zeros
                        scale = amount;
                        d.mat = 0.0f;
                        d.off1 = off(arr_d, tb1, dpad - 8);
                        d.gz1 = 1;
                    }
                } else {
                    scale = amount;
                    const double ix = lx > 0.0 ? 1.0 / lx : 0.0;
                    const double iy = ly > 0.0 ? 1.0 / ly : 0.0;
                    if (kind == K_ANN2) {
                        d.ix = (float)ix;
                        d.iy = (float)iy;
                    } else {   // state 0: both; 1: only the first life alive; 2: only the second
                        d.ix = r.state0 == 2 ? 0.0f : (float)ix;
                        d.iy = r.state0 == 1 ? 0.0f : (float)(rho * iy);
                    }
                }
                d.scale = scale;
                d.sc_h = (float)scale;
                d.sc_l = (float)(scale - (double)d.sc_h);
                ds[(size_t)f * W + k] = d;
            }
        }
        };
        {
            const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
            const int T = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::min(hw, 16), n_slots / 16384));
            run_parts(T, [&](int k) {
                fill((int)((long long)L.n_tiles * k / T), (int)((long long)L.n_tiles * (k + 1) / T));
            });
        }
        CU(c->d_defl_slots.ensure(std::max<size_t>(1, n_slots) * sizeof(DeflSlot)));
        CU(c->d_defl_kinds.ensure(std::max<size_t>(1, L.h_k2.size()) * sizeof(int32_t)));
        if (n_slots) {
            CU(c->h_defl_stage.upload(c->d_defl_slots.p, n_slots * sizeof(DeflSlot), c->stream));
            // pageable source: staged before the call returns
            CU(cudaMemcpyAsync(c->d_defl_kinds.p, L.h_k2.data(), L.h_k2.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, c->stream));
        }
        c->defl_lay_key = lkey;
        c->defl_W = W;
        c->defl_dpad = dpad;
        c->defl_n_st = L.n_tiles;
    }

    const int64_t n_pol = (int64_t)c->pols.size();
    const int NSc = c->n_scen, s_pad = c->s_pad;
    const size_t n_v0 = (size_t)n_pol * NSc;
    float* V0f = (outs & RSV_OUT_V0) ? out->V0 : nullptr;
    double* V0d = (outs & RSV_OUT_V0) ? out->V0d : nullptr;
    double* tot = (outs & RSV_OUT_SCEN_TOTAL) ? out->scen_total : nullptr;
    float* hV0f = V0f;
    double *hV0d = V0d, *htot = tot;
    // A page-locked host V0 that is mapped into the device's address space is
    // written by the kernel itself (coherent stores over the CPU-GPU link, at
    // a small fraction of the link's bandwidth for this kernel), so its 4 or 8
    // bytes per valuation are not staged in device memory and copied after.
    // Both ends of each buffer must lie in mapped page-locked memory, else the
    // staged copy is used.
    auto mapped = [](const void* p, size_t bytes) -> char* {
        cudaPointerAttributes a0{}, a1{};
        const char* q = static_cast<const char*>(p);
        if (cudaPointerGetAttributes(&a0, q) != cudaSuccess ||
            cudaPointerGetAttributes(&a1, q + bytes - 1) != cudaSuccess) {
            cudaGetLastError();   // not a CUDA allocation
            return nullptr;
        }
        if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
            return nullptr;
        char* d = static_cast<char*>(a0.devicePointer);
        return static_cast<char*>(a1.devicePointer) == d + bytes - 1 ? d : nullptr;
    };
    bool direct_v0 = false;
    if (!o->on_device && (V0f || V0d) && n_v0 > 0) {
        char* df = V0f ? mapped(V0f, n_v0 * sizeof(float)) : nullptr;
        char* dd = V0d ? mapped(V0d, n_v0 * sizeof(double)) : nullptr;
        if ((!V0f || df) && (!V0d || dd)) {
            direct_v0 = true;
            if (V0f) V0f = reinterpret_cast<float*>(df);
            if (V0d) V0d = reinterpret_cast<double*>(dd);
        }
    }
    if (!o->on_device) {
        if (V0f && !direct_v0) { CU(c->d_o_v0f.ensure(n_v0 * sizeof(float))); V0f = c->d_o_v0f.as<float>(); }
        if (V0d && !direct_v0) { CU(c->d_o_v0d.ensure(n_v0 * sizeof(double))); V0d = c->d_o_v0d.as<double>(); }
        if (tot) { CU(c->d_o_tot.ensure(NSc * sizeof(double))); tot = c->d_o_tot.as<double>(); }
    }
    CU(c->d_ctl.ensure(2 * sizeof(int32_t)));
    CU(cudaMemsetAsync(c->d_ctl.p, 0, 2 * sizeof(int32_t), c->stream));
    if (tot) CU(c->d_partial.ensure((size_t)std::max(1, L.n_tiles) * s_pad * sizeof(double)));
    if (tot && L.n_tiles == 0) CU(cudaMemsetAsync(tot, 0, NSc * sizeof(double), c->stream));

    // the deflator plane, rows of four steps, a whole number of staged blocks
    const int n_groups = std::max(1, (c->n_steps + DEFL_KB - 1) / DEFL_KB) * DEFL_G;
    CU(c->d_defl_plane.ensure((size_t)n_groups * s_pad * sizeof(float4)));

    DeflArgs a{};
    a.tab = c->d_defl_tab.as<float>();
    a.tab_bytes = (int32_t)tab_bytes;
    a.D = c->d_defl_plane.as<float4>();
    a.s_pad = s_pad;
    a.n_scen = NSc;
    a.n_groups = n_groups;
    a.slots = c->d_defl_slots.as<DeflSlot>();
    a.st_kind = c->d_defl_kinds.as<int32_t>();
    a.n_st = L.n_tiles;
    a.counter = c->d_ctl.as<int32_t>();
    a.status = c->d_ctl.as<int32_t>() + 1;
    a.V0f = V0f;
    a.V0d = V0d;
    a.v0_ld = NSc;
    a.partial = tot ? c->d_partial.as<double>() : nullptr;
    a.part_ld = s_pad;

    int bps = 0;
    CU(V.occupancy(&bps, smem));
    if (bps < 1) return fail(c, RSV_E_CUDA, "variant %s cannot be resident with %zu B smem", V.name, smem);
    // one launch on the scenario columns [s0, s0 + w)
    auto launch = [&](int s0, int w) -> rsv_status {
        DeflArgs b = a;
        b.D = a.D + s0;
        b.n_scen = w;
        b.n_chunks = (w + CH - 1) / CH;
        const long long items = (long long)L.n_tiles * b.n_chunks;
        if (items > 0x7fffffffLL) return fail(c, RSV_E_ARG, "too many work items (%lld)", items);
        b.n_items = (int32_t)items;
        b.V0f = a.V0f ? a.V0f + s0 : nullptr;
        b.V0d = a.V0d ? a.V0d + s0 : nullptr;
        b.partial = a.partial ? a.partial + s0 : nullptr;
        const long long grid = std::max(1LL, std::min((long long)c->sm_count * bps, items));
        CU(cudaMemsetAsync(c->d_ctl.p, 0, sizeof(int32_t), c->stream));
        CU(V.launch(b, (int)grid, smem, c->stream));
        return RSV_OK;
    };

    const bool pipelined =
        !o->on_device && !direct_v0 && ((hV0f != nullptr) != (hV0d != nullptr)) && L.n_tiles > 0 && NSc >= 256;
    CU(cudaEventRecord(c->ev0, c->stream));
    CU(launch_defl_plane(c->d_v64.as<double>(), c->n_steps, s_pad, n_groups, c->d_defl_plane.as<float4>(),
                         c->stream));
    bool copied_v0 = direct_v0;
    if (L.n_tiles > 0 && pipelined) {
        // V0 in column blocks, each copied to the host on a second stream
        // while the next block computes (the last block's copy is the tail
        // left after the last kernel: eight blocks keep it short)
        const int blocks = std::min(8, NSc / 128);
        const int width = ((NSc + blocks - 1) / blocks + 127) / 128 * 128;
        if (!c->copy_stream) CU(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->ev_block) CU(cudaEventCreateWithFlags(&c->ev_block, cudaEventDisableTiming));
        const size_t esz = hV0f ? sizeof(float) : sizeof(double);
        char* dV0 = hV0f ? reinterpret_cast<char*>(V0f) : reinterpret_cast<char*>(V0d);
        char* hV0 = hV0f ? reinterpret_cast<char*>(hV0f) : reinterpret_cast<char*>(hV0d);
        for (int s0 = 0; s0 < NSc; s0 += width) {
            const int w = std::min(width, NSc - s0);
            if ((st = launch(s0, w)) != RSV_OK) return st;
            CU(cudaEventRecord(c->ev_block, c->stream));
            CU(cudaStreamWaitEvent(c->copy_stream, c->ev_block, 0));
            CU(cudaMemcpy2DAsync(hV0 + (size_t)s0 * esz, (size_t)NSc * esz, dV0 + (size_t)s0 * esz, (size_t)NSc * esz,
                                 (size_t)w * esz, (size_t)n_pol, cudaMemcpyDeviceToHost, c->copy_stream));
        }
        CU(cudaEventRecord(c->ev1, c->stream));
        CU(cudaEventRecord(c->ev_block, c->copy_stream));
        CU(cudaStreamWaitEvent(c->stream, c->ev_block, 0));
        copied_v0 = true;
    } else {
        if (L.n_tiles > 0 && (st = launch(0, NSc)) != RSV_OK) return st;
        CU(cudaEventRecord(c->ev1, c->stream));
    }
    c->ev_recorded = true;
    if (tot && L.n_tiles > 0 && (st = scenario_totals(c, a.partial, L.n_tiles, s_pad, NSc, tot)) != RSV_OK) return st;
    if (!o->on_device) {
        if (hV0f && !copied_v0) CU(cudaMemcpyAsync(hV0f, V0f, n_v0 * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        if (hV0d && !copied_v0) CU(cudaMemcpyAsync(hV0d, V0d, n_v0 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        if (htot) CU(cudaMemcpyAsync(htot, tot, NSc * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        return rsv_synchronize(c);
    }
    return RSV_OK;
}

}  // namespace rsv
