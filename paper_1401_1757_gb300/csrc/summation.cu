// summation.cu -- the reserves by their summation definition (FP64), the
// O(S^2) method the paper's recurrence replaces (Eq. basicReserveSummation,
// Section 3.8.1): for every step t of a chain, one thread sums the cash flows
// of steps s = t .. S-1 discounted and weighted by the products of the
// one-step matrices from t to s,
//   r_t = sum_{s=t}^{S-1} (prod_{u=t}^{s} v_u) e_j^T (prod_{u=t}^{s} W_u) c_s
//         + (prod_{u=t}^{S-1} v_u) e_j^T (prod_{u=t}^{S-1} W_u) r_S,
// carrying the row vector e_j^T prod W (1 or 3 entries of the reduced model)
// forward from t.  A warp takes 32 consecutive t of one chain.  It exists to
// measure the summation against the recurrence on this hardware; its results
// equal the recurrence's to rounding.
#include <algorithm>
#include <cstdint>

#include "rsv_device.cuh"
#include "summation.cuh"

namespace rsv {
namespace {

// r_t of chain (slot rec, scenario column v) in the reduced state k
__device__ double sum_reserve(const double2* tab, const double* v, int s_pad, const SlotRec& rec, int kind, int t,
                              const double* cf) {
    const int S = rec.S;
    const double rho = (double)rec.rho_h + (double)rec.rho_l;
    if (kind != K_JL && kind != K_LS2) {
        const bool joint = kind == K_ANN2 || kind == K_ASS2, ann = kind == K_ANN || kind == K_ANN2;
        double D = 1.0, r = 0.0;   // D = prod_{u=t}^{s-1} v_u p_u
        for (int s = t; s < S; ++s) {
            const double vs = v[(size_t)s * s_pad];
            double p = tab[rec.idx1 + s].x, q = tab[rec.idx1 + s].y;
            if (joint) {   // joint status: p = px py, q = qx + px qy
                const double2 ey = tab[rec.idx2 + s];
                q = q + p * ey.y;
                p = p * ey.x;
            }
            const double cs = cf ? cf[s] : 1.0;   // c_s / c
            r += (ann ? D * vs * p : D * vs * q) * cs;   // annuity: paid if alive at s+1; assurance: death in s
            D *= vs * p;
        }
        return r + D * rec.bnd;
    }
    // three-state models: row x = e_k^T prod W over states (00, x only, y only),
    // W = [[px py, px qy, qx py], [0, px, 0], [0, 0, py]].  JL: c = (1, 1, rho)
    // on the states at the step's end, r_S = 0.  Second death: the benefit on
    // the transitions into "both dead", x (qx qy, qx, qy), r_S = bnd in every state.
    double x0 = rec.state0 == 0 ? 1.0 : 0.0, x1 = rec.state0 == 1 ? 1.0 : 0.0, x2 = rec.state0 == 2 ? 1.0 : 0.0;
    double D = 1.0, r = 0.0;
    for (int s = t; s < S; ++s) {
        const double vs = v[(size_t)s * s_pad];
        const double2 ex = tab[rec.idx1 + s], ey = tab[rec.idx2 + s];
        const double cs = cf ? cf[s] : 1.0;
        D *= vs;
        if (kind == K_LS2) r += D * (x0 * ex.y * ey.y + x1 * ex.y + x2 * ey.y) * cs;
        const double y0 = x0 * ex.x * ey.x;
        const double y1 = x0 * ex.x * ey.y + x1 * ex.x;
        const double y2 = x0 * ex.y * ey.x + x2 * ey.x;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        if (kind == K_JL) r += D * (x0 + x1 + x2 * rho) * cs;
    }
    if (kind == K_LS2) r += D * (x0 + x1 + x2) * rec.bnd;
    return r;
}

__global__ void __launch_bounds__(256) summation_kernel(const RecurArgs a, int warps_per_chain_max) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const double2* tab = reinterpret_cast<const double2*>(smem_raw);
    if (!stage_to_smem(smem_raw, a.tab, (uint32_t)a.tab_bytes, &bar, a.status)) return;
    const int lane = threadIdx.x & 31;
    const double* plane = static_cast<const double*>(a.v);
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(a.counter, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= a.n_items) break;
        // item = (tile * n_scen + s) * warps_per_chain_max + w: steps 32 w .. 32 w + 31
        const int w = item % warps_per_chain_max, chain = item / warps_per_chain_max;
        const int tile = chain / a.n_scen, s = chain - tile * a.n_scen;
        const SlotRec rec = a.slots[tile];
        if (rec.pol < 0) continue;
        const int t = 32 * w + lane;
        const bool want_all = a.traj != nullptr;
        if (t > rec.S || (!want_all && t != 0)) continue;
        const int kind = a.tile_kind[tile];
        const double amount = a.amount[rec.pol];
        const double* cf = a.cf ? static_cast<const double*>(a.cf) + (size_t)rec.pol * a.cf_ld : nullptr;
        const double bnd = (rec.state0 == 0 || kind == K_LS2) ? (double)rec.bnd : 0.0;   // r_S in the state
        const double x = amount * (t == rec.S ? bnd : sum_reserve(tab, plane + s, a.s_pad, rec, kind, t, cf));
        if (want_all && t <= a.n_steps)
            a.traj[((size_t)rec.pol * (a.n_steps + 1) + t) * a.n_scen + s] = x;
        if (t == 0) {
            const size_t o = (size_t)rec.pol * a.n_scen + s;
            if (a.V0f) a.V0f[o] = (float)x;
            if (a.V0d) a.V0d[o] = x;
            if (a.partial) a.partial[(size_t)tile * a.s_pad + s] = x;
        }
    }
}

}  // namespace

cudaError_t launch_summation(const RecurArgs& a, int warps_per_chain_max, int sm_count, size_t smem,
                             cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(summation_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, summation_kernel, 256, smem)) != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const long long need = ((long long)a.n_items + 7) / 8;
    const int grid = (int)std::max(1LL, std::min((long long)sm_count * bps, need));
    summation_kernel<<<grid, 256, smem, st>>>(a, warps_per_chain_max);
    return cudaGetLastError();
}

}  // namespace rsv
