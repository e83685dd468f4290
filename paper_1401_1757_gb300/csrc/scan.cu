// scan.cu -- the backward recurrence as a parallel-in-time scan (FP64): one
// warp per chain, its lanes over blocks of time steps.
//
// Each step of Eq. generalForm (f = 1) is an affine map of the next step's
// reduced reserve vector, r_t = a_t + B_t r_{t+1} with B_t = v_t W_t and
// a_t = B_t c_t (Section 3.1).  Affine maps compose associatively,
//   (a, B) o (a', B') = (a + B a', B B'),
// so a chain of S steps splits into 32 blocks: lane l composes the maps of
// steps [l L, (l+1) L) (L = ceil(S / 32)), a warp suffix scan of the 32
// composites (five shuffle levels, fixed order) gives every lane the map from
// the boundary r_S to the start of its block, and lane 0 holds r_0.  With the
// trajectory requested each lane then replays its block from r at its end.
//
// This fills a warp with one chain, where the scenario-parallel kernels need
// 32 scenarios per warp: it is the launch for few scenarios (one flat rate)
// and for very long projections.  For the 3-state models (joint life,
// second death) B keeps the structure [[b00, b01, b02], [0, b11, 0],
// [0, 0, b22]] under products.
#include <algorithm>
#include <cstdint>

#include "rsv_device.cuh"
#include "scan.cuh"

namespace rsv {
namespace {

struct Aff1 {   // 1 state
    double a, b;
};
struct Aff3 {   // JL states 00, 01, 10
    double a0, a1, a2, b00, b01, b02, b11, b22;
};

__device__ __forceinline__ Aff1 ident(Aff1) { return Aff1{0.0, 1.0}; }
__device__ __forceinline__ Aff3 ident(Aff3) { return Aff3{0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 1.0, 1.0}; }

// x o y: apply y first, then x
__device__ __forceinline__ Aff1 compose(const Aff1& x, const Aff1& y) { return Aff1{x.a + x.b * y.a, x.b * y.b}; }
__device__ __forceinline__ Aff3 compose(const Aff3& x, const Aff3& y) {
    Aff3 z;
    z.a0 = x.a0 + x.b00 * y.a0 + x.b01 * y.a1 + x.b02 * y.a2;
    z.a1 = x.a1 + x.b11 * y.a1;
    z.a2 = x.a2 + x.b22 * y.a2;
    z.b00 = x.b00 * y.b00;
    z.b01 = x.b00 * y.b01 + x.b01 * y.b11;
    z.b02 = x.b00 * y.b02 + x.b02 * y.b22;
    z.b11 = x.b11 * y.b11;
    z.b22 = x.b22 * y.b22;
    return z;
}

__device__ __forceinline__ Aff1 shfl_down(const Aff1& x, int d) {
    return Aff1{__shfl_down_sync(0xffffffffu, x.a, d), __shfl_down_sync(0xffffffffu, x.b, d)};
}
__device__ __forceinline__ Aff3 shfl_down(const Aff3& x, int d) {
    Aff3 z;
    z.a0 = __shfl_down_sync(0xffffffffu, x.a0, d);
    z.a1 = __shfl_down_sync(0xffffffffu, x.a1, d);
    z.a2 = __shfl_down_sync(0xffffffffu, x.a2, d);
    z.b00 = __shfl_down_sync(0xffffffffu, x.b00, d);
    z.b01 = __shfl_down_sync(0xffffffffu, x.b01, d);
    z.b02 = __shfl_down_sync(0xffffffffu, x.b02, d);
    z.b11 = __shfl_down_sync(0xffffffffu, x.b11, d);
    z.b22 = __shfl_down_sync(0xffffffffu, x.b22, d);
    return z;
}

// The map of step t of a chain (per unit amount).
struct StepMaps {
    const double2* tab;   // (p, q) entries in shared memory
    const double* v;      // scenario column: v[t * s_pad]
    int s_pad, idx1, idx2;
    double rho;
    const double* cf;     // the policy's cash-flow multipliers c_t / c, or null (level)

    __device__ __forceinline__ double c(int t) const { return cf ? cf[t] : 1.0; }

    __device__ __forceinline__ void at(int t, Aff1& m, int kind) const {
        const double vt = v[(size_t)t * s_pad];
        double p = tab[idx1 + t].x, q = tab[idx1 + t].y;
        if (kind == K_ANN2 || kind == K_ASS2) {   // joint status: p = px py, q = qx + px qy
            const double2 ey = tab[idx2 + t];
            q = q + p * ey.y;
            p = p * ey.x;
        }
        if (kind == K_ANN || kind == K_ANN2) {   // r = v p (c_t + r')
            const double g = vt * p;
            m = Aff1{g * c(t), g};
        } else {                                 // r = v (q c_t + p r')
            m = Aff1{vt * q * c(t), vt * p};
        }
    }
    __device__ __forceinline__ void at(int t, Aff3& m, int kind) const {
        // B = v [[px py, px qy, qx py], [0, px, 0], [0, 0, py]] for both three-state models
        const double vt = v[(size_t)t * s_pad];
        const double2 ex = tab[idx1 + t], ey = tab[idx2 + t];
        m.b00 = vt * ex.x * ey.x;
        m.b01 = vt * ex.x * ey.y;
        m.b02 = vt * ex.y * ey.x;
        m.b11 = vt * ex.x;
        m.b22 = vt * ey.x;
        const double ct = c(t);
        if (kind == K_JL) {   // r = v W (c_t + r'), c_t = (1, 1, rho) c_t / c
            m.a0 = (m.b00 + m.b01 + m.b02 * rho) * ct;
            m.a1 = m.b11 * ct;
            m.a2 = m.b22 * rho * ct;
        } else {              // second death in the step: v (qx qy, qx, qy) c_t / c
            m.a0 = vt * ex.y * ey.y * ct;
            m.a1 = vt * ex.y * ct;
            m.a2 = vt * ey.y * ct;
        }
    }
};

// r at the start of a map's steps, from the vector r at their end (in place)
__device__ __forceinline__ void apply(const Aff1& m, double (&r)[3]) { r[0] = m.a + m.b * r[0]; }
__device__ __forceinline__ void apply(const Aff3& m, double (&r)[3]) {
    const double r0 = m.a0 + m.b00 * r[0] + m.b01 * r[1] + m.b02 * r[2];
    const double r1 = m.a1 + m.b11 * r[1];
    const double r2 = m.a2 + m.b22 * r[2];
    r[0] = r0;
    r[1] = r1;
    r[2] = r2;
}

// r_S per unit amount: the endowment's maturity sum in state 0, or in every
// state of the second-death model (a life alive)
__device__ __forceinline__ void boundary(const SlotRec& rec, int kind, double (&r)[3]) {
    r[0] = rec.bnd;
    r[1] = r[2] = kind == K_LS2 ? (double)rec.bnd : 0.0;
}

// state k of r, selected among compile-time indices (keeps r in registers)
__device__ __forceinline__ double pick(const double (&r)[3], int k) { return k == 0 ? r[0] : (k == 1 ? r[1] : r[2]); }

// One chain (tile of one policy, scenario s); returns amount * r_0 in the
// policy's reported state (valid in lane 0).
template <class A>
__device__ double scan_chain(const StepMaps& sm, int kind, const SlotRec& rec, int s, double amount,
                             const RecurArgs& a, int lane) {
    const int S = rec.S;
    const int L = (S + 31) / 32;
    const int t0 = min(S, lane * L), t1 = min(S, t0 + L);
    A blk = ident(A{});
    for (int t = t1 - 1; t >= t0; --t) {
        A m;
        sm.at(t, m, kind);
        blk = compose(m, blk);
    }
    // suffix scan: lane l ends with blk_l o blk_{l+1} o ... o blk_31
    A suf = blk;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const A y = shfl_down(suf, d);
        if (lane + d < 32) suf = compose(suf, y);
    }
    const int k = rec.state0;
    if (a.traj) {
        // r at the end of this lane's block: the next lane's suffix applied to r_S
        A next = shfl_down(suf, 1);
        if (lane == 31) next = ident(A{});
        double r[3];
        boundary(rec, kind, r);
        apply(next, r);
        const size_t base = (size_t)rec.pol * (a.n_steps + 1);
        // the boundary row t = S, written by the lane whose block ends there
        if (S <= a.n_steps && ((t1 == S && t0 < t1) || (S == 0 && lane == 0)))
            a.traj[(base + S) * a.n_scen + s] = amount * pick(r, k);
        for (int t = t1 - 1; t >= t0; --t) {
            A m;
            sm.at(t, m, kind);
            apply(m, r);
            a.traj[(base + t) * a.n_scen + s] = amount * pick(r, k);
        }
    }
    double r[3];
    boundary(rec, kind, r);
    apply(suf, r);
    return amount * pick(r, k);
}

__global__ void __launch_bounds__(256) scan_kernel(const RecurArgs a) {
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
        const int tile = item / a.n_scen, s = item - tile * a.n_scen;   // tiles of one policy
        const SlotRec rec = a.slots[tile];
        if (rec.pol < 0) continue;
        const int kind = a.tile_kind[tile];
        const double* cf = a.cf ? static_cast<const double*>(a.cf) + (size_t)rec.pol * a.cf_ld : nullptr;
        StepMaps sm{tab, plane + s, a.s_pad, rec.idx1, rec.idx2, (double)rec.rho_h + (double)rec.rho_l, cf};
        const double amount = a.amount[rec.pol];
        const double x = (kind == K_JL || kind == K_LS2) ? scan_chain<Aff3>(sm, kind, rec, s, amount, a, lane)
                                                         : scan_chain<Aff1>(sm, kind, rec, s, amount, a, lane);
        if (lane == 0) {
            const size_t o = (size_t)rec.pol * a.n_scen + s;
            if (a.V0f) a.V0f[o] = (float)x;
            if (a.V0d) a.V0d[o] = x;
            if (a.partial) a.partial[(size_t)tile * a.s_pad + s] = x;
        }
    }
}

}  // namespace

// The time-scan launch: a persistent grid of 8-warp CTAs over n_tiles (one
// policy each) x n_scen chains.  The FP64 decrement tables are staged per CTA.
cudaError_t launch_scan(const RecurArgs& a, int sm_count, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(scan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int bps = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, scan_kernel, 256, smem)) != cudaSuccess) return e;
    if (bps < 1) return cudaErrorInvalidConfiguration;
    const long long need = ((long long)a.n_items + 7) / 8;
    const int grid = (int)std::max(1LL, std::min((long long)sm_count * bps, need));
    scan_kernel<<<grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace rsv
