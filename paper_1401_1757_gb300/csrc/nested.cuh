// nested.cuh -- arguments and launchers of the nested valuation kernels.
#pragma once

#include "recur_kernel.cuh"

namespace rsv {

struct NestedArgs {
    const void* tab;          // staged decrement tables (form's entry format)
    int32_t tab_bytes;
    const void* v;            // inner-path planes of this batch [B][n_nodes][Lmax][i_pad]
    int32_t i_pad, n_inner, Lmax, n_nodes, node_step, B, o0;
    const SlotRec* slots;     // policy tiles (valuation-time ages and steps)
    const int32_t* tile_kind;
    int32_t n_tiles;
    const double* wts;        // [n_pol][n_nodes][3] amount x in-force probability per reduced state
    int32_t n_chunks, n_items;
    int32_t* counter;
    int32_t* status;
    double* L_all;            // [n_outer][n_nodes][n_inner]
};

// Constants of one exact monthly Vasicek step of (r, integral of r):
// I = b dt + (r - b) k1 + l21 z1 + l22 z2, r' = b + (r - b) e + l11 z1.
struct VasStep {
    double e, k1, l11, l21, l22, b, dt;
};
VasStep vasicek_step_constants(double a, double b, double sigma, double dt);
int nested_tile_width(int form);
cudaError_t launch_nested(int form, const NestedArgs& a, int sm_count, size_t smem, cudaStream_t st);
// o_first: the global index of the first outer path (the key of its random
// streams); outputs and r_node are indexed from 0.
cudaError_t launch_outer_paths(const VasStep& s, uint64_t seed, int o_first, int n_outer, int n_nodes, int node_step, double r0,
                               double* r_node, double* d0, cudaStream_t st);
// Tables of the inner-path generator's Box-Muller step (FP64): (sin, cos) of
// 2 pi j / BM_SC for j < BM_SC, then for the BM_LG intervals of the logarithm
// (1/c_j to 18 significant bits, -ln(2^k_j / c_j)); built once on the host.
constexpr int BM_SC = 1024, BM_LG = 128;
constexpr int BM_LG_K0 = 53;   // first interval whose centre 1 + (j + 1/2)/128 exceeds sqrt 2
const double2* bm_tables_host();   // BM_SC + BM_LG entries
cudaError_t launch_inner_paths(int form, const VasStep& s, uint64_t seed, int o_first, int o0, int B, int n_nodes, int n_inner,
                               int i_pad, int Lmax, const int* Ln, const double* r_node, const double2* bm,
                               void* plane, int sm_count, cudaStream_t st);
// The curve mode with the outer paths on the lanes (planes [n_nodes][Lmax][o_pad])
// and the transpose of its [n_nodes][n_outer] liabilities to [n_outer][n_nodes].
cudaError_t launch_curve_planes_lanes(int form, double a, double b, double sigma, int n_outer, int n_nodes, int o_pad,
                                      int Lmax, const int* Ln, const double* r_node, void* plane, int sm_count,
                                      cudaStream_t st);
cudaError_t launch_transpose_on(const double* Lt, int n_outer, int n_nodes, double* L, cudaStream_t st);

// ---- the brute-force mode in deflated units (RSV_FORM_F32_DEFLATED) ---------
// The node liability is the policies' expected cash flows E_p(t) at valuation
// (the weights of the deflated valuation kernel, scaled by amount / l_x or
// amount) discounted along the inner path from the node:
//   L_{o,n,i} = sum_p scale_p [ sum_{t >= m} D_i(m, t+1) E_p(t) + D_i(m, S_p) mat_p ],
// D_i(m, t+1) = v_m ... v_t on inner path i, since sum_j pi_{p,n,j} r_{p,j}(node)
// is the expected value at the node of the cash flows after it.
struct NestSlot {   // 64 bytes, one policy slot of a tile
    int32_t base1, age1, z1;   // life 1: float4 index of copy 0 of its staged array, its age at valuation,
                               // the first table entry that is zero (the table's end, +1 for deaths)
    int32_t base2, age2, z2;   // life 2 (K_JL, K_ANN2)
    int32_t S, pol;            // steps from valuation; pol -1 = padding
    float ix, iy, mat;         // as DeflSlot
    int32_t kind;
    float sc_h, sc_l;          // the scale as an FP32 head and tail
    int32_t unit;              // 1: alive past its table's end at valuation (death in the first month)
    int32_t pad;
};
static_assert(sizeof(NestSlot) == 64, "NestSlot layout");

struct NestDeflArgs {
    const float* tab;          // the deflated form's staged tables
    int32_t tab_bytes, dpad;
    const float4* D;           // [B][n_nodes][G4][i_pad]: D_i(m, m+tau+1) for tau = 4g .. 4g+3
    int32_t i_pad, n_inner, G4, n_nodes, node_step, B, o0;
    const NestSlot* slots;     // [n_tiles * P]
    const int32_t* tile_kind;
    int32_t n_tiles, n_chunks, n_items;
    int32_t* counter;
    int32_t* status;
    double* L_all;
};
constexpr int kNestDeflP = 4;   // policies per tile of the deflated nested kernel
// The generator runs ctas_per_sm CTAs of 128 threads per SM (grid-stride);
// the valuation kernel at most max_per_sm CTAs per SM, so that both fit on
// every SM when they run concurrently on two streams.
cudaError_t launch_inner_paths_defl(const VasStep& s, uint64_t seed, int o_first, int o0, int B, int n_nodes, int n_inner,
                                    int i_pad, int G4, const int* Ln, const double* r_node, const double2* bm,
                                    float4* plane, int sm_count, int ctas_per_sm, cudaStream_t st);
cudaError_t launch_nested_defl(const NestDeflArgs& a, int sm_count, int max_per_sm, cudaStream_t st);
cudaError_t launch_node_stats(const double* L_all, int n_on, int n_inner, int k, double* mean, double* kth,
                              cudaStream_t st);

}  // namespace rsv
