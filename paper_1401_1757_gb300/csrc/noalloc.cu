// noalloc.cu -- rsv_reserves_noalloc: the compensated-FP32 valuation for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// is owned by another allocator (a fixed arena or pool that must stay the
// only owner), or latency-bound code that must not take cudaMalloc's implicit
// device-wide synchronisation in the middle of its work.  For them this entry
// point takes every input and output as the caller's device buffers and keeps
// its working memory in one file-scope device array, so it allocates nothing.
//
// Scratch (`g_rsv_noalloc_scratch`, kScratchBytes = 32 MiB; every GPU that
// loads the library holds it until the process exits), in this order:
//   control words                                 256 B
//   decrement table as (p hi, p lo, q hi, q lo)   4096 x 16 B = 64 KiB
//   scenario plane as (v hi, v lo), step-major     n_steps x s_pad x 8 B
//   one work record per policy (SlotRec)          n_pol x 32 B
//   reduced model per policy                      n_pol x 4 B
//   amount per policy                             n_pol x 8 B
//   per-group scenario sums (256 policies a group) ceil(n_pol / 256) x n_scen x 8 B
// (s_pad = n_scen rounded up to 128, every region aligned to 256 B.)
// Every call shares the array, which keeps the last call's contents; a call
// clears the control words first and rewrites every region before it reads
// it.  Calls whose GPU work overlaps (other streams, other host threads) race
// on the array and must be serialised by the caller.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "rsv.h"
#include "abi_guard.cuh"
#include "recur_kernel.cuh"

namespace rsv {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kTabEntries = 4096;                      // age + steps bound (as rsv_compute_reserves)
constexpr size_t kCtlBytes = 256;
constexpr int kGroup = 256;                            // policies per partial-sum group
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_rsv_noalloc_scratch[kScratchBytes];

// Control words.  CTL_BAD_ARG / CTL_BAD_ASM: the smallest index of a record
// that breaks an argument rule (RSV_E_ARG) / an assumption of Section 3.7
// (RSV_E_ASSUMPTION), INT32_MAX if none; the call reports the first bad record
// in portfolio order, as rsv_compute_reserves does.
enum { CTL_COUNTER = 0, CTL_STATUS = 1, CTL_BAD_ARG = 2, CTL_BAD_ASM = 3 };
enum : int32_t { NA_OK = 0, NA_TIMEOUT = DEV_TIMEOUT, NA_BAD_INPUT = 3 };

struct NaLayout {
    int32_t* ctl;
    float4* tab;
    float2* plane;
    SlotRec* slots;
    int32_t* kinds;
    double* amount;
    double* red;
    size_t end;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline size_t scen_pad(int n_scen) { return ((size_t)n_scen + 127) / 128 * 128; }

__host__ __device__ inline NaLayout carve(unsigned char* base, int n_pol, int n_scen, int n_steps) {
    NaLayout L;
    size_t off = 0;
    L.ctl = reinterpret_cast<int32_t*>(base + off);
    off += kCtlBytes;
    L.tab = reinterpret_cast<float4*>(base + off);
    off += align256((size_t)kTabEntries * sizeof(float4));
    L.plane = reinterpret_cast<float2*>(base + off);
    off += align256((size_t)n_steps * scen_pad(n_scen) * sizeof(float2));
    L.slots = reinterpret_cast<SlotRec*>(base + off);
    off += align256((size_t)n_pol * sizeof(SlotRec));
    L.kinds = reinterpret_cast<int32_t*>(base + off);
    off += align256((size_t)n_pol * sizeof(int32_t));
    L.amount = reinterpret_cast<double*>(base + off);
    off += align256((size_t)n_pol * sizeof(double));
    L.red = reinterpret_cast<double*>(base + off);
    off += ((size_t)n_pol + kGroup - 1) / kGroup * (size_t)n_scen * sizeof(double);
    L.end = off;
    return L;
}

// Bytes of scratch one call needs (the end of the carved layout).
inline size_t na_bytes(int n_pol, int n_scen, int n_steps) {
    return kCtlBytes + align256((size_t)kTabEntries * sizeof(float4)) +
           align256((size_t)n_steps * scen_pad(n_scen) * sizeof(float2)) + align256((size_t)n_pol * sizeof(SlotRec)) +
           align256((size_t)n_pol * sizeof(int32_t)) + align256((size_t)n_pol * sizeof(double)) +
           ((size_t)n_pol + kGroup - 1) / kGroup * (size_t)n_scen * sizeof(double);
}

// Table -> hi/lo pairs (zero survival past the table), scenarios -> hi/lo
// plane, one work record per policy; validation of all three.
__global__ void na_prepare_kernel(unsigned char* scratch, const rsv_policy* __restrict__ pols, int n_pol,
                                  const double* __restrict__ p_monthly, int n_ages, const double* __restrict__ v,
                                  int n_scen, int n_steps) {
    const NaLayout L = carve(scratch, n_pol, n_scen, n_steps);
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
    for (size_t k = tid; k < (size_t)kTabEntries; k += nth) {
        const double p = k < (size_t)n_ages ? p_monthly[k] : 0.0;
        if (!(p >= 0.0 && p <= 1.0)) atomicExch(&L.ctl[CTL_STATUS], NA_BAD_INPUT);
        const double q = 1.0 - p;
        const float ph = __double2float_rn(p), qh = __double2float_rn(q);
        L.tab[k] = make_float4(ph, __double2float_rn(p - (double)ph), qh, __double2float_rn(q - (double)qh));
    }
    const size_t sp = scen_pad(n_scen);
    for (size_t i = tid; i < (size_t)n_steps * sp; i += nth) {
        const int t = (int)(i / sp), s = (int)(i % sp);
        double x = 1.0;   // padding scenarios: any finite factor, never written out
        if (s < n_scen) {
            x = v[(size_t)t * n_scen + s];
            if (!(x > 0.0 && x < INFINITY)) atomicExch(&L.ctl[CTL_STATUS], NA_BAD_INPUT);
        }
        const float h = __double2float_rn(x);
        L.plane[i] = make_float2(h, __double2float_rn(x - (double)h));
    }
    for (size_t i = tid; i < (size_t)n_pol; i += nth) {
        const rsv_policy r = pols[i];
        const bool jl = r.product == RSV_JL_REVERSIONARY;
        // the checks of rsv_compute_reserves, in its order: argument rules,
        // then the assumptions (amount, reversion, scenario length), then the
        // table bound on age + steps
        bool ok = r.product >= RSV_SL_ANNUITY && r.product <= RSV_ENDOWMENT && r.reserved == 0 && r.table1 == 0 &&
                  (!jl || r.table2 == 0) && r.age1_m >= 0 && (!jl || r.age2_m >= 0) && r.term_m >= 0 &&
                  r.state0 >= 0 && r.state0 <= (jl ? 2 : 0);
        bool assumption = false;
        int S = 0;
        if (ok) {
            if (r.product == RSV_SL_ANNUITY) {
                S = max(0, n_ages - r.age1_m);
                if (r.term_m > 0) S = min(S, r.term_m);
            } else if (jl) {
                S = max(0, n_ages - min(r.age1_m, r.age2_m));
                if (r.term_m > 0) S = min(S, r.term_m);
            } else {
                S = r.term_m;
            }
            assumption = !isfinite(r.amount) || (jl && !(r.reversion >= 0.0 && r.reversion <= 1.0)) || S > n_steps;
            ok = !assumption && (long long)r.age1_m + S <= kTabEntries &&
                 (!jl || (long long)r.age2_m + S <= kTabEntries);
        }
        SlotRec s;
        s.idx1 = ok ? r.age1_m : 0;
        s.idx2 = (ok && jl) ? r.age2_m : 0;
        s.S = ok ? S : 0;
        s.pol = ok ? (int)i : -1;
        const double rho = (ok && jl) ? r.reversion : 0.0;
        s.rho_h = __double2float_rn(rho);
        s.rho_l = __double2float_rn(rho - (double)s.rho_h);
        s.state0 = ok ? r.state0 : 0;
        s.bnd = (ok && r.product == RSV_ENDOWMENT) ? 1.0f : 0.0f;
        L.slots[i] = s;
        L.kinds[i] = jl ? K_JL : (r.product == RSV_SL_ANNUITY ? K_ANN : K_ASS);
        L.amount[i] = ok ? r.amount : 0.0;
        if (!ok) atomicMin(&L.ctl[assumption ? CTL_BAD_ASM : CTL_BAD_ARG], (int)i);
    }
}

__global__ void na_init_ctl_kernel(int32_t* ctl) {
    if (threadIdx.x == 0) {
        ctl[CTL_COUNTER] = 0;
        ctl[CTL_STATUS] = NA_OK;
        ctl[CTL_BAD_ARG] = INT32_MAX;
        ctl[CTL_BAD_ASM] = INT32_MAX;
    }
}

// The compensated-form valuation kernel with its queue head, status word,
// table, plane and records in the scratch array: one policy x 32 scenarios
// per warp item, the tile template of the main kernels.
__global__ void __launch_bounds__(256) na_recur_kernel(unsigned char* scratch, int n_pol, int n_scen, int n_steps,
                                                       double* __restrict__ V0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const NaLayout L = carve(scratch, n_pol, n_scen, n_steps);
    float4* tab = reinterpret_cast<float4*>(smem_raw);
    if (!stage_to_smem(tab, L.tab, (uint32_t)(kTabEntries * sizeof(float4)), &bar, &L.ctl[CTL_STATUS])) return;
    const TileEnv env{L.slots, L.plane, scen_pad(n_scen), n_scen, n_steps, L.amount, nullptr, nullptr, n_scen};
    const int n_chunks = (n_scen + 31) / 32;
    const long long n_items = (long long)n_pol * n_chunks;
    const int lane = threadIdx.x & 31;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = atomicAdd(&L.ctl[CTL_COUNTER], 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int p = (int)(item / n_chunks), chunk = (int)(item % n_chunks);
        const int kind = L.kinds[p];
        if (kind == K_JL) {
            Tile<F_COMP, 1, 1, K_JL, false> w(env, tab, p, chunk, lane);
            w.run_steps();
            w.epilogue_v0(p, nullptr, V0, nullptr);
        } else if (kind == K_ANN) {
            Tile<F_COMP, 1, 1, K_ANN, false> w(env, tab, p, chunk, lane);
            w.run_steps();
            w.epilogue_v0(p, nullptr, V0, nullptr);
        } else {
            Tile<F_COMP, 1, 1, K_ASS, false> w(env, tab, p, chunk, lane);
            w.run_steps();
            w.epilogue_v0(p, nullptr, V0, nullptr);
        }
    }
}

// Per-scenario totals of V0 in a fixed order: sums over groups of 256
// policies into the scratch, then over the groups.
__global__ void na_group_sums_kernel(unsigned char* scratch, int n_pol, int n_scen, int n_steps,
                                     const double* __restrict__ V0) {
    const NaLayout L = carve(scratch, n_pol, n_scen, n_steps);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scen) return;
    const int g = blockIdx.y, p1 = min(n_pol, (g + 1) * kGroup);
    double acc = 0.0;
    for (int p = g * kGroup; p < p1; ++p) acc += V0[(size_t)p * n_scen + s];
    L.red[(size_t)g * n_scen + s] = acc;
}

__global__ void na_total_kernel(unsigned char* scratch, int n_pol, int n_scen, int n_steps, double* __restrict__ total) {
    const NaLayout L = carve(scratch, n_pol, n_scen, n_steps);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_scen) return;
    const int groups = (n_pol + kGroup - 1) / kGroup;
    double acc = 0.0;
    for (int g = 0; g < groups; ++g) acc += L.red[(size_t)g * n_scen + s];
    total[s] = acc;
}

// Device address of the scratch array, looked up once per device with that
// device current.  The name is only a host-side stand-in: the kernels are
// given this address, never the symbol.
std::mutex g_addr_mutex;
unsigned char* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int device, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_rsv_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

}  // namespace
}  // namespace rsv

using namespace rsv;

extern "C" rsv_status rsv_reserves_noalloc(int device, void* cuda_stream, const rsv_policy* pols, int32_t n_pol,
                                           const double* p_monthly, int32_t n_ages, const double* v, int32_t n_scen,
                                           int32_t n_steps, double* V0, double* scen_total) try {
    if (device < 0 || device >= kMaxDevices || n_pol < 0 || (n_pol > 0 && (!pols || !V0)) || !p_monthly ||
        n_ages < 1 || n_ages > kTabEntries || !v || n_scen < 1 || n_steps < 1)
        return RSV_E_ARG;
    // every size term is computed in 64-bit; a dimension that alone exceeds the
    // scratch is refused before the sum is formed
    if ((size_t)n_scen > kScratchBytes / sizeof(double) || (size_t)n_steps > kScratchBytes / sizeof(double) ||
        (size_t)n_pol > kScratchBytes / sizeof(SlotRec) || na_bytes(n_pol, n_scen, n_steps) > kScratchBytes)
        return RSV_E_LIMIT;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaSetDevice(device) != cudaSuccess) return RSV_E_CUDA;
    unsigned char* scratch = nullptr;
    if (scratch_address(device, &scratch) != cudaSuccess) return RSV_E_CUDA;
    int sms = 0, bps = 0;
    const size_t smem = (size_t)kTabEntries * sizeof(float4);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return RSV_E_CUDA;
    if (cudaFuncSetAttribute(na_recur_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSV_E_CUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, na_recur_kernel, 256, smem) != cudaSuccess || bps < 1)
        return RSV_E_CUDA;
    na_init_ctl_kernel<<<1, 32, 0, st>>>(reinterpret_cast<int32_t*>(scratch));
    if (cudaGetLastError() != cudaSuccess) return RSV_E_CUDA;
    na_prepare_kernel<<<sms * 4, 256, 0, st>>>(scratch, pols, n_pol, p_monthly, n_ages, v, n_scen, n_steps);
    if (cudaGetLastError() != cudaSuccess) return RSV_E_CUDA;
    if (n_pol > 0) {
        const long long items = (long long)n_pol * ((n_scen + 31) / 32);
        const long long grid = std::min<long long>((long long)sms * bps, (items * 32 + 255) / 256);
        na_recur_kernel<<<(int)grid, 256, smem, st>>>(scratch, n_pol, n_scen, n_steps, V0);
        if (cudaGetLastError() != cudaSuccess) return RSV_E_CUDA;
    }
    if (scen_total) {
        if (n_pol > 0) {
            dim3 g1((n_scen + 127) / 128, (n_pol + kGroup - 1) / kGroup);
            na_group_sums_kernel<<<g1, 128, 0, st>>>(scratch, n_pol, n_scen, n_steps, V0);
            if (cudaGetLastError() != cudaSuccess) return RSV_E_CUDA;
        }
        na_total_kernel<<<(n_scen + 127) / 128, 128, 0, st>>>(scratch, n_pol, n_scen, n_steps, scen_total);
        if (cudaGetLastError() != cudaSuccess) return RSV_E_CUDA;
    }
    int32_t ctl[4] = {0, 0, 0, 0};
    if (cudaMemcpyAsync(ctl, scratch, sizeof ctl, cudaMemcpyDeviceToHost, st) != cudaSuccess) return RSV_E_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RSV_E_CUDA;
    if (ctl[CTL_STATUS] == NA_TIMEOUT) return RSV_E_TIMEOUT;
    if (ctl[CTL_STATUS] == NA_BAD_INPUT) return RSV_E_ASSUMPTION;   // a table entry or discount factor
    if (ctl[CTL_BAD_ARG] != INT32_MAX || ctl[CTL_BAD_ASM] != INT32_MAX)
        return ctl[CTL_BAD_ARG] < ctl[CTL_BAD_ASM] ? RSV_E_ARG : RSV_E_ASSUMPTION;
    return RSV_OK;
} catch (...) {
    return rsv::host_error(nullptr);
}
