// probe.cu -- device diagnostics: the measured FP32 and FP64 fused
// multiply-add throughput (the denominators of the ALU rooflines beside the
// nominal ones, SMs x lanes x 2 x clock), and a self-test of the bounded
// device-side wait the kernels use for their bulk-copy staging.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "rsv.h"
#include "abi_guard.cuh"
#include "rsv_device.cuh"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread
constexpr int kIters = 4096;    // loop trips, 16 FMAs per chain each

__device__ __forceinline__ float fma_rn(float x, float a, float b) { return __fmaf_rn(x, a, b); }
__device__ __forceinline__ double fma_rn(double x, double a, double b) { return __fma_rn(x, a, b); }

// Each thread runs kChains independent chains x = fma(x, a, b); the result
// is written only if impossible (keeps the compiler from removing the work).
template <class T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T a, T b, T* sink) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma_rn(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-12345.0) sink[threadIdx.x] = s;
}

template <class T>
rsv_status probe(int device, cudaStream_t st, double* tflops) {
    int sms = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return RSV_E_CUDA;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fma_probe_kernel<T>, 256, 0) != cudaSuccess)
        return RSV_E_CUDA;
    T* sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(T)) != cudaSuccess) return RSV_E_NOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int grid = sms * bps;
    const T a = (T)0.999999, b = (T)1e-7;
    fma_probe_kernel<T><<<grid, 256, 0, st>>>(a, b, sink);   // warm-up
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, st);
        fma_probe_kernel<T><<<grid, 256, 0, st>>>(a, b, sink);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (err != cudaSuccess) return RSV_E_CUDA;
    const double flops = 2.0 * kChains * 16.0 * kIters * 256.0 * grid;
    *tflops = flops / (best * 1e-3) / 1e12;
    return RSV_OK;
}

// One CTA stages n16 x 16 bytes into shared memory with the bulk-copy and
// mbarrier primitives of the kernels' table staging, declaring extra_tx bytes
// more than it copies (0: a normal staging).  With extra_tx > 0 the barrier's
// phase cannot complete: the bounded wait runs out after `limit` polls, the
// kernel records DEV_TIMEOUT and returns.  Every copy it issued still lands
// (the second bounded wait gives them time), so nothing is left in flight.
// On success the staged bytes are copied back out for the host to compare.
__global__ void __launch_bounds__(128) wait_selftest_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                            int n16, uint32_t extra_tx, uint32_t limit,
                                                            int32_t* status) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t bar;
    const uint32_t bytes = (uint32_t)n16 * 16u;
    if (threadIdx.x == 0) {
        rsv::mbar_init(&bar, 1);
        rsv::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        rsv::mbar_arrive_expect_tx(&bar, bytes + extra_tx);
        for (uint32_t off = 0; off < bytes; off += rsv::kBulkChunk) {
            const uint32_t n = bytes - off < rsv::kBulkChunk ? bytes - off : rsv::kBulkChunk;
            rsv::bulk_g2s(smem + off, reinterpret_cast<const char*>(src) + off, n, &bar);
        }
    }
    bool ok = rsv::mbar_wait_bounded(&bar, 0, limit);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(status, rsv::DEV_TIMEOUT);
        rsv::mbar_wait_bounded(&bar, 0, limit);   // the copies issued land before the CTA exits
        __syncthreads();
        return;
    }
    const uint4* s4 = reinterpret_cast<const uint4*>(smem);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = s4[i];
}

}  // namespace

extern "C" rsv_status rsv_selftest_bounded_wait(int32_t device, void* cuda_stream, int32_t never_completes) try {
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (cudaSetDevice(device) != cudaSuccess) return RSV_E_CUDA;
    constexpr int n16 = 1024;   // 16 KiB
    uint4 *src = nullptr, *dst = nullptr;
    int32_t* status = nullptr;
    if (cudaMalloc(&src, n16 * 16) != cudaSuccess) return RSV_E_NOMEM;
    if (cudaMalloc(&dst, n16 * 16) != cudaSuccess || cudaMalloc(&status, 4) != cudaSuccess) {
        cudaFree(src);
        cudaFree(dst);
        return RSV_E_NOMEM;
    }
    std::vector<uint32_t> h(n16 * 4), back(n16 * 4);
    for (size_t i = 0; i < h.size(); ++i) h[i] = (uint32_t)(i * 2654435761u + 12345u);
    rsv_status rc = RSV_OK;
    int32_t dev_status = 0;
    if (cudaMemcpyAsync(src, h.data(), n16 * 16, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(dst, 0, n16 * 16, st) != cudaSuccess || cudaMemsetAsync(status, 0, 4, st) != cudaSuccess) {
        rc = RSV_E_CUDA;
    } else {
        wait_selftest_kernel<<<1, 128, n16 * 16, st>>>(src, dst, n16, never_completes ? 16u : 0u, 1u << 16, status);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(&dev_status, status, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(back.data(), dst, n16 * 16, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            rc = RSV_E_CUDA;
        else if (dev_status == rsv::DEV_TIMEOUT)
            rc = RSV_E_TIMEOUT;
        else if (back != h)
            rc = RSV_E_CUDA;   // the staged bytes did not round-trip
    }
    cudaFree(src);
    cudaFree(dst);
    cudaFree(status);
    return rc;
} catch (...) {
    return rsv::host_error(nullptr);
}

extern "C" rsv_status rsv_probe_fma_peak(int32_t device, void* cuda_stream, int32_t fp64, double* tflops) try {
    if (!tflops) return RSV_E_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return fp64 ? probe<double>(device, st, tflops) : probe<float>(device, st, tflops);
} catch (...) {
    return rsv::host_error(nullptr);
}
