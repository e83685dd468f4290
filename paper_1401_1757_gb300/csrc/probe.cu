// probe.cu -- measured FP32 and FP64 fused multiply-add throughput of the
// device, the denominators of the ALU rooflines beside the nominal ones
// (SMs x lanes x 2 x clock).
#include <cuda_runtime.h>

#include <cstdint>

#include "rsv.h"

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

}  // namespace

extern "C" rsv_status rsv_probe_fma_peak(int32_t device, void* cuda_stream, int32_t fp64, double* tflops) {
    if (!tflops) return RSV_E_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return fp64 ? probe<double>(device, st, tflops) : probe<float>(device, st, tflops);
}
