// scan.cuh -- launcher of the FP64 parallel-in-time scan (scan.cu).
#pragma once

#include <cuda_runtime.h>

#include "rsv_device.cuh"

namespace rsv {
// A persistent grid over tiles of one policy x scenarios (a.n_items of them);
// the FP64 decrement tables (smem bytes) are staged per CTA.
cudaError_t launch_scan(const RecurArgs& a, int sm_count, size_t smem, cudaStream_t st);
}  // namespace rsv
