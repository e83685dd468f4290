// summation.cuh -- launcher of the FP64 summation-definition kernel (summation.cu).
#pragma once

#include <cuda_runtime.h>

#include "rsv_device.cuh"

namespace rsv {
// A persistent grid over (tile of one policy, scenario, block of 32 steps)
// items, a.n_items = n_tiles * n_scen * warps_per_chain_max; the FP64
// decrement tables (smem bytes) are staged per CTA.
cudaError_t launch_summation(const RecurArgs& a, int warps_per_chain_max, int sm_count, size_t smem,
                             cudaStream_t st);
}  // namespace rsv
