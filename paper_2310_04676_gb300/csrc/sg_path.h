// Path-following waypoint tables built on the device (sg_path.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "sg_internal.h"

namespace sg {

constexpr int kPathDense = 64;      // polyline samples per spline segment
constexpr int kPathWarps = 4;       // envs (one per warp) per block

size_t path_smem_bytes(int K);      // dynamic shared memory of one block
cudaError_t prepare_path_kernel();  // one-time kernel attributes (not capturable)
// Builds path [E][W][3] from ctrl [E][K][3] for envs with mask[e] != 0 (all when mask is null).
cudaError_t launch_build_paths(const float* ctrl, int K, const uint8_t* mask, int E, int W,
                               float* path, cudaStream_t stream);

}  // namespace sg
