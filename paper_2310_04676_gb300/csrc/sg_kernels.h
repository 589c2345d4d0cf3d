// Kernel launchers (implemented in sg_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "sg_internal.h"

namespace sg {

struct StateArgs {
  const int32_t* slot_env;
  const int32_t* slot_info;
  float* q;
  float* qd;
  const float* q0;
  int32_t* step_count;
  float* track;             // [6][NS] goal offset / velocity (tracking task), or null
  int num_slots, max_joints;
};

constexpr int kMaxThreads = 256;   // largest step-kernel block

constexpr int kMaxObsDim = 127;    // widest observation row the step kernels stage

// Row pitch (floats) of the per-warp observation stage: rows keep 8-byte
// alignment when D is even; otherwise an odd pitch avoids bank conflicts.
SG_HD inline int stage_pitch(int obs_dim) {
  return (obs_dim & 1) ? obs_dim : (obs_dim % 4 == 0 ? obs_dim + 2 : obs_dim);
}

size_t step_smem_bytes(int threads, int obs_dim);
cudaError_t prepare_step_kernel();   // one-time kernel attributes (not capturable)
cudaError_t launch_step(const StepArgs& a, int threads, cudaStream_t stream);
// warp-pair variant (sg_pair.cu): threads must be a multiple of 64
size_t step_pair_smem_bytes(int threads, int obs_dim);
cudaError_t prepare_step_pair_kernel();
cudaError_t launch_step_pair(const StepArgs& a, int threads, cudaStream_t stream);
cudaError_t launch_reset(const StateArgs& s, const uint8_t* mask, cudaStream_t stream);
cudaError_t launch_get_state(const StateArgs& s, float* q, float* qd, int32_t* sc,
                             cudaStream_t stream);
cudaError_t launch_set_state(const StateArgs& s, const float* q, const float* qd,
                             const int32_t* sc, cudaStream_t stream);
// copies the tracking-task goal state out (off, vel) and/or in (off_in, vel_in)
cudaError_t launch_goal_state(const StateArgs& s, float* off, float* vel, const float* off_in,
                              const float* vel_in, cudaStream_t stream);

}  // namespace sg
