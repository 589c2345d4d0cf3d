// Differentiable rollout kernels (implemented in sg_diff.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "sg_internal.h"

namespace sg {

constexpr int kDiffThreads = 128;
constexpr int kDiffPairThreads = 64;       // warp-pair forward: one pair per block
constexpr int kDiffPairMaxWarpsPerSM = 2;  // warp-pair forward up to this many chain warps per SM
constexpr int kReplayWarps = 2;        // replay warps per group of 32 chains
constexpr int kDiffPipeThreads = 256;  // two groups (replay warps + adjoint) in 8 warp slots
// per substep record: q, qd, cos q, sin q, k_s, 1/L_ii (7 each), L (21), per
// link the inverse-dynamics sweep quantities w, wd, acc, F, N, f, n (21 each),
// and (in a step's last substep record) the tool-tip Jacobian of the state
// after the step (21)
constexpr int kReplayFields = 231;
constexpr int kReplayBufs = kReplayWarps + 1;   // segment buffers in flight
constexpr int kMaxCkptEvery = 32;      // checkpoint interval limit (thread-local segment buffer)
constexpr int kMaxDiffSubsteps = 16;   // substeps limit of the differentiable rollout

struct DiffArgs {
  const float* params;
  const int32_t* slot_env;
  const int32_t* slot_info;
  const int32_t* warp_class;
  const float* q;          // start state [kMaxLinks][NS]
  const float* qd;
  float* ckpt;             // [nseg + 1][2 * kMaxLinks][NS]
  const float* actions;    // [T][E][J]
  float* ee;               // [T][E][kMaxChains][3]   (forward output)
  const float* dl_dee;     // [T][E][kMaxChains][3]   (backward input)
  float* dactions;         // [T][E][J]         (backward output)
  float* dmass;            // [E][J]            (backward output)
  float* dq0;              // [E][J] or null    (backward output)
  float* dqd0;             // [E][J] or null    (backward output)
  float* replay;           // [kReplayBufs][groups][ckpt_every * substeps][kReplayFields][32] or null
  int32_t* err;
  int prefilled;           // backward: buffer 0 holds the last segment's records (forward wrote them)
  int num_warps, num_slots, num_envs, max_joints, T, substeps, ckpt_every, nseg;
  float h;
};

constexpr size_t kMaxReplayFloats = (size_t)1 << 28;   // 1 GiB of replay buffers at most

// Floats of the replay buffers of the pipelined backward kernel.
inline size_t replay_floats(int ckpt_every, int substeps, int num_slots) {
  return (size_t)kReplayBufs * ckpt_every * substeps * kReplayFields * num_slots;
}

struct MassArgs {
  float* params;
  const int32_t* slot_env;
  const int32_t* slot_info;
  const float* mass;       // caller [E][J]
  const float* mass0;      // [kMaxLinks][NS] masses of the description
  const float* inertia0;   // [3][kMaxLinks][NS] inertias of the description
  int num_slots, max_joints;
};

// Context accessors for entry points implemented outside sg_api.cu:
// the context's parameter/state/slot pointers and sizes (shape fields zero).
DiffArgs context_diff_args(sg_ctx* ctx);
void context_set_error(sg_ctx* ctx, const char* msg);
// SG_OK if the context's device is current; else an error (message set) naming fn
sg_status context_check_device(sg_ctx* ctx, const char* fn);
cudaStream_t context_stream(sg_ctx* ctx);
// the context's device error word (DEVERR_* flags, read by sg_sync_status)
int32_t* context_err(sg_ctx* ctx);
// total joints of every env [E] (host copy of the description)
const std::vector<int32_t>& context_env_dof(sg_ctx* ctx);

cudaError_t prepare_diff_kernels();
cudaError_t launch_diff_forward(const DiffArgs& a, cudaStream_t s);
// Reverse pass: with a.replay set, the pipelined kernel (kReplayWarps warps
// replay the next segments' substeps while another runs the adjoint of the
// current one); otherwise the one-warp kernel.
cudaError_t launch_diff_backward(const DiffArgs& a, cudaStream_t s);
cudaError_t launch_set_mass(const MassArgs& m, cudaStream_t s);

}  // namespace sg
