// sg_diff_track_noalloc: the tracking-loss gradient of the differentiable
// rollout without any device allocation.
//
// Why: sg_diff_forward allocates its checkpoint buffer with cudaMalloc on
// first use.  Some callers cannot allocate device memory at the point where
// they need gradients -- e.g. a control or training loop embedded in a host
// application that hands out all device memory from its own pre-reserved
// pool and forbids allocations after start-up, or code that must not
// synchronise the device (cudaMalloc/cudaFree may).  This entry point takes
// its scratch space (checkpoints and the loss cotangent) from a fixed,
// file-scope __device__ array instead, so it allocates nothing.
//
// The scratch array is part of the library image: every GPU that loads
// libsg.so holds kNoAllocScratchBytes (32 MiB) of device memory for it until
// the process exits.  All calls on a device share that one array, which
// keeps the last call's contents; calls whose GPU work overlaps (two
// streams, two host threads, or two contexts on the same device) race on it
// and must be serialised by the caller.  Every entry that a call reads is
// written earlier in the same call, so nothing needs clearing between calls.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "sg.h"
#include "sg_diff.h"
#include "sg_internal.h"

namespace sg {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kNoAllocScratchFloats = kNoAllocScratchBytes / sizeof(float);

// The scratch array.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress (noalloc_scratch()).
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on
// the first call of the entry point on that device and cached.  The cached
// address is checked against the runtime before use (it becomes invalid if
// the program resets the device, which unloads the library's module); an
// address the runtime no longer knows is looked up again.
cudaError_t noalloc_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (g_scratch_ptr[dev]) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, g_scratch_ptr[dev]) != cudaSuccess ||
        attr.type != cudaMemoryTypeDevice || attr.device != dev) {
      cudaGetLastError();          // clear the error of an unknown pointer
      g_scratch_ptr[dev] = nullptr;
    }
  }
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// One thread per chain slot (warps aligned with the packing): dL/d(ee) =
// 2 (ee - target) for the slot's chain, and the per-env loss
// sum_t sum_c ||ee_c - target_c||^2 (the chains of a multi-arm env sit in
// one lane group and are summed with shuffles).
__global__ void track_seed_kernel(DiffArgs a, const float* ee, const float* target,
                                  float* dl_dee, float* loss) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  const int gw = slot / kWarp;
  if (gw >= a.num_warps) return;                 // whole warps only (slots are warp-padded)
  const int glog = group_log2(a.warp_class[gw]);
  const int env = a.slot_env[slot];
  const int c = decode_slot(a.slot_info[slot]).c;
  const size_t E = (size_t)a.num_envs;
  float acc = 0.f;
  if (env >= 0) {
    for (int t = 0; t < a.T; ++t) {
      const size_t base = (((size_t)t * E + env) * kMaxChains + c) * 3;
      for (int k = 0; k < 3; ++k) {
        const float d = ee[base + k] - target[base + k];
        dl_dee[base + k] = 2.f * d;
        acc += d * d;
      }
    }
  }
  for (int off = 1; off < (1 << glog); off <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (env >= 0 && c == 0) loss[env] = acc;
}

}  // namespace
}  // namespace sg

extern "C" sg_status sg_diff_track_noalloc(sg_ctx* ctx, const float* actions_dev, int32_t T,
                                           float dt, int32_t substeps, int32_t ckpt_every,
                                           const float* target_dev, float* ee_dev,
                                           float* loss_dev, float* dactions_dev,
                                           float* dmass_dev) {
  using namespace sg;
  if (!ctx) return SG_ERR_INVALID_ARG;
  const sg_status st_dev = context_check_device(ctx, "sg_diff_track_noalloc");
  if (st_dev != SG_OK) return st_dev;
  auto fail = [&](sg_status st, const char* msg) {
    context_set_error(ctx, msg);
    return st;
  };
  if (!actions_dev || !target_dev || !ee_dev || !loss_dev || !dactions_dev || !dmass_dev)
    return fail(SG_ERR_INVALID_ARG, "sg_diff_track_noalloc: all arrays must be non-NULL");
  if (T < 1 || T > 4096) return fail(SG_ERR_INVALID_ARG, "sg_diff_track_noalloc: T must be 1..4096");
  if (!(dt > 0.f) || !std::isfinite(dt))
    return fail(SG_ERR_INVALID_ARG, "sg_diff_track_noalloc: dt must be > 0");
  if (substeps < 1 || substeps > kMaxDiffSubsteps)
    return fail(SG_ERR_INVALID_ARG, "sg_diff_track_noalloc: substeps must be 1..16");
  if (ckpt_every < 1 || ckpt_every > kMaxCkptEvery)
    return fail(SG_ERR_INVALID_ARG, "sg_diff_track_noalloc: ckpt_every must be 1..32");
  DiffArgs a = context_diff_args(ctx);
  const int nseg = (T + ckpt_every - 1) / ckpt_every;
  const size_t ckpt_floats = (size_t)(nseg + 1) * 2 * kMaxLinks * a.num_slots;
  const size_t seed_floats = (size_t)T * a.num_envs * 3 * kMaxChains;
  if (ckpt_floats + seed_floats > kNoAllocScratchFloats)
    return fail(SG_ERR_INVALID_ARG,
                "sg_diff_track_noalloc: checkpoints + loss cotangent exceed the 32 MiB static "
                "scratch (reduce T, envs, or raise ckpt_every)");
  float* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) {
    context_set_error(ctx, cudaGetErrorString(e));
    return SG_ERR_CUDA;
  }
  cudaStream_t s = context_stream(ctx);
  a.T = T;
  a.substeps = substeps;
  a.ckpt_every = ckpt_every;
  a.nseg = nseg;
  a.h = dt / (float)substeps;
  a.ckpt = scratch;
  a.actions = actions_dev;
  a.ee = ee_dev;
  e = launch_diff_forward(a, s);
  float* dl_dee = scratch + ckpt_floats;
  if (e == cudaSuccess) {
    const int threads = 128;
    track_seed_kernel<<<(a.num_slots + threads - 1) / threads, threads, 0, s>>>(
        a, ee_dev, target_dev, dl_dee, loss_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    a.dl_dee = dl_dee;
    a.dactions = dactions_dev;
    a.dmass = dmass_dev;
    a.dq0 = nullptr;
    a.dqd0 = nullptr;
    e = launch_diff_backward(a, s);
  }
  if (e != cudaSuccess) {
    context_set_error(ctx, cudaGetErrorString(e));
    return SG_ERR_CUDA;
  }
  return SG_OK;
}
