// C ABI of libsg.so (declared in include/sg.h): context management, argument
// validation and kernel launches.  All device work goes to the context's
// stream; no call synchronises except sg_create, sg_destroy and
// sg_sync_status.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg.h"
#include "sg_devcheck.h"
#include "sg_internal.h"
#include "sg_pack.h"
#include "sg_diff.h"
#include "sg_kernels.h"
#include "sg_path.h"

struct sg_ctx {
  sg::Plan plan;
  int device = -1;                 // CUDA device current at sg_create (owns everything below)
  cudaStream_t stream = nullptr;
  float* d_params = nullptr;
  float* d_q = nullptr;
  float* d_qd = nullptr;
  float* d_q0 = nullptr;
  float* d_path = nullptr;
  int32_t* d_slot_env = nullptr;
  int32_t* d_slot_info = nullptr;
  int32_t* d_warp_class = nullptr;
  int32_t* d_step_count = nullptr;
  int32_t* d_err = nullptr;
  float* d_track = nullptr;        // [6][NS] goal offset / velocity (tracking task)
  int threads = 128;
  int rollout_mode = SG_ROLLOUT_PERSISTENT;
  int split = 1;
  int packing = SG_PACK_CLASS;
  std::vector<int32_t> warp_order;   // position w holds warp warp_order[w] of the plan's order
  int host_io = SG_HOST_IO_AUTO;
  int fault = sg::FAULT_NONE;      // test hook (sg_debug_set_fault)
  unsigned long long wait_ns = sg::kDefaultWaitNs;
  // pipelined host rollout: copy streams and events
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  cudaEvent_t host_ev[2 + 2 * 8] = {};
  std::string last_error;
  // captured rollout (CUDA graph) and the arguments it was captured for
  cudaStream_t capture_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  struct Key {
    const float* actions;
    float* obs;
    float* reward;
    uint8_t* done;
    int T, substeps, threads, mode, split, fault;
    unsigned long long wait_ns;
    float dt;
    bool operator==(const Key& o) const {
      return actions == o.actions && obs == o.obs && reward == o.reward && done == o.done &&
             T == o.T && substeps == o.substeps && threads == o.threads && mode == o.mode &&
             split == o.split && fault == o.fault && wait_ns == o.wait_ns && dt == o.dt;
    }
  } graph_key{};
  // device staging for sg_rollout_host
  float* d_stage_act = nullptr;
  float* d_stage_obs = nullptr;
  float* d_stage_rew = nullptr;
  uint8_t* d_stage_done = nullptr;
  int stage_T = 0;
  // description masses / inertias (for sg_set_link_mass)
  float* d_mass0 = nullptr;
  float* d_inertia0 = nullptr;
  // differentiable rollout: checkpoint scratch and the last forward's shape
  float* d_ckpt = nullptr;
  size_t ckpt_floats = 0;
  float* d_replay = nullptr;       // pipelined backward: segment buffers of substep records
  size_t replay_floats = 0;
  bool use_replay = false;
  bool replay_prefilled = false;   // replay buffer 0 holds the last forward's last segment
  bool diff_ready = false;
  int diff_T = 0, diff_substeps = 0, diff_every = 0;
  float diff_dt = 0.f;
  // state snapshot for the autotuner
  float* d_snap_q = nullptr;
  float* d_snap_qd = nullptr;
  int32_t* d_snap_sc = nullptr;
};

namespace {

thread_local std::string g_create_error;

constexpr int kHostChunks = 8;                    // pipelined host rollout: chunks of steps
constexpr int kHostEvents = 2 + 2 * kHostChunks;

sg_status set_err(sg_ctx* ctx, sg_status code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

// SG_OK if the context's device is current, else an error naming entry point fn.
sg_status on_device(sg_ctx* ctx, const char* fn) {
  std::string msg;
  const sg_status st = sg::check_device(
      ctx->device, [](int* d) { return (int)cudaGetDevice(d); }, fn, &msg);
  if (st != SG_OK) set_err(ctx, st, msg);
  return st;
}

#define SG_CHECK_DEVICE(ctx, fn)                   \
  do {                                             \
    const sg_status st_dev_ = on_device(ctx, fn);  \
    if (st_dev_ != SG_OK) return st_dev_;          \
  } while (0)

sg_status cuda_err(sg_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SG_OK;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return set_err(ctx, e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA, m);
}

template <class T>
cudaError_t upload(T** dst, const T* src, size_t n, cudaStream_t s) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), sizeof(T) * (n ? n : 1));
  if (e != cudaSuccess) return e;
  if (n && src) return cudaMemcpyAsync(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, s);
  return cudaSuccess;
}

// Device address of page-locked host memory the current device can access,
// or null (pageable or unknown memory: use staged copies).
void* device_view(const void* host) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, host) != cudaSuccess) {
    cudaGetLastError();   // clear the sticky-free error of an unknown pointer
    return nullptr;
  }
  if (attr.type != cudaMemoryTypeHost || !attr.devicePointer) return nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  int mapped = 0;
  if (cudaDeviceGetAttribute(&mapped, cudaDevAttrCanMapHostMemory, dev) != cudaSuccess || !mapped)
    return nullptr;
  return attr.devicePointer;
}

void free_ctx(sg_ctx* c) {
  if (!c) return;
  for (cudaEvent_t ev : c->host_ev)
    if (ev) cudaEventDestroy(ev);
  if (c->h2d_stream) cudaStreamDestroy(c->h2d_stream);
  if (c->d2h_stream) cudaStreamDestroy(c->d2h_stream);
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  void* ptrs[] = {c->d_params, c->d_q, c->d_qd, c->d_q0, c->d_path, c->d_slot_env, c->d_track,
                  c->d_slot_info, c->d_warp_class, c->d_step_count, c->d_err,
                  c->d_stage_act, c->d_stage_obs, c->d_stage_rew, c->d_stage_done,
                  c->d_snap_q, c->d_snap_qd, c->d_snap_sc, c->d_mass0, c->d_inertia0,
                  c->d_ckpt, c->d_replay};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

sg::StateArgs state_args(sg_ctx* c) {
  sg::StateArgs s;
  s.slot_env = c->d_slot_env;
  s.slot_info = c->d_slot_info;
  s.q = c->d_q;
  s.qd = c->d_qd;
  s.q0 = c->d_q0;
  s.step_count = c->d_step_count;
  s.track = c->d_track;
  s.num_slots = c->plan.num_slots;
  s.max_joints = c->plan.max_joints;
  return s;
}

sg::StepArgs step_args(sg_ctx* c, float dt, int substeps, int T) {
  sg::StepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.params = c->d_params;
  a.slot_env = c->d_slot_env;
  a.slot_info = c->d_slot_info;
  a.warp_class = c->d_warp_class;
  a.q = c->d_q;
  a.qd = c->d_qd;
  a.step_count = c->d_step_count;
  a.path = c->d_path;
  a.err = c->d_err;
  a.num_warps = c->plan.num_warps;
  a.num_slots = c->plan.num_slots;
  a.num_envs = c->plan.num_envs;
  a.max_joints = c->plan.max_joints;
  a.obs_dim = c->plan.obs_dim;
  a.task = c->plan.task;
  a.path_len = c->plan.path_len;
  a.episode_len = c->plan.episode_len;
  a.alpha = c->plan.alpha;
  a.track = c->d_track;
  a.seed = c->plan.seed;
  a.track_sigma = c->plan.track_sigma;
  a.track_limit = c->plan.track_limit;
  a.substeps = substeps;
  a.T = T;
  a.h = dt / (float)substeps;
  a.fault = c->fault;
  a.wait_ns = c->wait_ns;
  return a;
}

sg_status check_step_args(sg_ctx* ctx, const void* actions, float dt, int substeps,
                          const void* obs, const void* rew, const void* done) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  if (!actions || !obs || !rew || !done)
    return set_err(ctx, SG_ERR_INVALID_ARG, "actions, obs, reward and done must be non-NULL");
  if (!(dt > 0.f) || !std::isfinite(dt)) return set_err(ctx, SG_ERR_INVALID_ARG, "dt must be > 0");
  if (substeps < 1 || substeps > 64)
    return set_err(ctx, SG_ERR_INVALID_ARG, "substeps must be 1..64");
  return SG_OK;
}

bool valid_threads(int t) { return t == 32 || t == 64 || t == 128 || t == 256; }

cudaError_t launch_plan(const sg_ctx* c, const sg::StepArgs& a, cudaStream_t s) {
  return c->split == 2 ? sg::launch_step_pair(a, c->threads, s)
                       : sg::launch_step(a, c->threads, s);
}

// Host rollout as a pipeline of chunks of steps: copy-in of chunk c + 1 (h2d
// stream), the persistent kernel of chunk c (context stream) and copy-out of
// chunk c - 1 (d2h stream) overlap; events order each chunk's three stages,
// and the context stream waits for the last copy-out.  The chunked launches
// compute the same bits as one launch (state is stored and reloaded exactly
// between launches).
sg_status pipelined_host_rollout(sg_ctx* c, const float* act_h, int T, float dt, int substeps,
                                 float* obs_h, float* rew_h, uint8_t* done_h) {
  const size_t E = c->plan.num_envs, J = c->plan.max_joints, D = c->plan.obs_dim;
  const int nch = T < kHostChunks ? T : kHostChunks;
  const int len = (T + nch - 1) / nch;
  cudaError_t e = cudaSuccess;
  if (!c->h2d_stream) e = cudaStreamCreateWithFlags(&c->h2d_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && !c->d2h_stream)
    e = cudaStreamCreateWithFlags(&c->d2h_stream, cudaStreamNonBlocking);
  for (int k = 0; k < kHostEvents && e == cudaSuccess; ++k)
    if (!c->host_ev[k]) e = cudaEventCreateWithFlags(&c->host_ev[k], cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_err(c, e, "sg_rollout_host: streams");
  // both copy streams start after the work already queued on the context stream
  cudaEvent_t start = c->host_ev[0], fin = c->host_ev[1];
  e = cudaEventRecord(start, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->h2d_stream, start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->d2h_stream, start, 0);
  for (int k = 0; k < nch && e == cudaSuccess; ++k) {
    const int t0 = k * len, t1 = t0 + len < T ? t0 + len : T;
    if (t0 >= t1) break;
    const size_t n = (size_t)(t1 - t0);
    cudaEvent_t in = c->host_ev[2 + 2 * k], done_k = c->host_ev[3 + 2 * k];
    e = cudaMemcpyAsync(c->d_stage_act + (size_t)t0 * E * J, act_h + (size_t)t0 * E * J,
                        sizeof(float) * n * E * J, cudaMemcpyHostToDevice, c->h2d_stream);
    if (e == cudaSuccess) e = cudaEventRecord(in, c->h2d_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, in, 0);
    if (e == cudaSuccess) {
      sg::StepArgs a = step_args(c, dt, substeps, (int)n);
      a.actions = c->d_stage_act + (size_t)t0 * E * J;
      a.obs = c->d_stage_obs + (size_t)t0 * E * D;
      a.reward = c->d_stage_rew + (size_t)t0 * E;
      a.done = c->d_stage_done + (size_t)t0 * E;
      e = launch_plan(c, a, c->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(done_k, c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->d2h_stream, done_k, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(obs_h + (size_t)t0 * E * D, c->d_stage_obs + (size_t)t0 * E * D,
                          sizeof(float) * n * E * D, cudaMemcpyDeviceToHost, c->d2h_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(rew_h + (size_t)t0 * E, c->d_stage_rew + (size_t)t0 * E,
                          sizeof(float) * n * E, cudaMemcpyDeviceToHost, c->d2h_stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(done_h + (size_t)t0 * E, c->d_stage_done + (size_t)t0 * E, n * E,
                          cudaMemcpyDeviceToHost, c->d2h_stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(fin, c->d2h_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, fin, 0);
  return cuda_err(c, e, "sg_rollout_host");
}

// Enqueue (capturing first if needed) the rollout graph on the context's stream.
sg_status run_rollout(sg_ctx* c, const float* actions, int T, float dt, int substeps, float* obs,
                      float* rew, uint8_t* done) {
  const sg_ctx::Key key{actions, obs, rew, done, T, substeps, c->threads, c->rollout_mode,
                        c->split, c->fault, c->wait_ns, dt};
  if (!c->graph_exec || !(key == c->graph_key)) {
    if (c->graph_exec) {
      cudaGraphExecDestroy(c->graph_exec);
      c->graph_exec = nullptr;
    }
    cudaError_t e = cudaSuccess;
    if (!c->capture_stream) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_err(c, e, "sg_rollout: capture stream");
    e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_err(c, e, "sg_rollout: begin capture");
    cudaError_t le = cudaSuccess;
    const size_t E = c->plan.num_envs, J = c->plan.max_joints, D = c->plan.obs_dim;
    if (c->rollout_mode == SG_ROLLOUT_PERSISTENT) {
      sg::StepArgs a = step_args(c, dt, substeps, T);
      a.actions = actions;
      a.obs = obs;
      a.reward = rew;
      a.done = done;
      le = launch_plan(c, a, c->capture_stream);
    } else {
      for (int t = 0; t < T && le == cudaSuccess; ++t) {
        sg::StepArgs a = step_args(c, dt, substeps, 1);
        a.actions = actions + (size_t)t * E * J;
        a.obs = obs + (size_t)t * E * D;
        a.reward = rew + (size_t)t * E;
        a.done = done + (size_t)t * E;
        le = launch_plan(c, a, c->capture_stream);
      }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->capture_stream, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->graph_exec = nullptr;
      return cuda_err(c, e, "sg_rollout: capture");
    }
    c->graph_key = key;
  }
  return cuda_err(c, cudaGraphLaunch(c->graph_exec, c->stream), "sg_rollout: graph launch");
}

sg_status check_rollout_args(sg_ctx* ctx, const void* actions, int T, float dt, int substeps,
                             const void* obs, const void* rew, const void* done) {
  sg_status st = check_step_args(ctx, actions, dt, substeps, obs, rew, done);
  if (st != SG_OK) return st;
  if (T < 1 || T > 4096) return set_err(ctx, SG_ERR_INVALID_ARG, "T must be 1..4096");
  return SG_OK;
}

template <class T>
cudaError_t ensure(T** p, size_t n) {
  if (*p) return cudaSuccess;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * n);
}

cudaError_t snapshot(sg_ctx* c, bool save) {
  const size_t n = (size_t)sg::kMaxLinks * c->plan.num_slots, E = c->plan.num_envs;
  cudaError_t e = ensure(&c->d_snap_q, n);
  if (e == cudaSuccess) e = ensure(&c->d_snap_qd, n);
  if (e == cudaSuccess) e = ensure(&c->d_snap_sc, E);
  if (e != cudaSuccess) return e;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  if (save) {
    e = cudaMemcpyAsync(c->d_snap_q, c->d_q, n * 4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_snap_qd, c->d_qd, n * 4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_snap_sc, c->d_step_count, E * 4, k, c->stream);
  } else {
    e = cudaMemcpyAsync(c->d_q, c->d_snap_q, n * 4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_qd, c->d_snap_qd, n * 4, k, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_step_count, c->d_snap_sc, E * 4, k, c->stream);
  }
  return e;
}

// dst[f][w][i] = src[f][perm[w]][i] over F x NW x B 32-bit words (the warp
// reorder of a packing change); src and dst do not overlap
__global__ void permute_warps_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst,
                                     const int32_t* __restrict__ perm, int F, int NW, int B) {
  const long long per = (long long)NW * B, n = (long long)F * per;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long f = idx / per, rem = idx - f * per;
    const int w = (int)(rem / B), i = (int)(rem - (long long)w * B);
    dst[idx] = src[f * per + (long long)perm[w] * B + i];
  }
}

cudaError_t launch_permute_warps(const void* src, void* dst, const int32_t* perm, int F, int NW,
                                 int B, cudaStream_t stream) {
  const long long n = (long long)F * NW * B;
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  permute_warps_kernel<<<(int)blocks, 256, 0, stream>>>(static_cast<const uint32_t*>(src),
                                                        static_cast<uint32_t*>(dst), perm, F, NW, B);
  return cudaGetLastError();
}

// Put the warps in `packing`'s order: the parameter records, slot tables,
// per-slot state and the autotuner's state snapshot are gathered into a
// temporary buffer and copied back in place (the pointers captured in a
// rollout graph stay valid).  A pending differentiable forward refers to the
// old order and is discarded.
cudaError_t apply_packing(sg_ctx* c, int packing) {
  const std::vector<int32_t> target = sg::packing_order(c->plan, packing);
  const int NW = c->plan.num_warps;
  std::vector<int32_t> inv(NW), rel(NW);
  for (int w = 0; w < NW; ++w) inv[c->warp_order[w]] = w;
  bool identity = true;
  for (int w = 0; w < NW; ++w) {
    rel[w] = inv[target[w]];
    identity = identity && rel[w] == w;
  }
  c->packing = packing;
  if (identity) return cudaSuccess;
  struct Arr {
    void* p;
    int F, B;
  };
  const int W = sg::kWarp;
  const Arr arrs[] = {{c->d_params, 1, sg::kRecordFloats}, {c->d_q, sg::kMaxLinks, W},
                      {c->d_qd, sg::kMaxLinks, W},          {c->d_q0, sg::kMaxLinks, W},
                      {c->d_slot_env, 1, W},                {c->d_slot_info, 1, W},
                      {c->d_warp_class, 1, 1},              {c->d_track, 6, W},
                      {c->d_mass0, sg::kMaxLinks, W},       {c->d_inertia0, 3 * sg::kMaxLinks, W},
                      {c->d_snap_q, sg::kMaxLinks, W},      {c->d_snap_qd, sg::kMaxLinks, W}};
  size_t words = 0;
  for (const Arr& a : arrs) words = std::max(words, (size_t)a.F * NW * a.B);
  void* tmp = nullptr;
  int32_t* d_rel = nullptr;
  cudaError_t e = cudaMalloc(&tmp, words * 4 + (size_t)NW * 4 + 16);
  if (e != cudaSuccess) return e;
  d_rel = reinterpret_cast<int32_t*>(static_cast<char*>(tmp) + words * 4);
  e = cudaMemcpyAsync(d_rel, rel.data(), (size_t)NW * 4, cudaMemcpyHostToDevice, c->stream);
  for (const Arr& a : arrs) {
    if (!a.p || e != cudaSuccess) continue;
    e = launch_permute_warps(a.p, tmp, d_rel, a.F, NW, a.B, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(a.p, tmp, (size_t)a.F * NW * a.B * 4, cudaMemcpyDeviceToDevice,
                          c->stream);
  }
  const cudaError_t es = cudaStreamSynchronize(c->stream);   // rel and tmp are released below
  if (e == cudaSuccess) e = es;
  cudaFree(tmp);
  if (e == cudaSuccess) {
    c->warp_order = target;
    c->diff_ready = false;
    c->replay_prefilled = false;
  }
  return e;
}

}  // namespace

extern "C" {

sg_status sg_plan_packing(const sg_desc* desc, int32_t packing, int32_t* order,
                          int32_t num_warps, char* err, int32_t err_len) {
  sg::Plan p;
  std::string msg;
  sg_status st;
  try {
    st = sg::build_plan(desc, &p, &msg);
    if (st == SG_OK && (packing != SG_PACK_CLASS && packing != SG_PACK_INTERLEAVE)) {
      st = SG_ERR_INVALID_ARG;
      msg = "packing must be SG_PACK_CLASS or SG_PACK_INTERLEAVE";
    } else if (st == SG_OK && (!order || num_warps != p.num_warps)) {
      st = SG_ERR_INVALID_ARG;
      msg = "order must hold num_slots / 32 entries";
    }
    if (st == SG_OK) {
      const std::vector<int32_t> o = sg::packing_order(p, packing);
      std::copy(o.begin(), o.end(), order);
    }
  } catch (const std::bad_alloc&) {
    st = SG_ERR_OOM;
    msg = "host allocation failed";
  }
  if (err && err_len > 0) {
    std::strncpy(err, msg.c_str(), (size_t)err_len - 1);
    err[err_len - 1] = '\0';
  }
  return st;
}

sg_status sg_set_packing(sg_ctx* ctx, int32_t packing) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_set_packing");
  if (packing != SG_PACK_CLASS && packing != SG_PACK_INTERLEAVE)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_set_packing: unknown packing");
  return cuda_err(ctx, apply_packing(ctx, packing), "sg_set_packing");
}

int32_t sg_get_packing(const sg_ctx* ctx) { return ctx ? ctx->packing : -1; }

sg_status sg_plan(const sg_desc* desc, sg_plan_info* info, char* err, int32_t err_len) {
  sg::Plan p;
  std::string msg;
  sg_status st;
  try {
    st = sg::build_plan(desc, &p, &msg);
  } catch (const std::bad_alloc&) {
    st = SG_ERR_OOM;
    msg = "host allocation failed";
  }
  if (err && err_len > 0) {
    std::strncpy(err, msg.c_str(), (size_t)err_len - 1);
    err[err_len - 1] = '\0';
  }
  if (st != SG_OK) return st;
  if (info) {
    info->obs_dim = p.obs_dim;
    info->num_slots = p.num_slots;
    info->num_chains = p.num_chains;
    for (int k = 0; k < 4; ++k) info->class_slots[k] = p.class_slots[k];
  }
  return SG_OK;
}

sg_status sg_create(const sg_desc* desc, void* stream, sg_ctx** out) {
  if (!out) {
    g_create_error = "out is NULL";
    return SG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  sg_ctx* c = new (std::nothrow) sg_ctx();
  if (!c) {
    g_create_error = "host allocation failed";
    return SG_ERR_OOM;
  }
  std::string msg;
  sg_status st;
  try {
    st = sg::build_plan(desc, &c->plan, &msg);
  } catch (const std::bad_alloc&) {
    st = SG_ERR_OOM;
    msg = "host allocation failed";
  }
  if (st != SG_OK) {
    g_create_error = msg;
    free_ctx(c);
    return st;
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    cudaGetLastError();
    g_create_error = "sg_create: no CUDA device is available";
    free_ctx(c);
    return SG_ERR_CUDA;
  }
  c->stream = static_cast<cudaStream_t>(stream);
  const sg::Plan& P = c->plan;
  c->warp_order = sg::packing_order(P, SG_PACK_CLASS);
  const size_t NS = P.num_slots;
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  step(upload(&c->d_params, P.params.data(), P.params.size(), c->stream));
  step(upload(&c->d_slot_env, P.slot_env.data(), NS, c->stream));
  step(upload(&c->d_slot_info, P.slot_info.data(), NS, c->stream));
  step(upload(&c->d_warp_class, P.warp_class.data(), P.warp_class.size(), c->stream));
  step(upload(&c->d_q0, P.q0.data(), P.q0.size(), c->stream));
  step(upload(&c->d_mass0, P.mass0.data(), P.mass0.size(), c->stream));
  step(upload(&c->d_inertia0, P.inertia0.data(), P.inertia0.size(), c->stream));
  step(upload<float>(&c->d_q, nullptr, (size_t)sg::kMaxLinks * NS, c->stream));
  step(upload<float>(&c->d_qd, nullptr, (size_t)sg::kMaxLinks * NS, c->stream));
  step(upload<int32_t>(&c->d_step_count, nullptr, (size_t)P.num_envs, c->stream));
  step(upload<int32_t>(&c->d_err, nullptr, 1, c->stream));
  const size_t path_floats = (size_t)P.num_envs * P.path_len * 3;
  step(upload(&c->d_path, P.path.empty() ? nullptr : P.path.data(), path_floats, c->stream));
  float* d_ctrl = nullptr;     // control points of device-built paths (freed below)
  if (e == cudaSuccess && P.task == SG_TASK_PATH) e = sg::prepare_path_kernel();
  if (!P.path_ctrl.empty()) {
    step(upload(&d_ctrl, P.path_ctrl.data(), P.path_ctrl.size(), c->stream));
    if (e == cudaSuccess)
      e = sg::launch_build_paths(d_ctrl, P.path_ctrl_len, nullptr, P.num_envs, P.path_len,
                                 c->d_path, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_q, 0, sizeof(float) * sg::kMaxLinks * NS, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_qd, 0, sizeof(float) * sg::kMaxLinks * NS, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int32_t), c->stream);
  if (e == cudaSuccess && P.task == SG_TASK_TRACK) {
    e = cudaMalloc(&c->d_track, sizeof(float) * 6 * NS);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_track, 0, sizeof(float) * 6 * NS, c->stream);
  }
  if (e == cudaSuccess) e = sg::prepare_step_kernel();
  if (e == cudaSuccess) e = sg::prepare_step_pair_kernel();
  if (e == cudaSuccess) e = sg::prepare_diff_kernels();
  if (e == cudaSuccess) e = sg::launch_reset(state_args(c), nullptr, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (d_ctrl) {
    cudaStreamSynchronize(c->stream);
    cudaFree(d_ctrl);
  }
  if (e != cudaSuccess) {
    g_create_error = std::string("sg_create: ") + cudaGetErrorString(e);
    sg_status code = e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
    free_ctx(c);
    return code;
  }
  *out = c;
  return SG_OK;
}

void sg_destroy(sg_ctx* ctx) {
  if (!ctx) return;
  // release on the owning device, then restore the caller's current device
  int cur = -1;
  const bool have = cudaGetDevice(&cur) == cudaSuccess;
  const bool other = have && cur != ctx->device && ctx->device >= 0;
  if (other) cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
  if (other) cudaSetDevice(cur);
}

sg_status sg_debug_set_fault(sg_ctx* ctx, int32_t mode, int64_t wait_limit_ns) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  if (mode != SG_FAULT_NONE && mode != SG_FAULT_SKIP_PARAM_COPY && mode != SG_FAULT_SKIP_PARTNER)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_debug_set_fault: unknown mode");
  if (wait_limit_ns < 0 || wait_limit_ns > (int64_t)sg::kDefaultWaitNs)
    return set_err(ctx, SG_ERR_INVALID_ARG,
                   "sg_debug_set_fault: wait_limit_ns must be 0 (default) .. 2e9");
  ctx->fault = mode;
  ctx->wait_ns = wait_limit_ns ? (unsigned long long)wait_limit_ns : sg::kDefaultWaitNs;
  return SG_OK;
}

int32_t sg_device(const sg_ctx* ctx) { return ctx ? ctx->device : -1; }

sg_status sg_set_stream(sg_ctx* ctx, void* stream) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return SG_OK;
}

int32_t sg_obs_dim(const sg_ctx* ctx) { return ctx ? ctx->plan.obs_dim : 0; }
int32_t sg_num_envs(const sg_ctx* ctx) { return ctx ? ctx->plan.num_envs : 0; }
int32_t sg_max_joints(const sg_ctx* ctx) { return ctx ? ctx->plan.max_joints : 0; }

sg_status sg_reset(sg_ctx* ctx, const uint8_t* env_mask_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_reset");
  return cuda_err(ctx, sg::launch_reset(state_args(ctx), env_mask_dev, ctx->stream), "sg_reset");
}

sg_status sg_step(sg_ctx* ctx, const float* actions_dev, float dt, int32_t substeps,
                  float* obs_dev, float* reward_dev, uint8_t* done_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_step");
  sg_status st = check_step_args(ctx, actions_dev, dt, substeps, obs_dev, reward_dev, done_dev);
  if (st != SG_OK) return st;
  sg::StepArgs a = step_args(ctx, dt, substeps, 1);
  a.actions = actions_dev;
  a.obs = obs_dev;
  a.reward = reward_dev;
  a.done = done_dev;
  return cuda_err(ctx, launch_plan(ctx, a, ctx->stream), "sg_step");
}

sg_status sg_observe(sg_ctx* ctx, const float* targets_dev, const uint8_t* env_mask_dev,
                     float* obs_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_observe");
  if (!targets_dev || !obs_dev)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_observe: targets and obs must be non-NULL");
  sg::StepArgs a = step_args(ctx, 1.f, 1, 1);
  a.actions = targets_dev;
  a.obs = obs_dev;
  a.obs_mask = env_mask_dev;
  a.observe = 1;
  a.substeps = 0;
  return cuda_err(ctx, sg::launch_step(a, ctx->threads, ctx->stream), "sg_observe");
}

sg_status sg_rollout(sg_ctx* ctx, const float* actions_dev, int32_t T, float dt,
                     int32_t substeps, float* obs_dev, float* reward_dev, uint8_t* done_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_rollout");
  sg_status st = check_rollout_args(ctx, actions_dev, T, dt, substeps, obs_dev, reward_dev, done_dev);
  if (st != SG_OK) return st;
  return run_rollout(ctx, actions_dev, T, dt, substeps, obs_dev, reward_dev, done_dev);
}

sg_status sg_set_host_io(sg_ctx* ctx, int32_t mode) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  if (mode != SG_HOST_IO_AUTO && mode != SG_HOST_IO_STAGED && mode != SG_HOST_IO_DIRECT)
    return set_err(ctx, SG_ERR_INVALID_ARG,
                   "sg_set_host_io: mode must be 0 (pipelined), 1 (staged) or 2 (direct)");
  ctx->host_io = mode;
  return SG_OK;
}

sg_status sg_rollout_host(sg_ctx* ctx, const float* actions_host, int32_t T, float dt,
                          int32_t substeps, float* obs_host, float* reward_host,
                          uint8_t* done_host) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_rollout_host");
  sg_status st =
      check_rollout_args(ctx, actions_host, T, dt, substeps, obs_host, reward_host, done_host);
  if (st != SG_OK) return st;
  if (ctx->host_io == SG_HOST_IO_DIRECT) {
    // page-locked host memory the device can address: the kernel moves the data itself
    void *a_d = device_view(actions_host), *o_d = device_view(obs_host);
    void *r_d = device_view(reward_host), *d_d = device_view(done_host);
    if (a_d && o_d && r_d && d_d)
      return run_rollout(ctx, static_cast<const float*>(a_d), T, dt, substeps,
                         static_cast<float*>(o_d), static_cast<float*>(r_d),
                         static_cast<uint8_t*>(d_d));
  }
  const size_t E = ctx->plan.num_envs, J = ctx->plan.max_joints, D = ctx->plan.obs_dim;
  cudaError_t e = cudaSuccess;
  if (T > ctx->stage_T) {
    e = cudaStreamSynchronize(ctx->stream);
    void* old[] = {ctx->d_stage_act, ctx->d_stage_obs, ctx->d_stage_rew, ctx->d_stage_done};
    for (void* p : old)
      if (p) cudaFree(p);
    ctx->d_stage_act = ctx->d_stage_obs = ctx->d_stage_rew = nullptr;
    ctx->d_stage_done = nullptr;
    ctx->stage_T = 0;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stage_act, sizeof(float) * T * E * J);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stage_obs, sizeof(float) * T * E * D);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stage_rew, sizeof(float) * T * E);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stage_done, (size_t)T * E);
    if (e != cudaSuccess) return cuda_err(ctx, e, "sg_rollout_host: staging");
    ctx->stage_T = T;
  }
  if (ctx->host_io == SG_HOST_IO_STAGED || ctx->host_io == SG_HOST_IO_DIRECT) {
    // serial: copy in, rollout, copy out, all on the context's stream
    e = cudaMemcpyAsync(ctx->d_stage_act, actions_host, sizeof(float) * T * E * J,
                        cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "sg_rollout_host: copy in");
    st = run_rollout(ctx, ctx->d_stage_act, T, dt, substeps, ctx->d_stage_obs, ctx->d_stage_rew,
                     ctx->d_stage_done);
    if (st != SG_OK) return st;
    e = cudaMemcpyAsync(obs_host, ctx->d_stage_obs, sizeof(float) * T * E * D,
                        cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(reward_host, ctx->d_stage_rew, sizeof(float) * T * E,
                          cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(done_host, ctx->d_stage_done, (size_t)T * E, cudaMemcpyDeviceToHost,
                          ctx->stream);
    return cuda_err(ctx, e, "sg_rollout_host: copy out");
  }
  return pipelined_host_rollout(ctx, actions_host, T, dt, substeps, obs_host, reward_host,
                                done_host);
}

sg_status sg_set_launch(sg_ctx* ctx, int32_t threads_per_block, int32_t rollout_mode,
                        int32_t chain_split) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  if (!valid_threads(threads_per_block))
    return set_err(ctx, SG_ERR_INVALID_ARG, "threads_per_block must be 32, 64, 128 or 256");
  if (rollout_mode != SG_ROLLOUT_PERSISTENT && rollout_mode != SG_ROLLOUT_STEP_GRAPH)
    return set_err(ctx, SG_ERR_INVALID_ARG, "unknown rollout mode");
  if (chain_split != 1 && chain_split != 2)
    return set_err(ctx, SG_ERR_INVALID_ARG, "chain_split must be 1 or 2");
  if (chain_split == 2 && threads_per_block < 64)
    return set_err(ctx, SG_ERR_INVALID_ARG, "chain_split 2 needs threads_per_block >= 64");
  ctx->threads = threads_per_block;
  ctx->rollout_mode = rollout_mode;
  ctx->split = chain_split;
  return SG_OK;
}

sg_status sg_get_launch(const sg_ctx* ctx, int32_t* threads_per_block, int32_t* rollout_mode,
                        int32_t* chain_split) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  if (threads_per_block) *threads_per_block = ctx->threads;
  if (rollout_mode) *rollout_mode = ctx->rollout_mode;
  if (chain_split) *chain_split = ctx->split;
  return SG_OK;
}

sg_status sg_autotune(sg_ctx* ctx, const float* actions_dev, int32_t T, float dt,
                      int32_t substeps, float* obs_dev, float* reward_dev, uint8_t* done_dev,
                      int32_t repeats, float* best_ms) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_autotune");
  sg_status st = check_rollout_args(ctx, actions_dev, T, dt, substeps, obs_dev, reward_dev, done_dev);
  if (st != SG_OK) return st;
  if (repeats < 1 || repeats > 1000) return set_err(ctx, SG_ERR_INVALID_ARG, "repeats must be 1..1000");
  cudaError_t e = snapshot(ctx, true);
  if (e != cudaSuccess) return cuda_err(ctx, e, "sg_autotune: snapshot");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return cuda_err(ctx, e, "sg_autotune: events");
  const int threads_list[] = {32, 64, 128, 256};
  const int modes[] = {SG_ROLLOUT_PERSISTENT, SG_ROLLOUT_STEP_GRAPH};
  float best = -1.f;
  int best_t = ctx->threads, best_m = ctx->rollout_mode, best_s = ctx->split;
  int best_p = ctx->packing;
  // time every launch plan of the current packing
  auto time_plans = [&]() {
    for (int m : modes) {
      for (int plan = 0; plan < 8; ++plan) {
        const int th = threads_list[plan & 3], sp = 1 + (plan >> 2);
        if (sp == 2 && th < 64) continue;
        ctx->threads = th;
        ctx->rollout_mode = m;
        ctx->split = sp;
        std::vector<float> times;
        for (int r = -1; r < repeats && st == SG_OK; ++r) {
          e = snapshot(ctx, false);
          if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
          if (e != cudaSuccess) break;
          st = run_rollout(ctx, actions_dev, T, dt, substeps, obs_dev, reward_dev, done_dev);
          if (st != SG_OK) break;
          e = cudaEventRecord(e1, ctx->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) break;
          if (r >= 0) times.push_back(ms);
        }
        if (e != cudaSuccess || st != SG_OK) return;
        std::sort(times.begin(), times.end());
        const float med = times[times.size() / 2];
        if (best < 0.f || med < best) {
          best = med;
          best_t = th;
          best_m = m;
          best_s = sp;
          best_p = ctx->packing;
        }
      }
    }
  };
  const int packings[2] = {SG_PACK_CLASS, SG_PACK_INTERLEAVE};
  const int npack = sg::packing_order(ctx->plan, SG_PACK_INTERLEAVE) !=
                            sg::packing_order(ctx->plan, SG_PACK_CLASS)
                        ? 2
                        : 1;
  for (int i = 0; i < npack && e == cudaSuccess && st == SG_OK; ++i) {
    e = apply_packing(ctx, packings[i]);
    if (e == cudaSuccess) time_plans();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->threads = best_t;
  ctx->rollout_mode = best_m;
  ctx->split = best_s;
  if (e == cudaSuccess && ctx->packing != best_p) e = apply_packing(ctx, best_p);
  if (st != SG_OK) return st;
  if (e == cudaSuccess) e = snapshot(ctx, false);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "sg_autotune");
  if (best_ms) *best_ms = best;
  return SG_OK;
}

sg_status sg_get_state(sg_ctx* ctx, float* q_dev, float* qd_dev, int32_t* step_count_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_get_state");
  return cuda_err(ctx, sg::launch_get_state(state_args(ctx), q_dev, qd_dev, step_count_dev,
                                            ctx->stream),
                  "sg_get_state");
}

sg_status sg_set_state(sg_ctx* ctx, const float* q_dev, const float* qd_dev,
                       const int32_t* step_count_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_set_state");
  return cuda_err(ctx, sg::launch_set_state(state_args(ctx), q_dev, qd_dev, step_count_dev,
                                            ctx->stream),
                  "sg_set_state");
}

namespace {
sg::DiffArgs diff_args(sg_ctx* c) {
  sg::DiffArgs a;
  std::memset(&a, 0, sizeof(a));
  a.params = c->d_params;
  a.slot_env = c->d_slot_env;
  a.slot_info = c->d_slot_info;
  a.warp_class = c->d_warp_class;
  a.q = c->d_q;
  a.qd = c->d_qd;
  a.ckpt = c->d_ckpt;
  a.replay = c->use_replay ? c->d_replay : nullptr;
  a.err = c->d_err;
  a.num_warps = c->plan.num_warps;
  a.num_slots = c->plan.num_slots;
  a.num_envs = c->plan.num_envs;
  a.max_joints = c->plan.max_joints;
  a.T = c->diff_T;
  a.substeps = c->diff_substeps;
  a.ckpt_every = c->diff_every;
  a.nseg = (c->diff_T + c->diff_every - 1) / c->diff_every;
  a.h = c->diff_dt / (float)c->diff_substeps;
  return a;
}
}  // namespace

}  // extern "C"

namespace sg {
DiffArgs context_diff_args(sg_ctx* c) {
  DiffArgs a;
  std::memset(&a, 0, sizeof(a));
  a.params = c->d_params;
  a.slot_env = c->d_slot_env;
  a.slot_info = c->d_slot_info;
  a.warp_class = c->d_warp_class;
  a.q = c->d_q;
  a.qd = c->d_qd;
  a.err = c->d_err;
  a.num_warps = c->plan.num_warps;
  a.num_slots = c->plan.num_slots;
  a.num_envs = c->plan.num_envs;
  a.max_joints = c->plan.max_joints;
  return a;
}
void context_set_error(sg_ctx* c, const char* msg) { c->last_error = msg; }
sg_status context_check_device(sg_ctx* c, const char* fn) { return on_device(c, fn); }
cudaStream_t context_stream(sg_ctx* c) { return c->stream; }
int32_t* context_err(sg_ctx* c) { return c->d_err; }
const std::vector<int32_t>& context_env_dof(sg_ctx* c) { return c->plan.env_dof; }
}  // namespace sg

extern "C" {

sg_status sg_diff_forward(sg_ctx* ctx, const float* actions_dev, int32_t T, float dt,
                          int32_t substeps, int32_t ckpt_every, float* ee_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_diff_forward");
  if (!actions_dev || !ee_dev)
    return set_err(ctx, SG_ERR_INVALID_ARG, "actions and ee must be non-NULL");
  if (T < 1 || T > 4096) return set_err(ctx, SG_ERR_INVALID_ARG, "T must be 1..4096");
  if (!(dt > 0.f) || !std::isfinite(dt)) return set_err(ctx, SG_ERR_INVALID_ARG, "dt must be > 0");
  if (substeps < 1 || substeps > sg::kMaxDiffSubsteps)
    return set_err(ctx, SG_ERR_INVALID_ARG, "substeps must be 1..16 for the differentiable rollout");
  if (ckpt_every < 1 || ckpt_every > sg::kMaxCkptEvery)
    return set_err(ctx, SG_ERR_INVALID_ARG, "ckpt_every must be 1..32");
  const int nseg = (T + ckpt_every - 1) / ckpt_every;
  const size_t need = (size_t)(nseg + 1) * 2 * sg::kMaxLinks * ctx->plan.num_slots;
  if (need > ctx->ckpt_floats) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (ctx->d_ckpt) cudaFree(ctx->d_ckpt);
    ctx->d_ckpt = nullptr;
    ctx->ckpt_floats = 0;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_ckpt, need * sizeof(float));
    if (e != cudaSuccess) return cuda_err(ctx, e, "sg_diff_forward: checkpoint buffer");
    ctx->ckpt_floats = need;
  }
  // replay buffers of the pipelined backward (above the cap: the one-warp backward)
  const size_t rneed = sg::replay_floats(ckpt_every, substeps, ctx->plan.num_slots);
  ctx->use_replay = rneed <= sg::kMaxReplayFloats;
  if (ctx->use_replay && rneed > ctx->replay_floats) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (ctx->d_replay) cudaFree(ctx->d_replay);
    ctx->d_replay = nullptr;
    ctx->replay_floats = 0;
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_replay, rneed * sizeof(float));
    if (e != cudaSuccess) {
      ctx->use_replay = false;
      return cuda_err(ctx, e, "sg_diff_forward: replay buffer");
    }
    ctx->replay_floats = rneed;
  }
  ctx->diff_T = T;
  ctx->diff_dt = dt;
  ctx->diff_substeps = substeps;
  ctx->diff_every = ckpt_every;
  ctx->diff_ready = true;
  sg::DiffArgs a = diff_args(ctx);
  a.actions = actions_dev;
  a.ee = ee_dev;
  ctx->replay_prefilled = ctx->use_replay;
  return cuda_err(ctx, sg::launch_diff_forward(a, ctx->stream), "sg_diff_forward");
}

sg_status sg_diff_backward(sg_ctx* ctx, const float* actions_dev, const float* dl_dee_dev,
                           float* dactions_dev, float* dmass_dev, float* dq0_dev,
                           float* dqd0_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_diff_backward");
  if (!ctx->diff_ready)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_diff_backward needs a preceding sg_diff_forward");
  if (!actions_dev || !dl_dee_dev || !dactions_dev || !dmass_dev)
    return set_err(ctx, SG_ERR_INVALID_ARG, "actions, dl_dee, dactions and dmass must be non-NULL");
  sg::DiffArgs a = diff_args(ctx);
  a.actions = actions_dev;
  a.dl_dee = dl_dee_dev;
  a.dactions = dactions_dev;
  a.dmass = dmass_dev;
  a.dq0 = dq0_dev;
  a.dqd0 = dqd0_dev;
  // the first reverse pass after a forward starts from the records the forward
  // left in buffer 0; later ones (which overwrote it) replay that segment too
  a.prefilled = ctx->replay_prefilled ? 1 : 0;
  ctx->replay_prefilled = false;
  return cuda_err(ctx, sg::launch_diff_backward(a, ctx->stream), "sg_diff_backward");
}

sg_status sg_set_link_mass(sg_ctx* ctx, const float* mass_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_set_link_mass");
  if (!mass_dev) return set_err(ctx, SG_ERR_INVALID_ARG, "mass must be non-NULL");
  sg::MassArgs m;
  m.params = ctx->d_params;
  m.slot_env = ctx->d_slot_env;
  m.slot_info = ctx->d_slot_info;
  m.mass = mass_dev;
  m.mass0 = ctx->d_mass0;
  m.inertia0 = ctx->d_inertia0;
  m.num_slots = ctx->plan.num_slots;
  m.max_joints = ctx->plan.max_joints;
  return cuda_err(ctx, sg::launch_set_mass(m, ctx->stream), "sg_set_link_mass");
}

sg_status sg_get_goal_state(sg_ctx* ctx, float* offset_dev, float* velocity_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_get_goal_state");
  if (!ctx->d_track) return set_err(ctx, SG_ERR_INVALID_ARG, "goal state exists only for SG_TASK_TRACK");
  return cuda_err(ctx, sg::launch_goal_state(state_args(ctx), offset_dev, velocity_dev, nullptr,
                                             nullptr, ctx->stream),
                  "sg_get_goal_state");
}

sg_status sg_set_goal_state(sg_ctx* ctx, const float* offset_dev, const float* velocity_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_set_goal_state");
  if (!ctx->d_track) return set_err(ctx, SG_ERR_INVALID_ARG, "goal state exists only for SG_TASK_TRACK");
  return cuda_err(ctx, sg::launch_goal_state(state_args(ctx), nullptr, nullptr, offset_dev,
                                             velocity_dev, ctx->stream),
                  "sg_set_goal_state");
}

sg_status sg_set_paths(sg_ctx* ctx, const float* ctrl_dev, int32_t K,
                       const uint8_t* env_mask_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_set_paths");
  if (ctx->plan.task != SG_TASK_PATH)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_set_paths: not a path-following context");
  if (!ctrl_dev) return set_err(ctx, SG_ERR_INVALID_ARG, "sg_set_paths: ctrl_dev is NULL");
  if (K < 2 || K > sg::kMaxPathCtrl)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_set_paths: K must be 2..64");
  return cuda_err(ctx,
                  sg::launch_build_paths(ctrl_dev, K, env_mask_dev, ctx->plan.num_envs,
                                         ctx->plan.path_len, ctx->d_path, ctx->stream),
                  "sg_set_paths");
}

sg_status sg_get_paths(sg_ctx* ctx, float* path_dev) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_get_paths");
  if (ctx->plan.task != SG_TASK_PATH)
    return set_err(ctx, SG_ERR_INVALID_ARG, "sg_get_paths: not a path-following context");
  if (!path_dev) return set_err(ctx, SG_ERR_INVALID_ARG, "sg_get_paths: path_dev is NULL");
  const size_t bytes = sizeof(float) * (size_t)ctx->plan.num_envs * ctx->plan.path_len * 3;
  return cuda_err(ctx, cudaMemcpyAsync(path_dev, ctx->d_path, bytes, cudaMemcpyDeviceToDevice,
                                       ctx->stream),
                  "sg_get_paths");
}

sg_status sg_sync_status(sg_ctx* ctx) {
  if (!ctx) return SG_ERR_INVALID_ARG;
  SG_CHECK_DEVICE(ctx, "sg_sync_status");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "sg_sync_status");
  int32_t flags = 0;
  e = cudaMemcpy(&flags, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int32_t));
  if (e != cudaSuccess) return cuda_err(ctx, e, "sg_sync_status");
  if (flags & sg::DEVERR_TIMEOUT)
    return set_err(ctx, SG_ERR_TIMEOUT, "a bounded device wait for a parameter copy gave up");
  if (flags & sg::DEVERR_NONFINITE)
    return set_err(ctx, SG_ERR_NONFINITE, "an environment produced a non-finite state");
  return SG_OK;
}

const char* sg_last_error(const sg_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : g_create_error.c_str();
}

}  // extern "C"
