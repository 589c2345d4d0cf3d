// Step / rollout kernel and the small state kernels (reset, state I/O).
//
// Launch shape: one thread per chain slot, warps of one chain class, any
// number of warps per block.  Each warp stages its own parameter record in
// shared memory with one bulk asynchronous copy (cp.async.bulk, completion
// on an mbarrier) and then runs T control steps with the chain state held in
// registers: T = 1 is the plain per-step launch, T > 1 the persistent
// rollout, and both execute the same instructions per step.
#include <cuda_runtime.h>

#include "sg_chain.cuh"
#include "sg_device.cuh"
#include "sg_internal.h"
#include "sg_kernels.h"
#include "sg_rng.cuh"

namespace sg {

// Stage the warp's parameter record into shared memory; false if the copy
// did not complete within the wait bound (error flag set).  With the test
// hook FAULT_SKIP_PARAM_COPY no copy is started, so the wait runs out.
__device__ __forceinline__ bool stage_record(const StepArgs& a, int gw, int cls, float* rec,
                                             uint64_t* bar, int lane) {
  if (lane == 0) {
    mbar_init(bar, 1);
    if (a.fault != FAULT_SKIP_PARAM_COPY) {
      const unsigned bytes = (unsigned)record_bytes_dev(cls);
      mbar_expect_tx(bar, bytes);
      bulk_g2s(rec, a.params + (size_t)gw * kRecordFloats, bytes, bar);
    }
  }
  __syncwarp();
  // warp-uniform verdict: either every lane proceeds or the whole warp leaves
  if (__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0, a.wait_ns))) return true;
  if (lane == 0) atomicOr(a.err, DEVERR_TIMEOUT);
  mbar_wait_bounded(bar, 0, a.wait_ns);   // give an in-flight copy a second bounded chance
  __syncwarp();
  return false;
}

// Observation rows are first assembled in a per-warp shared-memory stage
// (one row per env of the warp, odd row pitch: no bank conflicts), then the
// warp writes each row to HBM with consecutive lanes on consecutive floats.
// kGlog: log2 of the lanes per env (1, 2 or 4 chains in a lane group), a
// compile-time constant so that the group reductions and the row write-out
// unroll completely.  block: the warp's rows belong to consecutive envs and
// are written as one contiguous block (write_block), else row by row -- a
// run-time choice, so that the dynamics are compiled once and every warp
// rounds alike whatever its env order (a permuted batch gives the same bits).
template <int kGlog, class Pat>
__device__ __forceinline__ void run_chain(const StepArgs& a, const Pat& pat, const Rec& rec,
                                          float* stage, int slot, int lane, bool block) {
  constexpr int glog = kGlog;
  constexpr int N = Pat::N;
  const int env = a.slot_env[slot];
  const bool valid = env >= 0;
  const SlotFields f = decode_slot(a.slot_info[slot]);
  const int c = f.c, nc = f.nc, jo = f.jo, ntot = f.ntot, obs_len = f.obs_len;
  const int NS = a.num_slots;
  const int D = a.obs_dim, DP = stage_pitch(a.obs_dim);
  constexpr int g = 1 << glog;                    // lanes per env
  constexpr int nrows = kWarp >> glog;
  float* srow = stage + (lane >> glog) * DP;
  // env owning stage row `lane` (rows >= nrows unused; -1: row not written)
  const int sel_env = (valid && (!a.obs_mask || a.obs_mask[env])) ? env : -1;
  const int row_env = __shfl_sync(0xffffffffu, sel_env, (lane << glog) & 31);

  float q[7], qd[7], qs[7], qn[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    q[i] = 0.f;
    qd[i] = 0.f;
    qs[i] = 0.f;
    qn[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    q[i] = a.q[(size_t)i * NS + slot];
    qd[i] = a.qd[(size_t)i * NS + slot];
  }
  int sc = valid ? a.step_count[env] : 0;
  const float goal_x = rec.cf(CF_GX), goal_y = rec.cf(CF_GY), goal_z = rec.cf(CF_GZ);
  // moving goal of the tracking task: offset and velocity
  const bool track = a.task == SG_TASK_TRACK;
  float gd[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
  if (track && valid) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gd[k] = a.track[(size_t)k * NS + slot];
      gv[k] = a.track[(size_t)(3 + k) * NS + slot];
    }
  }
  const size_t E = (size_t)a.num_envs;
  if (valid) load_targets(pat, a, 0, env, jo, qn);
  // padding of this env's observation row (constant zero, written once)
  if (valid && c == 0)
    for (int k = obs_len; k < D; ++k) srow[k] = 0.f;
  float cq[N], sq[N];
  joint_sincos(pat, q, cq, sq);

  for (int t = 0; t < a.T; ++t) {
#pragma unroll
    for (int i = 0; i < 7; ++i) qs[i] = qn[i];
    if (valid && t + 1 < a.T) load_targets(pat, a, t + 1, env, jo, qn);   // prefetch
    for (int k = 0; k < a.substeps; ++k)
      chain_substep_trig(pat, rec, q, qd, qs, cq, sq, a.h, kGravity);

    // ---- epilogue: tip pose, reward, observation, done
    V3 tip, r0, r1, r2;
    chain_tip_trig(pat, rec, q, cq, sq, tip, r0, r1, r2);
    bool bad = false;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (pat.active(i)) bad = bad || !isfinite(q[i]) || !isfinite(qd[i]);
    bad = bad && valid;
    for (int off = 1; off < g; off <<= 1) bad = bad || __shfl_xor_sync(0xffffffffu, bad ? 1 : 0, off) != 0;
    if (__any_sync(0xffffffffu, bad) && lane == 0 && !a.observe) atomicOr(a.err, DEVERR_NONFINITE);
    if (!a.observe) ++sc;

    float reward;
    if (a.task == SG_TASK_PATH) {
      const int W = a.path_len;
      const float* P = a.path + (size_t)(valid ? env : 0) * W * 3;
      const int t0 = max(sc, 0);
      const float* p0 = P + (size_t)min(t0, W - 1) * 3;
      const float dx = tip.x - p0[0], dy = tip.y - p0[1], dz = tip.z - p0[2];
      reward = -a.alpha * sqrtf(dx * dx + dy * dy + dz * dz);
      const int n = ntot;
      if (valid) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        if (!pat.active(i)) continue;
        srow[i] = q[i];
        srow[n + i] = qd[i];
      }
      srow[2 * n + 0] = tip.x;
      srow[2 * n + 1] = tip.y;
      srow[2 * n + 2] = tip.z;
      float quat[4];
      rot_to_quat(r0, r1, r2, quat);
#pragma unroll
      for (int k = 0; k < 4; ++k) srow[2 * n + 3 + k] = quat[k];
#pragma unroll
      for (int k = 1; k <= 3; ++k) {
        const float* pk = P + (size_t)min(t0 + k, W - 1) * 3;
        srow[2 * n + 4 + 3 * k] = pk[0];
        srow[2 * n + 5 + 3 * k] = pk[1];
        srow[2 * n + 6 + 3 * k] = pk[2];
      }
      }
    } else {
      float gx = goal_x, gy = goal_y, gz = goal_z;
      if (track && !a.observe) {
        float z[3];
        goal_noise(a.seed, valid ? env : 0, c, sc, z[0], z[1], z[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          gd[k] = fminf(fmaxf(gd[k] + gv[k], -a.track_limit), a.track_limit);
          gv[k] += a.track_sigma * z[k];
        }
      }
      if (track) {
        gx += gd[0];
        gy += gd[1];
        gz += gd[2];
      }
      const float dx = tip.x - gx, dy = tip.y - gy, dz = tip.z - gz;
      reward = valid ? -sqrtf(dx * dx + dy * dy + dz * dz) : 0.f;
      for (int off = 1; off < g; off <<= 1) reward += __shfl_xor_sync(0xffffffffu, reward, off);
      if (valid) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (!pat.active(i)) continue;
          srow[jo + i] = q[i];
          srow[ntot + jo + i] = qd[i];
          srow[2 * ntot + 3 * nc + jo + i] = qs[i];
        }
        srow[2 * ntot + 3 * c + 0] = tip.x;
        srow[2 * ntot + 3 * c + 1] = tip.y;
        srow[2 * ntot + 3 * c + 2] = tip.z;
        srow[3 * ntot + 3 * nc + 3 * c + 0] = gx;
        srow[3 * ntot + 3 * nc + 3 * c + 1] = gy;
        srow[3 * ntot + 3 * nc + 3 * c + 2] = gz;
      }
    }
    if (c == 0 && !a.observe) {
      if (valid) {
        a.reward[(size_t)t * E + env] = reward;
        a.done[(size_t)t * E + env] =
            (uint8_t)((sc >= a.episode_len ? SG_DONE_TIMEOUT : 0) | (bad ? SG_DONE_NONFINITE : 0));
      }
    }
    __syncwarp();
    if (block) write_block<nrows>(a.obs + (size_t)t * E * D, stage,
                                  __shfl_sync(0xffffffffu, row_env, 0), D, lane);
    else write_rows_n<nrows>(a.obs + (size_t)t * E * D, stage, row_env, D, DP, lane);
    __syncwarp();
  }

  if (valid && !a.observe) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      a.q[(size_t)i * NS + slot] = q[i];
      a.qd[(size_t)i * NS + slot] = qd[i];
    }
    if (c == 0) a.step_count[env] = sc;
    if (track) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        a.track[(size_t)k * NS + slot] = gd[k];
        a.track[(size_t)(3 + k) * NS + slot] = gv[k];
      }
    }
  }
}

__global__ void __launch_bounds__(kMaxThreads) step_kernel(StepArgs a) {
  extern __shared__ __align__(128) float smem[];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + wib;
  if (gw >= a.num_warps) return;
  const int wc = a.warp_class[gw];
  const int stage_floats = kWarp * stage_pitch(a.obs_dim);
  float* rec = smem + (size_t)wib * kRecordFloats;
  float* stage = smem + (size_t)wpb * kRecordFloats + (size_t)wib * stage_floats;
  uint64_t* bar =
      reinterpret_cast<uint64_t*>(smem + (size_t)wpb * (kRecordFloats + stage_floats)) + wib;
  if (!stage_record(a, gw, wc, rec, bar, lane)) return;
  const Rec r{rec + lane};
  const int slot = gw * kWarp + lane;
  const int glog = group_log2(wc);
  // rows of consecutive envs (homogeneous batches in caller order): block write
  const int my_env = a.slot_env[slot];
  const int my_row = (my_env >= 0 && (!a.obs_mask || a.obs_mask[my_env])) ? my_env : -1;
  const int row_env = __shfl_sync(0xffffffffu, my_row, (lane << glog) & 31);
  const bool block =
      rows_contiguous(row_env, kWarp >> glog, a.obs_dim, stage_pitch(a.obs_dim), lane);
  auto run = [&](const auto& pat) {
    if (glog == 0) run_chain<0>(a, pat, r, stage, slot, lane, block);
    else if (glog == 1) run_chain<1>(a, pat, r, stage, slot, lane, block);
    else run_chain<2>(a, pat, r, stage, slot, lane, block);
  };
  switch (wc & 3) {
    case CLS_7R: run(Pat7R{}); break;
    case CLS_7P: run(Pat7P{}); break;
    case CLS_4R: run(Pat4R{}); break;
    default: {
      int code;
      const float cf = r.cf(CF_CODE);
      memcpy(&code, &cf, 4);
      const int n = decode_slot(a.slot_info[slot]).nchain;
      run(PatGen{code, n});
    }
  }
}

// ---- reset and state I/O --------------------------------------------------
__global__ void reset_kernel(StateArgs s, const uint8_t* mask) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= s.num_slots) return;
  const int env = s.slot_env[slot];
  if (env < 0) return;
  if (mask && !mask[env]) return;
  const SlotFields f = decode_slot(s.slot_info[slot]);
  for (int i = 0; i < f.nchain; ++i) {
    s.q[(size_t)i * s.num_slots + slot] = s.q0[(size_t)i * s.num_slots + slot];
    s.qd[(size_t)i * s.num_slots + slot] = 0.f;
  }
  if (f.c == 0) s.step_count[env] = 0;
  if (s.track)
    for (int k = 0; k < 6; ++k) s.track[(size_t)k * s.num_slots + slot] = 0.f;
}

// goal offset / velocity of the tracking task <-> caller layout [E][4][3]
__global__ void goal_state_kernel(StateArgs s, float* off, float* vel, const float* off_in,
                                  const float* vel_in) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= s.num_slots) return;
  const int env = s.slot_env[slot];
  if (env < 0) return;
  const SlotFields f = decode_slot(s.slot_info[slot]);
  const size_t base = ((size_t)env * kMaxChains + f.c) * 3;
  for (int k = 0; k < 3; ++k) {
    float* d = s.track + (size_t)k * s.num_slots + slot;
    float* v = s.track + (size_t)(3 + k) * s.num_slots + slot;
    if (off) off[base + k] = *d;
    if (vel) vel[base + k] = *v;
    if (off_in) *d = off_in[base + k];
    if (vel_in) *v = vel_in[base + k];
  }
  if (f.c == 0) {               // chains the env does not have
    for (int k = 3 * f.nc; k < 3 * kMaxChains; ++k) {
      if (off) off[(size_t)env * kMaxChains * 3 + k] = 0.f;
      if (vel) vel[(size_t)env * kMaxChains * 3 + k] = 0.f;
    }
  }
}

__global__ void get_state_kernel(StateArgs s, float* q_out, float* qd_out, int32_t* sc_out) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= s.num_slots) return;
  const int env = s.slot_env[slot];
  if (env < 0) return;
  const SlotFields f = decode_slot(s.slot_info[slot]);
  const int n = f.nchain, c = f.c, jo = f.jo, ntot = f.ntot;
  const size_t row = (size_t)env * s.max_joints;
  for (int i = 0; i < n; ++i) {
    if (q_out) q_out[row + jo + i] = s.q[(size_t)i * s.num_slots + slot];
    if (qd_out) qd_out[row + jo + i] = s.qd[(size_t)i * s.num_slots + slot];
  }
  if (c == 0) {
    for (int j = ntot; j < s.max_joints; ++j) {
      if (q_out) q_out[row + j] = 0.f;
      if (qd_out) qd_out[row + j] = 0.f;
    }
    if (sc_out) sc_out[env] = s.step_count[env];
  }
}

__global__ void set_state_kernel(StateArgs s, const float* q_in, const float* qd_in,
                                 const int32_t* sc_in) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= s.num_slots) return;
  const int env = s.slot_env[slot];
  if (env < 0) return;
  const SlotFields f = decode_slot(s.slot_info[slot]);
  const int n = f.nchain, c = f.c, jo = f.jo;
  const size_t row = (size_t)env * s.max_joints;
  for (int i = 0; i < n; ++i) {
    if (q_in) s.q[(size_t)i * s.num_slots + slot] = q_in[row + jo + i];
    if (qd_in) s.qd[(size_t)i * s.num_slots + slot] = qd_in[row + jo + i];
  }
  if (c == 0 && sc_in) s.step_count[env] = sc_in[env];
}

// ---- launchers ------------------------------------------------------------
size_t step_smem_bytes(int threads, int obs_dim) {
  const int wpb = threads / kWarp;
  const size_t stage = (size_t)kWarp * stage_pitch(obs_dim);
  return (size_t)wpb * (kRecordFloats + stage) * sizeof(float) + (size_t)wpb * sizeof(uint64_t);
}

cudaError_t prepare_step_kernel() {
  return cudaFuncSetAttribute(step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)step_smem_bytes(kMaxThreads, kMaxObsDim));
}

cudaError_t launch_step(const StepArgs& a, int threads, cudaStream_t stream) {
  const int wpb = threads / kWarp;
  const int blocks = (a.num_warps + wpb - 1) / wpb;
  step_kernel<<<blocks, threads, step_smem_bytes(threads, a.obs_dim), stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reset(const StateArgs& s, const uint8_t* mask, cudaStream_t stream) {
  const int threads = 256, blocks = (s.num_slots + threads - 1) / threads;
  reset_kernel<<<blocks, threads, 0, stream>>>(s, mask);
  return cudaGetLastError();
}

cudaError_t launch_goal_state(const StateArgs& s, float* off, float* vel, const float* off_in,
                              const float* vel_in, cudaStream_t stream) {
  const int threads = 256, blocks = (s.num_slots + threads - 1) / threads;
  goal_state_kernel<<<blocks, threads, 0, stream>>>(s, off, vel, off_in, vel_in);
  return cudaGetLastError();
}

cudaError_t launch_get_state(const StateArgs& s, float* q, float* qd, int32_t* sc,
                             cudaStream_t stream) {
  const int threads = 256, blocks = (s.num_slots + threads - 1) / threads;
  get_state_kernel<<<blocks, threads, 0, stream>>>(s, q, qd, sc);
  return cudaGetLastError();
}

cudaError_t launch_set_state(const StateArgs& s, const float* q, const float* qd,
                             const int32_t* sc, cudaStream_t stream) {
  const int threads = 256, blocks = (s.num_slots + threads - 1) / threads;
  set_state_kernel<<<blocks, threads, 0, stream>>>(s, q, qd, sc);
  return cudaGetLastError();
}

}  // namespace sg
