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
#include "sg_internal.h"
#include "sg_kernels.h"

namespace sg {

constexpr float kGravity = 9.81f;
constexpr int kWaitLimit = 1 << 20;   // bounded mbarrier polling

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (int it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Stage the warp's parameter record into shared memory; false if the copy
// did not complete within the polling bound (error flag set).
__device__ __forceinline__ bool stage_record(const StepArgs& a, int gw, int cls, float* rec,
                                             uint64_t* bar, int lane) {
  if (lane == 0) {
    mbar_init(bar, 1);
    const unsigned bytes = (unsigned)record_bytes_dev(cls);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(rec, a.params + (size_t)gw * kRecordFloats, bytes, bar);
  }
  __syncwarp();
  // warp-uniform verdict: either every lane proceeds or the whole warp leaves
  if (__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0))) return true;
  if (lane == 0) atomicOr(a.err, DEVERR_TIMEOUT);
  mbar_wait_bounded(bar, 0);   // give an in-flight copy a second bounded chance
  __syncwarp();
  return false;
}

template <class Pat>
__device__ __forceinline__ void run_chain(const StepArgs& a, const Pat& pat, const Rec& rec,
                                          int slot, int lane, bool paired) {
  constexpr int N = Pat::N;
  const int env = a.slot_env[slot];
  const bool valid = env >= 0;
  const int info = a.slot_info[slot];
  const int c = (info >> SI_C_SHIFT) & 1;
  const int nc = (info >> SI_NC_SHIFT) & 3;
  const int jo = (info >> SI_JO_SHIFT) & 15;
  const int ntot = (info >> SI_NTOT_SHIFT) & 31;
  const int obs_len = (info >> SI_OBSLEN_SHIFT) & 127;
  const int NS = a.num_slots;

  float q[7], qd[7], qs[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    q[i] = 0.f;
    qd[i] = 0.f;
    qs[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    q[i] = a.q[(size_t)i * NS + slot];
    qd[i] = a.qd[(size_t)i * NS + slot];
  }
  int sc = (valid && c == 0) ? a.step_count[env] : 0;
  const float goal_x = rec.cf(CF_GX), goal_y = rec.cf(CF_GY), goal_z = rec.cf(CF_GZ);
  const size_t E = (size_t)a.num_envs;
  const int J = a.max_joints, D = a.obs_dim;

  for (int t = 0; t < a.T; ++t) {
    if (valid) {
      const float* arow = a.actions + ((size_t)t * E + env) * J + jo;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (pat.active(i)) qs[i] = __ldg(arow + i);
    }
    for (int k = 0; k < a.substeps; ++k) chain_substep(pat, rec, q, qd, qs, a.h, kGravity);

    // ---- epilogue: tip pose, reward, observation, done
    V3 tip, r0, r1, r2;
    chain_tip(pat, rec, q, tip, r0, r1, r2);
    bool bad = false;
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (pat.active(i)) bad = bad || !isfinite(q[i]) || !isfinite(qd[i]);
    bad = bad && valid;
    if (paired) bad = bad || __shfl_xor_sync(0xffffffffu, bad ? 1 : 0, 1) != 0;
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, DEVERR_NONFINITE);
    ++sc;

    float reward;
    float* row = a.obs + ((size_t)t * E + (valid ? env : 0)) * D;
    if (a.task == SG_TASK_PATH) {
      const int W = a.path_len;
      const float* P = a.path + (size_t)(valid ? env : 0) * W * 3;
      const int t0 = max(sc, 0);
      const float* p0 = P + (size_t)min(t0, W - 1) * 3;
      const float dx = tip.x - p0[0], dy = tip.y - p0[1], dz = tip.z - p0[2];
      reward = -a.alpha * sqrtf(dx * dx + dy * dy + dz * dz);
      if (valid) {
        const int n = ntot;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (!pat.active(i)) continue;
          row[i] = q[i];
          row[n + i] = qd[i];
        }
        row[2 * n + 0] = tip.x;
        row[2 * n + 1] = tip.y;
        row[2 * n + 2] = tip.z;
        float quat[4];
        rot_to_quat(r0, r1, r2, quat);
#pragma unroll
        for (int k = 0; k < 4; ++k) row[2 * n + 3 + k] = quat[k];
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
          const float* pk = P + (size_t)min(t0 + k, W - 1) * 3;
          row[2 * n + 4 + 3 * k] = pk[0];
          row[2 * n + 5 + 3 * k] = pk[1];
          row[2 * n + 6 + 3 * k] = pk[2];
        }
      }
    } else {
      const float dx = tip.x - goal_x, dy = tip.y - goal_y, dz = tip.z - goal_z;
      reward = -sqrtf(dx * dx + dy * dy + dz * dz);
      if (paired) reward += __shfl_xor_sync(0xffffffffu, reward, 1);
      if (valid) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (!pat.active(i)) continue;
          row[jo + i] = q[i];
          row[ntot + jo + i] = qd[i];
          row[2 * ntot + 3 * nc + jo + i] = qs[i];
        }
        row[2 * ntot + 3 * c + 0] = tip.x;
        row[2 * ntot + 3 * c + 1] = tip.y;
        row[2 * ntot + 3 * c + 2] = tip.z;
        row[3 * ntot + 3 * nc + 3 * c + 0] = goal_x;
        row[3 * ntot + 3 * nc + 3 * c + 1] = goal_y;
        row[3 * ntot + 3 * nc + 3 * c + 2] = goal_z;
      }
    }
    if (valid && c == 0) {
      for (int k = obs_len; k < D; ++k) row[k] = 0.f;
      a.reward[(size_t)t * E + env] = reward;
      a.done[(size_t)t * E + env] =
          (uint8_t)((sc >= a.episode_len ? SG_DONE_TIMEOUT : 0) | (bad ? SG_DONE_NONFINITE : 0));
    }
  }

  if (valid) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      a.q[(size_t)i * NS + slot] = q[i];
      a.qd[(size_t)i * NS + slot] = qd[i];
    }
    if (c == 0) a.step_count[env] = sc;
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
  float* rec = smem + (size_t)wib * kRecordFloats;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)wpb * kRecordFloats) + wib;
  if (!stage_record(a, gw, wc, rec, bar, lane)) return;
  const Rec r{rec + lane};
  const int slot = gw * kWarp + lane;
  const bool paired = (wc & kPairedBit) != 0;
  switch (wc & 3) {
    case CLS_7R: run_chain(a, Pat7R{}, r, slot, lane, paired); break;
    case CLS_7P: run_chain(a, Pat7P{}, r, slot, lane, paired); break;
    case CLS_4R: run_chain(a, Pat4R{}, r, slot, lane, paired); break;
    default: {
      int code;
      const float cf = r.cf(CF_CODE);
      memcpy(&code, &cf, 4);
      const int n = (a.slot_info[slot] >> SI_NCHAIN_SHIFT) & 7;
      run_chain(a, PatGen{code, n}, r, slot, lane, paired);
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
  const int info = s.slot_info[slot];
  const int n = (info >> SI_NCHAIN_SHIFT) & 7;
  for (int i = 0; i < n; ++i) {
    s.q[(size_t)i * s.num_slots + slot] = s.q0[(size_t)i * s.num_slots + slot];
    s.qd[(size_t)i * s.num_slots + slot] = 0.f;
  }
  if (((info >> SI_C_SHIFT) & 1) == 0) s.step_count[env] = 0;
}

__global__ void get_state_kernel(StateArgs s, float* q_out, float* qd_out, int32_t* sc_out) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= s.num_slots) return;
  const int env = s.slot_env[slot];
  if (env < 0) return;
  const int info = s.slot_info[slot];
  const int n = (info >> SI_NCHAIN_SHIFT) & 7;
  const int c = (info >> SI_C_SHIFT) & 1;
  const int jo = (info >> SI_JO_SHIFT) & 15;
  const int ntot = (info >> SI_NTOT_SHIFT) & 31;
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
  const int info = s.slot_info[slot];
  const int n = (info >> SI_NCHAIN_SHIFT) & 7;
  const int c = (info >> SI_C_SHIFT) & 1;
  const int jo = (info >> SI_JO_SHIFT) & 15;
  const size_t row = (size_t)env * s.max_joints;
  for (int i = 0; i < n; ++i) {
    if (q_in) s.q[(size_t)i * s.num_slots + slot] = q_in[row + jo + i];
    if (qd_in) s.qd[(size_t)i * s.num_slots + slot] = qd_in[row + jo + i];
  }
  if (c == 0 && sc_in) s.step_count[env] = sc_in[env];
}

// ---- launchers ------------------------------------------------------------
size_t step_smem_bytes(int threads) {
  const int wpb = threads / kWarp;
  return (size_t)wpb * kRecordFloats * sizeof(float) + (size_t)wpb * sizeof(uint64_t);
}

cudaError_t prepare_step_kernel() {
  return cudaFuncSetAttribute(step_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)step_smem_bytes(kMaxThreads));
}

cudaError_t launch_step(const StepArgs& a, int threads, cudaStream_t stream) {
  const int wpb = threads / kWarp;
  const int blocks = (a.num_warps + wpb - 1) / wpb;
  step_kernel<<<blocks, threads, step_smem_bytes(threads), stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reset(const StateArgs& s, const uint8_t* mask, cudaStream_t stream) {
  const int threads = 256, blocks = (s.num_slots + threads - 1) / threads;
  reset_kernel<<<blocks, threads, 0, stream>>>(s, mask);
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
