// Warp-pair step kernel: two warps share one block of 32 chains.
//
// When a batch has fewer chains than the GPU has warp schedulers (16384
// mixed envs are ~590 warps of chains for 608 schedulers), one thread per
// chain leaves each scheduler with a single dependent instruction stream.
// Here the substep of every chain is split across two warps that run
// concurrently on the same SM (sg_pair.cuh: role 0 the bias forces and the
// drive right-hand side, role 1 the mass matrix and its Cholesky factor,
// swapped through a double-buffered shared-memory exchange; bounded waits:
// no block barrier after start-up, and a wait that runs out sets
// DEVERR_TIMEOUT and the warp leaves, so a partner is never left waiting
// forever).  Both roles then execute the same triangular solve on the same
// operands and apply the same update, so their copies of the chain state
// stay bit-identical.  The
// observation rows are staged by both roles and written out half by each.
// The arithmetic is that of the one-thread-per-chain kernel; the two kernels
// agree to rounding (separately compiled code may contract multiply-adds
// differently).
#include <cuda_runtime.h>

#include "sg_chain.cuh"
#include "sg_device.cuh"
#include "sg_internal.h"
#include "sg_kernels.h"
#include "sg_pair.cuh"
#include "sg_rng.cuh"

namespace sg {

namespace {

constexpr int kPairBars = 3;                      // tma, exchange, stage

// kGlog: log2 of the lanes per env, a compile-time constant; block: rows of
// consecutive envs, written as contiguous blocks (a run-time choice, see
// run_chain)
template <int kGlog, class Pat>
__device__ __forceinline__ void run_pair(const StepArgs& a, const Pat& pat, const Rec& rec,
                                         float* stage, float* xbuf, uint64_t* bars, int group,
                                         int lane, int role, bool block) {
  constexpr int glog = kGlog;
  constexpr int N = Pat::N;
  const int slot = group * kWarp + lane;
  const int env = a.slot_env[slot];
  const bool valid = env >= 0;
  const SlotFields f = decode_slot(a.slot_info[slot]);
  const int c = f.c, nc = f.nc, jo = f.jo, ntot = f.ntot, obs_len = f.obs_len;
  const int NS = a.num_slots;
  const int D = a.obs_dim, DP = stage_pitch(a.obs_dim);
  constexpr int g = 1 << glog;                    // lanes per env
  constexpr int nrows = kWarp >> glog;
  float* srow = stage + (lane >> glog) * DP;
  const int row_env = __shfl_sync(0xffffffffu, env, (lane << glog) & 31);
  uint64_t* bar_x = bars + 1;
  uint64_t* bar_stage = bars + 2;
  unsigned ph_x = 0, ph_stage = 0;
  unsigned xphase = 0;

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
  const size_t E = (size_t)a.num_envs;
  const bool track = a.task == SG_TASK_TRACK;
  float gd[3] = {0.f, 0.f, 0.f}, gv[3] = {0.f, 0.f, 0.f};
  if (track && valid && role == 1) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gd[k] = a.track[(size_t)k * NS + slot];
      gv[k] = a.track[(size_t)(3 + k) * NS + slot];
    }
  }
  if (valid && role == 0) load_targets(pat, a, 0, env, jo, qn);
  if (valid && role == 0 && c == 0)
    for (int k = obs_len; k < D; ++k) srow[k] = 0.f;   // padding, written once
  float cq[N], sq[N];
  joint_sincos(pat, q, cq, sq);

  for (int t = 0; t < a.T; ++t) {
    if (role == 0) {
#pragma unroll
      for (int i = 0; i < 7; ++i) qs[i] = qn[i];
      if (valid && t + 1 < a.T) load_targets(pat, a, t + 1, env, jo, qn);
    }
    for (int k = 0; k < a.substeps; ++k, ++xphase) {
      float* xb = xbuf + (xphase & 1) * kXHalf;   // double-buffered exchange
      float L[N][N], inv[N], dqd[N];
      const bool skip = a.fault == FAULT_SKIP_PARTNER && role == 0 && xphase == 0;
      if (!pair_substep(pat, rec, q, qd, qs, cq, sq, a.h, xb, bar_x, ph_x, a.err, lane, role, L,
                        inv, dqd, a.wait_ns, skip))
        return;
      integrate(pat, q, qd, dqd, a.h);
      joint_sincos(pat, q, cq, sq);
    }

    // ---- epilogue: role 0 stages q, qd, q* and writes done; role 1 the tip
    // pose, goal / waypoints and the reward.
    ++sc;
    if (role == 0) {
      bool bad = false;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (pat.active(i)) bad = bad || !isfinite(q[i]) || !isfinite(qd[i]);
      bad = bad && valid;
      for (int off = 1; off < g; off <<= 1)
        bad = bad || __shfl_xor_sync(0xffffffffu, bad ? 1 : 0, off) != 0;
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.err, DEVERR_NONFINITE);
      const int n = ntot;
      if (valid) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (!pat.active(i)) continue;
          srow[jo + i] = q[i];
          srow[n + jo + i] = qd[i];
          if (a.task != SG_TASK_PATH) srow[2 * n + 3 * nc + jo + i] = qs[i];
        }
      }
      if (c == 0) {
        if (valid)
          a.done[(size_t)t * E + env] = (uint8_t)((sc >= a.episode_len ? SG_DONE_TIMEOUT : 0) |
                                                  (bad ? SG_DONE_NONFINITE : 0));
      }
    } else {
      V3 tip, r0, r1, r2;
      chain_tip_trig(pat, rec, q, cq, sq, tip, r0, r1, r2);
      float reward;
      if (a.task == SG_TASK_PATH) {
        const int W = a.path_len, n = ntot;
        const float* P = a.path + (size_t)(valid ? env : 0) * W * 3;
        const int t0 = max(sc, 0);
        const float* p0 = P + (size_t)min(t0, W - 1) * 3;
        const float dx = tip.x - p0[0], dy = tip.y - p0[1], dz = tip.z - p0[2];
        reward = -a.alpha * sqrtf(dx * dx + dy * dy + dz * dz);
        if (valid) {
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
        float gx = rec.cf(CF_GX), gy = rec.cf(CF_GY), gz = rec.cf(CF_GZ);
        if (track) {
          float z[3];
          goal_noise(a.seed, valid ? env : 0, c, sc, z[0], z[1], z[2]);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            gd[k] = fminf(fmaxf(gd[k] + gv[k], -a.track_limit), a.track_limit);
            gv[k] += a.track_sigma * z[k];
          }
          gx += gd[0];
          gy += gd[1];
          gz += gd[2];
        }
        const float dx = tip.x - gx, dy = tip.y - gy, dz = tip.z - gz;
        reward = valid ? -sqrtf(dx * dx + dy * dy + dz * dz) : 0.f;
        for (int off = 1; off < g; off <<= 1) reward += __shfl_xor_sync(0xffffffffu, reward, off);
        if (valid) {
          srow[2 * ntot + 3 * c + 0] = tip.x;
          srow[2 * ntot + 3 * c + 1] = tip.y;
          srow[2 * ntot + 3 * c + 2] = tip.z;
          srow[3 * ntot + 3 * nc + 3 * c + 0] = gx;
          srow[3 * ntot + 3 * nc + 3 * c + 1] = gy;
          srow[3 * ntot + 3 * nc + 3 * c + 2] = gz;
        }
      }
      if (valid && c == 0) a.reward[(size_t)t * E + env] = reward;
    }
    mbar_arrive(bar_stage);
    if (!pair_wait(bar_stage, ph_stage, a.err, lane, a.wait_ns)) return;
    // each role writes half of the staged rows
    constexpr int half = nrows >> 1;
    const int r0 = role * half;
    if (block) {
      write_block<half>(a.obs + (size_t)t * E * D, stage + r0 * DP,
                        __shfl_sync(0xffffffffu, row_env, 0) + r0, D, lane);
    } else {
      const int ev = __shfl_sync(0xffffffffu, row_env, (lane + r0) & 31);
      write_rows_n<half>(a.obs + (size_t)t * E * D, stage + r0 * DP, ev, D, DP, lane);
    }
  }

  if (valid && role == 0) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      a.q[(size_t)i * NS + slot] = q[i];
      a.qd[(size_t)i * NS + slot] = qd[i];
    }
    if (c == 0) a.step_count[env] = sc;
  }
  if (valid && role == 1 && track) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a.track[(size_t)k * NS + slot] = gd[k];
      a.track[(size_t)(3 + k) * NS + slot] = gv[k];
    }
  }
}

}  // namespace

__global__ void __launch_bounds__(kMaxThreads) step_kernel_pair(StepArgs a) {
  extern __shared__ __align__(128) float smem[];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int pairs = blockDim.x >> 6;
  // the first `pairs` warps take role 0, the rest role 1: with four pairs
  // per block, warps w and w + 4 share one of the SM's four schedulers, so
  // each scheduler holds one warp of each role instead of two of the same
  const int pair = w % pairs, role = w / pairs;
  const int stage_floats = kWarp * stage_pitch(a.obs_dim);
  float* rec = smem + (size_t)pair * kRecordFloats;
  float* stage = smem + (size_t)pairs * kRecordFloats + (size_t)pair * stage_floats;
  float* xbuf = smem + (size_t)pairs * (kRecordFloats + stage_floats) + (size_t)pair * kXFloats;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)pairs * (kRecordFloats + stage_floats + kXFloats)) +
                   (size_t)pair * kPairBars;
  // start-up: warp 0 initialises every pair's barriers before any warp leaves
  if (w == 0 && lane < pairs) {
    uint64_t* b = reinterpret_cast<uint64_t*>(smem + (size_t)pairs * (kRecordFloats + stage_floats + kXFloats)) +
                  (size_t)lane * kPairBars;
    mbar_init(b + 0, 1);
    mbar_init(b + 1, 2 * kWarp);
    mbar_init(b + 2, 2 * kWarp);
  }
  __syncthreads();
  const int group = blockIdx.x * pairs + pair;
  if (group >= a.num_warps) return;
  const int wc = a.warp_class[group];
  if (role == 0 && lane == 0) {
    const unsigned bytes = (unsigned)record_bytes_dev(wc);
    mbar_expect_tx(bars, bytes);
    bulk_g2s(rec, a.params + (size_t)group * kRecordFloats, bytes, bars);
  }
  unsigned ph_tma = 0;
  if (!pair_wait(bars, ph_tma, a.err, lane, a.wait_ns)) {
    mbar_wait_bounded(bars, 0, a.wait_ns);   // second bounded chance for an in-flight copy
    return;
  }
  const Rec r{rec + lane};
  const int glog = group_log2(wc);
  // rows of consecutive envs (homogeneous batches in caller order): block writes
  const int my_env = a.slot_env[group * kWarp + lane];
  const int row_env = __shfl_sync(0xffffffffu, my_env, (lane << glog) & 31);
  const bool block =
      rows_contiguous(row_env, kWarp >> glog, a.obs_dim, stage_pitch(a.obs_dim), lane);
  auto run = [&](const auto& pat) {
    if (glog == 0) run_pair<0>(a, pat, r, stage, xbuf, bars, group, lane, role, block);
    else if (glog == 1) run_pair<1>(a, pat, r, stage, xbuf, bars, group, lane, role, block);
    else run_pair<2>(a, pat, r, stage, xbuf, bars, group, lane, role, block);
  };
  switch (wc & 3) {
    case CLS_7R: run(Pat7R{}); break;
    case CLS_7P: run(Pat7P{}); break;
    case CLS_4R: run(Pat4R{}); break;
    default: {
      int code;
      const float cf = r.cf(CF_CODE);
      memcpy(&code, &cf, 4);
      const int n = decode_slot(a.slot_info[group * kWarp + lane]).nchain;
      run(PatGen{code, n});
    }
  }
}

size_t step_pair_smem_bytes(int threads, int obs_dim) {
  const int pairs = threads / (2 * kWarp);
  const size_t per = kRecordFloats + (size_t)kWarp * stage_pitch(obs_dim) + kXFloats;
  return (size_t)pairs * per * sizeof(float) + (size_t)pairs * kPairBars * sizeof(uint64_t);
}

cudaError_t prepare_step_pair_kernel() {
  return cudaFuncSetAttribute(step_kernel_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)step_pair_smem_bytes(kMaxThreads, kMaxObsDim));
}

cudaError_t launch_step_pair(const StepArgs& a, int threads, cudaStream_t stream) {
  const int pairs = threads / (2 * kWarp);
  const int blocks = (a.num_warps + pairs - 1) / pairs;
  step_kernel_pair<<<blocks, threads, step_pair_smem_bytes(threads, a.obs_dim), stream>>>(a);
  return cudaGetLastError();
}

}  // namespace sg
