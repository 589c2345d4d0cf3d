// Differentiable rollout: forward with state checkpoints, and the adjoint
// (reverse) pass with segment recomputation.  One thread per chain; the
// parameter record of each warp is staged in shared memory by one bulk copy.
//
// Forward: T control steps from the context state (which is left unchanged),
// writing the tool-tip position after every step and the chain state
// (q, qd) every `ckpt_every` steps plus the final state into a checkpoint
// buffer [nseg + 1][2 * 7][slots].
// Backward: for each segment, last first, the step-start states are
// recomputed from its checkpoint into thread-local memory; each step is then
// reversed substep by substep (the substep's input states are recomputed
// from the step-start state), accumulating the cotangents of the targets and
// of the link masses (see sg_adjoint.cuh for the substep adjoint).
#include <cuda_runtime.h>

#include "sg_adjoint.cuh"
#include "sg_chain.cuh"
#include "sg_device.cuh"
#include "sg_diff.h"
#include "sg_internal.h"

namespace sg {

namespace {

constexpr int kStateFloats = 2 * kMaxLinks;

__device__ __forceinline__ bool stage_params(const float* params, int* err, int gw, int cls,
                                             float* rec, uint64_t* bar, int lane) {
  if (lane == 0) {
    mbar_init(bar, 1);
    const unsigned bytes = (unsigned)record_bytes_dev(cls);
    mbar_expect_tx(bar, bytes);
    bulk_g2s(rec, params + (size_t)gw * kRecordFloats, bytes, bar);
  }
  __syncwarp();
  if (__all_sync(0xffffffffu, mbar_wait_bounded(bar, 0))) return true;
  if (lane == 0) atomicOr(err, DEVERR_TIMEOUT);
  mbar_wait_bounded(bar, 0);
  __syncwarp();
  return false;
}

struct SlotInfo {
  int env, c, nc, jo, ntot;
  bool valid;
};

__device__ __forceinline__ SlotInfo slot_info(const DiffArgs& a, int slot) {
  SlotInfo s;
  s.env = a.slot_env[slot];
  s.valid = s.env >= 0;
  const SlotFields f = decode_slot(a.slot_info[slot]);
  s.c = f.c;
  s.nc = f.nc;
  s.jo = f.jo;
  s.ntot = f.ntot;
  return s;
}

template <class Pat>
__device__ __forceinline__ void read_targets(const Pat& pat, const DiffArgs& a, int t,
                                             const SlotInfo& s, float (&qs)[7]) {
#pragma unroll
  for (int i = 0; i < 7; ++i) qs[i] = 0.f;
  if (!s.valid) return;
  const float* row = a.actions + ((size_t)t * a.num_envs + s.env) * a.max_joints + s.jo;
#pragma unroll
  for (int i = 0; i < Pat::N; ++i)
    if (pat.active(i)) qs[i] = __ldg(row + i);
}

template <class Pat>
__device__ __forceinline__ void put_ckpt(const Pat& pat, const DiffArgs& a, int k, int slot,
                                         const float (&q)[7], const float (&qd)[7]) {
  float* base = a.ckpt + (size_t)k * kStateFloats * a.num_slots;
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (!pat.active(i)) continue;
    base[(size_t)i * a.num_slots + slot] = q[i];
    base[(size_t)(kMaxLinks + i) * a.num_slots + slot] = qd[i];
  }
}

template <class Pat>
__device__ __forceinline__ void get_ckpt(const Pat& pat, const DiffArgs& a, int k, int slot,
                                         float (&q)[7], float (&qd)[7]) {
  const float* base = a.ckpt + (size_t)k * kStateFloats * a.num_slots;
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    q[i] = 0.f;
    qd[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (!pat.active(i)) continue;
    q[i] = base[(size_t)i * a.num_slots + slot];
    qd[i] = base[(size_t)(kMaxLinks + i) * a.num_slots + slot];
  }
}

template <class Pat>
__device__ __forceinline__ void diff_forward_chain(const DiffArgs& a, const Pat& pat,
                                                   const Rec& rec, int slot) {
  const SlotInfo s = slot_info(a, slot);
  float q[7], qd[7], qs[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    q[i] = 0.f;
    qd[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (!pat.active(i)) continue;
    q[i] = a.q[(size_t)i * a.num_slots + slot];
    qd[i] = a.qd[(size_t)i * a.num_slots + slot];
  }
  const size_t E = (size_t)a.num_envs;
  for (int t = 0; t < a.T; ++t) {
    if (t % a.ckpt_every == 0) put_ckpt(pat, a, t / a.ckpt_every, slot, q, qd);
    read_targets(pat, a, t, s, qs);
    for (int k = 0; k < a.substeps; ++k) chain_substep(pat, rec, q, qd, qs, a.h, kGravity);
    V3 tip, r0, r1, r2;
    chain_tip(pat, rec, q, tip, r0, r1, r2);
    if (s.valid) {
      float* e = a.ee + (((size_t)t * E + s.env) * kMaxChains + s.c) * 3;
      e[0] = tip.x;
      e[1] = tip.y;
      e[2] = tip.z;
      if (s.c == 0)                                  // chains the env does not have
        for (int k = 3 * s.nc; k < 3 * kMaxChains; ++k) e[k] = 0.f;
    }
  }
  put_ckpt(pat, a, a.nseg, slot, q, qd);
}

template <class Pat>
__device__ __forceinline__ void diff_backward_chain(const DiffArgs& a, const Pat& pat,
                                                    const Rec& rec, int slot) {
  constexpr int N = Pat::N;
  const SlotInfo s = slot_info(a, slot);
  const size_t E = (size_t)a.num_envs;
  const int J = a.max_joints;
  float lq[7], lqd[7], lm[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    lq[i] = 0.f;
    lqd[i] = 0.f;
    lm[i] = 0.f;
  }
  float seg_q[kMaxCkptEvery][kMaxLinks], seg_qd[kMaxCkptEvery][kMaxLinks];   // thread-local
  float sub_q[kMaxDiffSubsteps][kMaxLinks], sub_qd[kMaxDiffSubsteps][kMaxLinks];
  for (int seg = a.nseg - 1; seg >= 0; --seg) {
    const int t0 = seg * a.ckpt_every;
    const int t1 = min(a.T, t0 + a.ckpt_every);
    float q[7], qd[7], qs[7];
    get_ckpt(pat, a, seg, slot, q, qd);
    for (int j = 0; j < t1 - t0; ++j) {
#pragma unroll
      for (int i = 0; i < N; ++i) {
        seg_q[j][i] = q[i];
        seg_qd[j][i] = qd[i];
      }
      if (j + 1 < t1 - t0) {
        read_targets(pat, a, t0 + j, s, qs);
        for (int k = 0; k < a.substeps; ++k) chain_substep(pat, rec, q, qd, qs, a.h, kGravity);
      }
    }
    // state after the segment's last step
    float qn[7], qdn[7];
    get_ckpt(pat, a, seg + 1, slot, qn, qdn);
    for (int t = t1 - 1; t >= t0; --t) {
      // tool-tip cotangent of the state after step t
      if (s.valid) {
        const float* g = a.dl_dee + (((size_t)t * E + s.env) * kMaxChains + s.c) * 3;
        float gq[N];
#pragma unroll
        for (int i = 0; i < N; ++i) gq[i] = 0.f;
        tip_vjp(pat, rec, qn, V3{g[0], g[1], g[2]}, gq);
#pragma unroll
        for (int i = 0; i < N; ++i) lq[i] += gq[i];
      }
      // reverse step t from its start state
      read_targets(pat, a, t, s, qs);
#pragma unroll
      for (int i = 0; i < 7; ++i) {
        q[i] = 0.f;
        qd[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) {
        q[i] = seg_q[t - t0][i];
        qd[i] = seg_qd[t - t0][i];
      }
#pragma unroll
      for (int i = 0; i < 7; ++i) qn[i] = q[i];
      for (int k = 0; k < a.substeps; ++k) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          sub_q[k][i] = q[i];
          sub_qd[k][i] = qd[i];
        }
        if (k + 1 < a.substeps) chain_substep(pat, rec, q, qd, qs, a.h, kGravity);
      }
      float lqs[7];
#pragma unroll
      for (int i = 0; i < 7; ++i) lqs[i] = 0.f;
      for (int k = a.substeps - 1; k >= 0; --k) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          q[i] = sub_q[k][i];
          qd[i] = sub_qd[k][i];
        }
        substep_adjoint(pat, rec, q, qd, qs, a.h, kGravity, lq, lqd, lqs, lm);
      }
      if (s.valid) {
        float* row = a.dactions + ((size_t)t * E + s.env) * J;
#pragma unroll
        for (int i = 0; i < N; ++i)
          if (pat.active(i)) row[s.jo + i] = lqs[i];
        if (s.c == 0)
          for (int j = s.ntot; j < J; ++j) row[j] = 0.f;
      }
    }
  }
  if (s.valid) {
    float* mrow = a.dmass + (size_t)s.env * J;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      mrow[s.jo + i] = lm[i];
      if (a.dq0) a.dq0[(size_t)s.env * J + s.jo + i] = lq[i];
      if (a.dqd0) a.dqd0[(size_t)s.env * J + s.jo + i] = lqd[i];
    }
    if (s.c == 0) {
      for (int j = s.ntot; j < J; ++j) {
        mrow[j] = 0.f;
        if (a.dq0) a.dq0[(size_t)s.env * J + j] = 0.f;
        if (a.dqd0) a.dqd0[(size_t)s.env * J + j] = 0.f;
      }
    }
  }
}

template <bool kBackward>
__device__ __forceinline__ void diff_dispatch(const DiffArgs& a) {
  extern __shared__ __align__(128) float smem[];
  const int wib = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int gw = blockIdx.x * wpb + wib;
  if (gw >= a.num_warps) return;
  const int wc = a.warp_class[gw];
  float* rec = smem + (size_t)wib * kRecordFloats;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)wpb * kRecordFloats) + wib;
  if (!stage_params(a.params, a.err, gw, wc, rec, bar, lane)) return;
  const Rec r{rec + lane};
  const int slot = gw * kWarp + lane;
  auto run = [&](const auto& pat) {
    if constexpr (kBackward) diff_backward_chain(a, pat, r, slot);
    else diff_forward_chain(a, pat, r, slot);
  };
  switch (wc & 3) {
    case CLS_7R: run(Pat7R{}); break;
    case CLS_7P: run(Pat7P{}); break;
    case CLS_4R: run(Pat4R{}); break;
    default: {
      int code;
      const float cf = r.cf(CF_CODE);
      memcpy(&code, &cf, 4);
      run(PatGen{code, decode_slot(a.slot_info[slot]).nchain});
    }
  }
}

__global__ void __launch_bounds__(kDiffThreads) diff_forward_kernel(DiffArgs a) {
  diff_dispatch<false>(a);
}

__global__ void __launch_bounds__(kDiffThreads) diff_backward_kernel(DiffArgs a) {
  diff_dispatch<true>(a);
}

// link masses (and inertias, which scale with mass) from a caller array [E][J]
__global__ void set_mass_kernel(MassArgs m) {
  const int slot = blockIdx.x * blockDim.x + threadIdx.x;
  if (slot >= m.num_slots) return;
  const int env = m.slot_env[slot];
  if (env < 0) return;
  const SlotFields f = decode_slot(m.slot_info[slot]);
  const int n = f.nchain, jo = f.jo;
  float* rec = m.params + (size_t)(slot / kWarp) * kRecordFloats + (slot % kWarp);
  for (int i = 0; i < n; ++i) {
    const float mnew = m.mass[(size_t)env * m.max_joints + jo + i];
    const size_t k = (size_t)i * m.num_slots + slot;
    const float ratio = mnew / m.mass0[k];
    rec[(kChainFields + i * kLinkFields + LF_M) * kWarp] = mnew;
    rec[(kChainFields + i * kLinkFields + LF_IX) * kWarp] = m.inertia0[k] * ratio;
    rec[(kChainFields + i * kLinkFields + LF_IY) * kWarp] = m.inertia0[k + (size_t)kMaxLinks * m.num_slots] * ratio;
    rec[(kChainFields + i * kLinkFields + LF_IZ) * kWarp] = m.inertia0[k + (size_t)2 * kMaxLinks * m.num_slots] * ratio;
  }
}

size_t diff_smem_bytes(int threads) {
  const int wpb = threads / kWarp;
  return (size_t)wpb * kRecordFloats * sizeof(float) + (size_t)wpb * sizeof(uint64_t);
}

}  // namespace

cudaError_t prepare_diff_kernels() {
  cudaError_t e = cudaFuncSetAttribute(diff_forward_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)diff_smem_bytes(kDiffThreads));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(diff_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)diff_smem_bytes(kDiffThreads));
}

cudaError_t launch_diff_forward(const DiffArgs& a, cudaStream_t s) {
  const int wpb = kDiffThreads / kWarp;
  diff_forward_kernel<<<(a.num_warps + wpb - 1) / wpb, kDiffThreads, diff_smem_bytes(kDiffThreads),
                        s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diff_backward(const DiffArgs& a, cudaStream_t s) {
  const int wpb = kDiffThreads / kWarp;
  diff_backward_kernel<<<(a.num_warps + wpb - 1) / wpb, kDiffThreads,
                         diff_smem_bytes(kDiffThreads), s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_set_mass(const MassArgs& m, cudaStream_t s) {
  const int threads = 256;
  set_mass_kernel<<<(m.num_slots + threads - 1) / threads, threads, 0, s>>>(m);
  return cudaGetLastError();
}

}  // namespace sg
