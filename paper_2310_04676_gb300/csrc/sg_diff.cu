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
// Pipelined backward: the same arithmetic split between three warps that
// share 32 chains.  Two replay warps recompute, segment by segment, every
// substep from the segment's checkpoint -- state, joint trigonometry,
// Cholesky factor, drive stiffness and the inverse-dynamics sweeps at the
// substep's acceleration (the part of the substep adjoint that does not
// depend on the cotangent) -- into global segment buffers; the adjoint warp
// stages each substep's record in shared memory with one bulk copy and runs
// only the triangular solve and the reversed sweeps.  mbarriers hand the
// buffers back and forth (bounded waits: a wait that runs out sets
// DEVERR_TIMEOUT and the warps leave).  With replay buffers the forward
// kernel writes the last segment's records itself, so the first reverse pass
// after it starts without waiting for a replay.
#include <cuda_runtime.h>

#include "sg_adjoint.cuh"
#include "sg_chain.cuh"
#include "sg_device.cuh"
#include "sg_diff.h"
#include "sg_internal.h"
#include "sg_pair.cuh"

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

// dL/d(actions) of step t (the env's padding joints as 0, written by chain 0)
template <class Pat>
__device__ __forceinline__ void write_action_grads(const Pat& pat, const DiffArgs& a,
                                                   const SlotInfo& s, int t,
                                                   const float (&lqs)[7]) {
  if (!s.valid) return;
  const int J = a.max_joints;
  float* row = a.dactions + ((size_t)t * a.num_envs + s.env) * J;
#pragma unroll
  for (int i = 0; i < Pat::N; ++i)
    if (pat.active(i)) row[s.jo + i] = lqs[i];
  if (s.c == 0)
    for (int j = s.ntot; j < J; ++j) row[j] = 0.f;
}

// dL/d(link mass) (lm holds it times the mass, see rnea_vjp_rev) and, when
// requested, dL/d(initial q, qd)
template <class Pat>
__device__ __forceinline__ void write_final_grads(const Pat& pat, const DiffArgs& a,
                                                  const Rec& rec, const SlotInfo& s,
                                                  const float (&lq)[7], const float (&lqd)[7],
                                                  const float (&lm)[7]) {
  if (!s.valid) return;
  const int J = a.max_joints;
  const size_t r = (size_t)s.env * J;
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (!pat.active(i)) continue;
    a.dmass[r + s.jo + i] = lm[i] / rec.lf(i, LF_M);
    if (a.dq0) a.dq0[r + s.jo + i] = lq[i];
    if (a.dqd0) a.dqd0[r + s.jo + i] = lqd[i];
  }
  if (s.c == 0) {
    for (int j = s.ntot; j < J; ++j) {
      a.dmass[r + j] = 0.f;
      if (a.dq0) a.dq0[r + j] = 0.f;
      if (a.dqd0) a.dqd0[r + j] = 0.f;
    }
  }
}

// ---- substep records of the pipelined backward (see below) --------------
enum RecordField {
  RF_Q = 0, RF_QD = 7, RF_CQ = 14, RF_SQ = 21, RF_KS = 28, RF_INV = 35, RF_L = 42,
  RF_W = 63, RF_WD = 84, RF_ACC = 105, RF_F = 126, RF_NM = 147, RF_FL = 168, RF_NL = 189,
  RF_JT = 210
};
static_assert(RF_JT + 3 * kMaxLinks == kReplayFields, "record layout");
static_assert((kReplayFields * kWarp * sizeof(float)) % 16 == 0, "bulk copies of records");

constexpr int kPipeGroups = 2;     // chain groups per block
static_assert(kReplayWarps == 2 && kDiffPipeThreads == 8 * kWarp, "warp map of the block");
constexpr int kPipeBars = 3 + 2 * kReplayBufs;   // params, ready[B], freed[B], full[2]
constexpr unsigned kRecordBytes = kReplayFields * kWarp * sizeof(float);
constexpr unsigned long long kHandoffNs = 2000000000ull;   // bound of every wait (2 s)

// strictly lower triangle of L, row by row: (i, j), i > j
__device__ __forceinline__ constexpr int tri_lo(int i, int j) { return i * (i - 1) / 2 + j; }

// record of buffer b, chain group g, substep j of the segment: [field][lane]
__device__ __forceinline__ float* record_at(const DiffArgs& a, int b, int g, int j) {
  const size_t per_seg = (size_t)a.ckpt_every * a.substeps;
  return a.replay + (((size_t)b * a.num_warps + g) * per_seg + j) * (kReplayFields * kWarp);
}

__device__ __forceinline__ void fence_proxy_async_global() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Wait for completion `m` (0-based) of a barrier's phases, i.e. parity m & 1,
// bounded in time; warp-uniform verdict, DEVERR_TIMEOUT on failure.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, unsigned m, int* err, int lane) {
  const bool ok = __all_sync(0xffffffffu, mbar_wait_timed(bar, m & 1u, kHandoffNs));
  if (!ok && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
  return ok;
}

// id_sweeps output written straight into a record (p: record + lane)
struct RecordStore {
  float* p;
  __device__ __forceinline__ void put(int f, V3 v) const {
    p[f * kWarp] = v.x;
    p[(f + 1) * kWarp] = v.y;
    p[(f + 2) * kWarp] = v.z;
  }
  __device__ __forceinline__ void fwd(int i, V3 w, V3 wd, V3 acc, V3 f, V3 n) const {
    put(RF_W + 3 * i, w);
    put(RF_WD + 3 * i, wd);
    put(RF_ACC + 3 * i, acc);
    put(RF_F + 3 * i, f);
    put(RF_NM + 3 * i, n);
  }
  __device__ __forceinline__ void bwd(int i, V3 f, V3 n) const {
    put(RF_FL + 3 * i, f);
    put(RF_NL + 3 * i, n);
  }
};

// tip_jacobian output written into a record (p: record + lane)
struct JacStore {
  float* p;
  __device__ __forceinline__ void jac(int i, V3 v) const {
    p[(RF_JT + 3 * i) * kWarp] = v.x;
    p[(RF_JT + 3 * i + 1) * kWarp] = v.y;
    p[(RF_JT + 3 * i + 2) * kWarp] = v.z;
  }
};

// the sweeps of a record in shared memory (p: record + lane), as read by
// rnea_vjp_rev
struct RecordView {
  const float* p;
  __device__ __forceinline__ V3 at(int f) const {
    return V3{p[f * kWarp], p[(f + 1) * kWarp], p[(f + 2) * kWarp]};
  }
  __device__ __forceinline__ V3 w(int i) const { return at(RF_W + 3 * i); }
  __device__ __forceinline__ V3 wd(int i) const { return at(RF_WD + 3 * i); }
  __device__ __forceinline__ V3 acc(int i) const { return at(RF_ACC + 3 * i); }
  __device__ __forceinline__ V3 f(int i) const { return at(RF_F + 3 * i); }
  __device__ __forceinline__ V3 nm(int i) const { return at(RF_NM + 3 * i); }
  __device__ __forceinline__ V3 fl(int i) const { return at(RF_FL + 3 * i); }
  __device__ __forceinline__ V3 nl(int i) const { return at(RF_NL + 3 * i); }
};

template <class Pat>
__device__ __forceinline__ void put_state(const Pat& pat, float* p, const float (&q)[7],
                                          const float (&qd)[7], const float (&cq)[Pat::N],
                                          const float (&sq)[Pat::N], const float (&ks)[Pat::N],
                                          const float (&inv)[Pat::N],
                                          const float (&M)[Pat::N][Pat::N]) {
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (!pat.active(i)) continue;
    p[(RF_Q + i) * kWarp] = q[i];
    p[(RF_QD + i) * kWarp] = qd[i];
    p[(RF_CQ + i) * kWarp] = cq[i];
    p[(RF_SQ + i) * kWarp] = sq[i];
    p[(RF_KS + i) * kWarp] = ks[i];
    p[(RF_INV + i) * kWarp] = inv[i];
#pragma unroll
    for (int k = 0; k < i; ++k)
      if (pat.active(k)) p[(RF_L + tri_lo(i, k)) * kWarp] = M[i][k];
  }
}

template <class Pat>
__device__ __forceinline__ void get_state(const Pat& pat, const float* p, float (&q)[7],
                                          float (&qd)[7], float (&cq)[Pat::N],
                                          float (&sq)[Pat::N], float (&ks)[Pat::N],
                                          float (&inv)[Pat::N], float (&M)[Pat::N][Pat::N]) {
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    q[i] = 0.f;
    qd[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    cq[i] = 1.f;
    sq[i] = 0.f;
    ks[i] = 0.f;
    inv[i] = 0.f;
#pragma unroll
    for (int k = 0; k < Pat::N; ++k) M[i][k] = 0.f;
    if (!pat.active(i)) continue;
    q[i] = p[(RF_Q + i) * kWarp];
    qd[i] = p[(RF_QD + i) * kWarp];
    cq[i] = p[(RF_CQ + i) * kWarp];
    sq[i] = p[(RF_SQ + i) * kWarp];
    ks[i] = p[(RF_KS + i) * kWarp];
    inv[i] = p[(RF_INV + i) * kWarp];
#pragma unroll
    for (int k = 0; k < i; ++k)
      if (pat.active(k)) M[i][k] = p[(RF_L + tri_lo(i, k)) * kWarp];
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
  constexpr int N = Pat::N;
  const size_t E = (size_t)a.num_envs;
  // with replay buffers, the last segment's substep records go to buffer 0
  // (the reverse pass starts from them instead of replaying that segment)
  const int t_rec = a.replay ? (a.nseg - 1) * a.ckpt_every : a.T;
  const int g = slot / kWarp, lane = slot % kWarp;
  float cq[N], sq[N];                      // trigonometry of q, carried across substeps
  joint_sincos(pat, q, cq, sq);
  for (int t = 0; t < a.T; ++t) {
    if (t % a.ckpt_every == 0) put_ckpt(pat, a, t / a.ckpt_every, slot, q, qd);
    read_targets(pat, a, t, s, qs);
    if (t < t_rec) {
      for (int k = 0; k < a.substeps; ++k)
        chain_substep_trig(pat, rec, q, qd, qs, cq, sq, a.h, kGravity);
    } else {
      for (int k = 0; k < a.substeps; ++k) {
        float M[N][N], inv[N], acc[N], ks[N], dqd[N];
        substep_record(pat, rec, q, qd, qs, a.h, kGravity, cq, sq, M, inv, acc, ks, dqd);
        float* p = record_at(a, 0, g, (t - t_rec) * a.substeps + k) + lane;
        put_state(pat, p, q, qd, cq, sq, ks, inv, M);
        RecordStore st{p};
        id_sweeps(pat, rec, q, qd, acc, cq, sq, kGravity, st);
        integrate(pat, q, qd, dqd, a.h);
      }
      joint_sincos(pat, q, cq, sq);
      JacStore js{record_at(a, 0, g, (t - t_rec + 1) * a.substeps - 1) + lane};
      tip_jacobian(pat, rec, q, cq, sq, js);
    }
    V3 tip, r0, r1, r2;
    chain_tip_trig(pat, rec, q, cq, sq, tip, r0, r1, r2);
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

// Warp-pair forward (batches with a few warps of chains per SM): the substep
// of every chain is split across two warps as in the warp-pair step kernel
// (sg_pair.cuh).  Role 0 writes the checkpoints, role 1 the tool-tip
// positions; with replay buffers, the last segment's substep records are
// written as in the one-thread forward, role 1 the state part (state,
// trigonometry, stiffness, factor) and role 0 the inverse-dynamics sweeps.
template <class Pat>
__device__ __forceinline__ void diff_forward_pair(const DiffArgs& a, const Pat& pat,
                                                  const Rec& rec, int g, int lane, int role,
                                                  float* xbuf, uint64_t* bar_x) {
  constexpr int N = Pat::N;
  const int slot = g * kWarp + lane;
  const SlotInfo s = slot_info(a, slot);
  float q[7], qd[7], qs[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    q[i] = 0.f;
    qd[i] = 0.f;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    q[i] = a.q[(size_t)i * a.num_slots + slot];
    qd[i] = a.qd[(size_t)i * a.num_slots + slot];
  }
  const size_t E = (size_t)a.num_envs;
  const int t_rec = a.replay ? (a.nseg - 1) * a.ckpt_every : a.T;
  float cq[N], sq[N];
  joint_sincos(pat, q, cq, sq);
  unsigned ph_x = 0, xphase = 0;
  for (int t = 0; t < a.T; ++t) {
    if (role == 0 && t % a.ckpt_every == 0) put_ckpt(pat, a, t / a.ckpt_every, slot, q, qd);
    read_targets(pat, a, t, s, qs);
    for (int k = 0; k < a.substeps; ++k, ++xphase) {
      float* xb = xbuf + (xphase & 1) * kXHalf;   // double-buffered exchange
      float L[N][N], inv[N], dqd[N];
      if (!pair_substep(pat, rec, q, qd, qs, cq, sq, a.h, xb, bar_x, ph_x, a.err, lane, role, L,
                        inv, dqd))
        return;
      if (t >= t_rec) {
        float* p = record_at(a, 0, g, (t - t_rec) * a.substeps + k) + lane;
        if (role == 1) {
          float ks[N];
#pragma unroll
          for (int i = 0; i < N; ++i) {
            ks[i] = 0.f;
            if (!pat.active(i)) continue;
            const float kp = rec.lf(i, LF_KP), kl = rec.lf(i, LF_KLIM);
            const float lo = rec.lf(i, LF_QLO), hi = rec.lf(i, LF_QHI);
            ks[i] = kp + ((q[i] > hi || q[i] < lo) ? kl : 0.f);
          }
          put_state(pat, p, q, qd, cq, sq, ks, inv, L);
        } else {
          const float hinv = 1.f / a.h;
          float acc[N];
#pragma unroll
          for (int i = 0; i < N; ++i) acc[i] = pat.active(i) ? dqd[i] * hinv : 0.f;
          RecordStore st{p};
          id_sweeps(pat, rec, q, qd, acc, cq, sq, kGravity, st);
        }
      }
      integrate(pat, q, qd, dqd, a.h);
      joint_sincos(pat, q, cq, sq);
    }
    if (role == 1) {
      if (t >= t_rec) {
        JacStore js{record_at(a, 0, g, (t - t_rec + 1) * a.substeps - 1) + lane};
        tip_jacobian(pat, rec, q, cq, sq, js);
      }
      V3 tip, r0, r1, r2;
      chain_tip_trig(pat, rec, q, cq, sq, tip, r0, r1, r2);
      if (s.valid) {
        float* e = a.ee + (((size_t)t * E + s.env) * kMaxChains + s.c) * 3;
        e[0] = tip.x;
        e[1] = tip.y;
        e[2] = tip.z;
        if (s.c == 0)
          for (int k = 3 * s.nc; k < 3 * kMaxChains; ++k) e[k] = 0.f;
      }
    }
  }
  if (role == 0) put_ckpt(pat, a, a.nseg, slot, q, qd);
}

template <class Pat>
__device__ __forceinline__ void diff_backward_chain(const DiffArgs& a, const Pat& pat,
                                                    const Rec& rec, int slot) {
  constexpr int N = Pat::N;
  const SlotInfo s = slot_info(a, slot);
  const size_t E = (size_t)a.num_envs;
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
      write_action_grads(pat, a, s, t, lqs);
    }
  }
  write_final_grads(pat, a, rec, s, lq, lqd, lm);
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

constexpr int kFwdPairBars = 2;   // params, exchange

__global__ void __launch_bounds__(kDiffPairThreads) diff_forward_pair_kernel(DiffArgs a) {
  extern __shared__ __align__(128) float smem[];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int pairs = blockDim.x >> 6;
  // the first `pairs` warps take role 0, the rest role 1 (as in the step kernel)
  const int pair = w % pairs, role = w / pairs;
  float* rec = smem + (size_t)pair * kRecordFloats;
  float* xbuf = smem + (size_t)pairs * kRecordFloats + (size_t)pair * kXFloats;
  uint64_t* bar0 = reinterpret_cast<uint64_t*>(smem + (size_t)pairs * (kRecordFloats + kXFloats));
  uint64_t* bars = bar0 + (size_t)pair * kFwdPairBars;
  if (w == 0 && lane < pairs) {
    mbar_init(bar0 + (size_t)lane * kFwdPairBars, 1);
    mbar_init(bar0 + (size_t)lane * kFwdPairBars + 1, 2 * kWarp);
  }
  __syncthreads();
  const int g = blockIdx.x * pairs + pair;
  if (g >= a.num_warps) return;
  const int wc = a.warp_class[g];
  if (role == 0 && lane == 0) {
    const unsigned bytes = (unsigned)record_bytes_dev(wc);
    mbar_expect_tx(bars, bytes);
    bulk_g2s(rec, a.params + (size_t)g * kRecordFloats, bytes, bars);
  }
  unsigned ph_tma = 0;
  if (!pair_wait(bars, ph_tma, a.err, lane)) {
    mbar_wait_bounded(bars, 0);   // second bounded chance for an in-flight copy
    return;
  }
  const Rec r{rec + lane};
  auto run = [&](const auto& pat) { diff_forward_pair(a, pat, r, g, lane, role, xbuf, bars + 1); };
  switch (wc & 3) {
    case CLS_7R: run(Pat7R{}); break;
    case CLS_7P: run(Pat7P{}); break;
    case CLS_4R: run(Pat4R{}); break;
    default: {
      int code;
      const float cf = r.cf(CF_CODE);
      memcpy(&code, &cf, 4);
      run(PatGen{code, decode_slot(a.slot_info[g * kWarp + lane]).nchain});
    }
  }
}

size_t diff_fwd_pair_smem_bytes(int threads) {
  const int pairs = threads / (2 * kWarp);
  return (size_t)pairs * (kRecordFloats + kXFloats) * sizeof(float) +
         (size_t)pairs * kFwdPairBars * sizeof(uint64_t);
}

// ---- pipelined backward ----------------------------------------------------
// kReplayWarps + 1 warps share a group of 32 chains: the replay warps and the
// adjoint warp.  Replay warp r takes the segments of order r, r + R, ... (R
// replay warps; order 0 = the last segment): from the segment's checkpoint
// it recomputes every
// substep -- start state, joint trigonometry, Cholesky factor, drive
// stiffness -- and the inverse-dynamics sweeps at the substep's acceleration
// (link velocities, accelerations, inertial and transmitted wrenches: the
// part of the substep adjoint that does not depend on the cotangent), and
// writes them as one record per substep into buffer order % (R + 1).  The adjoint
// warp takes the orders in sequence; it copies each substep's record into
// shared memory with one bulk copy, one substep ahead, and runs the solve and
// the reversed sweeps only.
// Replay warp r: segments of order r, r + R, ..., each into buffer order % (R + 1).
template <class Pat>
__device__ __forceinline__ void replay_role(const DiffArgs& a, const Pat& pat, const Rec& rec,
                                            int g, int slot, int lane, int r, uint64_t* ready,
                                            uint64_t* freed) {
  constexpr int N = Pat::N;
  const SlotInfo s = slot_info(a, slot);
  // order 0 was written by the forward kernel when a.prefilled
  for (int order = (a.prefilled ? 1 : 0) + r; order < a.nseg; order += kReplayWarps) {
    const int seg = a.nseg - 1 - order, b = order % kReplayBufs;
    // the buffer's previous segment (order - R - 1) has been consumed
    if (order >= kReplayBufs && !wait_phase(freed + b, order / kReplayBufs - 1, a.err, lane))
      return;
    const int t0 = seg * a.ckpt_every;
    const int t1 = min(a.T, t0 + a.ckpt_every);
    float q[7], qd[7], qs[7];
    get_ckpt(pat, a, seg, slot, q, qd);
    for (int t = t0; t < t1; ++t) {
      read_targets(pat, a, t, s, qs);
      for (int k = 0; k < a.substeps; ++k) {
        float cq[N], sq[N], M[N][N], inv[N], acc[N], ks[N], dqd[N];
        substep_record(pat, rec, q, qd, qs, a.h, kGravity, cq, sq, M, inv, acc, ks, dqd);
        float* p = record_at(a, b, g, (t - t0) * a.substeps + k) + lane;
        put_state(pat, p, q, qd, cq, sq, ks, inv, M);
        RecordStore st{p};
        id_sweeps(pat, rec, q, qd, acc, cq, sq, kGravity, st);
        integrate(pat, q, qd, dqd, a.h);
      }
      // tool-tip Jacobian of the state after step t (for the tip cotangent)
      float cq[N], sq[N];
      joint_sincos(pat, q, cq, sq);
      JacStore js{record_at(a, b, g, (t - t0 + 1) * a.substeps - 1) + lane};
      tip_jacobian(pat, rec, q, cq, sq, js);
    }
    // the records are visible to the adjoint warp's bulk copies before it is told
    fence_proxy_async_global();
    __threadfence();
    mbar_arrive(ready + b);
  }
}

// Adjoint warp: the reverse sweep, segment by segment, substep records
// staged in shared memory (two slots, one substep ahead).
template <class Pat>
__device__ __forceinline__ void adjoint_role(const DiffArgs& a, const Pat& pat, const Rec& rec,
                                             int g, int slot, int lane, uint64_t* ready,
                                             uint64_t* freed, uint64_t* full, float* stage) {
  constexpr int N = Pat::N;
  const SlotInfo s = slot_info(a, slot);
  const size_t E = (size_t)a.num_envs;
  float lq[7], lqd[7], lm[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    lq[i] = 0.f;
    lqd[i] = 0.f;
    lm[i] = 0.f;
  }
  V3 gnext{0.f, 0.f, 0.f};                     // tip cotangent of the step about to be reversed
  if (s.valid) {
    const float* gp = a.dl_dee + (((size_t)(a.T - 1) * E + s.env) * kMaxChains + s.c) * 3;
    gnext = V3{gp[0], gp[1], gp[2]};
  }
  // record (buffer b, substep j) into slot m & 1
  auto fetch = [&](int b, int j, unsigned m) {
    __syncwarp();                              // every lane is done with the slot
    if (lane == 0) {
      fence_proxy_async_shared();
      mbar_expect_tx(full + (m & 1u), kRecordBytes);
      bulk_g2s(stage + (m & 1u) * (kReplayFields * kWarp), record_at(a, b, g, j), kRecordBytes,
               full + (m & 1u));
    }
  };
  unsigned n = 0;                              // substeps consumed so far
  if (a.prefilled) mbar_arrive(ready);         // buffer 0 holds order 0 already
  for (int order = 0; order < a.nseg; ++order) {
    const int seg = a.nseg - 1 - order, b = order % kReplayBufs;
    if (!wait_phase(ready + b, order / kReplayBufs, a.err, lane)) return;
    __threadfence();
    fence_proxy_async_global();
    const int t0 = seg * a.ckpt_every;
    const int t1 = min(a.T, t0 + a.ckpt_every);
    fetch(b, (t1 - t0) * a.substeps - 1, n);
    for (int t = t1 - 1; t >= t0; --t) {
      float lqs[7];
#pragma unroll
      for (int i = 0; i < 7; ++i) lqs[i] = 0.f;
      for (int k = a.substeps - 1; k >= 0; --k, ++n) {
        const int j = (t - t0) * a.substeps + k;
        if (!wait_phase(full + (n & 1u), n >> 1, a.err, lane)) {
          mbar_wait_timed(full + (n & 1u), (n >> 1) & 1u, kHandoffNs);   // the copy in flight
          return;
        }
        if (j > 0) fetch(b, j - 1, n + 1);
        const float* p = stage + (n & 1u) * (kReplayFields * kWarp) + lane;
        if (k == a.substeps - 1 && s.valid) {
          // tip cotangent of the state after step t: lq += J^T g
#pragma unroll
          for (int i = 0; i < N; ++i) {
            if (!pat.active(i)) continue;
            lq[i] += gnext.x * p[(RF_JT + 3 * i) * kWarp] +
                     gnext.y * p[(RF_JT + 3 * i + 1) * kWarp] +
                     gnext.z * p[(RF_JT + 3 * i + 2) * kWarp];
          }
          if (t > 0) {                         // the next step's, loaded ahead
            const float* gp = a.dl_dee + (((size_t)(t - 1) * E + s.env) * kMaxChains + s.c) * 3;
            gnext = V3{gp[0], gp[1], gp[2]};
          }
        }
        float q[7], qd[7], cq[N], sq[N], M[N][N], inv[N], ks[N];
        get_state(pat, p, q, qd, cq, sq, ks, inv, M);
        substep_adjoint_sw(pat, rec, q, qd, cq, sq, M, inv, ks, RecordView{p}, a.h, lq, lqd, lqs,
                           lm);
      }
      write_action_grads(pat, a, s, t, lqs);
    }
    __syncwarp();
    mbar_arrive(freed + b);
  }
  write_final_grads(pat, a, rec, s, lq, lqd, lm);
}

__global__ void __launch_bounds__(kDiffPipeThreads) diff_backward_pipe_kernel(DiffArgs a) {
  extern __shared__ __align__(128) float smem[];
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  // Two groups per block of 8 warps.  The adjoint warps (the critical path)
  // take warps 0 and 1, the replay warps 2, 3 (first) and 6, 7 (second);
  // warps 4 and 5 leave at once.  With warps spread over the SM's four
  // schedulers by index, each adjoint warp has a scheduler of its own
  // (measured 2.5% faster than three warps per group back to back).
  constexpr int groups = kPipeGroups;
  const int grp = w & 1;
  const int role = w < 2 ? kReplayWarps : (w < 4 ? 0 : (w < 6 ? -1 : 1));
  float* rec = smem + (size_t)grp * kRecordFloats;
  float* stage = smem + (size_t)groups * kRecordFloats + (size_t)grp * 2 * kReplayFields * kWarp;
  uint64_t* bar0 = reinterpret_cast<uint64_t*>(
      smem + (size_t)groups * (kRecordFloats + 2 * kReplayFields * kWarp));
  uint64_t* bars = bar0 + (size_t)grp * kPipeBars;
  // start-up: warp 0 initialises every group's barriers before any warp leaves
  if (w == 0 && lane < groups) {
    uint64_t* bb = bar0 + (size_t)lane * kPipeBars;
    mbar_init(bb + 0, 1);
    for (int k = 1; k < 1 + 2 * kReplayBufs; ++k) mbar_init(bb + k, kWarp);   // ready, freed
    mbar_init(bb + 1 + 2 * kReplayBufs, 1);                                   // full[2]
    mbar_init(bb + 2 + 2 * kReplayBufs, 1);
  }
  __syncthreads();
  if (role < 0) return;
  const int g = blockIdx.x * groups + grp;
  if (g >= a.num_warps) return;
  const int wc = a.warp_class[g];
  if (role == 0 && lane == 0) {
    const unsigned bytes = (unsigned)record_bytes_dev(wc);
    mbar_expect_tx(bars, bytes);
    bulk_g2s(rec, a.params + (size_t)g * kRecordFloats, bytes, bars);
  }
  unsigned ph_tma = 0;
  if (!pair_wait(bars, ph_tma, a.err, lane)) {
    mbar_wait_bounded(bars, 0);   // second bounded chance for an in-flight copy
    return;
  }
  const Rec r{rec + lane};
  const int slot = g * kWarp + lane;
  auto run = [&](const auto& pat) {
    if (role < kReplayWarps)
      replay_role(a, pat, r, g, slot, lane, role, bars + 1, bars + 1 + kReplayBufs);
    else
      adjoint_role(a, pat, r, g, slot, lane, bars + 1, bars + 1 + kReplayBufs,
                   bars + 1 + 2 * kReplayBufs, stage);
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

size_t diff_pipe_smem_bytes() {
  return (size_t)kPipeGroups * (kRecordFloats + 2 * kReplayFields * kWarp) * sizeof(float) +
         (size_t)kPipeGroups * kPipeBars * sizeof(uint64_t);
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
  e = cudaFuncSetAttribute(diff_forward_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)diff_fwd_pair_smem_bytes(kDiffPairThreads));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(diff_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)diff_smem_bytes(kDiffThreads));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(diff_backward_pipe_kernel,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)diff_pipe_smem_bytes());
}

cudaError_t launch_diff_forward(const DiffArgs& a, cudaStream_t s) {
  // a few warps of chains per SM: split each substep across a warp pair
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return cudaGetLastError();
  if (a.num_warps <= kDiffPairMaxWarpsPerSM * sms) {
    const int pairs = kDiffPairThreads / (2 * kWarp);
    diff_forward_pair_kernel<<<(a.num_warps + pairs - 1) / pairs, kDiffPairThreads,
                               diff_fwd_pair_smem_bytes(kDiffPairThreads), s>>>(a);
    return cudaGetLastError();
  }
  const int wpb = kDiffThreads / kWarp;
  diff_forward_kernel<<<(a.num_warps + wpb - 1) / wpb, kDiffThreads, diff_smem_bytes(kDiffThreads),
                        s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diff_backward(const DiffArgs& a, cudaStream_t s) {
  if (a.replay) {
    diff_backward_pipe_kernel<<<(a.num_warps + kPipeGroups - 1) / kPipeGroups, kDiffPipeThreads,
                                diff_pipe_smem_bytes(), s>>>(a);
    return cudaGetLastError();
  }
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
