// Host-side robot-description packer: validates an sg_desc and lays the
// environments out as warp-sized blocks of chain slots for the step kernel.
//
// Layout decisions (GB300-first):
//  * one CUDA thread integrates one serial chain; the chains of a
//    multi-arm env occupy a lane group of 2 or 4 adjacent lanes (a 3-arm env
//    leaves the fourth lane of its group idle);
//  * every warp holds chains of a single class (7R, 7P, generic, 4R) so the
//    kernel dispatches once per warp with no divergence;
//  * chains are grouped by class, longest chains first (their warps are
//    scheduled first), caller env order kept within a class;
//  * the parameters of one warp form a contiguous record
//    [chain fields][link][link fields] x 32 lanes (structure of arrays per
//    warp), so one bulk copy stages a warp's parameters in shared memory and
//    every lane then reads its own column without bank conflicts.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <sstream>

#include "sg_internal.h"
#include "sg_pack.h"

namespace sg {
namespace {

const int kAxes7[7] = {2, 1, 2, 1, 2, 1, 2};

int classify(int n, const int32_t* types, const int32_t* axes) {
  bool zy = true;
  for (int i = 0; i < n; ++i) zy = zy && axes[i] == kAxes7[i];
  if (!zy) return CLS_GEN;
  bool all_rev = true;
  for (int i = 0; i < n; ++i) all_rev = all_rev && types[i] == SG_JOINT_REVOLUTE;
  if (n == 7 && all_rev) return CLS_7R;
  if (n == 4 && all_rev) return CLS_4R;
  if (n == 7) {
    bool p = true;
    for (int i = 0; i < 7; ++i) p = p && types[i] == (i == 2 ? SG_JOINT_PRISMATIC : SG_JOINT_REVOLUTE);
    if (p) return CLS_7P;
  }
  return CLS_GEN;
}

bool finite(float x) { return std::isfinite(x); }

}  // namespace

sg_status build_plan(const sg_desc* d, Plan* P, std::string* err) {
  auto fail = [&](sg_status code, const std::string& m) {
    *err = m;
    return code;
  };
  if (!d) return fail(SG_ERR_INVALID_ARG, "desc is NULL");
  const int E = d->num_envs, J = d->max_joints;
  if (E < 1 || E > (1 << 26)) return fail(SG_ERR_INVALID_ARG, "num_envs out of range");
  if (J < 1 || J > kMaxDof) return fail(SG_ERR_INVALID_ARG, "max_joints must be 1..28");
  if (!d->env_num_chains || !d->chain_num_joints || !d->joint_type || !d->joint_axis ||
      !d->link_len || !d->link_mass || !d->link_inertia || !d->link_com || !d->q_lo ||
      !d->q_hi || !d->kp || !d->kd || !d->damping || !d->k_limit || !d->base_offset || !d->q0)
    return fail(SG_ERR_INVALID_ARG, "a required desc array is NULL");
  if (d->episode_len < 1) return fail(SG_ERR_INVALID_ARG, "episode_len must be >= 1");
  if (d->task != SG_TASK_REACH && d->task != SG_TASK_PATH && d->task != SG_TASK_TRACK)
    return fail(SG_ERR_INVALID_ARG, "unknown task");
  if (d->task != SG_TASK_PATH && !d->goal) return fail(SG_ERR_INVALID_ARG, "goal is NULL");
  if (d->task == SG_TASK_TRACK &&
      (!(d->track_sigma > 0.f) || !(d->track_limit > 0.f) || !finite(d->track_sigma) ||
       !finite(d->track_limit)))
    return fail(SG_ERR_INVALID_ARG, "tracking needs track_sigma > 0 and track_limit > 0");
  if (d->task == SG_TASK_PATH) {
    if (d->path_len < 4) return fail(SG_ERR_INVALID_ARG, "path task needs path_len >= 4");
    if ((d->path != nullptr) == (d->path_ctrl != nullptr))
      return fail(SG_ERR_INVALID_ARG, "path task needs exactly one of path and path_ctrl");
    if (d->path_ctrl) {
      if (d->path_ctrl_len < 2 || d->path_ctrl_len > kMaxPathCtrl)
        return fail(SG_ERR_INVALID_ARG, "path_ctrl_len must be 2..64");
      const size_t n = (size_t)E * d->path_ctrl_len * 3;
      for (size_t i = 0; i < n; ++i)
        if (!finite(d->path_ctrl[i])) return fail(SG_ERR_INVALID_ARG, "non-finite path_ctrl");
    }
    if (!finite(d->alpha)) return fail(SG_ERR_INVALID_ARG, "alpha not finite");
  }

  // ---- validate envs and classify chains --------------------------------
  std::vector<int> env_cls(E), env_ntot(E), env_nc(E);
  for (int e = 0; e < E; ++e) {
    const int nc = d->env_num_chains[e];
    if (nc < 1 || nc > SG_MAX_CHAINS) {
      std::ostringstream o;
      o << "env " << e << ": env_num_chains must be 1..4";
      return fail(SG_ERR_INVALID_ARG, o.str());
    }
    if (d->task == SG_TASK_PATH && nc != 1)
      return fail(SG_ERR_UNSUPPORTED, "path following is defined for single-chain envs");
    int ntot = 0, cls[kMaxChains] = {0, 0, 0, 0};
    for (int c = 0; c < nc; ++c) {
      const int n = d->chain_num_joints[kMaxChains * e + c];
      if (n < 1 || n > kMaxLinks) {
        std::ostringstream o;
        o << "env " << e << ": chain_num_joints must be 1..7";
        return fail(SG_ERR_INVALID_ARG, o.str());
      }
      if (ntot + n > J) return fail(SG_ERR_INVALID_ARG, "env DOF exceeds max_joints");
      const int32_t* ty = d->joint_type + (size_t)e * J + ntot;
      const int32_t* ax = d->joint_axis + (size_t)e * J + ntot;
      for (int i = 0; i < n; ++i) {
        if (ty[i] != SG_JOINT_REVOLUTE && ty[i] != SG_JOINT_PRISMATIC)
          return fail(SG_ERR_INVALID_ARG, "joint_type must be 0 or 1");
        if (ax[i] < 0 || ax[i] > 2) return fail(SG_ERR_INVALID_ARG, "joint_axis must be 0..2");
        if (ty[i] == SG_JOINT_PRISMATIC && ax[i] != 2)
          return fail(SG_ERR_UNSUPPORTED, "prismatic joints translate along local z only (axis 2)");
        const size_t k = (size_t)e * J + ntot + i;
        const float* in = d->link_inertia + 3 * k;
        const float vals[] = {d->link_len[k], d->link_com[k], d->q_lo[k], d->q_hi[k], d->kp[k],
                              d->kd[k], d->damping[k], d->k_limit[k], d->q0[k]};
        for (float v : vals)
          if (!finite(v)) return fail(SG_ERR_INVALID_ARG, "non-finite joint parameter");
        if (!(d->link_mass[k] > 0.f) || !finite(d->link_mass[k]))
          return fail(SG_ERR_INVALID_ARG, "link_mass must be > 0");
        if (!(in[0] > 0.f && in[1] > 0.f && in[2] > 0.f) || !finite(in[0] + in[1] + in[2]))
          return fail(SG_ERR_INVALID_ARG, "link_inertia entries must be > 0");
        if (d->kp[k] < 0.f || d->kd[k] < 0.f || d->damping[k] < 0.f || d->k_limit[k] < 0.f)
          return fail(SG_ERR_INVALID_ARG, "gains and damping must be >= 0");
        if (d->joint_drive && (d->joint_drive[k] < SG_DRIVE_POSITION || d->joint_drive[k] > SG_DRIVE_TORQUE))
          return fail(SG_ERR_INVALID_ARG, "joint_drive must be 0 (position), 1 (velocity) or 2 (torque)");
      }
      cls[c] = classify(n, ty, ax);
      ntot += n;
    }
    int k = cls[0];
    for (int c = 1; c < nc; ++c)
      if (cls[c] != cls[0]) k = CLS_GEN;
    env_cls[e] = k;
    env_ntot[e] = ntot;
    env_nc[e] = nc;
  }

  // ---- order the chain slots ---------------------------------------------
  P->env_dof.assign(env_ntot.begin(), env_ntot.end());
  P->num_envs = E;
  P->max_joints = J;
  P->task = d->task;
  P->path_len = d->task == SG_TASK_PATH ? d->path_len : 0;
  P->episode_len = d->episode_len;
  P->alpha = d->alpha;
  P->seed = d->seed;
  P->track_sigma = d->task == SG_TASK_TRACK ? d->track_sigma : 0.f;
  P->track_limit = d->task == SG_TASK_TRACK ? d->track_limit : 0.f;
  P->obs_dim = 0;
  auto obs_len = [&](int e) {
    return d->task == SG_TASK_PATH ? 2 * env_ntot[e] + 16 : 3 * env_ntot[e] + 6 * env_nc[e];
  };
  for (int e = 0; e < E; ++e) P->obs_dim = std::max(P->obs_dim, obs_len(e));
  if (P->obs_dim > 127) return fail(SG_ERR_UNSUPPORTED, "observation rows wider than 127 floats");

  static const int kOrder[CLS_COUNT] = {CLS_7R, CLS_7P, CLS_GEN, CLS_4R};
  P->slot_env.clear();
  P->slot_info.clear();
  P->warp_class.clear();
  std::vector<int> slot_chain;   // chain index (lane in its group) of each slot
  P->num_chains = 0;
  for (int k : kOrder) {
    for (int glog = 2; glog >= 0; --glog) {
      const int g = 1 << glog;
      const int first = (int)P->slot_env.size();
      for (int e = 0; e < E; ++e) {
        if (env_cls[e] != k || group_log2_of(env_nc[e]) != glog) continue;
        for (int c = 0; c < g; ++c) {
          P->slot_env.push_back(c < env_nc[e] ? e : -1 - e);   // idle lane of a 3-arm group
          slot_chain.push_back(c);
        }
        P->class_slots[k] += env_nc[e];
        P->num_chains += env_nc[e];
      }
      const int cnt = (int)P->slot_env.size() - first;
      if (cnt == 0) continue;
      const int padded = (cnt + kWarp - 1) / kWarp * kWarp;
      const int ref_env = P->slot_env[first];
      for (int s = cnt; s < padded; ++s) {
        P->slot_env.push_back(-1 - ref_env);       // padding: copy of a real chain
        slot_chain.push_back(s % g);
      }
      for (int w = 0; w < padded / kWarp; ++w) P->warp_class.push_back(k | (glog << kGroupShift));
    }
  }
  const int NS = (int)P->slot_env.size();
  P->num_slots = NS;
  P->num_warps = NS / kWarp;

  // ---- fill records, slot info and q0 ------------------------------------
  P->params.assign((size_t)P->num_warps * kRecordFloats, 0.f);
  P->q0.assign((size_t)kMaxLinks * NS, 0.f);
  P->mass0.assign((size_t)kMaxLinks * NS, 1.f);
  P->inertia0.assign((size_t)3 * kMaxLinks * NS, 1.f);
  P->slot_info.assign(NS, 0);
  for (int s = 0; s < NS; ++s) {
    const bool pad = P->slot_env[s] < 0;
    const int e = pad ? -1 - P->slot_env[s] : P->slot_env[s];
    const int c = slot_chain[s];
    const int cc = c < env_nc[e] ? c : 0;          // chain whose parameters the slot holds
    const int n = d->chain_num_joints[kMaxChains * e + cc];
    int jo = 0;
    for (int j = 0; j < cc; ++j) jo += d->chain_num_joints[kMaxChains * e + j];
    P->slot_info[s] = (n << SI_NCHAIN_SHIFT) | (c << SI_C_SHIFT) | (env_nc[e] << SI_NC_SHIFT) |
                      (jo << SI_JO_SHIFT) | (env_ntot[e] << SI_NTOT_SHIFT) |
                      (obs_len(e) << SI_OBSLEN_SHIFT);
    if (pad) P->slot_env[s] = -1;
    float* rec = P->params.data() + (size_t)(s / kWarp) * kRecordFloats;
    const int lane = s % kWarp;
    auto CF = [&](int f) -> float& { return rec[f * kWarp + lane]; };
    auto LF = [&](int i, int f) -> float& {
      return rec[(kChainFields + i * kLinkFields + f) * kWarp + lane];
    };
    for (int a = 0; a < 3; ++a) {
      CF(CF_BX + a) = d->base_offset[(size_t)(kMaxChains * e + cc) * 3 + a];
      CF(CF_GX + a) = d->goal ? d->goal[(size_t)(kMaxChains * e + cc) * 3 + a] : 0.f;
    }
    int code = 0;
    for (int i = 0; i < n; ++i) {
      const size_t k = (size_t)e * J + jo + i;
      code |= joint_code_bits(d->joint_type[k], d->joint_axis[k]) << (3 * i);
      LF(i, LF_L) = d->link_len[k];
      LF(i, LF_C) = d->link_com[k];
      LF(i, LF_M) = d->link_mass[k];
      LF(i, LF_IX) = d->link_inertia[3 * k + 0];
      LF(i, LF_IY) = d->link_inertia[3 * k + 1];
      LF(i, LF_IZ) = d->link_inertia[3 * k + 2];
      LF(i, LF_QLO) = d->q_lo[k];
      LF(i, LF_QHI) = d->q_hi[k];
      const int mode = d->joint_drive ? d->joint_drive[k] : SG_DRIVE_POSITION;
      LF(i, LF_KP) = mode == SG_DRIVE_POSITION ? d->kp[k] : 0.f;
      LF(i, LF_D) = mode == SG_DRIVE_TORQUE ? d->damping[k] : d->kd[k] + d->damping[k];
      LF(i, LF_KLIM) = d->k_limit[k];
      LF(i, LF_GA) = mode == SG_DRIVE_POSITION ? 0.f : (mode == SG_DRIVE_VELOCITY ? d->kd[k] : 1.f);
      P->q0[(size_t)i * NS + s] = d->q0[k];
      P->mass0[(size_t)i * NS + s] = d->link_mass[k];
      for (int a = 0; a < 3; ++a)
        P->inertia0[((size_t)a * kMaxLinks + i) * NS + s] = d->link_inertia[3 * k + a];
    }
    std::memcpy(&CF(CF_CODE), &code, 4);
  }
  P->path.clear();
  P->path_ctrl.clear();
  P->path_ctrl_len = 0;
  if (d->task == SG_TASK_PATH && d->path) {
    P->path.assign(d->path, d->path + (size_t)E * d->path_len * 3);
  } else if (d->task == SG_TASK_PATH) {
    P->path_ctrl.assign(d->path_ctrl, d->path_ctrl + (size_t)E * d->path_ctrl_len * 3);
    P->path_ctrl_len = d->path_ctrl_len;
  }
  return SG_OK;
}

std::vector<int32_t> packing_order(const Plan& P, int packing) {
  const int NW = P.num_warps;
  std::vector<int32_t> order(NW);
  for (int w = 0; w < NW; ++w) order[w] = w;
  if (packing != SG_PACK_INTERLEAVE) return order;
  // the class-grouped order's runs of one warp class; warp i of a run of n
  // warps goes to fractional position (2 i + 1) / (2 n), ties in run order
  // (exact integer comparisons, so every platform builds the same order)
  struct Key {
    long long num, den;
    int run, w;
  };
  std::vector<Key> keys;
  keys.reserve(NW);
  int run = 0;
  for (int w0 = 0; w0 < NW;) {
    int w1 = w0;
    while (w1 < NW && P.warp_class[w1] == P.warp_class[w0]) ++w1;
    const int n = w1 - w0;
    for (int i = 0; i < n; ++i) keys.push_back(Key{2LL * i + 1, 2LL * n, run, w0 + i});
    ++run;
    w0 = w1;
  }
  std::stable_sort(keys.begin(), keys.end(), [](const Key& a, const Key& b) {
    const long long l = a.num * b.den, r = b.num * a.den;
    return l < r || (l == r && a.run < b.run);
  });
  for (int w = 0; w < NW; ++w) order[w] = keys[w].w;
  return order;
}

}  // namespace sg
