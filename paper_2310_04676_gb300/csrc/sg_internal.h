// Internal declarations shared by the host packer, the C ABI and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "sg.h"

#ifdef __CUDACC__
#define SG_HD __host__ __device__
#else
#define SG_HD
#endif

namespace sg {

constexpr int kWarp = 32;
constexpr int kMaxLinks = 7;          // joints per chain (SG_MAX_CHAIN_JOINTS)
constexpr int kMaxChains = 4;         // chains per env (SG_MAX_CHAINS)
constexpr int kMaxDof = kMaxLinks * kMaxChains;   // joints per env
constexpr int kMaxPathCtrl = 64;      // control points of a device-built path
constexpr int kChainFields = 8;       // per chain slot: base xyz, goal xyz, joint code, pad
constexpr int kLinkFields = 12;       // per link: see LinkField
constexpr int kRecordFloats = (kChainFields + kMaxLinks * kLinkFields) * kWarp;

enum ChainField { CF_BX = 0, CF_BY, CF_BZ, CF_GX, CF_GY, CF_GZ, CF_CODE, CF_PAD };
enum LinkField {
  LF_L = 0,     // link length
  LF_C,         // COM offset along local z
  LF_M,         // mass
  LF_IX, LF_IY, LF_IZ,   // rotational inertia about the COM
  LF_QLO, LF_QHI,
  LF_KP,        // position stiffness kp (0 for velocity / torque commands)
  LF_D,         // implicit damping: kd + damping (position, velocity) or damping (torque)
  LF_KLIM,
  LF_GA         // command gain: 0 (position), kd (velocity), 1 (torque)
};

// Chain classes: a warp holds 32 chain slots of one class.  The chains of
// one env occupy a lane group of 1, 2 or 4 adjacent lanes (an env with 3
// chains leaves the fourth lane of its group idle); every env of a warp has
// the same group size.
enum ChainClass { CLS_7R = 0, CLS_7P = 1, CLS_GEN = 2, CLS_4R = 3, CLS_COUNT = 4 };
constexpr int kGroupShift = 2;        // warp_class = cls | (log2(group size) << kGroupShift)
SG_HD inline int group_log2(int warp_class) { return (warp_class >> kGroupShift) & 3; }
SG_HD inline int group_log2_of(int num_chains) { return num_chains == 1 ? 0 : (num_chains == 2 ? 1 : 2); }

// slot_info bit fields
constexpr int SI_NCHAIN_SHIFT = 0;    // joints of this chain (3 bits)
constexpr int SI_C_SHIFT = 3;         // chain index within the env / lane in its group (2 bits)
constexpr int SI_NC_SHIFT = 5;        // chains of the env (3 bits)
constexpr int SI_JO_SHIFT = 8;        // first joint of this chain in env joint order (5 bits)
constexpr int SI_NTOT_SHIFT = 13;     // total DOF of the env (5 bits)
constexpr int SI_OBSLEN_SHIFT = 18;   // observation length of the env (7 bits)
struct SlotFields {
  int nchain, c, nc, jo, ntot, obs_len;
};
SG_HD inline SlotFields decode_slot(int info) {
  return SlotFields{(info >> SI_NCHAIN_SHIFT) & 7, (info >> SI_C_SHIFT) & 3,
                    (info >> SI_NC_SHIFT) & 7,     (info >> SI_JO_SHIFT) & 31,
                    (info >> SI_NTOT_SHIFT) & 31,  (info >> SI_OBSLEN_SHIFT) & 127};
}

// Joint code of a generic chain: per joint 3 bits = axis (2 bits) | type << 2.
SG_HD inline int joint_code_bits(int type, int axis) { return (axis & 3) | ((type & 1) << 2); }

// Default wall-clock bound of every device-side wait (2 s)
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;

// Device error flags
constexpr int DEVERR_NONFINITE = 1;
constexpr int DEVERR_TIMEOUT = 2;

struct Plan {
  int num_envs = 0, max_joints = 0, obs_dim = 0, task = 0, path_len = 0, episode_len = 0;
  float alpha = 1.f;
  uint32_t seed = 0;
  float track_sigma = 0.f, track_limit = 0.f;
  int num_slots = 0, num_warps = 0, num_chains = 0;
  int class_slots[CLS_COUNT] = {0, 0, 0, 0};
  std::vector<int32_t> slot_env;    // [NS] caller env index, -1 for padding
  std::vector<int32_t> slot_info;   // [NS] SI_* fields
  std::vector<int32_t> warp_class;  // [NW]
  std::vector<int32_t> env_dof;     // [E] total joints of each env
  std::vector<float> params;        // [NW][kRecordFloats]
  std::vector<float> q0;            // [kMaxLinks][NS]
  std::vector<float> mass0;         // [kMaxLinks][NS] link masses of the description
  std::vector<float> inertia0;      // [3][kMaxLinks][NS] link inertias of the description
  std::vector<float> path;          // [E][W][3] (path task, table given)
  std::vector<float> path_ctrl;     // [E][K][3] (path task, table built on the device)
  int path_ctrl_len = 0;
};

// Validate `d` and build the packing plan; returns SG_OK or an error with *err set.
sg_status build_plan(const sg_desc* d, Plan* plan, std::string* err);

SG_HD inline int record_links(int warp_class) {
  return (warp_class & 3) == CLS_4R ? 4 : kMaxLinks;
}
// bytes of a warp's record that hold data (what one bulk copy moves)
SG_HD inline int record_bytes_dev(int warp_class) {
  return (kChainFields + record_links(warp_class) * kLinkFields) * kWarp * 4;
}

// ---- kernel launch arguments -------------------------------------------
struct StepArgs {
  const float* params;
  const int32_t* slot_env;
  const int32_t* slot_info;
  const int32_t* warp_class;
  float* q;                 // [kMaxLinks][NS]
  float* qd;                // [kMaxLinks][NS]
  int32_t* step_count;      // [E]
  const float* path;        // [E][W][3]
  int32_t* err;             // device error word
  float* track;             // [6][NS] goal offset xyz, goal velocity xyz (tracking task)
  const float* actions;     // [T][E][J]
  float* obs;               // [T][E][D]
  float* reward;            // [T][E]
  uint8_t* done;            // [T][E]
  const uint8_t* obs_mask;  // observe mode: envs whose rows are written (null: all)
  int num_warps, num_slots, num_envs, max_joints, obs_dim, task, path_len, episode_len;
  int substeps, T;
  int observe;              // 1: write the observation of the current state only (T = 1,
                            // no substeps, no reward/done, state and counters unchanged)
  float alpha, h;
  uint32_t seed;
  float track_sigma, track_limit;
  // test hook (sg_debug_set_fault): FAULT_* mode and the wall-clock bound
  // of every device-side wait of the step kernels
  int fault;
  unsigned long long wait_ns;
};

// Test-hook modes (sg.h, sg_debug_set_fault)
constexpr int FAULT_NONE = 0;
constexpr int FAULT_SKIP_PARAM_COPY = 1;   // step kernel: no parameter copy is started
constexpr int FAULT_SKIP_PARTNER = 2;      // warp-pair kernel: role 0 skips its first arrival

}  // namespace sg
