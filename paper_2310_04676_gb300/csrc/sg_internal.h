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
constexpr int kMaxDof = 14;           // joints per env
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

// Chain classes: a warp holds 32 chain slots of one class, all single-chain
// envs or all two-chain envs (lanes 2k, 2k+1 = chains 0, 1 of one env).
enum ChainClass { CLS_7R = 0, CLS_7P = 1, CLS_GEN = 2, CLS_4R = 3, CLS_COUNT = 4 };
constexpr int kPairedBit = 4;         // warp_class = cls | (paired ? kPairedBit : 0)

// slot_info bit fields
constexpr int SI_NCHAIN_SHIFT = 0;    // joints of this chain (3 bits)
constexpr int SI_C_SHIFT = 3;         // chain index within the env (1 bit)
constexpr int SI_NC_SHIFT = 4;        // chains of the env (2 bits)
constexpr int SI_JO_SHIFT = 6;        // first joint of this chain in env joint order (4 bits)
constexpr int SI_NTOT_SHIFT = 10;     // total DOF of the env (5 bits)
constexpr int SI_OBSLEN_SHIFT = 15;   // observation length of the env (7 bits)

// Joint code of a generic chain: per joint 3 bits = axis (2 bits) | type << 2.
SG_HD inline int joint_code_bits(int type, int axis) { return (axis & 3) | ((type & 1) << 2); }

// Device error flags
constexpr int DEVERR_NONFINITE = 1;
constexpr int DEVERR_TIMEOUT = 2;

struct Plan {
  int num_envs = 0, max_joints = 0, obs_dim = 0, task = 0, path_len = 0, episode_len = 0;
  float alpha = 1.f;
  int num_slots = 0, num_warps = 0, num_chains = 0;
  int class_slots[CLS_COUNT] = {0, 0, 0, 0};
  std::vector<int32_t> slot_env;    // [NS] caller env index, -1 for padding
  std::vector<int32_t> slot_info;   // [NS] SI_* fields
  std::vector<int32_t> warp_class;  // [NW]
  std::vector<float> params;        // [NW][kRecordFloats]
  std::vector<float> q0;            // [kMaxLinks][NS]
  std::vector<float> mass0;         // [kMaxLinks][NS] link masses of the description
  std::vector<float> inertia0;      // [3][kMaxLinks][NS] link inertias of the description
  std::vector<float> path;          // [E][W][3] (path task)
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
  const float* actions;     // [T][E][J]
  float* obs;               // [T][E][D]
  float* reward;            // [T][E]
  uint8_t* done;            // [T][E]
  int num_warps, num_slots, num_envs, max_joints, obs_dim, task, path_len, episode_len;
  int substeps, T;
  float alpha, h;
};

}  // namespace sg
