// Host build of the device chain code in double precision, for the CPU tests
// (test infrastructure, not part of the library).
//
// The device headers sg_chain.cuh, sg_adjoint.cuh and sg_rng.cuh are
// compiled for the host with `float` replaced by `double` (the copies are
// made by tests/test_host_chain.py); the parameter records are those of the
// library's own host packer (sg_pack.cpp).  The entry points run one
// substep, one substep adjoint, the tip kinematics of one chain of one env,
// or one draw of the counter-based noise, so the device algorithm can be
// compared with the FP64 oracle to double-precision rounding, without a
// GPU.
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>

inline void __sincosf(double x, double* s, double* c) {
  *s = std::sin(x);
  *c = std::cos(x);
}
inline double rsqrtf(double x) { return 1.0 / std::sqrt(x); }
inline double sqrtf(double x) { return std::sqrt(x); }
inline double fminf(double a, double b) { return a < b ? a : b; }
inline double fmaxf(double a, double b) { return a > b ? a : b; }
inline double logf(double x) { return std::log(x); }
inline void sincospif(double x, double* s, double* c) {
  const double pi = 3.14159265358979323846;
  *s = std::sin(pi * x);
  *c = std::cos(pi * x);
}

#define __device__
#define __forceinline__ inline
#include "sg_internal.h"
#include "chain_host.h"     // sg_chain.cuh with float -> double
#include "adjoint_host.h"   // sg_adjoint.cuh with float -> double
#include "rng_host.h"       // sg_rng.cuh with float -> double

using namespace sg;

namespace {

Plan g_plan;
double g_rec[kRecordFloats];
constexpr double kGrav = 9.81;

// Runs f(pattern, record view, number of joints) for chain c of env e.
template <class F>
int with_chain(int e, int c, F f) {
  int s = -1;
  for (int k = 0; k < g_plan.num_slots && s < 0; ++k)
    if (g_plan.slot_env[k] == e && decode_slot(g_plan.slot_info[k]).c == c) s = k;
  if (s < 0) return -1;
  const int w = s / kWarp, lane = s % kWarp;
  const float* src = g_plan.params.data() + (size_t)w * kRecordFloats;
  for (int i = 0; i < kRecordFloats; ++i) g_rec[i] = src[i];
  const Rec r{g_rec + lane};
  const int n = decode_slot(g_plan.slot_info[s]).nchain;
  switch (g_plan.warp_class[w] & 3) {
    case CLS_7R: return f(Pat7R{}, r, n);
    case CLS_7P: return f(Pat7P{}, r, n);
    case CLS_4R: return f(Pat4R{}, r, n);
    default: {
      int code;
      std::memcpy(&code, &src[CF_CODE * kWarp + lane], 4);
      return f(PatGen{code, n}, r, n);
    }
  }
}

void load(const double* src, int n, double (&dst)[7]) {
  for (int i = 0; i < 7; ++i) dst[i] = i < n ? src[i] : 0.0;
}

}  // namespace

extern "C" {

// Pack a description with the library's packer; returns the slot count or -1.
int host_plan(const sg_desc* d) {
  std::string err;
  return build_plan(d, &g_plan, &err) == SG_OK ? g_plan.num_slots : -1;
}

// One substep of chain c of env e from (q, qd) with commands qs: writes q',
// qd'; returns the chain's joint count (or -1).
int host_substep(int e, int c, const double* q_in, const double* qd_in, const double* qs_in,
                 double h, double* q_out, double* qd_out) {
  return with_chain(e, c, [&](auto pat, const Rec& r, int n) {
    double q[7], qd[7], qs[7];
    load(q_in, n, q);
    load(qd_in, n, qd);
    load(qs_in, n, qs);
    chain_substep(pat, r, q, qd, qs, h, kGrav);
    for (int i = 0; i < n; ++i) {
      q_out[i] = q[i];
      qd_out[i] = qd[i];
    }
    return n;
  });
}

// Adjoint of that substep: lq, lqd hold the cotangents of (q', qd') on entry
// and those of (q, qd) on exit; lqs, lm receive those of the commands and the
// link masses.
int host_substep_adjoint(int e, int c, const double* q_in, const double* qd_in,
                         const double* qs_in, double h, double* lq_io, double* lqd_io,
                         double* lqs_out, double* lm_out) {
  return with_chain(e, c, [&](auto pat, const Rec& r, int n) {
    double q[7], qd[7], qs[7], lq[7], lqd[7], lqs[7] = {0}, lm[7] = {0};
    load(q_in, n, q);
    load(qd_in, n, qd);
    load(qs_in, n, qs);
    load(lq_io, n, lq);
    load(lqd_io, n, lqd);
    substep_adjoint(pat, r, q, qd, qs, h, kGrav, lq, lqd, lqs, lm);
    for (int i = 0; i < n; ++i) {
      lq_io[i] = lq[i];
      lqd_io[i] = lqd[i];
      lqs_out[i] = lqs[i];
      lm_out[i] = lm[i] / r.lf(i, LF_M);   // lm holds dL/dm times the mass
    }
    return n;
  });
}

// Tool-tip position and tip-frame quaternion (x, y, z, w) of chain c of env e.
int host_tip(int e, int c, const double* q_in, double* tip_out, double* quat_out) {
  return with_chain(e, c, [&](auto pat, const Rec& r, int n) {
    double q[7];
    load(q_in, n, q);
    V3 tip, r0, r1, r2;
    chain_tip(pat, r, q, tip, r0, r1, r2);
    tip_out[0] = tip.x;
    tip_out[1] = tip.y;
    tip_out[2] = tip.z;
    rot_to_quat(r0, r1, r2, quat_out);
    return n;
  });
}

// gq = J_tip(q)^T gbar for chain c of env e.
int host_tip_vjp(int e, int c, const double* q_in, const double* gbar, double* gq_out) {
  return with_chain(e, c, [&](auto pat, const Rec& r, int n) {
    constexpr int N = std::decay_t<decltype(pat)>::N;
    double q[7], gq[N];
    load(q_in, n, q);
    for (int i = 0; i < N; ++i) gq[i] = 0.0;
    tip_vjp(pat, r, q, V3{gbar[0], gbar[1], gbar[2]}, gq);
    for (int i = 0; i < n; ++i) gq_out[i] = gq[i];
    return n;
  });
}

// Joint torques tau = ID(q, qd, qdd) of chain c of env e from the adjoint's
// inverse-dynamics sweeps: the wrench each link transmits to its parent,
// about the joint axis (revolute) or along it (prismatic).
int host_inverse_dynamics(int e, int c, const double* q_in, const double* qd_in,
                          const double* qdd_in, double* tau_out) {
  return with_chain(e, c, [&](auto pat, const Rec& r, int n) {
    constexpr int N = std::decay_t<decltype(pat)>::N;
    double q[7], qd[7], qdd[N], cq[N], sq[N];
    load(q_in, n, q);
    load(qd_in, n, qd);
    for (int i = 0; i < N; ++i) qdd[i] = i < n ? qdd_in[i] : 0.0;
    joint_sincos(pat, q, cq, sq);
    SweepArrays<N> sw;
    id_sweeps(pat, r, q, qd, qdd, cq, sq, kGrav, sw);
    for (int i = 0; i < n; ++i)
      tau_out[i] = pat.type(i) == 1 ? sw.FL[i].z : compc(sw.NL[i], pat.axis(i));
    return n;
  });
}

// One substep computed as the warp pair splits it (role 0: bias forces and
// right-hand side; role 1: mass matrix, armature and factor; then the shared
// solve), run one role after the other.
int host_substep_split(int e, int c, const double* q_in, const double* qd_in,
                       const double* qs_in, double h, double* q_out, double* qd_out) {
  return with_chain(e, c, [&](auto pat, const Rec& r, int n) {
    constexpr int N = std::decay_t<decltype(pat)>::N;
    double q[7], qd[7], qs[7], cq[N], sq[N];
    load(q_in, n, q);
    load(qd_in, n, qd);
    load(qs_in, n, qs);
    joint_sincos(pat, q, cq, sq);
    double bias[N], rhs[N], arm[N], Mdummy[N][N];
    V3 F[N], Nm[N];
    rnea_forward(pat, r, q, qd, cq, sq, kGrav, F, Nm);
    backward_sweep<decltype(pat), true, false>(pat, r, q, cq, sq, F, Nm, bias, Mdummy);
    drive_terms(pat, r, q, qd, qs, h, bias, rhs, arm);
    double M[N][N], inv[N], bias1[N] = {}, rhs1[N], arm1[N];
    V3 Fd[N] = {}, Nd[N] = {};
    backward_sweep<decltype(pat), false, true>(pat, r, q, cq, sq, Fd, Nd, bias1, M);
    drive_terms(pat, r, q, qd, qs, h, bias1, rhs1, arm1);
    chol_factor(pat, M, arm1, inv);
    chol_apply(pat, M, inv, rhs);
    integrate(pat, q, qd, rhs, h);
    for (int i = 0; i < n; ++i) {
      q_out[i] = q[i];
      qd_out[i] = qd[i];
    }
    return n;
  });
}

// Counter-based noise draws (tracking goals, policy exploration).
void host_goal_noise(uint32_t seed, int env, int chain, int step, double* z) {
  goal_noise(seed, env, chain, step, z[0], z[1], z[2]);
}

void host_action_noise(uint32_t seed, int env, int block, long long step, double* z) {
  double zz[4];
  action_noise(seed, env, block, step, zz);
  for (int k = 0; k < 4; ++k) z[k] = zz[k];
}

}  // extern "C"
