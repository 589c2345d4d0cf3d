// Per-chain dynamics in FP32 registers: one thread integrates one serial chain.
//
// Formulation (body frames, coordinate-axis joints):
//   * every joint rotates about a coordinate axis of its own frame (or
//     translates along its z), so a frame change is a 2x2 rotation of two
//     vector components and the joint offset (0, 0, l) is a sparse vector;
//   * bias forces c(q, qd) = RNEA(q, qd, 0) with gravity as a base
//     acceleration (Luh-Walker-Paul recursion; Featherstone 2008, ch. 5);
//   * joint-space inertia M(q) by composite rigid bodies carried in body
//     frames (mass, first moment, rotational inertia about the frame origin),
//     with each column force propagated to the ancestors (Featherstone 2008,
//     ch. 6);
//   * the implicit-drive substep solves (M + h d I + h^2 k_s I) dqd =
//     h (tau_d - h k_s qd - c) by an in-register Cholesky factorisation;
//     qd += dqd, q += h qd (semi-implicit Euler; the paper's engine
//     sub-steps each control step, Methods "Simulation Setup").
// All per-link arrays are indexed by compile-time link indices (fully
// unrolled loops), so they live in registers.
#pragma once

#include <cuda_runtime.h>

#include "sg_internal.h"

namespace sg {

struct V3 {
  float x, y, z;
};

__device__ __forceinline__ void add_comp(V3& v, int a, float t) {
  if (a == 0) v.x += t;
  else if (a == 1) v.y += t;
  else v.z += t;
}
__device__ __forceinline__ float compc(const V3& v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

// v <- R^T v for R = Rot(axis a, angle with cosine c, sine s): parent -> child coordinates
__device__ __forceinline__ V3 to_child(int a, float c, float s, V3 v) {
  if (a == 2) return V3{c * v.x + s * v.y, -s * v.x + c * v.y, v.z};
  if (a == 1) return V3{-s * v.z + c * v.x, v.y, c * v.z + s * v.x};
  return V3{v.x, c * v.y + s * v.z, -s * v.y + c * v.z};
}

// v <- R v: child -> parent coordinates
__device__ __forceinline__ V3 to_parent(int a, float c, float s, V3 v) {
  if (a == 2) return V3{c * v.x - s * v.y, s * v.x + c * v.y, v.z};
  if (a == 1) return V3{s * v.z + c * v.x, v.y, c * v.z - s * v.x};
  return V3{v.x, c * v.y - s * v.z, s * v.y + c * v.z};
}

// w x e_a
__device__ __forceinline__ V3 cross_axis(const V3& w, int a) {
  if (a == 2) return V3{w.y, -w.x, 0.f};
  if (a == 1) return V3{-w.z, 0.f, w.x};
  return V3{0.f, w.z, -w.y};
}

// e_a x h
__device__ __forceinline__ V3 axis_cross(int a, const V3& h) {
  if (a == 2) return V3{-h.y, h.x, 0.f};
  if (a == 1) return V3{h.z, 0.f, -h.x};
  return V3{0.f, -h.z, h.y};
}

// symmetric 3x3
struct S3 {
  float xx, yy, zz, xy, xz, yz;
};

// column a of a symmetric matrix
__device__ __forceinline__ V3 sym_col(const S3& J, int a) {
  if (a == 2) return V3{J.xz, J.yz, J.zz};
  if (a == 1) return V3{J.xy, J.yy, J.yz};
  return V3{J.xx, J.xy, J.xz};
}

// J <- R J R^T (child -> parent) for a rotation about axis a.  With the
// in-plane pair (u, v) = ((a+1)%3, (a+2)%3): u' = c u - s v, v' = s u + c v.
__device__ __forceinline__ S3 sym_to_parent(int a, float c, float s, const S3& J) {
  float uu, vv, uv, ua, va, aa;
  if (a == 2) { uu = J.xx; vv = J.yy; uv = J.xy; ua = J.xz; va = J.yz; aa = J.zz; }
  else if (a == 1) { uu = J.zz; vv = J.xx; uv = J.xz; ua = J.yz; va = J.xy; aa = J.yy; }
  else { uu = J.yy; vv = J.zz; uv = J.yz; ua = J.xy; va = J.xz; aa = J.xx; }
  const float cc = c * c, ss = s * s, cs = c * s;
  const float nuu = cc * uu - 2.f * cs * uv + ss * vv;
  const float nvv = ss * uu + 2.f * cs * uv + cc * vv;
  const float nuv = cs * (uu - vv) + (cc - ss) * uv;
  const float nua = c * ua - s * va;
  const float nva = s * ua + c * va;
  S3 r;
  if (a == 2) { r.xx = nuu; r.yy = nvv; r.xy = nuv; r.xz = nua; r.yz = nva; r.zz = aa; }
  else if (a == 1) { r.zz = nuu; r.xx = nvv; r.xz = nuv; r.yz = nua; r.xy = nva; r.yy = aa; }
  else { r.yy = nuu; r.zz = nvv; r.yz = nuv; r.xy = nua; r.xz = nva; r.xx = aa; }
  return r;
}

// ---- chain patterns ------------------------------------------------------
// type(i): 0 revolute, 1 prismatic; axis(i): 0/1/2; active(i): link exists.
struct Pat7R {
  static constexpr int N = 7;
  __device__ __forceinline__ int type(int) const { return 0; }
  __device__ __forceinline__ int axis(int i) const { return (i & 1) ? 1 : 2; }
  __device__ __forceinline__ bool active(int) const { return true; }
};
struct Pat7P {
  static constexpr int N = 7;
  __device__ __forceinline__ int type(int i) const { return i == 2 ? 1 : 0; }
  __device__ __forceinline__ int axis(int i) const { return (i & 1) ? 1 : 2; }
  __device__ __forceinline__ bool active(int) const { return true; }
};
struct Pat4R {
  static constexpr int N = 4;
  __device__ __forceinline__ int type(int) const { return 0; }
  __device__ __forceinline__ int axis(int i) const { return (i & 1) ? 1 : 2; }
  __device__ __forceinline__ bool active(int) const { return true; }
};
struct PatGen {
  static constexpr int N = 7;
  int code, n;
  __device__ __forceinline__ int type(int i) const { return (code >> (3 * i + 2)) & 1; }
  __device__ __forceinline__ int axis(int i) const { return (code >> (3 * i)) & 3; }
  __device__ __forceinline__ bool active(int i) const { return i < n; }
};

// Parameter access: record of this warp in shared memory, column `lane`.
struct Rec {
  const float* base;   // shared-memory record of the warp, offset by lane
  __device__ __forceinline__ float cf(int f) const { return base[f * kWarp]; }
  __device__ __forceinline__ float lf(int i, int f) const {
    return base[(kChainFields + i * kLinkFields + f) * kWarp];
  }
};

// ---- pieces of one implicit-drive semi-implicit Euler substep ------------
template <class Pat>
__device__ __forceinline__ void joint_sincos(const Pat& pat, const float (&q)[7],
                                             float (&cq)[Pat::N], float (&sq)[Pat::N]) {
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (pat.active(i) && pat.type(i) == 0) {
      __sincosf(q[i], &sq[i], &cq[i]);
    } else {
      cq[i] = 1.f;
      sq[i] = 0.f;
    }
  }
}

// RNEA forward sweep (qdd = 0): body-frame velocities/accelerations and the
// inertial force F and moment Nm (about the COM) of every link.
template <class Pat>
__device__ __forceinline__ void rnea_forward(const Pat& pat, const Rec& rec, const float (&q)[7],
                                             const float (&qd)[7], const float (&cq)[Pat::N],
                                             const float (&sq)[Pat::N], float grav,
                                             V3 (&F)[Pat::N], V3 (&Nm)[Pat::N]) {
  constexpr int N = Pat::N;
  {
    V3 w{0.f, 0.f, 0.f}, wd{0.f, 0.f, 0.f}, acc{0.f, 0.f, grav};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      const int a = pat.axis(i);
      float ell = (i == 0) ? 0.f : rec.lf(i - 1, LF_L);
      if (pat.type(i) == 1) ell += q[i];
      // acceleration of the parent-fixed point at (0, 0, ell)
      V3 ap{acc.x + ell * (wd.y + w.z * w.x), acc.y + ell * (-wd.x + w.z * w.y),
            acc.z - ell * (w.x * w.x + w.y * w.y)};
      if (pat.type(i) == 0) {
        w = to_child(a, cq[i], sq[i], w);
        wd = to_child(a, cq[i], sq[i], wd);
        ap = to_child(a, cq[i], sq[i], ap);
        const V3 wxa = cross_axis(w, a);
        wd.x += qd[i] * wxa.x;
        wd.y += qd[i] * wxa.y;
        wd.z += qd[i] * wxa.z;
        add_comp(w, a, qd[i]);
      } else {
        const float t = 2.f * qd[i];
        ap.x += t * w.y;
        ap.y -= t * w.x;
      }
      acc = ap;
      const float c = rec.lf(i, LF_C), m = rec.lf(i, LF_M);
      const float Ix = rec.lf(i, LF_IX), Iy = rec.lf(i, LF_IY), Iz = rec.lf(i, LF_IZ);
      F[i] = V3{m * (acc.x + c * (wd.y + w.z * w.x)), m * (acc.y + c * (-wd.x + w.z * w.y)),
                m * (acc.z - c * (w.x * w.x + w.y * w.y))};
      Nm[i] = V3{Ix * wd.x + (Iz - Iy) * w.y * w.z, Iy * wd.y + (Ix - Iz) * w.z * w.x,
                 Iz * wd.z + (Iy - Ix) * w.x * w.y};
    }
  }

}

// Backward sweep from the tip: with kBias the RNEA wrenches give the bias
// forces c(q, qd); with kMass the composite bodies give M(q) (upper triangle
// and diagonal).
template <class Pat, bool kBias, bool kMass>
__device__ __forceinline__ void backward_sweep(const Pat& pat, const Rec& rec, const float (&q)[7],
                                               const float (&cq)[Pat::N],
                                               const float (&sq)[Pat::N],
                                               const V3 (&F)[Pat::N], const V3 (&Nm)[Pat::N],
                                               float (&bias)[Pat::N], float (&M)[Pat::N][Pat::N]) {
  constexpr int N = Pat::N;
  V3 fc{0.f, 0.f, 0.f}, nc{0.f, 0.f, 0.f};   // child wrench in the current frame
  float mc = 0.f;                             // composite mass
  V3 hc{0.f, 0.f, 0.f};                       // composite first moment
  S3 Jc{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};        // composite inertia about the origin
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    if (!pat.active(i)) continue;
    const int a = pat.axis(i);
    const float c = rec.lf(i, LF_C);
    V3 f{0.f, 0.f, 0.f}, n{0.f, 0.f, 0.f};
    if constexpr (kBias) {
      // RNEA: wrench on link i about its origin
      f = V3{F[i].x + fc.x, F[i].y + fc.y, F[i].z + fc.z};
      n = V3{Nm[i].x - c * F[i].y + nc.x, Nm[i].y + c * F[i].x + nc.y, Nm[i].z + nc.z};
      bias[i] = pat.type(i) == 0 ? compc(n, a) : f.z;
    }
    if constexpr (kMass) {
      // composite body of links i..N-1 about origin i
      const float m = rec.lf(i, LF_M);
      const float mcc = m * c;
      mc += m;
      hc.z += mcc;
      Jc.xx += rec.lf(i, LF_IX) + mcc * c;
      Jc.yy += rec.lf(i, LF_IY) + mcc * c;
      Jc.zz += rec.lf(i, LF_IZ);
      // column i: wrench that gives unit acceleration of joint i
      V3 cf, cn;
      if (pat.type(i) == 0) {
        cn = sym_col(Jc, a);
        cf = axis_cross(a, hc);
        M[i][i] = compc(cn, a);
      } else {
        cf = V3{0.f, 0.f, mc};
        cn = V3{hc.y, -hc.x, 0.f};
        M[i][i] = mc;
      }
#pragma unroll
      for (int j = i - 1; j >= 0; --j) {
        // frame j+1 -> frame j
        const int aj1 = pat.axis(j + 1);
        float ell = rec.lf(j, LF_L);
        if (pat.type(j + 1) == 0) {
          cf = to_parent(aj1, cq[j + 1], sq[j + 1], cf);
          cn = to_parent(aj1, cq[j + 1], sq[j + 1], cn);
        } else {
          ell += q[j + 1];
        }
        cn.x -= ell * cf.y;
        cn.y += ell * cf.x;
        M[j][i] = pat.type(j) == 0 ? compc(cn, pat.axis(j)) : cf.z;
      }
    }
    // carry the RNEA wrench and the composite body to the parent frame
    if (i > 0) {
      float ell = rec.lf(i - 1, LF_L);
      if (pat.type(i) == 1) ell += q[i];
      if constexpr (kBias) {
        V3 fp = f, np = n;
        if (pat.type(i) == 0) {
          fp = to_parent(a, cq[i], sq[i], f);
          np = to_parent(a, cq[i], sq[i], n);
        }
        np.x -= ell * fp.y;
        np.y += ell * fp.x;
        fc = fp;
        nc = np;
      }
      if constexpr (kMass) {
        V3 hp = hc;
        S3 Jp = Jc;
        if (pat.type(i) == 0) {
          hp = to_parent(a, cq[i], sq[i], hc);
          Jp = sym_to_parent(a, cq[i], sq[i], Jc);
        }
        // shift the composite from origin i to origin i-1 (offset (0,0,ell))
        const float t = 2.f * ell * hp.z + mc * ell * ell;
        Jp.xx += t;
        Jp.yy += t;
        Jp.xz -= ell * hp.x;
        Jp.yz -= ell * hp.y;
        hp.z += mc * ell;
        hc = hp;
        Jc = Jp;
      }
    }
  }
}

// Implicit drive terms: arm = h d + h^2 k_s (added to the diagonal of M) and
// rhs = h (tau_d - h k_s qd - c), with the drive torque
// tau_d = kp (q* - q) + g q* - d qd + tau_lim: the command q* is a position
// target (g = 0), a velocity target (kp = 0, g = kd) or a torque (kp = 0,
// g = 1, d = joint damping only), as packed per joint.
template <class Pat>
__device__ __forceinline__ void drive_terms(const Pat& pat, const Rec& rec, const float (&q)[7],
                                            const float (&qd)[7], const float (&qs)[7], float h,
                                            const float (&bias)[Pat::N], float (&rhs)[Pat::N],
                                            float (&arm)[Pat::N]) {
  constexpr int N = Pat::N;
  const float hh = h * h;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    const float kp = rec.lf(i, LF_KP), d = rec.lf(i, LF_D), kl = rec.lf(i, LF_KLIM);
    const float ga = rec.lf(i, LF_GA);
    const float lo = rec.lf(i, LF_QLO), hi = rec.lf(i, LF_QHI);
    // limit spring, active beyond either bound (selects, no branches)
    const bool over = q[i] > hi, under = q[i] < lo;
    const float bound = over ? hi : lo;
    const bool act = over || under;
    const float ks = kp + (act ? kl : 0.f);
    const float tl = act ? -kl * (q[i] - bound) : 0.f;
    const float tau = kp * (qs[i] - q[i]) + ga * qs[i] - d * qd[i] + tl;
    rhs[i] = h * (tau - h * ks * qd[i] - bias[i]);
    arm[i] = h * d + hh * ks;
  }

}

// (M + diag(arm)) = L L^T in registers: L overwrites the lower triangle of M
// (M[i][j], i > j; the upper triangle holds A on entry) and inv[i] = 1 / L_ii.
template <class Pat>
__device__ __forceinline__ void chol_factor(const Pat& pat, float (&M)[Pat::N][Pat::N],
                                            const float (&arm)[Pat::N], float (&inv)[Pat::N]) {
  constexpr int N = Pat::N;
#pragma unroll
  for (int i = 0; i < N; ++i)
    if (pat.active(i)) M[i][i] += arm[i];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (!pat.active(j)) continue;
    float s = M[j][j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= M[j][k] * M[j][k];
    inv[j] = rsqrtf(s);
#pragma unroll
    for (int i = j + 1; i < N; ++i) {
      if (!pat.active(i)) continue;
      float t = M[j][i];   // upper triangle holds A
#pragma unroll
      for (int k = 0; k < j; ++k) t -= M[i][k] * M[j][k];
      M[i][j] = t * inv[j];
    }
  }
}

// rhs <- (L L^T)^{-1} rhs (forward, then backward substitution).
template <class Pat>
__device__ __forceinline__ void chol_apply(const Pat& pat, const float (&M)[Pat::N][Pat::N],
                                           const float (&inv)[Pat::N], float (&rhs)[Pat::N]) {
  constexpr int N = Pat::N;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    float t = rhs[i];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= M[i][k] * rhs[k];
    rhs[i] = t * inv[i];
  }
#pragma unroll
  for (int i = N - 1; i >= 0; --i) {
    if (!pat.active(i)) continue;
    float t = rhs[i];
#pragma unroll
    for (int k = i + 1; k < N; ++k) {
      if (pat.active(k)) t -= M[k][i] * rhs[k];
    }
    rhs[i] = t * inv[i];
  }
}

// rhs <- (M + diag(arm))^{-1} rhs by an in-register Cholesky factorisation.
template <class Pat>
__device__ __forceinline__ void chol_solve(const Pat& pat, float (&M)[Pat::N][Pat::N],
                                           const float (&arm)[Pat::N], float (&rhs)[Pat::N]) {
  float inv[Pat::N];
  chol_factor(pat, M, arm, inv);
  chol_apply(pat, M, inv, rhs);
}

template <class Pat>
__device__ __forceinline__ void integrate(const Pat& pat, float (&q)[7], float (&qd)[7],
                                          const float (&dqd)[Pat::N], float h) {
#pragma unroll
  for (int i = 0; i < Pat::N; ++i) {
    if (!pat.active(i)) continue;
    qd[i] += dqd[i];
    q[i] += h * qd[i];
  }
}

// One implicit-drive semi-implicit Euler substep of one chain (one thread).
// cq, sq hold cos / sin of the joint angles q on entry and are updated to
// those of the new q on exit (the next substep and the tip kinematics reuse
// them).
template <class Pat>
__device__ __forceinline__ void chain_substep_trig(const Pat& pat, const Rec& rec, float (&q)[7],
                                                   float (&qd)[7], const float (&qs)[7],
                                                   float (&cq)[Pat::N], float (&sq)[Pat::N],
                                                   float h, float grav) {
  constexpr int N = Pat::N;
  float bias[N], M[N][N], rhs[N], arm[N];
  V3 F[N], Nm[N];
  rnea_forward(pat, rec, q, qd, cq, sq, grav, F, Nm);
  backward_sweep<Pat, true, true>(pat, rec, q, cq, sq, F, Nm, bias, M);
  drive_terms(pat, rec, q, qd, qs, h, bias, rhs, arm);
  chol_solve(pat, M, arm, rhs);
  integrate(pat, q, qd, rhs, h);
  joint_sincos(pat, q, cq, sq);
}

// One substep computing the joint trigonometry itself.
template <class Pat>
__device__ __forceinline__ void chain_substep(const Pat& pat, const Rec& rec, float (&q)[7],
                                              float (&qd)[7], const float (&qs)[7], float h,
                                              float grav) {
  float cq[Pat::N], sq[Pat::N];
  joint_sincos(pat, q, cq, sq);
  chain_substep_trig(pat, rec, q, qd, qs, cq, sq, h, grav);
}

// col_u' = c col_u + s col_v, col_v' = -s col_u + c col_v
__device__ __forceinline__ void rot_cols(V3& u, V3& v, float c, float s) {
  const V3 a = u, b = v;
  u = V3{c * a.x + s * b.x, c * a.y + s * b.y, c * a.z + s * b.z};
  v = V3{-s * a.x + c * b.x, -s * a.y + c * b.y, -s * a.z + c * b.z};
}

// World pose of the tool tip (and tip rotation columns) from q, given the
// cos / sin of the joint angles.
template <class Pat>
__device__ __forceinline__ void chain_tip_trig(const Pat& pat, const Rec& rec, const float (&q)[7],
                                               const float (&cq)[Pat::N],
                                               const float (&sq)[Pat::N], V3& tip, V3& r0,
                                               V3& r1, V3& r2) {
  constexpr int N = Pat::N;
  V3 p{rec.cf(CF_BX), rec.cf(CF_BY), rec.cf(CF_BZ)};
  V3 c0{1.f, 0.f, 0.f}, c1{0.f, 1.f, 0.f}, c2{0.f, 0.f, 1.f};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    if (pat.type(i) == 1) {
      p.x += q[i] * c2.x;
      p.y += q[i] * c2.y;
      p.z += q[i] * c2.z;
    } else {
      const float s = sq[i], c = cq[i];
      const int a = pat.axis(i);
      // R <- R Rot_a with the in-plane pair (u, v) = ((a+1)%3, (a+2)%3)
      if (a == 2) rot_cols(c0, c1, c, s);
      else if (a == 1) rot_cols(c2, c0, c, s);
      else rot_cols(c1, c2, c, s);
    }
    const float L = rec.lf(i, LF_L);
    p.x += L * c2.x;
    p.y += L * c2.y;
    p.z += L * c2.z;
  }
  tip = p;
  r0 = c0;
  r1 = c1;
  r2 = c2;
}

template <class Pat>
__device__ __forceinline__ void chain_tip(const Pat& pat, const Rec& rec, const float (&q)[7],
                                          V3& tip, V3& r0, V3& r1, V3& r2) {
  float cq[Pat::N], sq[Pat::N];
  joint_sincos(pat, q, cq, sq);
  chain_tip_trig(pat, rec, q, cq, sq, tip, r0, r1, r2);
}

// Unit quaternion (x, y, z, w), w >= 0, of the rotation with columns r0, r1, r2
// (Shepperd 1978: branch on the largest of trace and the diagonal).
__device__ __forceinline__ void rot_to_quat(const V3& r0, const V3& r1, const V3& r2, float* o) {
  const float m00 = r0.x, m11 = r1.y, m22 = r2.z;
  const float m01 = r1.x, m10 = r0.y, m02 = r2.x, m20 = r0.z, m12 = r2.y, m21 = r1.z;
  const float tr = m00 + m11 + m22;
  float x, y, z, w;
  if (tr >= m00 && tr >= m11 && tr >= m22) {
    w = 0.5f * sqrtf(1.f + tr);
    const float k = 0.25f / w;
    x = (m21 - m12) * k;
    y = (m02 - m20) * k;
    z = (m10 - m01) * k;
  } else if (m00 >= m11 && m00 >= m22) {
    x = 0.5f * sqrtf(1.f + m00 - m11 - m22);
    const float k = 0.25f / x;
    w = (m21 - m12) * k;
    y = (m01 + m10) * k;
    z = (m02 + m20) * k;
  } else if (m11 >= m22) {
    y = 0.5f * sqrtf(1.f - m00 + m11 - m22);
    const float k = 0.25f / y;
    w = (m02 - m20) * k;
    x = (m01 + m10) * k;
    z = (m12 + m21) * k;
  } else {
    z = 0.5f * sqrtf(1.f - m00 - m11 + m22);
    const float k = 0.25f / z;
    w = (m10 - m01) * k;
    x = (m02 + m20) * k;
    y = (m12 + m21) * k;
  }
  if (w < 0.f) {
    x = -x;
    y = -y;
    z = -z;
    w = -w;
  }
  o[0] = x;
  o[1] = y;
  o[2] = z;
  o[3] = w;
}

}  // namespace sg
