// Reverse-mode (adjoint) pieces of the implicit-drive substep, one thread per
// chain, FP32 registers / thread-local arrays.
//
// The substep solves A(q) dqd = rhs(q, qd, q*) with A = M(q) + diag(arm) and
// rhs = h (tau_d - h k_s qd - c(q, qd)).  Since M(q) dqd + h c(q, qd) =
// h ID(q, qd, a) with a = dqd / h (inverse dynamics), the implicit-function
// theorem gives, for a cotangent lambda on dqd and mu = A^{-1} lambda:
//   lambda_q  += -h k_s mu - h (dID/dq)^T mu
//   lambda_qd += -h d mu - h^2 k_s mu - h (dID/dqd)^T mu
//   lambda_q* +=  h (kp + g) mu            (g: command gain of the joint)
//   lambda_m  += -h (dID/dm)^T mu            (a held fixed)
// The vector-Jacobian product of ID is the reverse of the body-frame RNEA
// below: id_sweeps (forward sweep with qdd = a, backward sweep giving the
// link wrenches; independent of the cotangent), then rnea_vjp_rev (both
// sweeps reversed).  Link inertias scale with the link
// mass (fixed box size), so d(F, N)/dm = (F, N) / m.
#pragma once

#include "sg_chain.cuh"

namespace sg {

__device__ __forceinline__ V3 v3add(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ float dot3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// K(w, wd) = wd x e_z + w x (w x e_z) (times a length: acceleration of the
// body point at distance `length` along local z)
__device__ __forceinline__ V3 kz(V3 w, V3 wd) {
  return V3{wd.y + w.z * w.x, -wd.x + w.z * w.y, -(w.x * w.x + w.y * w.y)};
}

// Adjoint of K: accumulates d(Kbar . K)/dw and /dwd.
__device__ __forceinline__ void kz_adj(V3 w, V3 Kb, V3& wb, V3& wdb) {
  wdb.y += Kb.x;
  wdb.x -= Kb.y;
  wb.z += Kb.x * w.x + Kb.y * w.y;
  wb.x += Kb.x * w.z - 2.f * Kb.z * w.x;
  wb.y += Kb.y * w.z - 2.f * Kb.z * w.y;
}

// e_a x v
__device__ __forceinline__ V3 axis_x(int a, V3 v) { return axis_cross(a, v); }

// Inverse-dynamics sweeps of tau = ID(q, qd, qdd) (gravity by base
// acceleration; no cotangent involved): base to tip, every link's angular
// velocity w, angular acceleration wd, origin acceleration acc, inertial
// force F and moment Nm about its COM (out.fwd); tip to base, the wrench
// (f, n) it transmits about its origin (out.bwd).
template <class Pat, class Out>
__device__ __forceinline__ void id_sweeps(const Pat& pat, const Rec& rec, const float (&q)[7],
                                          const float (&qd)[7], const float (&qdd)[Pat::N],
                                          const float (&cq)[Pat::N], const float (&sq)[Pat::N],
                                          float grav, Out& out) {
  constexpr int N = Pat::N;
  V3 F[N], Nm[N];
  float ell[N];
  {
    V3 w{0.f, 0.f, 0.f}, wd{0.f, 0.f, 0.f}, acc{0.f, 0.f, grav};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      const int a = pat.axis(i);
      ell[i] = (i == 0 ? 0.f : rec.lf(i - 1, LF_L)) + (pat.type(i) == 1 ? q[i] : 0.f);
      const V3 K = kz(w, wd);
      V3 ap{acc.x + ell[i] * K.x, acc.y + ell[i] * K.y, acc.z + ell[i] * K.z};
      if (pat.type(i) == 0) {
        w = to_child(a, cq[i], sq[i], w);
        wd = to_child(a, cq[i], sq[i], wd);
        ap = to_child(a, cq[i], sq[i], ap);
        const V3 wxa = cross_axis(w, a);
        wd.x += qd[i] * wxa.x;
        wd.y += qd[i] * wxa.y;
        wd.z += qd[i] * wxa.z;
        add_comp(wd, a, qdd[i]);
        add_comp(w, a, qd[i]);
      } else {
        const float t = 2.f * qd[i];
        ap.x += t * w.y;
        ap.y -= t * w.x;
        ap.z += qdd[i];
      }
      acc = ap;
      const float c = rec.lf(i, LF_C), m = rec.lf(i, LF_M);
      const float Ix = rec.lf(i, LF_IX), Iy = rec.lf(i, LF_IY), Iz = rec.lf(i, LF_IZ);
      const V3 Kc = kz(w, wd);
      F[i] = V3{m * (acc.x + c * Kc.x), m * (acc.y + c * Kc.y), m * (acc.z + c * Kc.z)};
      Nm[i] = V3{Ix * wd.x + (Iz - Iy) * w.y * w.z, Iy * wd.y + (Ix - Iz) * w.z * w.x,
                 Iz * wd.z + (Iy - Ix) * w.x * w.y};
      out.fwd(i, w, wd, acc, F[i], Nm[i]);
    }
  }
  {
    V3 fc{0.f, 0.f, 0.f}, nc{0.f, 0.f, 0.f};
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      if (!pat.active(i)) continue;
      const float c = rec.lf(i, LF_C);
      const V3 f = v3add(F[i], fc);
      const V3 n{Nm[i].x - c * F[i].y + nc.x, Nm[i].y + c * F[i].x + nc.y, Nm[i].z + nc.z};
      out.bwd(i, f, n);
      if (i > 0) {
        V3 fp = f, np = n;
        if (pat.type(i) == 0) {
          fp = to_parent(pat.axis(i), cq[i], sq[i], f);
          np = to_parent(pat.axis(i), cq[i], sq[i], n);
        }
        np.x -= ell[i] * fp.y;
        np.y += ell[i] * fp.x;
        fc = fp;
        nc = np;
      }
    }
  }
}

// id_sweeps output kept in thread-local arrays; also the accessor
// rnea_vjp_rev reads them through.
template <int N>
struct SweepArrays {
  V3 W[N], WD[N], ACC[N], F[N], Nm[N], FL[N], NL[N];
  __device__ __forceinline__ void fwd(int i, V3 w, V3 wd, V3 acc, V3 f, V3 n) {
    W[i] = w;
    WD[i] = wd;
    ACC[i] = acc;
    F[i] = f;
    Nm[i] = n;
  }
  __device__ __forceinline__ void bwd(int i, V3 f, V3 n) {
    FL[i] = f;
    NL[i] = n;
  }
  __device__ __forceinline__ V3 w(int i) const { return W[i]; }
  __device__ __forceinline__ V3 wd(int i) const { return WD[i]; }
  __device__ __forceinline__ V3 acc(int i) const { return ACC[i]; }
  __device__ __forceinline__ V3 f(int i) const { return F[i]; }
  __device__ __forceinline__ V3 nm(int i) const { return Nm[i]; }
  __device__ __forceinline__ V3 fl(int i) const { return FL[i]; }
  __device__ __forceinline__ V3 nl(int i) const { return NL[i]; }
};

// Reverse of id_sweeps: given mu and the sweeps' quantities (accessor sw),
// accumulates gq += (dID/dq)^T mu, gqd += (dID/dqd)^T mu and
// gm += m (dID/dm)^T mu -- the mass cotangent times the link mass, since
// ID is linear in m (F, N / m); callers divide by m once at the end of a
// rollout (the masses are constant over it), not once per substep.
template <class Pat, class Sw>
__device__ __forceinline__ void rnea_vjp_rev(const Pat& pat, const Rec& rec, const float (&q)[7],
                                             const float (&qd)[7], const float (&cq)[Pat::N],
                                             const float (&sq)[Pat::N], const Sw& sw,
                                             const float (&mu)[Pat::N], float (&gq)[Pat::N],
                                             float (&gqd)[Pat::N], float (&gm)[Pat::N]) {
  constexpr int N = Pat::N;
  float ell[N], ellb[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    ellb[i] = 0.f;
    ell[i] = (i == 0 ? 0.f : rec.lf(i - 1, LF_L)) + (pat.type(i) == 1 ? q[i] : 0.f);
  }
  // ---- reverse of the backward sweep (base to tip): link wrench adjoints
  V3 Fb[N], Nb[N];
  {
    V3 fb{0.f, 0.f, 0.f}, nb{0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      if (pat.type(i) == 0) add_comp(nb, pat.axis(i), mu[i]);
      else fb.z += mu[i];
      const float c = rec.lf(i, LF_C);
      Fb[i] = V3{fb.x + c * nb.y, fb.y - c * nb.x, fb.z};
      Nb[i] = nb;
      // the wrench of link i+1, carried into frame i, fed f_i and n_i
      if (i + 1 < N && pat.active(i + 1)) {
        const int j = i + 1;
        const float e = ell[j];
        const V3 flj = sw.fl(j);
        V3 gb{fb.x + e * nb.y, fb.y - e * nb.x, fb.z};
        V3 g = flj;
        if (pat.type(j) == 0) g = to_parent(pat.axis(j), cq[j], sq[j], flj);
        ellb[j] += -nb.x * g.y + nb.y * g.x;
        V3 nbj = nb, fbj = gb;
        if (pat.type(j) == 0) {
          const int a = pat.axis(j);
          nbj = to_child(a, cq[j], sq[j], nb);
          fbj = to_child(a, cq[j], sq[j], gb);
          gq[j] += dot3(nbj, axis_x(a, sw.nl(j))) + dot3(fbj, axis_x(a, flj));
        }
        fb = fbj;
        nb = nbj;
      }
    }
  }
  // ---- reverse of the forward sweep (tip to base)
  {
    V3 wb{0.f, 0.f, 0.f}, wdb{0.f, 0.f, 0.f}, accb{0.f, 0.f, 0.f};
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
      if (!pat.active(i)) continue;
      const float c = rec.lf(i, LF_C), m = rec.lf(i, LF_M);
      const float Ix = rec.lf(i, LF_IX), Iy = rec.lf(i, LF_IY), Iz = rec.lf(i, LF_IZ);
      const V3 w = sw.w(i), wd = sw.wd(i);
      // F = m (acc + c K(w, wd)), N = I wd + w x (I w)
      accb.x += m * Fb[i].x;
      accb.y += m * Fb[i].y;
      accb.z += m * Fb[i].z;
      kz_adj(w, V3{m * c * Fb[i].x, m * c * Fb[i].y, m * c * Fb[i].z}, wb, wdb);
      gm[i] += dot3(Fb[i], sw.f(i)) + dot3(Nb[i], sw.nm(i));
      const V3 nb = Nb[i];
      wdb.x += Ix * nb.x;
      wdb.y += Iy * nb.y;
      wdb.z += Iz * nb.z;
      wb.x += nb.y * (Ix - Iz) * w.z + nb.z * (Iy - Ix) * w.y;
      wb.y += nb.x * (Iz - Iy) * w.z + nb.z * (Iy - Ix) * w.x;
      wb.z += nb.x * (Iz - Iy) * w.y + nb.y * (Ix - Iz) * w.x;
      // joint i: parent quantities (link i-1, or the fixed base)
      const V3 wp = i > 0 ? sw.w(i - 1) : V3{0.f, 0.f, 0.f};
      const V3 wdp = i > 0 ? sw.wd(i - 1) : V3{0.f, 0.f, 0.f};
      V3 wpb, wdpb, apb;
      if (pat.type(i) == 0) {
        const int a = pat.axis(i);
        const V3 wr = to_child(a, cq[i], sq[i], wp);
        const V3 wdr = to_child(a, cq[i], sq[i], wdp);
        const V3 apr = sw.acc(i);
        const V3 wrxa = cross_axis(wr, a);
        gqd[i] += compc(wb, a) + dot3(wdb, wrxa);
        const V3 axwdb = axis_x(a, wdb);
        const V3 wrb{wb.x + qd[i] * axwdb.x, wb.y + qd[i] * axwdb.y, wb.z + qd[i] * axwdb.z};
        gq[i] += dot3(wrb, wrxa) + dot3(wdb, cross_axis(wdr, a)) + dot3(accb, cross_axis(apr, a));
        wpb = to_parent(a, cq[i], sq[i], wrb);
        wdpb = to_parent(a, cq[i], sq[i], wdb);
        apb = to_parent(a, cq[i], sq[i], accb);
      } else {
        apb = accb;
        const float t = 2.f * qd[i];
        // acc = ap + 2 qd (wp x e_z): d/dwp of accb . (wp x e_z) = e_z x accb
        wpb = V3{wb.x - t * accb.y, wb.y + t * accb.x, wb.z};
        wdpb = wdb;
        gqd[i] += 2.f * (accb.x * wp.y - accb.y * wp.x);
      }
      // ap = acc_parent + ell K(wp, wdp)
      const V3 K = kz(wp, wdp);
      ellb[i] += dot3(apb, K);
      kz_adj(wp, V3{ell[i] * apb.x, ell[i] * apb.y, ell[i] * apb.z}, wpb, wdpb);
      if (pat.type(i) == 1) gq[i] += ellb[i];
      wb = wpb;
      wdb = wdpb;
      accb = apb;
    }
  }
}

// gq += J_tip(q)^T gbar: world-frame tip Jacobian transpose of one chain.
template <class Pat>
__device__ __forceinline__ void tip_vjp(const Pat& pat, const Rec& rec, const float (&q)[7],
                                        V3 gbar, float (&gq)[Pat::N]) {
  constexpr int N = Pat::N;
  V3 P[N], Z[N];
  V3 p{rec.cf(CF_BX), rec.cf(CF_BY), rec.cf(CF_BZ)};
  V3 c0{1.f, 0.f, 0.f}, c1{0.f, 1.f, 0.f}, c2{0.f, 0.f, 1.f};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    if (pat.type(i) == 1) {
      Z[i] = c2;
      p = V3{p.x + q[i] * c2.x, p.y + q[i] * c2.y, p.z + q[i] * c2.z};
    } else {
      float s, c;
      __sincosf(q[i], &s, &c);
      const int a = pat.axis(i);
      if (a == 2) rot_cols(c0, c1, c, s);
      else if (a == 1) rot_cols(c2, c0, c, s);
      else rot_cols(c1, c2, c, s);
      Z[i] = a == 0 ? c0 : (a == 1 ? c1 : c2);
    }
    P[i] = p;
    const float L = rec.lf(i, LF_L);
    p = V3{p.x + L * c2.x, p.y + L * c2.y, p.z + L * c2.z};
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    if (pat.type(i) == 1) {
      gq[i] += dot3(gbar, Z[i]);
    } else {
      const V3 r{p.x - P[i].x, p.y - P[i].y, p.z - P[i].z};
      const V3 zr{Z[i].y * r.z - Z[i].z * r.y, Z[i].z * r.x - Z[i].x * r.z,
                  Z[i].x * r.y - Z[i].y * r.x};
      gq[i] += dot3(gbar, zr);
    }
  }
}

// World-frame tool-tip Jacobian of one chain, J_i = d(tip)/dq_i: z_i x
// (tip - p_i) for a revolute joint i, z_i for a prismatic one (z_i its axis,
// p_i its origin), given the joint trigonometry; out.jac(i, J_i).  Two
// passes of the kinematics (the tip, then each joint's column as its frame
// is reached) keep no per-link arrays.  J^T g is the tip cotangent's
// contribution to the joint-position cotangent (tip_vjp computes it from q).
template <class Pat>
__device__ __forceinline__ void tip_frames_step(const Pat& pat, const Rec& rec, const float (&q)[7],
                                                const float (&cq)[Pat::N],
                                                const float (&sq)[Pat::N], int i, V3& p, V3& c0,
                                                V3& c1, V3& c2) {
  if (pat.type(i) == 1) {
    p = V3{p.x + q[i] * c2.x, p.y + q[i] * c2.y, p.z + q[i] * c2.z};
  } else {
    const int a = pat.axis(i);
    if (a == 2) rot_cols(c0, c1, cq[i], sq[i]);
    else if (a == 1) rot_cols(c2, c0, cq[i], sq[i]);
    else rot_cols(c1, c2, cq[i], sq[i]);
  }
}

template <class Pat, class Out>
__device__ __forceinline__ void tip_jacobian(const Pat& pat, const Rec& rec, const float (&q)[7],
                                             const float (&cq)[Pat::N], const float (&sq)[Pat::N],
                                             Out& out) {
  constexpr int N = Pat::N;
  const V3 base{rec.cf(CF_BX), rec.cf(CF_BY), rec.cf(CF_BZ)};
  V3 tip = base;
  {
    V3 c0{1.f, 0.f, 0.f}, c1{0.f, 1.f, 0.f}, c2{0.f, 0.f, 1.f};
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      tip_frames_step(pat, rec, q, cq, sq, i, tip, c0, c1, c2);
      const float L = rec.lf(i, LF_L);
      tip = V3{tip.x + L * c2.x, tip.y + L * c2.y, tip.z + L * c2.z};
    }
  }
  V3 p = base;
  V3 c0{1.f, 0.f, 0.f}, c1{0.f, 1.f, 0.f}, c2{0.f, 0.f, 1.f};
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    tip_frames_step(pat, rec, q, cq, sq, i, p, c0, c1, c2);
    if (pat.type(i) == 1) {
      out.jac(i, c2);
    } else {
      const int a = pat.axis(i);
      const V3 z = a == 0 ? c0 : (a == 1 ? c1 : c2);
      const V3 r{tip.x - p.x, tip.y - p.y, tip.z - p.z};
      out.jac(i, V3{z.y * r.z - z.z * r.y, z.z * r.x - z.x * r.z, z.x * r.y - z.y * r.x});
    }
    const float L = rec.lf(i, LF_L);
    p = V3{p.x + L * c2.x, p.y + L * c2.y, p.z + L * c2.z};
  }
}

// Forward substep that also returns the Cholesky factor (L in the lower
// triangle of M, inv = 1 / L_ii), the velocity increment dqd, the
// acceleration a = dqd / h and the drive stiffness k_s of every joint
// (needed by the adjoint).
template <class Pat>
__device__ __forceinline__ void substep_record(const Pat& pat, const Rec& rec, const float (&q)[7],
                                               const float (&qd)[7], const float (&qs)[7], float h,
                                               float grav, float (&cq)[Pat::N], float (&sq)[Pat::N],
                                               float (&M)[Pat::N][Pat::N], float (&inv)[Pat::N],
                                               float (&acc)[Pat::N], float (&ks)[Pat::N],
                                               float (&dqd)[Pat::N]) {
  constexpr int N = Pat::N;
  float bias[N], rhs[N], arm[N];
  V3 F[N], Nm[N];
  joint_sincos(pat, q, cq, sq);
  rnea_forward(pat, rec, q, qd, cq, sq, grav, F, Nm);
  backward_sweep<Pat, true, true>(pat, rec, q, cq, sq, F, Nm, bias, M);
  drive_terms(pat, rec, q, qd, qs, h, bias, rhs, arm);
  chol_factor(pat, M, arm, inv);
  chol_apply(pat, M, inv, rhs);
  const float hinv = 1.f / h;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    dqd[i] = rhs[i];
    if (!pat.active(i)) continue;
    acc[i] = rhs[i] * hinv;
    // k_s = (arm - h d) / h^2 recomputed directly from the limit test
    const float kp = rec.lf(i, LF_KP), kl = rec.lf(i, LF_KLIM);
    const float lo = rec.lf(i, LF_QLO), hi = rec.lf(i, LF_QHI);
    ks[i] = kp + ((q[i] > hi || q[i] < lo) ? kl : 0.f);
  }
}

// Adjoint of one substep given its start state (q, qd, joint trigonometry),
// the Cholesky factor, the drive stiffness and the inverse-dynamics sweeps
// (accessor sw).
template <class Pat, class Sw>
__device__ __forceinline__ void substep_adjoint_sw(
    const Pat& pat, const Rec& rec, const float (&q)[7], const float (&qd)[7],
    const float (&cq)[Pat::N], const float (&sq)[Pat::N], const float (&M)[Pat::N][Pat::N],
    const float (&inv)[Pat::N], const float (&ks)[Pat::N], const Sw& sw, float h,
    float (&lq)[7], float (&lqd)[7], float (&lqs)[7], float (&lm)[7]) {
  constexpr int N = Pat::N;
  float mu[N], gq[N], gqd[N], gm[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    mu[i] = 0.f;
    gq[i] = 0.f;
    gqd[i] = 0.f;
    gm[i] = 0.f;
    if (!pat.active(i)) continue;
    lqd[i] += h * lq[i];   // q' = q + h qd'
    mu[i] = lqd[i];        // qd' = qd + dqd
  }
  chol_apply(pat, M, inv, mu);
  rnea_vjp_rev(pat, rec, q, qd, cq, sq, sw, mu, gq, gqd, gm);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    const float kp = rec.lf(i, LF_KP), d = rec.lf(i, LF_D), ga = rec.lf(i, LF_GA);
    lq[i] += -h * ks[i] * mu[i] - h * gq[i];
    lqd[i] += -h * d * mu[i] - h * h * ks[i] * mu[i] - h * gqd[i];
    lqs[i] += h * (kp + ga) * mu[i];
    lm[i] += -h * gm[i];
  }
}

// Adjoint of one substep.  On entry lq, lqd are the cotangents of the
// substep's outputs (q', qd'); on exit those of its inputs (q, qd).  lqs and
// lm accumulate the cotangents of the targets q* and of the link masses,
// the latter times the link mass (divide by m for dL/dm).
template <class Pat>
__device__ __forceinline__ void substep_adjoint(const Pat& pat, const Rec& rec, const float (&q)[7],
                                                const float (&qd)[7], const float (&qs)[7],
                                                float h, float grav, float (&lq)[7],
                                                float (&lqd)[7], float (&lqs)[7],
                                                float (&lm)[7]) {
  constexpr int N = Pat::N;
  float cq[N], sq[N], M[N][N], inv[N], acc[N], ks[N], dqd[N];
  substep_record(pat, rec, q, qd, qs, h, grav, cq, sq, M, inv, acc, ks, dqd);
  SweepArrays<N> sw;
  id_sweeps(pat, rec, q, qd, acc, cq, sq, grav, sw);
  substep_adjoint_sw(pat, rec, q, qd, cq, sq, M, inv, ks, sw, h, lq, lqd, lqs, lm);
}

}  // namespace sg
