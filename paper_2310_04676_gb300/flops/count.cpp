// Algorithmic FP32 operation counts of the chain code (host build).
//
// The device headers sg_chain.cuh and sg_adjoint.cuh are compiled for the
// host with `float` replaced by the counting scalar CF below (the copies are
// made by flops/count.py).  CF counts additions/subtractions and
// multiplications; like the compiler it does not count an operation it can
// fold: an operand that is a literal 0, a factor of +-1, or two literal
// operands.  Special functions (sin/cos, rsqrt, sqrt, division) are counted
// apart.  Output: one line per chain pattern with the FLOPs (an FMA is a
// multiplication and an addition: 2) of one substep, the tip kinematics,
// one substep adjoint and the tip Jacobian-transpose product.
#include <cmath>
#include <cstdio>

struct Cnt {
  long add = 0, mul = 0, sfu = 0;
} g;

struct CF {
  double v;
  bool k;   // a literal (compile-time constant)
  CF() : v(0), k(true) {}
  CF(double x) : v(x), k(true) {}
  CF(int x) : v(x), k(true) {}
  static CF var(double x) {
    CF c(x);
    c.k = false;
    return c;
  }
};
inline CF mk(double v, bool k) {
  CF c(v);
  c.k = k;
  return c;
}
inline CF addsub(CF a, CF b, double r) {
  if (a.k && b.k) return mk(r, true);
  if ((a.k && a.v == 0) || (b.k && b.v == 0)) return mk(r, false);
  g.add++;
  return mk(r, false);
}
inline CF operator+(CF a, CF b) { return addsub(a, b, a.v + b.v); }
inline CF operator-(CF a, CF b) { return addsub(a, b, a.v - b.v); }
inline CF operator*(CF a, CF b) {
  const double r = a.v * b.v;
  if (a.k && b.k) return mk(r, true);
  if ((a.k && a.v == 0) || (b.k && b.v == 0)) return mk(0.0, true);
  if ((a.k && std::fabs(a.v) == 1) || (b.k && std::fabs(b.v) == 1)) return mk(r, false);
  g.mul++;
  return mk(r, false);
}
inline CF operator/(CF a, CF b) {
  g.sfu++;
  return mk(a.v / b.v, a.k && b.k);
}
inline CF operator-(CF a) { return mk(-a.v, a.k); }
inline CF& operator+=(CF& a, CF b) { return a = a + b; }
inline CF& operator-=(CF& a, CF b) { return a = a - b; }
inline CF& operator*=(CF& a, CF b) { return a = a * b; }
inline bool operator<(CF a, CF b) { return a.v < b.v; }
inline bool operator>(CF a, CF b) { return a.v > b.v; }
inline bool operator<=(CF a, CF b) { return a.v <= b.v; }
inline bool operator>=(CF a, CF b) { return a.v >= b.v; }
inline bool operator==(CF a, CF b) { return a.v == b.v; }
inline bool operator!=(CF a, CF b) { return a.v != b.v; }
inline void __sincosf(CF x, CF* s, CF* c) {
  g.sfu++;
  *s = mk(std::sin(x.v), false);
  *c = mk(std::cos(x.v), false);
}
inline CF rsqrtf(CF x) {
  g.sfu++;
  return mk(1.0 / std::sqrt(x.v), false);
}
inline CF sqrtf(CF x) {
  g.sfu++;
  return mk(std::sqrt(x.v), false);
}
inline CF fminf(CF a, CF b) { return mk(a.v < b.v ? a.v : b.v, a.k && b.k); }
inline CF fmaxf(CF a, CF b) { return mk(a.v > b.v ? a.v : b.v, a.k && b.k); }

#define __device__
#define __forceinline__ inline
#include "sg_internal.h"
#include "chain_host.h"     // sg_chain.cuh with float -> CF
#include "adjoint_host.h"   // sg_adjoint.cuh with float -> CF

using namespace sg;

template <class P>
void count(const char* name, P pat) {
  static CF rec[kRecordFloats];
  for (int i = 0; i < kRecordFloats; ++i) rec[i] = CF::var(0.1 + 0.001 * i);
  const Rec r{rec};
  CF q[7], qd[7], qs[7], lq[7], lqd[7], lqs[7], lm[7];
  for (int i = 0; i < 7; ++i) {
    q[i] = CF::var(0.1 * i);
    qd[i] = CF::var(0.2);
    qs[i] = CF::var(0.3);
    lq[i] = CF::var(0.01 * i);
    lqd[i] = CF::var(0.02);
    lqs[i] = CF::var(0.0);
    lm[i] = CF::var(0.0);
  }
  const CF h = CF::var(1.0 / 120), grav = CF::var(9.81);
  // the substep as the kernels run it: trigonometry carried in from the
  // previous substep (chain_substep_trig recomputes it for the new state)
  CF cq[P::N], sq[P::N];
  joint_sincos(pat, q, cq, sq);
  g = Cnt();
  chain_substep_trig(pat, r, q, qd, qs, cq, sq, h, grav);
  const Cnt sub = g;
  g = Cnt();
  V3 tip, r0, r1, r2;
  chain_tip_trig(pat, r, q, cq, sq, tip, r0, r1, r2);
  const Cnt tp = g;
  g = Cnt();
  substep_adjoint(pat, r, q, qd, qs, h, grav, lq, lqd, lqs, lm);
  const Cnt adj = g;
  // the replay part of a substep adjoint: the recomputed substep with its
  // factor, then the inverse-dynamics sweeps (replay warps, or the forward
  // kernel for the last segment)
  g = Cnt();
  {
    CF cq2[P::N], sq2[P::N], M[P::N][P::N], inv[P::N], acc[P::N], ks[P::N], dqd[P::N];
    substep_record(pat, r, q, qd, qs, h, grav, cq2, sq2, M, inv, acc, ks, dqd);
    SweepArrays<P::N> sw;
    id_sweeps(pat, r, q, qd, acc, cq2, sq2, grav, sw);
  }
  const Cnt rp = g;
  g = Cnt();
  CF gq[P::N];
  for (int i = 0; i < P::N; ++i) gq[i] = CF::var(0.0);
  tip_vjp(pat, r, q, V3{CF::var(0.1), CF::var(0.2), CF::var(0.3)}, gq);
  const Cnt tv = g;
  std::printf("%s substep %ld tip %ld substep_adjoint %ld tip_vjp %ld substep_replay %ld\n", name,
              sub.add + sub.mul, tp.add + tp.mul, adj.add + adj.mul, tv.add + tv.mul,
              rp.add + rp.mul);
}

int main() {
  count("7R", Pat7R{});
  count("7P", Pat7P{});
  count("4R", Pat4R{});
  return 0;
}
