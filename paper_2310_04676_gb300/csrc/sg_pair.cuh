// One implicit-drive substep of 32 chains split across a warp pair (used by
// the warp-pair step kernel and the warp-pair forward of the differentiable
// rollout).
//   role 0 (dynamics): RNEA bias forces and the implicit drive right-hand side;
//   role 1 (inertia):  composite-rigid-body mass matrix plus the drive
//                      armature, then its Cholesky factorisation.
// The two halves run concurrently and meet in a shared-memory exchange (one
// mbarrier phase per substep, bounded wait); both roles then run the same
// triangular solve on the same operands, so their copies of the chain state
// stay bit-identical.
#pragma once

#include "sg_chain.cuh"
#include "sg_device.cuh"

namespace sg {

// exchange per pair and substep: the Cholesky factor (lower triangle with
// 1/L_ii on the diagonal, packed row by row) and the right-hand side; the
// caller alternates two such buffers between substeps
constexpr int kTri = kMaxLinks * (kMaxLinks + 1) / 2;
constexpr int kXHalf = (kTri + kMaxLinks) * kWarp;
constexpr int kXFloats = 2 * kXHalf;

__device__ __forceinline__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Computes this role's half of the substep from (q, qd, q*, cos q, sin q),
// exchanges it through xb and returns in (L, inv, dqd) the factor, the
// reciprocal diagonal and the solved velocity increment (state not yet
// advanced).  False (error flag set) if the partner did not arrive within
// wait_ns.  skip_arrival (a test hook) leaves out this warp's arrival, so
// that both warps' waits run out.
template <class Pat>
__device__ __forceinline__ bool pair_substep(const Pat& pat, const Rec& rec, const float (&q)[7],
                                             const float (&qd)[7], const float (&qs)[7],
                                             const float (&cq)[Pat::N], const float (&sq)[Pat::N],
                                             float h, float* xb, uint64_t* bar_x, unsigned& ph_x,
                                             int* err, int lane, int role,
                                             float (&L)[Pat::N][Pat::N], float (&inv)[Pat::N],
                                             float (&dqd)[Pat::N],
                                             unsigned long long wait_ns = kWaitNs,
                                             bool skip_arrival = false) {
  constexpr int N = Pat::N;
  if (role == 0) {
    float bias[N], rhs[N], arm[N], Mdummy[N][N];
    V3 F[N], Nm[N];
    rnea_forward(pat, rec, q, qd, cq, sq, kGravity, F, Nm);
    backward_sweep<Pat, true, false>(pat, rec, q, cq, sq, F, Nm, bias, Mdummy);
    drive_terms(pat, rec, q, qd, qs, h, bias, rhs, arm);
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (pat.active(i)) xb[(kTri + i) * kWarp + lane] = rhs[i];
  } else {
    float M[N][N], minv[N], bias_dummy[N], rhs_dummy[N], arm[N];
    V3 Fd[N], Nd[N];
    backward_sweep<Pat, false, true>(pat, rec, q, cq, sq, Fd, Nd, bias_dummy, M);
    drive_terms(pat, rec, q, qd, qs, h, bias_dummy, rhs_dummy, arm);
    chol_factor(pat, M, arm, minv);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      if (!pat.active(i)) continue;
      xb[tri(i, i) * kWarp + lane] = minv[i];
#pragma unroll
      for (int j = 0; j < i; ++j) xb[tri(i, j) * kWarp + lane] = M[i][j];
    }
  }
  if (!skip_arrival) mbar_arrive(bar_x);
  if (!pair_wait(bar_x, ph_x, err, lane, wait_ns)) return false;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (!pat.active(i)) continue;
    dqd[i] = xb[(kTri + i) * kWarp + lane];
    inv[i] = xb[tri(i, i) * kWarp + lane];
#pragma unroll
    for (int j = 0; j < i; ++j) L[i][j] = xb[tri(i, j) * kWarp + lane];
  }
  chol_apply(pat, L, inv, dqd);
  return true;
}

}  // namespace sg
