// Device helpers shared by the step kernels: mbarrier / bulk-copy PTX
// wrappers with bounded waits, action loads and the observation write-out.
#pragma once

#include <cuda_runtime.h>

#include "sg_chain.cuh"
#include "sg_internal.h"

namespace sg {

constexpr float kGravity = 9.81f;
// Default wall-clock bound of every device-side wait (2 s); a test hook can
// shorten it per context (StepArgs::wait_ns).
constexpr unsigned long long kWaitNs = kDefaultWaitNs;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// One poll of a barrier phase; the thread may be suspended for at most
// about 20 us (the suspend-time hint) while the phase is incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for a barrier phase, bounded by wall time (limit_ns, read from
// %globaltimer after every unsuccessful poll) and, should the timer not
// advance, by an iteration count.
__device__ __forceinline__ bool mbar_wait_timed(uint64_t* bar, unsigned parity,
                                                unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned it = 0; it < (1u << 24); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
  return false;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  unsigned long long limit_ns = kWaitNs) {
  return mbar_wait_timed(bar, parity, limit_ns);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait with a warp-uniform verdict; false (and the error flag set)
// if the partner did not arrive within limit_ns.
__device__ __forceinline__ bool pair_wait(uint64_t* bar, unsigned& parity, int* err, int lane,
                                          unsigned long long limit_ns = kWaitNs) {
  const bool ok = __all_sync(0xffffffffu, mbar_wait_timed(bar, parity, limit_ns));
  parity ^= 1u;
  if (!ok && lane == 0) atomicOr(err, DEVERR_TIMEOUT);
  return ok;
}

template <class Pat>
__device__ __forceinline__ void load_targets(const Pat& pat, const StepArgs& a, int t, int env,
                                             int jo, float (&dst)[7]) {
  const float* arow = a.actions + ((size_t)t * a.num_envs + env) * a.max_joints + jo;
#pragma unroll
  for (int i = 0; i < Pat::N; ++i)
    if (pat.active(i)) dst[i] = __ldg(arow + i);
}

// Copy the warp's staged observation rows to HBM: one warp-wide store per row
// (8-byte vectors when rows are 8-byte aligned and D <= 64, else 4-byte).
__device__ __forceinline__ void write_rows(float* obs_t, const float* stage, int row_env, int nrows,
                                           int D, int DP, int lane) {
  if ((D & 1) == 0 && D <= 2 * kWarp) {
    const int half = D >> 1;
#pragma unroll 4
    for (int rr = 0; rr < nrows; ++rr) {
      const int er = __shfl_sync(0xffffffffu, row_env, rr);
      if (er >= 0 && lane < half) {
        const float2 v = reinterpret_cast<const float2*>(stage + rr * DP)[lane];
        reinterpret_cast<float2*>(obs_t + (size_t)er * D)[lane] = v;
      }
    }
  } else {
#pragma unroll 4
    for (int rr = 0; rr < nrows; ++rr) {
      const int er = __shfl_sync(0xffffffffu, row_env, rr);
      if (er >= 0) {
        const float* src = stage + rr * DP;
        float* dst = obs_t + (size_t)er * D;
        for (int k = lane; k < D; k += kWarp) dst[k] = src[k];
      }
    }
  }
}

// The warp's kRows staged rows when they belong to consecutive envs (env0 ..
// env0 + kRows - 1) and the stage pitch equals D: one contiguous block of
// kRows * D floats in shared and in global memory, copied with all lanes on
// consecutive addresses -- 16-byte vectors when both ends are 16-byte
// aligned, else 4-byte words.  (Row by row, a single-arm env of odd width
// D = 27 cost about 280 cycles per row; the block copy a few per row.)
template <int kRows>
__device__ __forceinline__ void write_block(float* obs_t, const float* stage, int env0, int D,
                                            int lane) {
  float* dst = obs_t + (size_t)env0 * D;
  const int n = kRows * D;
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(stage)) & 15) == 0 &&
      (n & 3) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(stage);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = lane; i < (n >> 2); i += kWarp) d4[i] = s4[i];
  } else {
    for (int i = lane; i < n; i += kWarp) dst[i] = stage[i];
  }
}

// Whether a warp's kRows observation rows (row r: env row_env of lane r,
// -1 if not written) are consecutive envs whose staged rows are contiguous
// (stage pitch D), i.e. can be written by write_block; warp-uniform.
__device__ __forceinline__ bool rows_contiguous(int row_env, int nrows, int D, int DP, int lane) {
  const int env0 = __shfl_sync(0xffffffffu, row_env, 0);
  return DP == D && env0 >= 0 &&
         __all_sync(0xffffffffu, lane >= nrows || row_env == env0 + lane);
}

// write_rows with the row count known at compile time (loop fully unrolled)
template <int kRows>
__device__ __forceinline__ void write_rows_n(float* obs_t, const float* stage, int row_env, int D,
                                             int DP, int lane) {
  if ((D & 1) == 0 && D <= 2 * kWarp) {
    const int half = D >> 1;
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) {
      const int er = __shfl_sync(0xffffffffu, row_env, rr);
      if (er >= 0 && lane < half) {
        const float2 v = reinterpret_cast<const float2*>(stage + rr * DP)[lane];
        reinterpret_cast<float2*>(obs_t + (size_t)er * D)[lane] = v;
      }
    }
  } else {
    write_rows(obs_t, stage, row_env, kRows, D, DP, lane);
  }
}

}  // namespace sg
