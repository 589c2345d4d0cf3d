// Waypoint tables of the path-following task (Results, "Path following"):
// a cubic spline through each env's control points, sampled at regular
// intervals of distance along the curve.
//
// One warp builds one env's table, in FP32 throughout:
//   1. natural-spline second derivatives M (uniform knots t_i = i, M = 0 at
//      both ends) from the tridiagonal system M_{i-1} + 4 M_i + M_{i+1} =
//      6 (P_{i+1} - 2 P_i + P_{i-1}), by the Thomas algorithm (lanes 0..2,
//      one coordinate each), then the per-segment coefficients
//      S_i(s) = a s^3 + b s^2 + c s + d, s = t - t_i in [0, 1];
//   2. a dense polyline of kPathDense points per segment (s = j / 64) plus
//      the end point; chord lengths and their running sum within each
//      segment by warp scans, and the arc length at each segment start as
//      an unevaluated float sum hi + lo (error-free TwoSum accumulation,
//      Knuth, TAOCP vol. 2, 4.2.2), so that the table does not lose
//      precision with the number of segments;
//   3. waypoint w at arc length x = w L / (W - 1), also as hi + lo: the
//      segment by binary search over the segment starts, then the polyline
//      piece by binary search within the segment, and linear interpolation
//      between its two points.
// FP64 is not used: on this part it runs at a small fraction of the FP32 rate.
#include "sg_path.h"

namespace sg {
namespace {

struct PathLayout {
  size_t lc, off, m, cp, coef, ctrl, bytes;  // byte offsets within a warp's region
};

// Per warp: in-segment running chord sums lc [K-1][64], segment-start arc
// lengths off [K] (float2 hi, lo), M [K][3], Thomas multipliers [K],
// coefficients [K-1][12], control points [K][3].
__host__ __device__ inline PathLayout path_layout(int K) {
  PathLayout L;
  L.off = 0;
  L.lc = L.off + sizeof(float2) * K;
  L.m = L.lc + sizeof(float) * kPathDense * (K - 1);
  L.cp = L.m + sizeof(float) * 3 * K;
  L.coef = L.cp + sizeof(float) * K;
  L.ctrl = L.coef + sizeof(float) * 12 * (K - 1);
  L.bytes = (L.ctrl + sizeof(float) * 3 * K + 15) & ~size_t(15);
  return L;
}

// Point n (0 .. 64 (K-1)) of the dense polyline: segment min(n / 64, K - 2)
// at s = (n - 64 seg) / 64, so the last point is the end of the last segment.
__device__ __forceinline__ void dense_point(const float* coef, int K, int n, float& x, float& y,
                                            float& z) {
  const int seg = min(n / kPathDense, K - 2);
  const float s = (float)(n - kPathDense * seg) * (1.f / kPathDense);
  const float* c = coef + 12 * seg;   // a(3) b(3) c(3) d(3)
  x = ((c[0] * s + c[3]) * s + c[6]) * s + c[9];
  y = ((c[1] * s + c[4]) * s + c[7]) * s + c[10];
  z = ((c[2] * s + c[5]) * s + c[8]) * s + c[11];
}

__device__ __forceinline__ float warp_inclusive_scan(float v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const float u = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += u;
  }
  return v;
}

// s + e = a + b exactly (TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (a.x + a.y) <= (b.x + b.y) for normalised float pairs.
__device__ __forceinline__ bool ff_le(float2 a, float2 b) {
  return a.x < b.x || (a.x == b.x && a.y <= b.y);
}

__global__ void __launch_bounds__(32 * kPathWarps)
build_paths_kernel(const float* __restrict__ ctrl, int K, const uint8_t* __restrict__ mask,
                   int E, int W, float* __restrict__ path) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int e = blockIdx.x * kPathWarps + warp;
  if (e >= E) return;                       // warp-uniform
  if (mask && !mask[e]) return;             // warp-uniform
  const PathLayout L = path_layout(K);
  unsigned char* base = smem + L.bytes * warp;
  float2* off = reinterpret_cast<float2*>(base + L.off);  // [K]
  float* lc = reinterpret_cast<float*>(base + L.lc);      // [K-1][64]
  float* M = reinterpret_cast<float*>(base + L.m);        // [K][3]
  float* cp = reinterpret_cast<float*>(base + L.cp);      // [K]
  float* coef = reinterpret_cast<float*>(base + L.coef);  // [K-1][12]
  float* P = reinterpret_cast<float*>(base + L.ctrl);     // [K][3]

  const float* src = ctrl + (size_t)e * K * 3;
  for (int i = lane; i < 3 * K; i += 32) P[i] = src[i];
  __syncwarp();

  // 1. natural-spline second derivatives (interior unknowns 1..K-2)
  if (lane < 3) {
    const int k = lane;
    M[k] = 0.f;
    M[3 * (K - 1) + k] = 0.f;
    float cprev = 0.f, dprev = 0.f;
    for (int i = 1; i <= K - 2; ++i) {
      const float r = 6.f * ((P[3 * (i + 1) + k] - P[3 * i + k]) - (P[3 * i + k] - P[3 * (i - 1) + k]));
      const float den = 4.f - cprev;
      cprev = 1.f / den;
      dprev = (r - dprev) * cprev;
      if (k == 0) cp[i] = cprev;
      M[3 * i + k] = dprev;
    }
    __syncwarp(0x7u);
    for (int i = K - 3; i >= 1; --i) M[3 * i + k] -= cp[i] * M[3 * (i + 1) + k];
  }
  __syncwarp();
  for (int idx = lane; idx < 3 * (K - 1); idx += 32) {
    const int i = idx / 3, k = idx - 3 * i;
    const float m0 = M[3 * i + k], m1 = M[3 * (i + 1) + k];
    const float p0 = P[3 * i + k], p1 = P[3 * (i + 1) + k];
    float* c = coef + 12 * i;
    c[k] = (m1 - m0) * (1.f / 6.f);
    c[3 + k] = 0.5f * m0;
    c[6 + k] = (p1 - p0) - (2.f * m0 + m1) * (1.f / 6.f);
    c[9 + k] = p0;
  }
  __syncwarp();

  // 2. chord lengths, their running sum within each segment
  for (int seg = 0; seg < K - 1; ++seg) {
    float carry = 0.f;
#pragma unroll
    for (int half = 0; half < kPathDense; half += 32) {
      const int n = kPathDense * seg + half + lane;
      float x0, y0, z0, x1, y1, z1;
      dense_point(coef, K, n, x0, y0, z0);
      dense_point(coef, K, n + 1, x1, y1, z1);
      const float dx = x1 - x0, dy = y1 - y0, dz = z1 - z0;
      const float s = carry + warp_inclusive_scan(sqrtf(dx * dx + dy * dy + dz * dz), lane);
      lc[n] = s;
      carry = __shfl_sync(0xffffffffu, s, 31);
    }
  }
  __syncwarp();
  // arc length at each segment start, hi + lo
  if (lane == 0) {
    float hi = 0.f, lo = 0.f;
    off[0] = make_float2(0.f, 0.f);
    for (int seg = 0; seg < K - 1; ++seg) {
      float s, err;
      two_sum(hi, lc[kPathDense * seg + kPathDense - 1], s, err);
      two_sum(s, __fadd_rn(lo, err), hi, lo);
      off[seg + 1] = make_float2(hi, lo);
    }
  }
  __syncwarp();

  // 3. waypoints at equal arc-length spacing: x = w * (step_hi + step_lo)
  const float2 total = off[K - 1];
  const float wm1 = (float)max(W - 1, 1);
  const float step_hi = __fdiv_rn(total.x, wm1);
  const float step_lo = __fdiv_rn(__fadd_rn(__fmaf_rn(-step_hi, wm1, total.x), total.y), wm1);
  float* dst = path + (size_t)e * W * 3;
  for (int w = lane; w < W; w += 32) {
    float2 x;
    if (w == W - 1) {
      x = total;
    } else {
      const float fw = (float)w;
      const float xh = __fmul_rn(fw, step_hi);
      const float xl = __fadd_rn(__fmaf_rn(fw, step_hi, -xh), __fmul_rn(fw, step_lo));
      two_sum(xh, xl, x.x, x.y);
    }
    int lo = 0, hi = K - 2;                 // largest segment with off[seg] <= x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (ff_le(off[mid], x)) lo = mid; else hi = mid - 1;
    }
    const int seg = lo;
    const float r = __fadd_rn(__fsub_rn(x.x, off[seg].x), __fsub_rn(x.y, off[seg].y));
    const float* c = lc + kPathDense * seg;  // c[j] = length from the segment start to point j+1
    int a = 0, b = kPathDense - 1;          // largest j in [0, 63] with len(j) <= r, len(0) = 0
    while (a < b) {
      const int mid = (a + b + 1) >> 1;
      if (c[mid - 1] <= r) a = mid; else b = mid - 1;
    }
    const float l0 = a > 0 ? c[a - 1] : 0.f, l1 = c[a];
    const float span = l1 - l0;
    const float f = span > 0.f ? fminf(fmaxf((r - l0) / span, 0.f), 1.f) : 0.f;
    float x0, y0, z0, x1, y1, z1;
    const int n = kPathDense * seg + a;
    dense_point(coef, K, n, x0, y0, z0);
    dense_point(coef, K, n + 1, x1, y1, z1);
    dst[3 * w + 0] = x0 + f * (x1 - x0);
    dst[3 * w + 1] = y0 + f * (y1 - y0);
    dst[3 * w + 2] = z0 + f * (z1 - z0);
  }
}

}  // namespace

size_t path_smem_bytes(int K) { return path_layout(K).bytes * kPathWarps; }
cudaError_t prepare_path_kernel() {
  return cudaFuncSetAttribute(build_paths_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)path_smem_bytes(kMaxPathCtrl));
}

cudaError_t launch_build_paths(const float* ctrl, int K, const uint8_t* mask, int E, int W,
                               float* path, cudaStream_t stream) {
  if (K < 2 || K > kMaxPathCtrl || E < 1 || W < 1) return cudaErrorInvalidValue;
  const int blocks = (E + kPathWarps - 1) / kPathWarps;
  build_paths_kernel<<<blocks, 32 * kPathWarps, path_smem_bytes(K), stream>>>(ctrl, K, mask, E,
                                                                               W, path);
  return cudaGetLastError();
}

}  // namespace sg
