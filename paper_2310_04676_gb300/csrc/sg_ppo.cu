// GPU-resident PPO loop (include/sg_ppo.h): the policy and value networks,
// action sampling, env stepping, time-out bootstrapping, resets, GAE and the
// clipped PPO update, all on the env context's stream.
//
// Layout: activations are row-major [rows][width] (rows = envs while
// collecting, minibatch rows while updating); weights row-major [out][in].
// The dense layers run on this library's tensor-core contraction (sg_mlp.cu:
// tcgen05 kind::tf32 with three-product split precision, FP32-grade; one
// TF32 product per term with tf32 = 1): forward products with the bias and
// ELU in their epilogue, input gradients with the ELU derivative and the
// bias-gradient partial sums of the layer below in theirs, and weight
// gradients split over the minibatch rows with a fixed-order sum of the
// partials.  The Gaussian head and its gradient, GAE, the gathers, the
// reductions (fixed-order, so results do not depend on scheduling) and Adam
// are the kernels below.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sg.h"
#include "sg_diff.h"
#include "sg_internal.h"
#include "sg_mlp.h"
#include "sg_ppo.h"
#include "sg_rng.cuh"

namespace sg {
namespace {

constexpr int kH1 = 256, kH2 = 128, kH3 = 64;
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 512;            // partial sums of the two-stage reductions
constexpr float kHalfLog2Pi = 0.91893853320467274f;

// ---- parameter layout ------------------------------------------------------
struct Layer {
  size_t w, b;       // offsets of W [out][in] and b [out]
  int in, out;
  // offsets of W's TF32 parts in the pre-split buffer: as the forward
  // product's B (n = out, k = in) and as the input gradient's (n = in, k = out)
  size_t pre_fwd = 0, pre_dx = 0;
};
struct Net {
  Layer l[4];
};
struct Layout {
  Net actor, critic;
  size_t log_std, total;
};

Layout make_layout(int D, int A) {
  Layout L;
  size_t k = 0;
  const int dims[4] = {D, kH1, kH2, kH3};
  auto net = [&](Net& n, int out_last) {
    for (int i = 0; i < 4; ++i) {
      n.l[i].in = dims[i];
      n.l[i].out = i < 3 ? dims[i + 1] : out_last;
      n.l[i].w = k;
      k += (size_t)n.l[i].in * n.l[i].out;
      n.l[i].b = k;
      k += n.l[i].out;
    }
  };
  net(L.actor, A);
  L.log_std = k;
  k += A;
  net(L.critic, 1);
  L.total = k;
  return L;
}

// ---- kernels -----------------------------------------------------------------
// Zero-padded copy of rows [rows][w] -> [rows][wp]
__global__ void pad_rows_kernel(const float* __restrict__ src, int rows, int w, int wp,
                                float* __restrict__ dst) {
  const long long n = (long long)rows * wp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / wp), c = (int)(i - (long long)r * wp);
    dst[i] = c < w ? src[(size_t)r * w + c] : 0.f;
  }
}

// Public <-> internal (padded) parameter layouts: internal[map[i]] = public[i]
__global__ void scatter_kernel(const float* __restrict__ pub, const int32_t* __restrict__ map,
                               int n, float* __restrict__ in) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    in[map[i]] = pub[i];
}
__global__ void gather_params_kernel(const float* __restrict__ in, const int32_t* __restrict__ map,
                                     int n, float* __restrict__ pub) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    pub[i] = in[map[i]];
}

// Actions, log-probabilities and values of one collect step (thread per env).
__global__ void sample_kernel(const float* __restrict__ mu, const float* __restrict__ log_std,
                              const float* __restrict__ mask, const long long* __restrict__ step,
                              int t, uint32_t seed, int E, int A, int Ap,
                              float* __restrict__ actions, float* __restrict__ logp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const long long gstep = *step + t;
  float lp = 0.f;
  for (int blk = 0; blk * 4 < A; ++blk) {
    float z[4];
    action_noise(seed, e, blk, gstep, z);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * blk + c;
      if (j >= A) break;
      const float ls = log_std[j];
      actions[(size_t)e * A + j] = mu[(size_t)e * Ap + j] + expf(ls) * z[c];
      if (mask[(size_t)e * A + j] != 0.f) lp += -0.5f * z[c] * z[c] - ls - kHalfLog2Pi;
    }
  }
  logp[e] = lp;
}

// Bootstrap time-outs into the reward and mark envs to reset.
__global__ void bootstrap_kernel(float* __restrict__ reward, const uint8_t* __restrict__ done,
                                 const float* __restrict__ value, float gamma, int E,
                                 uint8_t* __restrict__ reset) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const uint8_t d = done[e];
  if (d & SG_DONE_TIMEOUT) reward[e] += gamma * value[e];
  reset[e] = d != 0 ? 1 : 0;
}

// GAE over the n steps of every env (thread per env).
__global__ void gae_kernel(const float* __restrict__ reward, const float* __restrict__ value,
                           const uint8_t* __restrict__ done, int n, int E, float gamma, float lam,
                           float* __restrict__ adv, float* __restrict__ ret) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  float next = 0.f;
  for (int t = n - 1; t >= 0; --t) {
    const size_t i = (size_t)t * E + e;
    const float keep = done[i] ? 0.f : 1.f;
    const float delta = reward[i] + gamma * value[i + E] * keep - value[i];
    next = delta + gamma * lam * keep * next;
    adv[i] = next;
    ret[i] = next + value[i];
  }
}

__global__ void advance_kernel(long long* step, int n) { *step += n; }

// Block reduction of a double (all threads get the result).
__device__ double block_sum(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_down_sync(0xffffffffu, r, off);
    if (threadIdx.x == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// blocks of the bias-gradient partial sums of the output layers
constexpr int kBGradBlocks = 608;

// Per-block column sums of Y [rows][w] for narrow w (the output layers' bias
// gradient): block b takes rows [b*chunk, (b+1)*chunk); thread t sums column
// t % w over every (256 / w)-th row; partial sums then combine in thread order.
__global__ void __launch_bounds__(256)
colsum_partial_kernel(const float* __restrict__ Y, int rows, int w, float* __restrict__ part) {
  __shared__ float sh[256];
  const int groups = blockDim.x / w;
  const int c = threadIdx.x % w, g = threadIdx.x / w;
  const int chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  float acc = 0.f;
  if (g < groups)
    for (int r = r0 + g; r < r1; r += groups) acc += Y[(size_t)r * w + c];
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < w) {
    float t = 0.f;
    for (int k = 0; k < groups; ++k) t += sh[k * w + threadIdx.x];
    part[(size_t)blockIdx.x * w + threadIdx.x] = t;
  }
}

// The bias gradients of one network's four layers in one launch: job j
// sums part_j[b][c] over b < nblk_j for its w_j columns (a block per column,
// columns of the jobs in order).
struct BGradJobs {
  const float* part[4];
  float* grad[4];
  int nblk[4], w[4];
};
__global__ void __launch_bounds__(128) bgrad_final_multi_kernel(BGradJobs J) {
  __shared__ double sh[32];
  int c = blockIdx.x, j = 0;
  while (j < 3 && c >= J.w[j]) c -= J.w[j++];
  const float* part = J.part[j];
  const int w = J.w[j];
  double s = 0.0;
  for (int b = threadIdx.x; b < J.nblk[j]; b += blockDim.x) s += part[(size_t)b * w + c];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) J.grad[j][c] = (float)s;
}

// Stage 1: per-block sums of x and x^2 (fixed grid, fixed order).
__global__ void __launch_bounds__(kRedThreads)
moments_partial_kernel(const float* __restrict__ x, long long n, double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0, q = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    s += v;
    q += v * v;
  }
  s = block_sum(s, sh);
  q = block_sum(q, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s;
    part[2 * blockIdx.x + 1] = q;
  }
}

// Stage 2: mean and 1 / (unbiased std + 1e-8) of the advantages.
__global__ void __launch_bounds__(kRedThreads)
moments_final_kernel(const double* __restrict__ part, int nblk, long long n,
                     float* __restrict__ norm) {
  __shared__ double sh[32];
  double s = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    s += part[2 * i];
    q += part[2 * i + 1];
  }
  s = block_sum(s, sh);
  q = block_sum(q, sh);
  if (threadIdx.x == 0) {
    const double mean = s / (double)n;
    const double var = n > 1 ? (q - (double)n * mean * mean) / (double)(n - 1) : 0.0;
    norm[0] = (float)mean;
    norm[1] = (float)(1.0 / (sqrt(var > 0.0 ? var : 0.0) + 1e-8));
  }
}

struct Batch {
  const float *obs, *act, *logp, *value, *adv, *ret, *jmask, *norm;
};
struct MiniBatch {
  float *obs, *act, *logp, *value, *adv, *ret, *mask;
};

// Gather minibatch rows (warp per row): row index b = t * E + e.
__global__ void gather_kernel(Batch src, MiniBatch dst, const int32_t* __restrict__ idx, int M,
                              int E, int D, int Dp, int A) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= M) return;
  const long long b = idx[row];
  const int e = (int)(b % E);
  for (int k = lane; k < Dp; k += 32)
    dst.obs[(size_t)row * Dp + k] = k < D ? src.obs[(size_t)b * D + k] : 0.f;
  for (int k = lane; k < A; k += 32) {
    dst.act[(size_t)row * A + k] = src.act[(size_t)b * A + k];
    dst.mask[(size_t)row * A + k] = src.jmask[(size_t)e * A + k];
  }
  if (lane == 0) {
    dst.logp[row] = src.logp[b];
    dst.value[row] = src.value[b];
    dst.adv[row] = (src.adv[b] - src.norm[0]) * src.norm[1];
    dst.ret[row] = src.ret[b];
  }
}

struct HeadArgs {
  const float *mu, *v, *log_std;
  MiniBatch mb;
  float *d_mu, *d_v;
  float* part;          // [blocks][2 + 2A]: surrogate sum, value-loss sum, dlogstd_j, count_j
  int M, A, Ap;
  float clip, value_coef;
};

// Losses of the minibatch and their gradients with respect to the actor's
// mean, the critic's value and log_std (thread per row; per-block partials).
__global__ void __launch_bounds__(kRedThreads) head_kernel(HeadArgs h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool ok = i < h.M;
  const int A = h.A;
  const float inv_m = 1.f / (float)h.M;
  float surr = 0.f, vl = 0.f;
  float g_logp = 0.f;
  float zz[kMaxDof];
  if (ok) {
    float lp = 0.f;
    for (int j = 0; j < A; ++j) {
      const float ls = h.log_std[j];
      const float z = (h.mb.act[(size_t)i * A + j] - h.mu[(size_t)i * h.Ap + j]) * expf(-ls);
      zz[j] = z;
      if (h.mb.mask[(size_t)i * A + j] != 0.f) lp += -0.5f * z * z - ls - kHalfLog2Pi;
    }
    const float ratio = expf(lp - h.mb.logp[i]);
    const float adv = h.mb.adv[i];
    const float s1 = -adv * ratio;
    const float s2 = -adv * fminf(fmaxf(ratio, 1.f - h.clip), 1.f + h.clip);
    surr = fmaxf(s1, s2);
    // d max(s1, s2) / d logp: the clipped branch is flat where it is the larger
    g_logp = (s2 > s1) ? 0.f : -adv * ratio;
    const float v = h.v[i], vo = h.mb.value[i], R = h.mb.ret[i];
    const float dv = fminf(fmaxf(v - vo, -h.clip), h.clip);
    const float vc = vo + dv;
    const float l1 = (v - R) * (v - R), l2 = (vc - R) * (vc - R);
    vl = fmaxf(l1, l2);
    float gv;
    if (l1 > l2) gv = 2.f * (v - R);
    else if (l2 > l1) gv = (v - vo >= -h.clip && v - vo <= h.clip) ? 2.f * (vc - R) : 0.f;
    else gv = 0.5f * (2.f * (v - R) + ((v - vo >= -h.clip && v - vo <= h.clip) ? 2.f * (vc - R) : 0.f));
    h.d_v[i] = h.value_coef * gv * inv_m;
    const float g = g_logp * inv_m;
    for (int j = 0; j < h.Ap; ++j) {
      const float m = j < A ? h.mb.mask[(size_t)i * A + j] : 0.f;
      h.d_mu[(size_t)i * h.Ap + j] = m != 0.f ? g * zz[j] * expf(-h.log_std[j]) : 0.f;
    }
  }
  // per-block sums of (surrogate, value loss, dlogstd_j, count_j): warp
  // shuffles per column, then the warps' partials in a fixed order
  const int stride = 2 + 2 * A;
  __shared__ float wpart[kRedThreads / 32][2 + 2 * kMaxDof];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int col = 0; col < stride; ++col) {
    float x;
    if (col == 0) x = ok ? surr : 0.f;
    else if (col == 1) x = ok ? vl : 0.f;
    else {
      const int j = col < 2 + A ? col - 2 : col - 2 - A;
      const float m = ok ? h.mb.mask[(size_t)i * A + j] : 0.f;
      x = col < 2 + A ? ((ok && m != 0.f) ? g_logp * inv_m * (zz[j] * zz[j] - 1.f) : 0.f) : m;
    }
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
    if (lane == 0) wpart[w][col] = x;
  }
  __syncthreads();
  if (threadIdx.x < stride) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += wpart[k][threadIdx.x];
    h.part[(size_t)blockIdx.x * stride + threadIdx.x] = (float)t;
  }
}

// Final reduction of the head partials: log_std gradient (surrogate +
// entropy terms) and the minibatch's loss statistics (one block; each warp
// sums whole columns with its lanes, fixed order).
__global__ void __launch_bounds__(kRedThreads)
head_final_kernel(const float* __restrict__ part, int nblk, int A, int M,
                  const float* __restrict__ log_std, float entropy_coef,
                  float* __restrict__ grad_log_std, float* __restrict__ stats) {
  const int stride = 2 + 2 * A;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __shared__ double col[2 + 2 * kMaxDof];
  for (int c = w; c < stride; c += nw) {
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(size_t)b * stride + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) col[c] = s;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j < A) {
    const double cnt = col[2 + A + j] / (double)M;          // mean over rows of the mask
    grad_log_std[j] = (float)(col[2 + j] - (double)entropy_coef * cnt);
  }
  if (j == 0 && stats) {
    double ent = 0.0;
    for (int k = 0; k < A; ++k) ent += (0.5 + kHalfLog2Pi + (double)log_std[k]) * col[2 + A + k] / M;
    stats[0] = (float)(col[0] / M);
    stats[1] = (float)(col[1] / M);
    stats[2] = (float)ent;
  }
}

// Sum of squares of the gradient: stage 1 per block, stage 2 the clip factor.
__global__ void __launch_bounds__(kRedThreads)
sumsq_partial_kernel(const float* __restrict__ g, long long n, double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    s += (double)g[i] * g[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedThreads)
clip_final_kernel(const double* __restrict__ part, int nblk, float max_norm,
                  float* __restrict__ clip_coef, float* __restrict__ stats) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double norm = sqrt(s);
    const double c = (double)max_norm / (norm + 1e-6);
    *clip_coef = (float)(c < 1.0 ? c : 1.0);
    if (stats) stats[3] = (float)norm;
  }
}

// Adam with bias correction on the clipped gradient.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ clip_coef, long long n, float lr, float bc1,
                            float bc2) {
  const float c = *clip_coef;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i] * c;
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
  }
}

int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace
}  // namespace sg

using sg::Layer;
using sg::Layout;
using sg::Net;

struct sg_ppo {
  sg_ctx* env = nullptr;
  sg_ppo_config cfg{};
  int E = 0, D = 0, A = 0, n = 0, M = 0;
  int Dp = 0, Ap = 0;                  // obs and action widths padded to multiples of 4
  long long B = 0;
  Layout L{};                          // internal (padded) parameter layout
  size_t public_params = 0;            // length of the caller's flat vector
  int32_t* pub2int = nullptr;          // [public_params] internal index of each public entry
  float* xin = nullptr;                // [E][Dp] padded observations of the collect step
  cudaStream_t stream = nullptr;       // the stream the collect graph was captured for
  // The actor's products run on `stream`, the critic's on `side`, forked
  // from and joined back to `stream` by events: the networks are
  // independent between the minibatch gather and the loss head, and between
  // the head and the gradient norm.  Scratch per network: the row-split
  // partial sums of the weight gradients, the bias-gradient partials, the
  // input-gradient buffers.
  // Within a network's backward the weight gradients run on a third stream
  // (Lane::sw), each after the event that its output gradient is ready
  // (Lane::ev_dy), joined back before the bias gradients are finished.
  struct Lane {
    cudaStream_t s = nullptr, sw = nullptr;
    cudaEvent_t ev_dy[4] = {nullptr, nullptr, nullptr, nullptr}, ev_w = nullptr;
    float* work = nullptr;
    float* bgrad_part = nullptr;
    float* dbuf[3] = {nullptr, nullptr, nullptr};   // input gradients of layers 3, 2, 1
  } lane[2];
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  long long mlp_work_floats = 0;
  float* pre = nullptr;                // the weights' TF32 parts (sg::launch_mlp_presplit)
  sg::PresplitJobs pre_jobs{};
  int32_t* err = nullptr;              // the env context's device error word
  float *params = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
  long long adam_t = 0;
  long long* d_step = nullptr;         // global step of the exploration noise
  float *obs = nullptr, *actions = nullptr, *logp = nullptr, *values = nullptr, *rewards = nullptr;
  uint8_t* dones = nullptr;
  float *adv = nullptr, *ret = nullptr;
  float* jmask = nullptr;              // [E][A]
  uint8_t* reset_mask = nullptr;       // [E]
  float* zero_targets = nullptr;       // [E][A]
  // activations and their gradients, [rows_max][width]
  float *ha[3] = {nullptr, nullptr, nullptr}, *hc[3] = {nullptr, nullptr, nullptr};
  float *mu = nullptr, *vout = nullptr;
  float *dmu = nullptr, *dv = nullptr;  // loss gradients w.r.t. the actor mean and the value
  sg::MiniBatch mb{};
  float* head_part = nullptr;
  // bias-gradient partial sums (per network, Lane::bgrad_part), a region per
  // layer: [row tiles][width] (hidden layers), [blocks][out] (output layer)
  size_t bgrad_off[4] = {0, 0, 0, 0};
  double* red_part = nullptr;
  float* norm = nullptr;               // advantage mean, 1 / std
  float* clip_coef = nullptr;
  cudaGraphExec_t collect_exec = nullptr;
  int fault = 0;                       // test hook (sg_ppo_debug_set_fault)
  unsigned long long wait_ns = 0;      // bound of the contraction's waits, 0 = default
  std::vector<void*> allocs;
};

namespace {

sg_status fail(sg_ppo* p, sg_status code, const std::string& msg) {
  if (p && p->env) sg::context_set_error(p->env, msg.c_str());
  return code;
}

sg_status cuda_fail(sg_ppo* p, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SG_OK;
  return fail(p, e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <class T>
cudaError_t dalloc(sg_ppo* p, T** ptr, size_t count) {
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(ptr), sizeof(T) * (count ? count : 1));
  if (e == cudaSuccess) p->allocs.push_back(*ptr);
  return e;
}

// Products of the networks: tensor-core contraction (3xTF32, or one TF32
// product in the tf32 mode); the narrow ones (the first layer's 28 inputs,
// the output layers, their weight and input gradients) as FP32 FMA loops.
sg::MlpGemmArgs gemm_args(const sg_ppo* p) {
  sg::MlpGemmArgs g{};
  g.split_tf32 = p->cfg.tf32 ? 0 : 1;
  g.narrow = 1;
  g.err = p->err;
  g.fault = p->fault == SG_FAULT_SKIP_WEIGHT_COPY ? 1 : 0;
  g.wait_ns = p->wait_ns;
  return g;
}

// Split every layer's weights into their TF32 parts, in both operand roles
// (one launch; after every change of the parameters, before the products)
bool presplit_weights(sg_ppo* p) {
  return sg::launch_mlp_presplit(p->pre_jobs, p->cfg.tf32 ? 0 : 1, p->stream) == cudaSuccess;
}

// Y[rows][out] = act(X[rows][in] W^T + b), act = ELU on hidden layers
bool gemm_fwd(sg_ppo* p, const sg_ppo::Lane& ln, const float* X, int rows, const Layer& l,
              float* Y, bool elu) {
  sg::MlpGemmArgs g = gemm_args(p);
  g.A = X, g.a_m = l.in, g.a_k = 1;
  g.B = p->params + l.w, g.b_n = l.in, g.b_k = 1;
  g.b_pre = p->pre + l.pre_fwd, g.b_npad = sg::presplit_npad(l.out);
  g.C = Y, g.c_m = l.out;
  g.bias = p->params + l.b, g.elu = elu ? 1 : 0;
  g.M = rows, g.N = l.out, g.K = l.in;
  return sg::launch_mlp_gemm(g, ln.s) == cudaSuccess;
}
// dZ[rows][in] = (dY[rows][out] W) * ELU'(y), y [rows][in] the output of the
// ELU layer below, and per 128-row tile the column sums of dZ (that layer's
// bias gradient) into colsum
bool gemm_bwd_data_elu(sg_ppo* p, const sg_ppo::Lane& ln, const float* dY, int rows,
                       const Layer& l, const float* y, float* dZ, float* colsum) {
  sg::MlpGemmArgs g = gemm_args(p);
  g.A = dY, g.a_m = l.out, g.a_k = 1;
  g.B = p->params + l.w, g.b_n = 1, g.b_k = l.in;       // B(n = in, k = out) = W[out][in]
  g.b_pre = p->pre + l.pre_dx, g.b_npad = sg::presplit_npad(l.in);
  g.C = dZ, g.c_m = l.in;
  g.M = rows, g.N = l.in, g.K = l.out;
  g.act_y = y;
  g.colsum = colsum;
  return sg::launch_mlp_gemm(g, ln.s) == cudaSuccess;
}
// dW[out][in] = dY^T X (rows split over CTAs); with a bias_part region:
// the column sums of dY (db[out] = dY^T 1) per block of rows into it
bool gemm_bwd_weight(sg_ppo* p, const sg_ppo::Lane& ln, const float* dY, const float* X,
                     int rows, const Layer& l, float* bias_part) {
  sg::MlpGemmArgs g = gemm_args(p);
  g.A = dY, g.a_m = 1, g.a_k = l.out;                   // A(m = out, k = row)
  g.B = X, g.b_n = 1, g.b_k = l.in;                     // B(n = in, k = row)
  g.C = p->grad + l.w, g.c_m = l.in;
  g.M = l.out, g.N = l.in, g.K = rows;
  if (sg::launch_mlp_gemm_split(g, ln.work, p->mlp_work_floats, ln.s) != cudaSuccess)
    return false;
  if (!bias_part) return true;
  sg::colsum_partial_kernel<<<sg::kBGradBlocks, 256, 0, ln.s>>>(dY, rows, l.out, bias_part);
  return cudaGetLastError() == cudaSuccess;
}

// Forward of one network over `rows` inputs; hidden outputs kept in h[0..2].
bool net_forward(sg_ppo* p, const sg_ppo::Lane& ln, const Net& net, const float* X, int rows,
                 float* const (&h)[3], float* out) {
  const float* in = X;
  for (int i = 0; i < 4; ++i) {
    float* y = i < 3 ? h[i] : out;
    if (!gemm_fwd(p, ln, in, rows, net.l[i], y, i < 3)) return false;
    in = y;
  }
  return true;
}

// Backward of one network from dOut [rows][out]; weight gradients into p->grad.
// Below the output layer the ELU backward also sums the bias gradient (per
// 128-row tile, each layer in its own region of the lane's partials); one
// launch then finishes all four bias gradients.  The input gradients run in
// order on ln.s, each layer's weight gradient on ln.sw once its output
// gradient is ready; every input gradient has a buffer of its own, so none
// is overwritten while a weight gradient still reads it.
bool net_backward(sg_ppo* p, const sg_ppo::Lane& ln, const Net& net, const float* X, int rows,
                  float* const (&h)[3], const float* dOut) {
  const float* dY = dOut;
  const int tiles = (rows + 127) / 128;
  sg::BGradJobs jobs{};
  int cols = 0;
  sg_ppo::Lane wl = ln;
  wl.s = ln.sw;                                // the weight gradients' stream
  for (int i = 3; i >= 0; --i) {
    const float* in = i > 0 ? h[i - 1] : X;
    float* part = ln.bgrad_part + p->bgrad_off[i];
    if (cudaEventRecord(ln.ev_dy[i], ln.s) != cudaSuccess ||
        cudaStreamWaitEvent(ln.sw, ln.ev_dy[i], 0) != cudaSuccess)
      return false;
    if (!gemm_bwd_weight(p, wl, dY, in, rows, net.l[i], i == 3 ? part : nullptr)) return false;
    if (i == 3) {
      jobs.part[0] = part, jobs.grad[0] = p->grad + net.l[3].b;
      jobs.nblk[0] = sg::kBGradBlocks, jobs.w[0] = net.l[3].out;
      cols += net.l[3].out;
    }
    if (i == 0) break;
    float* dX = ln.dbuf[3 - i];
    // input gradient with the ELU backward and the bias-gradient partial sums
    // of layer i - 1 in the product's epilogue
    float* below = ln.bgrad_part + p->bgrad_off[i - 1];
    if (!gemm_bwd_data_elu(p, ln, dY, rows, net.l[i], h[i - 1], dX, below)) return false;
    const int j = 4 - i;
    jobs.part[j] = below, jobs.grad[j] = p->grad + net.l[i - 1].b;
    jobs.nblk[j] = tiles, jobs.w[j] = net.l[i].in;
    cols += net.l[i].in;
    dY = dX;
  }
  if (cudaEventRecord(ln.ev_w, ln.sw) != cudaSuccess ||
      cudaStreamWaitEvent(ln.s, ln.ev_w, 0) != cudaSuccess)
    return false;
  sg::bgrad_final_multi_kernel<<<cols, 128, 0, ln.s>>>(jobs);
  return cudaGetLastError() == cudaSuccess;
}

sg_status bind_stream(sg_ppo* p, cudaStream_t s) {
  p->stream = s;
  p->lane[0].s = s;
  p->lane[1].s = p->side;
  return SG_OK;
}

// The side stream waits for the work enqueued so far on p->stream.
bool fork(sg_ppo* p) {
  return cudaEventRecord(p->ev_fork, p->stream) == cudaSuccess &&
         cudaStreamWaitEvent(p->side, p->ev_fork, 0) == cudaSuccess;
}
// p->stream waits for the work enqueued so far on the side stream.
bool join(sg_ppo* p) {
  return cudaEventRecord(p->ev_join, p->side) == cudaSuccess &&
         cudaStreamWaitEvent(p->stream, p->ev_join, 0) == cudaSuccess;
}

// The collect loop as a sequence of launches on p->stream (captured once).
sg_status enqueue_collect(sg_ppo* p) {
  const int E = p->E, A = p->A, D = p->D, n = p->n;
  const sg_ppo_config& c = p->cfg;
  const int tb = 128, eb = (E + tb - 1) / tb;
  // the observations after the previous collect (or sg_ppo_reset) start this one
  cudaError_t ce = cudaMemcpyAsync(p->obs, p->obs + (size_t)n * E * D, (size_t)E * D * 4,
                                   cudaMemcpyDeviceToDevice, p->stream);
  if (ce != cudaSuccess) return cuda_fail(p, ce, "sg_ppo_collect");
  if (!presplit_weights(p)) return fail(p, SG_ERR_CUDA, "sg_ppo_collect: weight split failed");
  for (int t = 0; t < n; ++t) {
    float* o_t = p->obs + (size_t)t * E * D;
    float* o_next = p->obs + (size_t)(t + 1) * E * D;
    float* a_t = p->actions + (size_t)t * E * A;
    float* v_t = p->values + (size_t)t * E;
    sg::pad_rows_kernel<<<sg::grid_for((long long)E * p->Dp, 256), 256, 0, p->stream>>>(
        o_t, E, D, p->Dp, p->xin);
    // actor on this stream, critic on the side stream
    if (!fork(p) || !net_forward(p, p->lane[0], p->L.actor, p->xin, E, p->ha, p->mu) ||
        !net_forward(p, p->lane[1], p->L.critic, p->xin, E, p->hc, v_t) || !join(p))
      return fail(p, SG_ERR_CUDA, "sg_ppo_collect: network forward failed");
    sg::sample_kernel<<<eb, tb, 0, p->stream>>>(p->mu, p->params + p->L.log_std, p->jmask,
                                               p->d_step, t, c.seed, E, A, p->Ap, a_t,
                                               p->logp + (size_t)t * E);
    sg_status st = sg_step(p->env, a_t, c.dt, c.substeps, o_next, p->rewards + (size_t)t * E,
                           p->dones + (size_t)t * E);
    if (st != SG_OK) return st;
    sg::bootstrap_kernel<<<eb, tb, 0, p->stream>>>(p->rewards + (size_t)t * E,
                                                  p->dones + (size_t)t * E, v_t, c.gamma, E,
                                                  p->reset_mask);
    if ((st = sg_reset(p->env, p->reset_mask)) != SG_OK) return st;
    if ((st = sg_observe(p->env, a_t, p->reset_mask, o_next)) != SG_OK) return st;
  }
  sg::pad_rows_kernel<<<sg::grid_for((long long)E * p->Dp, 256), 256, 0, p->stream>>>(
      p->obs + (size_t)n * E * D, E, D, p->Dp, p->xin);
  if (!net_forward(p, p->lane[0], p->L.critic, p->xin, E, p->hc, p->values + (size_t)n * E))
    return fail(p, SG_ERR_CUDA, "sg_ppo_collect: critic forward failed");
  sg::gae_kernel<<<eb, tb, 0, p->stream>>>(p->rewards, p->values, p->dones, n, E, c.gamma, c.lam,
                                          p->adv, p->ret);
  sg::moments_partial_kernel<<<sg::kRedBlocks, sg::kRedThreads, 0, p->stream>>>(p->adv, p->B,
                                                                                p->red_part);
  sg::moments_final_kernel<<<1, sg::kRedThreads, 0, p->stream>>>(p->red_part, sg::kRedBlocks,
                                                                 p->B, p->norm);
  sg::advance_kernel<<<1, 1, 0, p->stream>>>(p->d_step, n);
  return cuda_fail(p, cudaGetLastError(), "sg_ppo_collect");
}

}  // namespace

// the environment context's device must be current (see sg_devcheck.h)
#define SG_PPO_CHECK_DEVICE(p, fn)                                         \
  do {                                                                     \
    const sg_status st_dev_ = sg::context_check_device((p)->env, fn);      \
    if (st_dev_ != SG_OK) return st_dev_;                                  \
  } while (0)

extern "C" {

sg_status sg_ppo_create(sg_ctx* env, const sg_ppo_config* cfg, sg_ppo** out) {
  if (!out) return SG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!env || !cfg) return SG_ERR_INVALID_ARG;
  const sg_status st_dev = sg::context_check_device(env, "sg_ppo_create");
  if (st_dev != SG_OK) return st_dev;
  sg_ppo* p = new (std::nothrow) sg_ppo();
  if (!p) return SG_ERR_OOM;
  p->env = env;
  p->cfg = *cfg;
  const sg_ppo_config& c = *cfg;
  p->E = sg_num_envs(env);
  p->D = sg_obs_dim(env);
  p->A = sg_max_joints(env);
  p->n = c.n_steps;
  p->B = (long long)p->E * c.n_steps;
  auto bad = [&](const char* m) {
    fail(p, SG_ERR_INVALID_ARG, std::string("sg_ppo_create: ") + m);
    delete p;
    return SG_ERR_INVALID_ARG;
  };
  if (c.n_steps < 1 || c.n_steps > 4096) return bad("n_steps must be 1..4096");
  if (c.epochs < 1 || c.minibatches < 1) return bad("epochs and minibatches must be >= 1");
  if (p->B % c.minibatches != 0) return bad("minibatches must divide num_envs * n_steps");
  if (p->B / c.minibatches > (1 << 30)) return bad("minibatch too large");
  if (!(c.gamma >= 0.f && c.gamma <= 1.f) || !(c.lam >= 0.f && c.lam <= 1.f))
    return bad("gamma and lam must be in [0, 1]");
  if (!(c.clip > 0.f) || !(c.lr > 0.f) || !(c.max_grad_norm > 0.f) || !(c.dt > 0.f))
    return bad("clip, lr, max_grad_norm and dt must be > 0");
  if (!std::isfinite(c.value_coef) || !std::isfinite(c.entropy_coef)) return bad("coefficients must be finite");
  if (c.substeps < 1 || c.substeps > 64) return bad("substeps must be 1..64");
  p->M = (int)(p->B / c.minibatches);
  p->Dp = (p->D + 3) & ~3;
  p->Ap = (p->A + 3) & ~3;
  p->L = sg::make_layout(p->Dp, p->Ap);
  const Layout Lpub = sg::make_layout(p->D, p->A);
  p->public_params = Lpub.total;
  const int rows = p->M > p->E ? p->M : p->E;
  const int E = p->E, A = p->A, D = p->D, n = p->n;
  cudaError_t e = cudaSuccess;
  auto step = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const size_t P = p->L.total;
  step(dalloc(p, &p->params, P));
  step(dalloc(p, &p->grad, P));
  step(dalloc(p, &p->adam_m, P));
  step(dalloc(p, &p->adam_v, P));
  step(dalloc(p, &p->d_step, 1));
  step(dalloc(p, &p->obs, (size_t)(n + 1) * E * D));
  step(dalloc(p, &p->actions, (size_t)n * E * A));
  step(dalloc(p, &p->logp, (size_t)n * E));
  step(dalloc(p, &p->values, (size_t)(n + 1) * E));
  step(dalloc(p, &p->rewards, (size_t)n * E));
  step(dalloc(p, &p->dones, (size_t)n * E));
  step(dalloc(p, &p->adv, (size_t)n * E));
  step(dalloc(p, &p->ret, (size_t)n * E));
  step(dalloc(p, &p->jmask, (size_t)E * A));
  step(dalloc(p, &p->reset_mask, (size_t)E));
  step(dalloc(p, &p->zero_targets, (size_t)E * A));
  const int widths[3] = {sg::kH1, sg::kH2, sg::kH3};
  for (int i = 0; i < 3; ++i) {
    step(dalloc(p, &p->ha[i], (size_t)rows * widths[i]));
    step(dalloc(p, &p->hc[i], (size_t)rows * widths[i]));
  }
  step(dalloc(p, &p->mu, (size_t)rows * p->Ap));
  step(dalloc(p, &p->xin, (size_t)E * p->Dp));
  step(dalloc(p, &p->pub2int, p->public_params));
  step(dalloc(p, &p->vout, (size_t)rows));
  for (sg_ppo::Lane& ln : p->lane) {
    for (float*& d : ln.dbuf) step(dalloc(p, &d, (size_t)rows * sg::kH1));
    step(cudaStreamCreateWithFlags(&ln.sw, cudaStreamNonBlocking));
    for (cudaEvent_t& ev : ln.ev_dy) step(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    step(cudaEventCreateWithFlags(&ln.ev_w, cudaEventDisableTiming));
  }
  step(dalloc(p, &p->dmu, (size_t)p->M * p->Ap));
  step(dalloc(p, &p->dv, (size_t)p->M));
  p->mlp_work_floats = (long long)2 * 152 * sg::kH1 * sg::kH2;   // row-split partial sums
  for (sg_ppo::Lane& ln : p->lane) step(dalloc(p, &ln.work, (size_t)p->mlp_work_floats));
  {
    // pre-split weights: every layer as a forward B, layers 2..4 as an input-gradient B
    size_t off = 0;
    Net* nets[2] = {&p->L.actor, &p->L.critic};
    int nj = 0;
    for (Net* net : nets)
      for (int i = 0; i < 4; ++i) {
        Layer& l = net->l[i];
        l.pre_fwd = off;
        off += (size_t)sg::presplit_floats(l.out, l.in);
        if (i > 0) {
          l.pre_dx = off;
          off += (size_t)sg::presplit_floats(l.in, l.out);
        }
      }
    step(dalloc(p, &p->pre, off));
    for (Net* net : nets)
      for (int i = 0; i < 4; ++i) {
        const Layer& l = net->l[i];
        p->pre_jobs.job[nj++] = sg::PresplitJob{p->params + l.w, l.in, 1, l.out, l.in,
                                                sg::presplit_npad(l.out), p->pre + l.pre_fwd};
        if (i > 0)
          p->pre_jobs.job[nj++] = sg::PresplitJob{p->params + l.w, 1, l.in, l.in, l.out,
                                                  sg::presplit_npad(l.in), p->pre + l.pre_dx};
      }
    p->pre_jobs.n = nj;
  }
  step(dalloc(p, &p->mb.obs, (size_t)p->M * p->Dp));
  step(dalloc(p, &p->mb.act, (size_t)p->M * A));
  step(dalloc(p, &p->mb.mask, (size_t)p->M * A));
  step(dalloc(p, &p->mb.logp, (size_t)p->M));
  step(dalloc(p, &p->mb.value, (size_t)p->M));
  step(dalloc(p, &p->mb.adv, (size_t)p->M));
  step(dalloc(p, &p->mb.ret, (size_t)p->M));
  const int head_blocks = (p->M + sg::kRedThreads - 1) / sg::kRedThreads;
  step(dalloc(p, &p->head_part, (size_t)head_blocks * (2 + 2 * A)));
  step(dalloc(p, &p->red_part, (size_t)2 * sg::kRedBlocks));
  const size_t part_rows = std::max<size_t>(sg::kBGradBlocks, ((size_t)rows + 127) / 128);
  p->bgrad_off[0] = 0;
  p->bgrad_off[1] = part_rows * sg::kH1;
  p->bgrad_off[2] = part_rows * (sg::kH1 + sg::kH2);
  p->bgrad_off[3] = part_rows * (sg::kH1 + sg::kH2 + sg::kH3);
  for (sg_ppo::Lane& ln : p->lane)
    step(dalloc(p, &ln.bgrad_part, p->bgrad_off[3] + part_rows * (size_t)p->Ap));
  step(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
  step(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
  step(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  step(dalloc(p, &p->norm, 2));
  step(dalloc(p, &p->clip_coef, 1));
  step(sg::prepare_mlp_kernels());
  if (e != cudaSuccess) {
    sg_status st = cuda_fail(p, e, "sg_ppo_create");
    sg_ppo_destroy(p);
    return st;
  }
  // host-built constants: joint mask, zero targets, public -> internal parameter map
  std::vector<float> jm((size_t)E * A, 0.f);
  std::vector<int32_t> map(p->public_params);
  {
    const Net* pn[2] = {&Lpub.actor, &Lpub.critic};
    const Net* in[2] = {&p->L.actor, &p->L.critic};
    for (int k = 0; k < 2; ++k)
      for (int i = 0; i < 4; ++i) {
        const Layer &a = pn[k]->l[i], &b = in[k]->l[i];
        for (int r = 0; r < a.out; ++r) {
          for (int q = 0; q < a.in; ++q) map[a.w + (size_t)r * a.in + q] = (int32_t)(b.w + (size_t)r * b.in + q);
          map[a.b + r] = (int32_t)(b.b + r);
        }
      }
    for (int j = 0; j < A; ++j) map[Lpub.log_std + j] = (int32_t)(p->L.log_std + j);
  }
  step(cudaMemcpyAsync(p->pub2int, map.data(), map.size() * 4, cudaMemcpyHostToDevice,
                       sg::context_stream(env)));
  const std::vector<int32_t>& dof = sg::context_env_dof(env);
  for (int k = 0; k < E; ++k)
    for (int j = 0; j < A && j < dof[k]; ++j) jm[(size_t)k * A + j] = 1.f;
  cudaStream_t s = sg::context_stream(env);
  step(cudaMemcpyAsync(p->jmask, jm.data(), jm.size() * 4, cudaMemcpyHostToDevice, s));
  step(cudaMemsetAsync(p->zero_targets, 0, (size_t)E * A * 4, s));
  step(cudaMemsetAsync(p->params, 0, P * 4, s));
  step(cudaMemsetAsync(p->grad, 0, P * 4, s));
  step(cudaMemsetAsync(p->adam_m, 0, P * 4, s));
  step(cudaMemsetAsync(p->adam_v, 0, P * 4, s));
  step(cudaMemsetAsync(p->d_step, 0, sizeof(long long), s));
  step(cudaStreamSynchronize(s));     // the host vectors above go out of scope
  if (e != cudaSuccess) {
    sg_status st = cuda_fail(p, e, "sg_ppo_create");
    sg_ppo_destroy(p);
    return st;
  }
  p->err = sg::context_err(env);
  bind_stream(p, s);
  *out = p;
  return SG_OK;
}

void sg_ppo_destroy(sg_ppo* p) {
  if (!p) return;
  // release on the env context's device, then restore the caller's current device
  const int owner = sg_device(p->env);
  int cur = -1;
  const bool other = cudaGetDevice(&cur) == cudaSuccess && owner >= 0 && cur != owner;
  if (other) cudaSetDevice(owner);
  // every stream of the handle finished before its memory is released
  if (p->stream) cudaStreamSynchronize(p->stream);
  if (p->side) cudaStreamSynchronize(p->side);
  for (sg_ppo::Lane& ln : p->lane)
    if (ln.sw) cudaStreamSynchronize(ln.sw);
  if (p->collect_exec) cudaGraphExecDestroy(p->collect_exec);
  for (void* a : p->allocs) cudaFree(a);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->side) cudaStreamDestroy(p->side);
  for (sg_ppo::Lane& ln : p->lane) {
    if (ln.sw) cudaStreamDestroy(ln.sw);
    for (cudaEvent_t ev : ln.ev_dy)
      if (ev) cudaEventDestroy(ev);
    if (ln.ev_w) cudaEventDestroy(ln.ev_w);
  }
  delete p;
  if (other) cudaSetDevice(cur);
}

int64_t sg_ppo_num_params(const sg_ppo* p) { return p ? (int64_t)p->public_params : 0; }

sg_status sg_ppo_set_params(sg_ppo* p, const float* src) {
  if (!p || !src) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_set_params");
  bind_stream(p, sg::context_stream(p->env));
  cudaError_t e = cudaMemsetAsync(p->params, 0, p->L.total * 4, p->stream);   // padding stays 0
  const int n = (int)p->public_params;
  if (e == cudaSuccess) {
    sg::scatter_kernel<<<sg::grid_for(n, 256), 256, 0, p->stream>>>(src, p->pub2int, n, p->params);
    e = cudaGetLastError();
  }
  return cuda_fail(p, e, "sg_ppo_set_params");
}

sg_status sg_ppo_get_params(sg_ppo* p, float* dst) {
  if (!p || !dst) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_get_params");
  bind_stream(p, sg::context_stream(p->env));
  const int n = (int)p->public_params;
  sg::gather_params_kernel<<<sg::grid_for(n, 256), 256, 0, p->stream>>>(p->params, p->pub2int, n,
                                                                         dst);
  return cuda_fail(p, cudaGetLastError(), "sg_ppo_get_params");
}

sg_status sg_ppo_reset(sg_ppo* p, int64_t step0) {
  if (!p) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_reset");
  bind_stream(p, sg::context_stream(p->env));
  sg_status st = sg_reset(p->env, nullptr);
  // the first observations go where a collect leaves its last ones
  if (st == SG_OK)
    st = sg_observe(p->env, p->zero_targets, nullptr, p->obs + (size_t)p->n * p->E * p->D);
  if (st != SG_OK) return st;
  cudaError_t e = cudaMemsetAsync(p->adam_m, 0, p->L.total * 4, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->adam_v, 0, p->L.total * 4, p->stream);
  const long long s0 = step0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->d_step, &s0, sizeof(long long), cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);   // s0 is a host local
  p->adam_t = 0;
  return cuda_fail(p, e, "sg_ppo_reset");
}

sg_status sg_ppo_collect(sg_ppo* p) {
  if (!p) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_collect");
  cudaStream_t s = sg::context_stream(p->env);
  if (!p->collect_exec) {
    // capture on a private stream, then replay on the env's stream
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(p, e, "sg_ppo_collect: stream");
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    sg_status st = SG_OK;
    if (e == cudaSuccess) {
      sg_set_stream(p->env, cap);
      bind_stream(p, cap);
      st = enqueue_collect(p);
      cudaGraph_t g = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cap, &g);
      if (e == cudaSuccess) e = ee;
      if (e == cudaSuccess && st == SG_OK) e = cudaGraphInstantiate(&p->collect_exec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    sg_set_stream(p->env, s);
    bind_stream(p, s);
    cudaStreamDestroy(cap);
    if (st != SG_OK) return st;
    if (e != cudaSuccess) return cuda_fail(p, e, "sg_ppo_collect: capture");
  }
  bind_stream(p, s);
  return cuda_fail(p, cudaGraphLaunch(p->collect_exec, s), "sg_ppo_collect");
}

sg_status sg_ppo_debug_set_fault(sg_ppo* p, int32_t mode, int64_t wait_limit_ns) {
  if (!p) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_debug_set_fault");
  if (mode != SG_FAULT_NONE && mode != SG_FAULT_SKIP_WEIGHT_COPY)
    return fail(p, SG_ERR_INVALID_ARG, "sg_ppo_debug_set_fault: unknown mode");
  if (wait_limit_ns < 0 || wait_limit_ns > 2000000000LL)
    return fail(p, SG_ERR_INVALID_ARG,
                "sg_ppo_debug_set_fault: wait_limit_ns must be 0 (default) .. 2e9");
  // the collect graph holds the products' arguments: capture it again
  if (p->collect_exec) {
    const cudaError_t e = cudaStreamSynchronize(sg::context_stream(p->env));
    if (e != cudaSuccess) return cuda_fail(p, e, "sg_ppo_debug_set_fault");
    cudaGraphExecDestroy(p->collect_exec);
    p->collect_exec = nullptr;
  }
  p->fault = mode;
  p->wait_ns = (unsigned long long)wait_limit_ns;
  return SG_OK;
}

sg_status sg_ppo_update(sg_ppo* p, const int32_t* perm, float* stats) {
  if (!p || !perm) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_update");
  bind_stream(p, sg::context_stream(p->env));
  const sg_ppo_config& c = p->cfg;
  const int M = p->M, A = p->A, D = p->D, E = p->E;
  const long long P = (long long)p->L.total;
  sg::Batch src{p->obs, p->actions, p->logp, p->values, p->adv, p->ret, p->jmask, p->norm};
  const int head_blocks = (M + sg::kRedThreads - 1) / sg::kRedThreads;
  for (int ep = 0; ep < c.epochs; ++ep) {
    for (int k = 0; k < c.minibatches; ++k) {
      const int32_t* idx = perm + (size_t)ep * p->B + (size_t)k * M;
      float* st = stats ? stats + 4 * ((size_t)ep * c.minibatches + k) : nullptr;
      sg::gather_kernel<<<(int)(((long long)M * 32 + 255) / 256), 256, 0, p->stream>>>(
          src, p->mb, idx, M, E, D, p->Dp, A);
      if (!presplit_weights(p)) return fail(p, SG_ERR_CUDA, "sg_ppo_update: weight split failed");
      if (!fork(p) || !net_forward(p, p->lane[0], p->L.actor, p->mb.obs, M, p->ha, p->mu) ||
          !net_forward(p, p->lane[1], p->L.critic, p->mb.obs, M, p->hc, p->vout) || !join(p))
        return fail(p, SG_ERR_CUDA, "sg_ppo_update: forward failed");
      sg::HeadArgs h{p->mu, p->vout, p->params + p->L.log_std, p->mb, p->dmu, p->dv,
                     p->head_part, M, A, p->Ap, c.clip, c.value_coef};
      sg::head_kernel<<<head_blocks, sg::kRedThreads, 0, p->stream>>>(h);
      sg::head_final_kernel<<<1, sg::kRedThreads, 0, p->stream>>>(p->head_part, head_blocks, A, M,
                                                     p->params + p->L.log_std, c.entropy_coef,
                                                     p->grad + p->L.log_std, st);
      if (!fork(p) || !net_backward(p, p->lane[0], p->L.actor, p->mb.obs, M, p->ha, p->dmu) ||
          !net_backward(p, p->lane[1], p->L.critic, p->mb.obs, M, p->hc, p->dv) || !join(p))
        return fail(p, SG_ERR_CUDA, "sg_ppo_update: backward failed");
      sg::sumsq_partial_kernel<<<sg::kRedBlocks, sg::kRedThreads, 0, p->stream>>>(p->grad, P,
                                                                                  p->red_part);
      sg::clip_final_kernel<<<1, sg::kRedThreads, 0, p->stream>>>(p->red_part, sg::kRedBlocks,
                                                                  c.max_grad_norm, p->clip_coef,
                                                                  st);
      ++p->adam_t;
      const float bc1 = (float)(1.0 - std::pow(0.9, (double)p->adam_t));
      const float bc2 = (float)(1.0 - std::pow(0.999, (double)p->adam_t));
      sg::adam_kernel<<<sg::grid_for(P, 256), 256, 0, p->stream>>>(
          p->params, p->grad, p->adam_m, p->adam_v, p->clip_coef, P, c.lr, bc1, bc2);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(p, e, "sg_ppo_update");
    }
  }
  return SG_OK;
}

namespace {
// (device pointer, bytes) of a rollout buffer
bool buffer_of(sg_ppo* p, int which, void** ptr, size_t* bytes) {
  const size_t nE = (size_t)p->n * p->E;
  switch (which) {
    case SG_PPO_OBS: *ptr = p->obs; *bytes = (nE + p->E) * p->D * 4; return true;
    case SG_PPO_ACTIONS: *ptr = p->actions; *bytes = nE * p->A * 4; return true;
    case SG_PPO_LOGP: *ptr = p->logp; *bytes = nE * 4; return true;
    case SG_PPO_VALUES: *ptr = p->values; *bytes = (nE + p->E) * 4; return true;
    case SG_PPO_REWARDS: *ptr = p->rewards; *bytes = nE * 4; return true;
    case SG_PPO_DONES: *ptr = p->dones; *bytes = nE; return true;
    case SG_PPO_ADVANTAGES: *ptr = p->adv; *bytes = nE * 4; return true;
    case SG_PPO_RETURNS: *ptr = p->ret; *bytes = nE * 4; return true;
    case SG_PPO_GRAD: *ptr = p->grad; *bytes = p->public_params * 4; return true;
    default: return false;
  }
}
}  // namespace

sg_status sg_ppo_get_buffer(sg_ppo* p, int32_t which, void* dst) {
  if (!p || !dst) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_get_buffer");
  void* ptr;
  size_t bytes;
  if (!buffer_of(p, which, &ptr, &bytes)) return fail(p, SG_ERR_INVALID_ARG, "unknown buffer");
  bind_stream(p, sg::context_stream(p->env));
  if (which == SG_PPO_GRAD) {
    const int n = (int)p->public_params;
    sg::gather_params_kernel<<<sg::grid_for(n, 256), 256, 0, p->stream>>>(
        p->grad, p->pub2int, n, static_cast<float*>(dst));
    return cuda_fail(p, cudaGetLastError(), "sg_ppo_get_buffer");
  }
  return cuda_fail(p, cudaMemcpyAsync(dst, ptr, bytes, cudaMemcpyDeviceToDevice, p->stream),
                   "sg_ppo_get_buffer");
}

sg_status sg_ppo_set_buffer(sg_ppo* p, int32_t which, const void* src) {
  if (!p || !src) return SG_ERR_INVALID_ARG;
  SG_PPO_CHECK_DEVICE(p, "sg_ppo_set_buffer");
  void* ptr;
  size_t bytes;
  if (!buffer_of(p, which, &ptr, &bytes) || which == SG_PPO_GRAD)
    return fail(p, SG_ERR_INVALID_ARG, "unknown or read-only buffer");
  bind_stream(p, sg::context_stream(p->env));
  cudaError_t e = cudaMemcpyAsync(ptr, src, bytes, cudaMemcpyDeviceToDevice, p->stream);
  if (e == cudaSuccess && which == SG_PPO_ADVANTAGES) {
    // the update normalises with the batch moments: recompute them
    sg::moments_partial_kernel<<<sg::kRedBlocks, sg::kRedThreads, 0, p->stream>>>(p->adv, p->B,
                                                                                  p->red_part);
    sg::moments_final_kernel<<<1, sg::kRedThreads, 0, p->stream>>>(p->red_part, sg::kRedBlocks,
                                                                   p->B, p->norm);
    e = cudaGetLastError();
  }
  return cuda_fail(p, e, "sg_ppo_set_buffer");
}

}  // extern "C"
