// Dense contraction of the PPO networks on tcgen05 tensor cores (sg_mlp.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace sg {

// C[m c_m + n] (+ split s at s c_split) = epilogue(sum_k A(m, k) B(n, k))
// with A(m, k) = A[m a_m + k a_k], B(n, k) = B[n b_n + k b_k].
struct MlpGemmArgs {
  const float* A;
  long long a_m, a_k;
  const float* B;
  long long b_n, b_k;
  float* C;
  long long c_m;
  const float* bias;    // [N] or null: added to every row
  int M, N, K;
  int elu;              // 1: ELU after the bias
  // input-gradient epilogue of an ELU layer: C = (A B^T) * ELU'(y) with
  // y[m c_m + n] the layer's activated output (ELU'(y) = 1 for y > 0, else
  // y + 1), and per CTA row tile the column sums of C (the bias gradient of
  // that layer) into colsum[blockIdx.x][N]; both null otherwise
  const float* act_y;
  float* colsum;
  int split_tf32;       // 1: three-product split precision (FP32-grade); 0: one TF32 product
  int k_per_split;      // K per CTA layer when c_split != 0 (a multiple of 32)
  long long c_split;    // 0: one output; else split s writes its partial sum at C + s c_split
  int n_tile;           // 0: chosen by the launcher
  int* err;             // device error word (bounded waits), or null
  // B already split into TF32 parts (launch_mlp_presplit), or null: b_pre
  // holds presplit_floats(N, K) floats for b_npad = presplit_npad(N) rows
  const float* b_pre;
  int b_npad;
  // 1: narrow products (K <= 32 with K N <= 2048, or N <= 16 with K <= 64)
  // run as FP32 FMA loops on the CUDA cores instead (mlp_narrow_kind)
  int narrow;
  // test hook: 1 = every CTA of a product with pre-split B leaves out the
  // copy of its first weight chunk, so the wait for it runs out
  int fault;
  unsigned long long wait_ns;   // bound of every wait, 0 = the default (2 s)
};

enum MlpNarrowKind { NARROW_NONE = 0, NARROW_K = 1, NARROW_N = 2 };
// which FP32 kernel serves a product when a.narrow is set (NARROW_NONE: the
// tensor-core contraction)
int mlp_narrow_kind(const MlpGemmArgs& a);

// One matrix to pre-split: B(n, k) = W[n wn + k wk], N x K, into dst
// (presplit_floats(N, K) floats, 16-byte aligned; npad = presplit_npad(N)).
struct PresplitJob {
  const float* W;
  long long wn, wk;
  int N, K, npad;
  float* dst;
};
constexpr int kMaxPresplitJobs = 16;
struct PresplitJobs {
  PresplitJob job[kMaxPresplitJobs];
  int n;
};

// output columns per CTA: up to 128; 64 for short contractions (K <= 32) or
// when wider tiles would leave fewer than two CTAs per SM
int mlp_tile_n(int M, int N, int K);
size_t mlp_smem_bytes(int n_tile, bool pre_b);
cudaError_t prepare_mlp_kernels();
// rows of a pre-split operand (N rounded up to the widest tile) and its size
int presplit_npad(int N);
long long presplit_floats(int N, int K);
// split every job's matrix into its TF32 parts (lo = 0 unless split_tf32),
// one launch for all jobs
cudaError_t launch_mlp_presplit(const PresplitJobs& jobs, int split_tf32, cudaStream_t s);
cudaError_t launch_mlp_gemm(const MlpGemmArgs& a, cudaStream_t s);
cudaError_t launch_mlp_split_reduce(const float* partial, int splits, long long split_len, float* C,
                                    long long n_total, cudaStream_t s);
// launch_mlp_gemm, splitting K over more CTAs (partial sums in `work`, then
// a fixed-order reduction) when the product has few output tiles, no bias
// and no activation, C is dense (c_m == N) and the partials fit in work.
cudaError_t launch_mlp_gemm_split(const MlpGemmArgs& a, float* work, long long work_floats,
                                  cudaStream_t s);

}  // namespace sg
