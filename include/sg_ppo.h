/*
 * sg_ppo.h -- GPU-resident PPO loop on top of an sg_ctx batch of envs.
 *
 * The paper trains its policies with a GPU implementation of PPO (Methods,
 * "Policy learning and control": batch B = n_robots x n_steps split into
 * large minibatches, generalized advantage estimation, time-outs handled by
 * adding the critic's value prediction to the reward) and times the loop
 * "with learning" with a policy of hidden layers 256, 128, 64 and ELU
 * activations (Results, Table II).  This API keeps the whole loop on the
 * device: policy and value networks, action sampling, env steps, resets,
 * advantages and the update.
 *
 * Networks: actor and critic are separate MLPs D -> 256 -> 128 -> 64 -> out
 * (ELU after each hidden layer; D = sg_obs_dim, actor out = A = J =
 * sg_max_joints, critic out = 1).  The policy is a diagonal Gaussian with a
 * state-independent log standard deviation per action; the action of a joint
 * is its drive command (sg_step's actions); joints an env does not have are
 * sampled but left out of log-probabilities and entropy.
 *
 * Flat parameter vector (float32), in order:
 *   actor  W1 [256][D], b1 [256], W2 [128][256], b2 [128], W3 [64][128],
 *          b3 [64], W4 [A][64], b4 [A], log_std [A],
 *   critic W1 [256][D], b1 [256], W2 [128][256], b2 [128], W3 [64][128],
 *          b3 [64], W4 [1][64], b4 [1]
 * (W row-major [out][in]: y = W x + b).
 *
 * One iteration = sg_ppo_collect + sg_ppo_update:
 *   collect, for t = 0 .. n_steps-1, from the current observations o_t:
 *     mu = actor(o_t), V_t = critic(o_t), a_t = mu + exp(log_std) * eps_t,
 *     eps_t[e][j] standard normal from the counter-based generator keyed by
 *     (seed, e, j / 4, global step) (component j % 4; SplitMix64 finaliser
 *     and Box-Muller, as the tracking task's goal noise);
 *     (o', r_t, done_t) = sg_step(a_t); r_t += gamma V_t on a time-out step;
 *     envs with any done bit are reset (sg_reset) and their next
 *     observation is that of the reset state (sg_observe with a_t as the
 *     current targets); o_{t+1} = o';
 *   then V_n = critic(o_n) and GAE: delta_t = r_t + gamma V_{t+1} k_t - V_t,
 *   A_t = delta_t + gamma lambda k_t A_{t+1} (k_t = 0 after a done step),
 *   R_t = A_t + V_t.
 *   update: advantages normalised over the batch (mean 0, unbiased std 1,
 *   + 1e-8); for each epoch e and minibatch k the rows perm[e][k*M .. k*M+M-1]
 *   (M = B / minibatches, row index t * E + env) give the loss
 *     L = mean max(-A r, -A clamp(r, 1-clip, 1+clip))
 *       + value_coef mean max((V - R)^2, (V_old + clamp(V - V_old, +-clip) - R)^2)
 *       - entropy_coef mean H,      r = exp(logp - logp_old);
 *   its gradient is clipped to global norm max_grad_norm and Adam (beta
 *   0.9 / 0.999, eps 1e-8, bias-corrected) takes one step of size lr.
 *
 * Threading and streams: all work is ordered on the env context's stream;
 * the critic's products run on a private second stream of the handle,
 * forked from and joined back to the context's stream by events around each
 * network pass (the two networks are independent there), and within each
 * network's backward pass the weight gradients run on a private stream of
 * their own, each after its output gradient is ready; everything is joined
 * back, so every call's work is complete when the context's stream reaches
 * its end.  The collect
 * loop is captured once into a CUDA graph (the two networks as parallel
 * branches) and replayed.  Every step is a kernel of this library; the dense
 * layers run on its tensor-core contraction (sg_mlp_gemm below: FP32-grade
 * split precision, or one TF32 product per term with tf32 = 1; the output
 * layers and the input gradients below them as FP32 FMA loops), forward
 * products with the bias and ELU in their epilogue, input gradients with the
 * ELU derivative and the bias gradient's partial sums in theirs.
 */
#ifndef SG_PPO_H
#define SG_PPO_H

#include <stdint.h>

#include "sg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_ppo sg_ppo;

typedef struct sg_ppo_config {
  int32_t n_steps;          /* steps per env per iteration, >= 1 */
  int32_t epochs;           /* passes over the batch per update, >= 1 */
  int32_t minibatches;      /* minibatches per epoch; must divide E * n_steps */
  float gamma, lam;         /* discount, GAE lambda, in [0, 1] */
  float clip;               /* ratio and value clip, > 0 */
  float value_coef, entropy_coef;
  float lr;                 /* Adam step size, > 0 */
  float max_grad_norm;      /* global gradient-norm clip, > 0 */
  float dt;                 /* control step of the env, > 0 */
  int32_t substeps;         /* env substeps per step, 1..64 */
  uint32_t seed;            /* exploration-noise stream */
  int32_t tf32;             /* 1: one TF32 product per term (10-bit mantissas),
                               0: split precision, FP32-grade (default) */
} sg_ppo_config;

/* Create a PPO loop over the envs of `env` (which it uses, not owns; the env
 * must outlive it).  Allocates parameters, Adam moments, rollout buffers
 * ((n_steps + 1) x E x D observations and the per-step arrays), minibatch
 * activations and the partial sums of the weight gradients on the current
 * device, which must be the
 * env context's device (as for every sg_ppo_* call that enqueues work:
 * otherwise SG_ERR_INVALID_ARG and nothing is enqueued).  Parameters start
 * at zero: set them with sg_ppo_set_params.  Invalid configurations return
 * SG_ERR_INVALID_ARG (message in sg_last_error(env)). */
sg_status sg_ppo_create(sg_ctx *env, const sg_ppo_config *cfg, sg_ppo **out);
void sg_ppo_destroy(sg_ppo *ppo);

/* Length of the flat parameter vector (layout above). */
int64_t sg_ppo_num_params(const sg_ppo *ppo);

/* Copy parameters in / out (device float arrays of sg_ppo_num_params). */
sg_status sg_ppo_set_params(sg_ppo *ppo, const float *params_dev);
sg_status sg_ppo_get_params(sg_ppo *ppo, float *params_dev);

/* Reset every env (sg_reset), take the first observations (sg_observe with
 * zero targets; the next collect starts from them), zero the Adam moments
 * and step counts and set the global step of the exploration noise to
 * step0. */
sg_status sg_ppo_reset(sg_ppo *ppo, int64_t step0);

/* n_steps of acting and stepping from the last observations of the previous
 * collect (or of sg_ppo_reset), then values and advantages (see above).
 * The first call captures the loop into a CUDA graph (not capturable
 * itself); later calls replay it.  Advances the global step by n_steps. */
sg_status sg_ppo_collect(sg_ppo *ppo);

/* The PPO update over the last collected batch.  perm_dev [epochs][B]
 * (int32, device, B = E * n_steps) holds, per epoch, a permutation of
 * 0 .. B-1; stats_dev (device, may be NULL) receives per minibatch
 * [epochs * minibatches][4] = (surrogate loss, value loss, mean entropy,
 * gradient norm before clipping). */
sg_status sg_ppo_update(sg_ppo *ppo, const int32_t *perm_dev, float *stats_dev);

/* Copy a rollout buffer of the last collect into dst_dev (device):
 *   SG_PPO_OBS        float [n_steps + 1][E][D]
 *   SG_PPO_ACTIONS    float [n_steps][E][A]
 *   SG_PPO_LOGP       float [n_steps][E]
 *   SG_PPO_VALUES     float [n_steps + 1][E]
 *   SG_PPO_REWARDS    float [n_steps][E]   (bootstrapped)
 *   SG_PPO_DONES      uint8 [n_steps][E]
 *   SG_PPO_ADVANTAGES float [n_steps][E]   (before normalisation)
 *   SG_PPO_RETURNS    float [n_steps][E]
 *   SG_PPO_GRAD       float [sg_ppo_num_params]: the loss gradient of the
 *                     last minibatch, before clipping (parameter layout) */
enum {
  SG_PPO_OBS = 0, SG_PPO_ACTIONS = 1, SG_PPO_LOGP = 2, SG_PPO_VALUES = 3, SG_PPO_REWARDS = 4,
  SG_PPO_DONES = 5, SG_PPO_ADVANTAGES = 6, SG_PPO_RETURNS = 7, SG_PPO_GRAD = 8
};
sg_status sg_ppo_get_buffer(sg_ppo *ppo, int32_t which, void *dst_dev);

/* Overwrite the rollout buffers with the caller's (same layouts; the
 * observations, actions, logp, values, advantages and returns are what the
 * update reads), e.g. to run the update on a batch collected elsewhere. */
sg_status sg_ppo_set_buffer(sg_ppo *ppo, int32_t which, const void *src_dev);

/*
 * Test hook (not part of the method): makes a bounded wait of the
 * tensor-core contraction run out, so that its give-up path can be
 * exercised without a GPU fault or hang.  mode:
 *   SG_FAULT_NONE              normal operation (the default);
 *   SG_FAULT_SKIP_WEIGHT_COPY  every CTA of a product with pre-split weights
 *                              (the hidden layers' forward and input-gradient
 *                              products) leaves out the bulk copy of its first
 *                              weight chunk, so the issuing thread's wait for
 *                              it runs out.
 * wait_limit_ns bounds every wait of the contraction in wall-clock time (0 =
 * the default, 2 s; at most 2e9).  A wait that runs out sets the env
 * context's timeout flag (sg_sync_status(env) returns SG_ERR_TIMEOUT); the
 * CTA then waits, bounded, for its copies and tensor-core operations in
 * flight, releases its tensor memory and leaves without writing its output
 * tile, so the outputs of those products -- and whatever the collect or
 * update computes from them -- are unspecified until the next collect and
 * update with the hook off.  The collect graph is captured again.
 * SG_ERR_INVALID_ARG for an unknown mode or a limit out of range.
 */
enum { SG_FAULT_SKIP_WEIGHT_COPY = 3 };
sg_status sg_ppo_debug_set_fault(sg_ppo *ppo, int32_t mode, int64_t wait_limit_ns);

/*
 * The dense contraction of the policy and value networks (Methods, "Policy
 * learning and control": MLPs of 256, 128 and 64 ELU units), exposed as a
 * building block: on `stream` (cudaStream_t, NULL = legacy default stream),
 *   C[m * c_m + n] = act( sum_k A[m * a_m + k * a_k] * B[n * b_n + k * b_k] + bias[n] )
 * for 0 <= m < M, 0 <= n < N, 0 <= k < K; all pointers are device float
 * arrays, strides in elements (row- or column-major operands, transposes);
 * bias [N] may be NULL; act is ELU when elu != 0, else the identity.  It
 * runs on the tcgen05 tensor cores in kind::tf32 with FP32 accumulation;
 * with split_tf32 = 1 every operand is split into two TF32 parts
 * (x = hi + lo) and three products are accumulated (hi*hi + hi*lo + lo*hi:
 * FP32-grade, about 2^-22 relative per product), with 0 one TF32 product
 * (10-bit mantissas).  split_tf32 = 2 is FP32-grade as 1, except that
 * narrow products with k-contiguous A (a_k = 1) run as FP32 FMA loops on
 * the CUDA cores (exact FP32 products, fixed summation order): K <= 32 with
 * K * N <= 2048, or N <= 16 with K <= 64 a multiple of 4 and A 16-byte
 * aligned with a_m a multiple of 4.  `work` (device scratch of work_floats floats, may be
 * NULL) serves two purposes.  A product with few output tiles (fewer than
 * two 128 x 128 tiles per SM of 152), more than 32 terms, no bias or
 * activation and a dense C (c_m == N) splits K over more CTAs, their partial
 * sums in work, added in a fixed order afterwards (results do not depend on
 * scheduling).  Any other product splits B into its TF32 parts once, into
 * work, when work holds ceil(K / 16) * 2 * 16 * (N rounded up to 128)
 * floats and is 16-byte aligned, and every CTA then copies its part of them
 * instead of splitting B itself (the PPO networks' forward and
 * input-gradient products take this path with their weights).
 * Asynchronous; C must not overlap A, B or work.  SG_ERR_INVALID_ARG for NULL operands or negative
 * sizes; SG_ERR_CUDA if a launch fails.  A bounded device wait that runs out
 * leaves C unspecified.
 */
sg_status sg_mlp_gemm(void *stream, const float *A, int64_t a_m, int64_t a_k, const float *B,
                      int64_t b_n, int64_t b_k, const float *bias, int32_t elu, int32_t M,
                      int32_t N, int32_t K, float *C, int64_t c_m, float *work,
                      int64_t work_floats, int32_t split_tf32);

#ifdef __cplusplus
}
#endif

#endif /* SG_PPO_H */
