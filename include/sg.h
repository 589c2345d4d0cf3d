/*
 * sg.h -- C ABI of the batched articulated-arm simulation step (libsg.so).
 *
 * The library steps thousands of independent robot environments on one
 * GPU: each environment is one to four serial chains of revolute/prismatic
 * joints on a fixed base under PD joint drives (Surgical Gym, Methods,
 * "Simulation Setup": actors of rigid bodies joined by revolute/prismatic
 * joints, PD position targets as actions; Results, "Multi-Tool Target
 * Reaching": two or three arms per environment).  One step integrates the
 * reduced-coordinate rigid-body dynamics with `substeps` implicit-drive
 * semi-implicit Euler substeps (Methods, "Simulation Setup": the engine
 * sub-steps every control step) and writes the per-environment
 * observation, reward and done tensors (Methods, "Observation Space";
 * Results, "Environments"; Methods, "Policy learning and control": time-outs
 * reported apart from terminations).
 *
 * Conventions (all entry points):
 *  - Pointers named *_dev are DEVICE pointers (e.g. torch tensor data_ptr()),
 *    contiguous, row-major, caller-owned; pointers named *_host are host
 *    pointers.  The library never frees caller memory.
 *  - All device work is enqueued asynchronously on the context's stream
 *    (sg_create / sg_set_stream); results are valid once that stream has
 *    reached the call.  Host-side argument errors are reported
 *    synchronously by the return code; nothing is enqueued then.
 *  - Environment index i in every array is the caller's env i, whatever
 *    internal packing the library uses.
 *  - Device-side faults are never raised as traps: a non-finite state sets
 *    done bit SG_DONE_NONFINITE for that env and a context error flag that
 *    sg_sync_status() reports.
 *  - No C++ exception crosses this ABI.  sg_last_error() describes the last
 *    failing call of a context.
 *  - A context belongs to the CUDA device that was current at sg_create
 *    (sg_device()).  Every call that enqueues work or reads device state
 *    first checks that this device is current; if another device is current
 *    it returns SG_ERR_INVALID_ARG (SG_ERR_CUDA if the current device cannot
 *    be queried) and enqueues nothing.  sg_destroy releases the context on
 *    its own device whatever device is current.
 */
#ifndef SG_H
#define SG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_ctx sg_ctx;   /* opaque; owned by the library */

typedef enum sg_status {
  SG_OK = 0,
  SG_ERR_INVALID_ARG = 1,   /* bad pointer, size, range or layout */
  SG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  SG_ERR_OOM = 3,           /* device or host allocation failed */
  SG_ERR_NONFINITE = 4,     /* a kernel saw a non-finite state (sg_sync_status) */
  SG_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up (sg_sync_status) */
  SG_ERR_UNSUPPORTED = 6    /* valid request outside what this library implements */
} sg_status;

enum {
  SG_TASK_REACH = 0,        /* Target Reaching / Multi-Tool Target Reaching */
  SG_TASK_PATH = 1,         /* Path Following (single-chain envs only) */
  SG_TASK_TRACK = 2         /* Active Tracking: reaching with moving goals */
};

enum {
  SG_JOINT_REVOLUTE = 0,
  SG_JOINT_PRISMATIC = 1    /* translation along the joint frame's local z */
};

enum {
  SG_DRIVE_POSITION = 0,    /* command = PD position target q* */
  SG_DRIVE_VELOCITY = 1,    /* command = velocity target qd* */
  SG_DRIVE_TORQUE = 2       /* command = joint torque / force */
};

enum {
  SG_DONE_TERMINATED = 1,   /* reserved: termination (never set by the tasks here) */
  SG_DONE_TIMEOUT = 2,      /* step count since reset reached episode_len */
  SG_DONE_NONFINITE = 4     /* q or qd became non-finite in this step */
};

enum {
  SG_MAX_CHAINS = 4,        /* chains (arms) per environment */
  SG_MAX_CHAIN_JOINTS = 7   /* joints per chain */
};

/*
 * Robot and task description.  All pointers are HOST pointers read during
 * sg_create / sg_plan only (the caller keeps ownership).  E = num_envs,
 * J = max_joints (row stride of every per-joint array, >= the total DOF of
 * every env).  Joint j of an env indexes chain 0's joints first, then
 * chain 1's.  Per-joint arrays beyond an env's DOF are ignored.
 *
 * Geometry: joint i of a chain sits at (0, 0, link_len[i-1]) in the frame
 * of link i-1 (at base_offset for i = 0, base axes aligned with the world);
 * a revolute joint rotates about its local axis joint_axis (0=x, 1=y,
 * 2=z); a prismatic joint translates along local z (joint_axis must be 2).
 * Link i extends along its local +z; its centre of mass is at
 * (0, 0, link_com[i]) with diagonal rotational inertia link_inertia[i]
 * about the centre of mass.  The tool tip of a chain is (0, 0, link_len)
 * of its last link.  Gravity is 9.81 m/s^2 along -z.
 *
 * Drive of joint i with command a (Methods, "Simulation Setup": PD position
 * or velocity targets, or torques), by joint_drive:
 *   SG_DRIVE_POSITION: tau = kp (a - q) - (kd + damping) qd + tau_lim
 *   SG_DRIVE_VELOCITY: tau = kd (a - qd) - damping qd + tau_lim
 *   SG_DRIVE_TORQUE:   tau = a - damping qd + tau_lim
 * where tau_lim = -k_limit (q - q_hi) above q_hi, -k_limit (q - q_lo) below
 * q_lo, 0 inside.  Stiffness and damping act implicitly (at the end of each
 * substep).  joint_drive may be NULL: all position targets.
 */
typedef struct sg_desc {
  int32_t num_envs;                 /* E >= 1 */
  int32_t max_joints;               /* J, 1..28 */
  const int32_t *env_num_chains;    /* [E]     1..4 */
  const int32_t *chain_num_joints;  /* [E][4]  1..7 (entries beyond env_num_chains unused) */
  const int32_t *joint_type;        /* [E][J]  SG_JOINT_* */
  const int32_t *joint_axis;        /* [E][J]  0=x 1=y 2=z */
  const float *link_len;            /* [E][J]  m */
  const float *link_mass;           /* [E][J]  kg, > 0 */
  const float *link_inertia;        /* [E][J][3] Ixx, Iyy, Izz about the COM, > 0 */
  const float *link_com;            /* [E][J]  COM offset along local z, m */
  const float *q_lo, *q_hi;         /* [E][J]  joint limits (rad or m) */
  const float *kp, *kd, *damping;   /* [E][J]  drive stiffness, drive damping, joint damping */
  const float *k_limit;             /* [E][J]  limit-spring stiffness (0 = no spring) */
  const float *base_offset;         /* [E][4][3] chain base positions (world) */
  const float *q0;                  /* [E][J]  state after reset (qd = 0) */
  int32_t episode_len;              /* steps until the time-out bit, >= 1 */
  int32_t task;                     /* SG_TASK_* */
  const float *goal;                /* [E][4][3] per-chain goal (SG_TASK_REACH) */
  const float *path;                /* [E][path_len][3] waypoints (SG_TASK_PATH), or NULL
                                       when path_ctrl is given, else NULL */
  int32_t path_len;                 /* W >= 4 for SG_TASK_PATH */
  float alpha;                      /* path reward scale */
  const int32_t *joint_drive;       /* [E][J] SG_DRIVE_*, or NULL (all position) */
  /* SG_TASK_TRACK (Results, "Active Tracking"): every step each chain's goal
   * offset d (from its initial goal) and goal velocity v move as
   *   d <- clamp(d + v, -track_limit, +track_limit) (per component),
   *   v <- v + track_sigma * N(0, 1)^3,
   * with the normal deviates drawn from a counter-based generator keyed by
   * (seed, env, chain, step count after the step); reset sets d = v = 0. */
  uint32_t seed;
  float track_sigma;                /* > 0 for SG_TASK_TRACK */
  float track_limit;                /* > 0 for SG_TASK_TRACK */
  /* SG_TASK_PATH with path == NULL: the library builds each env's waypoint
   * table on the device from these control points (see sg_set_paths). */
  const float *path_ctrl;           /* [E][path_ctrl_len][3], else NULL */
  int32_t path_ctrl_len;            /* K, 2..64 */
} sg_desc;

/*
 * Observation layout of env e (n = its total DOF, nc = its chains), padded
 * with zeros to D = sg_obs_dim():
 *   SG_TASK_REACH, SG_TASK_TRACK:
 *                  [q(n), qd(n), tip_c(3) per chain, q*(n), goal_c(3) per chain]
 *   SG_TASK_PATH:  [q(n), qd(n), tip(3), quat(4) = (x, y, z, w) with w >= 0,
 *                   waypoint[t+1](3), waypoint[t+2](3), waypoint[t+3](3)]
 * where t = steps since reset after this step and waypoint indices clamp at
 * path_len - 1.  Reward: REACH, TRACK  -sum_c ||tip_c - goal_c|| (the
 *                                       current, moved goal for TRACK);
 *                        PATH   -alpha ||tip - waypoint[t]||.
 */

typedef struct sg_plan_info {
  int32_t obs_dim;        /* D */
  int32_t num_slots;      /* internal chain slots (multiple of 32) */
  int32_t num_chains;     /* real chains (sum of env_num_chains) */
  int32_t class_slots[4]; /* slots per internal chain class: 7R, 7P, generic, 4R */
} sg_plan_info;

/* Validate a description and compute its packing plan on the host, with no
 * CUDA call.  Returns SG_ERR_INVALID_ARG / SG_ERR_UNSUPPORTED with a message
 * in err (NUL-terminated, truncated to err_len) when the description is
 * rejected.  info may be NULL. */
sg_status sg_plan(const sg_desc *desc, sg_plan_info *info, char *err, int32_t err_len);

/* Create a context: validate and pack the description, allocate the device
 * state and parameter slabs (cudaMalloc) and upload them on `stream`
 * (cudaStream_t, NULL = legacy default stream).  All envs start reset
 * (q = q0, qd = 0, step count 0).  On failure *out is NULL. */
sg_status sg_create(const sg_desc *desc, void *stream, sg_ctx **out);

/* Free a context and its device memory (synchronises its stream).  NULL is a no-op. */
void sg_destroy(sg_ctx *ctx);

/* The CUDA device the context belongs to (current at sg_create); -1 for NULL. */
int32_t sg_device(const sg_ctx *ctx);

/* Change the stream later calls enqueue on (a stream of the context's device). */
sg_status sg_set_stream(sg_ctx *ctx, void *stream);

int32_t sg_obs_dim(const sg_ctx *ctx);
int32_t sg_num_envs(const sg_ctx *ctx);
int32_t sg_max_joints(const sg_ctx *ctx);

/* Reset envs with env_mask_dev[e] != 0 (uint8 [E], device); NULL resets all.
 * Reset envs get q = q0, qd = 0, step count 0; others are untouched. */
sg_status sg_reset(sg_ctx *ctx, const uint8_t *env_mask_dev);

/* One control step of every env.
 *   actions_dev [E][J] float: joint commands (position / velocity targets or
 *               torques, per joint_drive; padding ignored)
 *   dt > 0 seconds, substeps 1..64 (substep length dt / substeps)
 *   obs_dev [E][D] float, reward_dev [E] float, done_dev [E] uint8 (outputs)
 * Does not reset envs: the caller passes done-derived masks to sg_reset. */
sg_status sg_step(sg_ctx *ctx, const float *actions_dev, float dt, int32_t substeps,
                  float *obs_dev, float *reward_dev, uint8_t *done_dev);

/* The observation of the current state, laid out as sg_step reports it,
 * without advancing time: q, qd, tool tips (and orientation) of the current
 * state, targets_dev [E][J] as the current commands q*, the current goals
 * (tracking: including their present offsets) or the waypoints after the
 * current step count (path).  Rows of envs with env_mask_dev[e] != 0 (uint8
 * [E], device; NULL = all) are written to obs_dev [E][D]; other rows are not
 * touched.  State, step counts, goals and the error flags are unchanged.  Use
 * it after sg_reset to obtain the first observation of new episodes. */
sg_status sg_observe(sg_ctx *ctx, const float *targets_dev, const uint8_t *env_mask_dev,
                     float *obs_dev);

/* Read / write the state in caller layout: q, qd [E][J] float (padding
 * joints are written as 0 by sg_get_state and ignored by sg_set_state),
 * step_count [E] int32.  Any of the three pointers may be NULL to skip it. */
sg_status sg_get_state(sg_ctx *ctx, float *q_dev, float *qd_dev, int32_t *step_count_dev);
sg_status sg_set_state(sg_ctx *ctx, const float *q_dev, const float *qd_dev,
                       const int32_t *step_count_dev);

/*
 * Rollout of T control steps (the batched form of sg_step):
 *   actions_dev [T][E][J], obs_dev [T][E][D], reward_dev [T][E], done_dev [T][E].
 * Results are identical, bit for bit, to T successive sg_step calls.  The
 * work is issued according to the context's launch plan:
 *   SG_ROLLOUT_PERSISTENT  one kernel runs all T steps with the chain state
 *                          held in registers (parameters staged once);
 *   SG_ROLLOUT_STEP_GRAPH  T single-step kernels.
 * Either way the launch sequence is captured once into a CUDA graph (on a
 * private capture stream) and replayed on the context's stream while T, dt,
 * substeps, the launch plan and all pointers stay the same; any change
 * re-captures.  T is 1..4096.
 */
enum { SG_ROLLOUT_PERSISTENT = 0, SG_ROLLOUT_STEP_GRAPH = 1 };

sg_status sg_rollout(sg_ctx *ctx, const float *actions_dev, int32_t T, float dt,
                     int32_t substeps, float *obs_dev, float *reward_dev, uint8_t *done_dev);

/* sg_rollout with HOST buffers (same shapes), enqueued on the context's
 * stream; the outputs are valid after sg_sync_status() or a stream
 * synchronisation.  The actions are copied to device staging buffers
 * (cudaMalloc on first use or growth) and the outputs back; how, by
 * sg_set_host_io:
 *   SG_HOST_IO_AUTO (default): pipelined -- the T steps run as up to 8
 *     chunks; copy-in of the next chunk, the rollout kernel of this one and
 *     copy-out of the previous one proceed together on two internal copy
 *     streams (page-locked host memory makes the copies asynchronous);
 *   SG_HOST_IO_STAGED: copy in, rollout, copy out, one after another;
 *   SG_HOST_IO_DIRECT: when all four buffers are page-locked host memory the
 *     device can address (cudaHostAlloc / cudaHostRegister), the rollout
 *     kernel reads the actions from and writes the outputs to host memory
 *     itself (NVLink-C2C on Grace-Blackwell); otherwise as STAGED.
 * All three compute the same bits as sg_rollout. */
sg_status sg_rollout_host(sg_ctx *ctx, const float *actions_host, int32_t T, float dt,
                          int32_t substeps, float *obs_host, float *reward_host,
                          uint8_t *done_host);

enum { SG_HOST_IO_AUTO = 0, SG_HOST_IO_STAGED = 1, SG_HOST_IO_DIRECT = 2 };
sg_status sg_set_host_io(sg_ctx *ctx, int32_t mode);

/* Launch plan: threads per block (32, 64, 128 or 256), the rollout mode
 * and the chain split: 1 = one thread integrates one chain (a warp holds 32
 * chains); 2 = two threads in two cooperating warps share each chain (one
 * computes the bias forces and drive terms, the other the mass matrix and
 * the solve), which doubles the parallelism of batches too small to fill
 * the GPU; threads_per_block must then be 64, 128 or 256.  Results do not
 * depend on the threads per block or the rollout mode (bit-identical); the
 * two chain splits round differently (they agree to FP32 rounding, not
 * bit for bit). */
sg_status sg_set_launch(sg_ctx *ctx, int32_t threads_per_block, int32_t rollout_mode,
                        int32_t chain_split);
sg_status sg_get_launch(const sg_ctx *ctx, int32_t *threads_per_block, int32_t *rollout_mode,
                        int32_t *chain_split);

/* Packing: the order of the warps of chain slots (each warp holds 32 chains
 * of one class; a block of the step kernel holds consecutive warps).
 *   SG_PACK_CLASS       warps grouped by chain class, longest chains first
 *                       (7R, 7P, generic, 4R), the order sg_create builds;
 *   SG_PACK_INTERLEAVE  the classes interleaved in proportion: warp i of a
 *                       class of n warps goes to the fractional position
 *                       (2 i + 1) / (2 n) of the sequence (ties in class
 *                       order), so every block holds a mix of long and short
 *                       chains.
 * Results do not depend on the packing (bit-identical).  sg_set_packing
 * reorders the context's parameters, slot tables and state in place
 * (a temporary device buffer; synchronises the stream) and discards a
 * pending sg_diff_forward (the next sg_diff_backward then fails with
 * SG_ERR_INVALID_ARG until sg_diff_forward runs again).  SG_ERR_INVALID_ARG
 * for an unknown packing. */
enum { SG_PACK_CLASS = 0, SG_PACK_INTERLEAVE = 1 };
sg_status sg_set_packing(sg_ctx *ctx, int32_t packing);
int32_t sg_get_packing(const sg_ctx *ctx);

/* Host only, no CUDA call: the warp order of `packing` for a description,
 * order[w] = the warp of the class-grouped order that position w holds, for
 * w < num_warps = sg_plan_info.num_slots / 32 (num_warps must equal it).
 * Errors as sg_plan (message in err), SG_ERR_INVALID_ARG for an unknown
 * packing or a wrong num_warps. */
sg_status sg_plan_packing(const sg_desc *desc, int32_t packing, int32_t *order,
                          int32_t num_warps, char *err, int32_t err_len);

/* Autotuner: times every launch plan (packing x threads per block x chain
 * split x rollout mode) on
 * a rollout with the given arguments (CUDA events, median of `repeats`
 * timed runs after one warm-up run each), keeps the fastest and writes its
 * time per rollout to *best_ms (may be NULL).  The interleaved packing is
 * tried only where it differs from the class-grouped one; the fastest
 * packing is left in place (sg_get_packing), which discards a pending
 * sg_diff_forward as sg_set_packing does.  The environment state and step
 * counts are restored afterwards; the output buffers hold the last trial's
 * results.  Synchronises the stream; allocates a state snapshot. */
sg_status sg_autotune(sg_ctx *ctx, const float *actions_dev, int32_t T, float dt,
                      int32_t substeps, float *obs_dev, float *reward_dev, uint8_t *done_dev,
                      int32_t repeats, float *best_ms);

/*
 * Differentiation of tool-tip trajectories (a hand-written adjoint of the
 * step; no counterpart in the paper, whose engine is not differentiable).
 *
 * sg_diff_forward: T control steps from the current state with
 * actions_dev [T][E][J], writing the tool-tip position of every chain after
 * every step to ee_dev [T][E][4][3] (entries of chains an env does not have
 * are 0).  The state (q, qd) is checkpointed every ckpt_every steps
 * (1..32) in context scratch memory (cudaMalloc on first use or growth),
 * together with the backward pass's replay buffers (3 * ckpt_every *
 * substeps * 210 * num_slots floats while that stays within 1 GiB; beyond it
 * the backward pass runs without them, more slowly; with them, the forward
 * also leaves the last segment's substep records there);
 * the context's own state and step counts are NOT changed.  substeps 1..16.
 *
 * sg_diff_backward: the reverse pass of the last sg_diff_forward on this
 * context.  Given dl_dee_dev [T][E][4][3] = dL/d(ee) it writes
 * dactions_dev [T][E][J] = dL/d(actions) and dmass_dev [E][J] = dL/d(link
 * mass) (link inertias scale with the mass, centre of mass fixed); dq0_dev
 * and dqd0_dev [E][J] (either may be NULL) receive dL/d(initial q, qd).
 * actions_dev must hold the same values as in the forward call (it may be
 * called more than once after one forward).  Each segment between
 * checkpoints is recomputed from its checkpoint (when the replay buffers
 * exist: by two further warps, ahead of the reverse sweep; the first call
 * after a forward takes the last segment from the forward's records).  Joint
 * limit springs switch on and off at the limits; the gradient is that of
 * the active branch.
 */
sg_status sg_diff_forward(sg_ctx *ctx, const float *actions_dev, int32_t T, float dt,
                          int32_t substeps, int32_t ckpt_every, float *ee_dev);
sg_status sg_diff_backward(sg_ctx *ctx, const float *actions_dev, const float *dl_dee_dev,
                           float *dactions_dev, float *dmass_dev, float *dq0_dev,
                           float *dqd0_dev);

/* Replace the link masses with mass_dev [E][J] (device, > 0); each link's
 * rotational inertia is rescaled by new mass / description mass (the link's
 * box dimensions and centre of mass stay fixed). */
sg_status sg_set_link_mass(sg_ctx *ctx, const float *mass_dev);

/*
 * sg_diff_track_noalloc -- the paper has no counterpart (its engine is not
 * differentiable); this is a no-allocation form of the differentiable
 * rollout above, fused with the tracking loss
 *     L_e = sum_t sum_c ||ee[t][e][c] - target[t][e][c]||^2 .
 * It runs sg_diff_forward's forward kernel, the loss cotangent and
 * sg_diff_backward's adjoint kernel in one call and writes ee_dev
 * [T][E][4][3], loss_dev [E], dactions_dev [T][E][J] = dL/d(actions) and
 * dmass_dev [E][J] = dL/d(link mass); target_dev is [T][E][4][3] (targets of
 * chains an env does not have are ignored).
 *
 * Who needs it: callers that cannot allocate device memory when they need
 * gradients -- a training or control loop inside a host program that owns
 * all device memory through its own pre-reserved pool and forbids further
 * allocation, or one that must not stall on the implicit device
 * synchronisation of cudaMalloc / cudaFree.  sg_diff_forward would
 * cudaMalloc its checkpoints; this call allocates nothing: its scratch (the
 * checkpoints and the loss cotangent) lives in a static __device__ array of
 * 32 MiB compiled into libsg.so, which every GPU that loads the library
 * holds until the process exits.  The context itself must have been created
 * beforehand (sg_create allocates).
 *
 * Limits: substeps 1..16, ckpt_every 1..32, T 1..4096, and
 * (ceil(T / ckpt_every) + 1) * 14 * sg_plan_info.num_slots + 12 * T * E
 * floats must fit in the 32 MiB (8388608 floats); larger requests return
 * SG_ERR_INVALID_ARG with a message and enqueue nothing.
 * All calls on a device share the one array and it keeps the last call's
 * contents (each call writes every entry it reads before reading it, so
 * nothing needs clearing); calls whose GPU work overlaps -- other streams,
 * other host threads, other contexts on the same device -- race on it, so
 * the caller must serialise them.  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  The context's
 * own state and its sg_diff_forward checkpoints are not touched.
 */
sg_status sg_diff_track_noalloc(sg_ctx *ctx, const float *actions_dev, int32_t T, float dt,
                                int32_t substeps, int32_t ckpt_every, const float *target_dev,
                                float *ee_dev, float *loss_dev, float *dactions_dev,
                                float *dmass_dev);

/* Goal state of SG_TASK_TRACK in caller layout: offset_dev (goal minus the
 * initial goal) and velocity_dev, both [E][4][3] float (entries of chains an
 * env does not have are written as 0 / ignored).  Either pointer may be
 * NULL.  SG_ERR_INVALID_ARG for other tasks. */
sg_status sg_get_goal_state(sg_ctx *ctx, float *offset_dev, float *velocity_dev);
sg_status sg_set_goal_state(sg_ctx *ctx, const float *offset_dev, const float *velocity_dev);

/*
 * Path-following waypoints built on the device (Results, "Path following":
 * a cubic spline S(t) = a (t - t_i)^3 + b (t - t_i)^2 + c (t - t_i) + d
 * through the path's points, sampled at regular intervals of distance along
 * it).  For every env with env_mask_dev[e] != 0 (uint8 [E], device; NULL =
 * all envs) the waypoint table is rebuilt from ctrl_dev [E][K][3] (device,
 * float; rows of unmasked envs are not read):
 *   - natural cubic spline through the K control points at t_i = i
 *     (S'' = 0 at both ends);
 *   - a polyline of 64 points per segment (t = t_i + j / 64) plus the end
 *     point, and its cumulative chord length;
 *   - waypoint w (0 <= w < path_len) at arc length w L / (path_len - 1)
 *     along that polyline (L its length), by linear interpolation.
 * K is 2..64 and need not equal path_ctrl_len.  Call it together with
 * sg_reset for new per-episode paths: waypoint w is the target at w steps
 * after reset.  Non-finite control points give non-finite waypoints.  The
 * table is rebuilt asynchronously on the context's stream.
 * SG_ERR_INVALID_ARG for other tasks, a NULL ctrl_dev or K out of range. */
sg_status sg_set_paths(sg_ctx *ctx, const float *ctrl_dev, int32_t K, const uint8_t *env_mask_dev);

/* Copy the waypoint tables [E][path_len][3] (float) into path_dev (device).
 * SG_ERR_INVALID_ARG for other tasks. */
sg_status sg_get_paths(sg_ctx *ctx, float *path_dev);

/* Synchronise the context's stream, then read and clear the device error
 * flags: SG_ERR_NONFINITE if any env produced a non-finite state since the
 * last call, SG_ERR_TIMEOUT if a bounded device wait gave up, else SG_OK
 * (or SG_ERR_CUDA if the stream reports an error). */
sg_status sg_sync_status(sg_ctx *ctx);

/* Measurement helper (not part of the method): the device's FP32 FMA rate in
 * TFLOP/s (an FMA counts 2), the denominator of the step kernels' ALU
 * roofline.  Runs `repeats` timed launches (after one warm-up) of a kernel
 * with 8 independent FMA chains per thread, 8 blocks of 256 threads per SM
 * and iters x 128 FMAs per thread, on `stream` (cudaStream_t, NULL = legacy
 * default stream) of the current device, and writes the best rate to
 * *tflops.  Synchronises the stream; allocates and frees a small buffer.
 * SG_ERR_INVALID_ARG for iters < 1, repeats < 1 or a NULL tflops. */
sg_status sg_measure_fp32_fma_rate(void *stream, int32_t iters, int32_t repeats, float *tflops);

/*
 * Test hook (not part of the method): makes a bounded device-side wait run
 * out, so that the give-up path of the step kernels can be exercised
 * without a GPU fault or hang.  mode:
 *   SG_FAULT_NONE            normal operation (the default);
 *   SG_FAULT_SKIP_PARAM_COPY the one-thread step kernel (chain split 1) does
 *                            not start the copy of each warp's parameter
 *                            record, so every warp's wait for it runs out;
 *   SG_FAULT_SKIP_PARTNER    in the warp-pair step kernel (chain split 2)
 *                            the dynamics warp of every pair leaves out its
 *                            first arrival at the pair's exchange, so both
 *                            warps' waits for it run out.
 * wait_limit_ns bounds every wait of the step kernels in wall-clock time
 * (0 = the default, 2 s; at most 2e9).  A wait that runs out sets the
 * context's timeout flag (sg_sync_status returns SG_ERR_TIMEOUT); the
 * warps then leave the kernel without writing outputs or state, so the
 * context's state and step counts are unchanged.  Applies to sg_step,
 * sg_rollout (re-captured when the hook changes) and sg_observe.
 * SG_ERR_INVALID_ARG for an unknown mode or a limit out of range.
 */
enum { SG_FAULT_NONE = 0, SG_FAULT_SKIP_PARAM_COPY = 1, SG_FAULT_SKIP_PARTNER = 2 };
sg_status sg_debug_set_fault(sg_ctx *ctx, int32_t mode, int64_t wait_limit_ns);

/* Message of the last failing call on ctx (never NULL; "" if none).
 * With ctx == NULL: the last sg_create failure of this thread. */
const char *sg_last_error(const sg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
