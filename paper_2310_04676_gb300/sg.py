"""Python binding of libsg.so (include/sg.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels; PyTorch
supplies device memory and the current CUDA stream.  There is no CPU
fallback: if libsg.so is missing or no GPU is present, construction fails.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsg.so")

TASK_REACH, TASK_PATH, TASK_TRACK = 0, 1, 2
SG_OK, SG_ERR_INVALID_ARG, SG_ERR_CUDA, SG_ERR_OOM, SG_ERR_NONFINITE, SG_ERR_TIMEOUT, \
    SG_ERR_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "SG_OK", 1: "SG_ERR_INVALID_ARG", 2: "SG_ERR_CUDA", 3: "SG_ERR_OOM",
                4: "SG_ERR_NONFINITE", 5: "SG_ERR_TIMEOUT", 6: "SG_ERR_UNSUPPORTED"}
DONE_TERMINATED, DONE_TIMEOUT, DONE_NONFINITE = 1, 2, 4
HOST_IO_AUTO, HOST_IO_STAGED, HOST_IO_DIRECT = 0, 1, 2
ROLLOUT_PERSISTENT, ROLLOUT_STEP_GRAPH = 0, 1
PACK_CLASS, PACK_INTERLEAVE = 0, 1
FAULT_NONE, FAULT_SKIP_PARAM_COPY, FAULT_SKIP_PARTNER, FAULT_SKIP_WEIGHT_COPY = 0, 1, 2, 3
DRIVE_POSITION, DRIVE_VELOCITY, DRIVE_TORQUE = 0, 1, 2
MAX_CHAINS = 4                     # chains per env (SG_MAX_CHAINS)


class SgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_f32p = ctypes.POINTER(ctypes.c_float)


class SgDesc(ctypes.Structure):
    _fields_ = [
        ("num_envs", ctypes.c_int32), ("max_joints", ctypes.c_int32),
        ("env_num_chains", _c_i32p), ("chain_num_joints", _c_i32p),
        ("joint_type", _c_i32p), ("joint_axis", _c_i32p),
        ("link_len", _c_f32p), ("link_mass", _c_f32p), ("link_inertia", _c_f32p),
        ("link_com", _c_f32p), ("q_lo", _c_f32p), ("q_hi", _c_f32p),
        ("kp", _c_f32p), ("kd", _c_f32p), ("damping", _c_f32p), ("k_limit", _c_f32p),
        ("base_offset", _c_f32p), ("q0", _c_f32p),
        ("episode_len", ctypes.c_int32), ("task", ctypes.c_int32),
        ("goal", _c_f32p), ("path", _c_f32p), ("path_len", ctypes.c_int32),
        ("alpha", ctypes.c_float),
        ("joint_drive", _c_i32p),
        ("seed", ctypes.c_uint32), ("track_sigma", ctypes.c_float), ("track_limit", ctypes.c_float),
        ("path_ctrl", _c_f32p), ("path_ctrl_len", ctypes.c_int32),
    ]


class SgPpoConfig(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("epochs", ctypes.c_int32),
                ("minibatches", ctypes.c_int32), ("gamma", ctypes.c_float), ("lam", ctypes.c_float),
                ("clip", ctypes.c_float), ("value_coef", ctypes.c_float),
                ("entropy_coef", ctypes.c_float), ("lr", ctypes.c_float),
                ("max_grad_norm", ctypes.c_float), ("dt", ctypes.c_float),
                ("substeps", ctypes.c_int32), ("seed", ctypes.c_uint32), ("tf32", ctypes.c_int32)]


PPO_OBS, PPO_ACTIONS, PPO_LOGP, PPO_VALUES, PPO_REWARDS, PPO_DONES, PPO_ADVANTAGES, PPO_RETURNS, \
    PPO_GRAD = range(9)

PPO_DEFAULTS = dict(n_steps=24, epochs=5, minibatches=4, gamma=0.99, lam=0.95, clip=0.2,
                    value_coef=1.0, entropy_coef=0.01, lr=1e-3, max_grad_norm=1.0, dt=1.0 / 60.0,
                    substeps=2, seed=1, tf32=0)


class SgPlanInfo(ctypes.Structure):
    _fields_ = [("obs_dim", ctypes.c_int32), ("num_slots", ctypes.c_int32),
                ("num_chains", ctypes.c_int32), ("class_slots", ctypes.c_int32 * 4)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libsg.so and declare its signatures (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libsg.so not built (%s): run paper_2310_04676_gb300.build" % path)
    lib = ctypes.CDLL(path)
    vp, i32, f32, u8p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p
    sig = {
        "sg_plan": (i32, [ctypes.POINTER(SgDesc), ctypes.POINTER(SgPlanInfo), ctypes.c_char_p, i32]),
        "sg_create": (i32, [ctypes.POINTER(SgDesc), vp, ctypes.POINTER(vp)]),
        "sg_destroy": (None, [vp]),
        "sg_set_stream": (i32, [vp, vp]),
        "sg_device": (i32, [vp]),
        "sg_debug_set_fault": (i32, [vp, i32, ctypes.c_int64]),
        "sg_obs_dim": (i32, [vp]),
        "sg_num_envs": (i32, [vp]),
        "sg_max_joints": (i32, [vp]),
        "sg_reset": (i32, [vp, u8p]),
        "sg_step": (i32, [vp, vp, f32, i32, vp, vp, u8p]),
        "sg_observe": (i32, [vp, vp, u8p, vp]),
        "sg_get_state": (i32, [vp, vp, vp, vp]),
        "sg_set_state": (i32, [vp, vp, vp, vp]),
        "sg_sync_status": (i32, [vp]),
        "sg_set_host_io": (i32, [vp, i32]),
        "sg_rollout": (i32, [vp, vp, i32, f32, i32, vp, vp, u8p]),
        "sg_rollout_host": (i32, [vp, vp, i32, f32, i32, vp, vp, u8p]),
        "sg_set_launch": (i32, [vp, i32, i32, i32]),
        "sg_get_launch": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "sg_autotune": (i32, [vp, vp, i32, f32, i32, vp, vp, u8p, i32, ctypes.POINTER(f32)]),
        "sg_set_packing": (i32, [vp, i32]),
        "sg_get_packing": (i32, [vp]),
        "sg_plan_packing": (i32, [ctypes.POINTER(SgDesc), i32, vp, i32, ctypes.c_char_p, i32]),
        "sg_diff_forward": (i32, [vp, vp, i32, f32, i32, i32, vp]),
        "sg_diff_backward": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "sg_set_link_mass": (i32, [vp, vp]),
        "sg_get_goal_state": (i32, [vp, vp, vp]),
        "sg_set_goal_state": (i32, [vp, vp, vp]),
        "sg_diff_track_noalloc": (i32, [vp, vp, i32, f32, i32, i32, vp, vp, vp, vp, vp]),
        "sg_set_paths": (i32, [vp, vp, i32, u8p]),
        "sg_get_paths": (i32, [vp, vp]),
        "sg_measure_fp32_fma_rate": (i32, [vp, i32, i32, ctypes.POINTER(f32)]),
        "sg_ppo_create": (i32, [vp, ctypes.POINTER(SgPpoConfig), ctypes.POINTER(vp)]),
        "sg_ppo_destroy": (None, [vp]),
        "sg_ppo_num_params": (ctypes.c_int64, [vp]),
        "sg_ppo_set_params": (i32, [vp, vp]),
        "sg_ppo_get_params": (i32, [vp, vp]),
        "sg_ppo_reset": (i32, [vp, ctypes.c_int64]),
        "sg_ppo_debug_set_fault": (i32, [vp, i32, ctypes.c_int64]),
        "sg_ppo_collect": (i32, [vp]),
        "sg_ppo_update": (i32, [vp, vp, vp]),
        "sg_ppo_get_buffer": (i32, [vp, i32, vp]),
        "sg_ppo_set_buffer": (i32, [vp, i32, vp]),
        "sg_mlp_gemm": (i32, [vp, vp, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_int64,
                             ctypes.c_int64, vp, i32, i32, i32, i32, vp, ctypes.c_int64, vp,
                             ctypes.c_int64, i32]),
        "sg_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _arr(desc, key, dtype, shape):
    a = np.ascontiguousarray(np.asarray(desc[key], dtype=dtype)).ravel()
    need = int(np.prod(shape))
    if a.size < need:
        raise ValueError("desc[%r] has %d elements, needs %d" % (key, a.size, need))
    return a


def make_c_desc(desc):
    """ctypes sg_desc over numpy copies of an ``sg_desc`` dictionary.
    Returns (struct, keepalive list)."""
    E, J = int(desc["num_envs"]), int(desc["max_joints"])
    keep = []

    def p(key, dtype, shape, ctype):
        if desc.get(key) is None:
            return ctypes.cast(None, ctype)
        a = _arr(desc, key, dtype, shape)
        keep.append(a)
        return a.ctypes.data_as(ctype)

    i32, f32 = np.int32, np.float32
    d = SgDesc()
    d.num_envs, d.max_joints = E, J
    d.env_num_chains = p("env_num_chains", i32, (E,), _c_i32p)
    d.chain_num_joints = p("chain_num_joints", i32, (E, MAX_CHAINS), _c_i32p)
    d.joint_type = p("joint_type", i32, (E, J), _c_i32p)
    d.joint_axis = p("joint_axis", i32, (E, J), _c_i32p)
    for k in ("link_len", "link_mass", "link_com", "q_lo", "q_hi", "kp", "kd", "damping",
              "k_limit", "q0"):
        setattr(d, k, p(k, f32, (E, J), _c_f32p))
    d.link_inertia = p("link_inertia", f32, (E, J, 3), _c_f32p)
    d.base_offset = p("base_offset", f32, (E, MAX_CHAINS, 3), _c_f32p)
    d.goal = p("goal", f32, (E, MAX_CHAINS, 3), _c_f32p)
    W = int(desc.get("path_len") or 0)
    d.path = p("path", f32, (E, W, 3), _c_f32p) if W else ctypes.cast(None, _c_f32p)
    d.path_len = W
    K = int(desc.get("path_ctrl_len") or 0)
    d.path_ctrl = p("path_ctrl", f32, (E, K, 3), _c_f32p) if K else ctypes.cast(None, _c_f32p)
    d.path_ctrl_len = K
    d.episode_len = int(desc["episode_len"])
    d.task = int(desc["task"])
    d.alpha = float(desc.get("alpha", 1.0))
    d.joint_drive = p("joint_drive", i32, (E, J), _c_i32p)
    d.seed = int(desc.get("seed", 0)) & 0xFFFFFFFF
    d.track_sigma = float(desc.get("track_sigma", 0.0))
    d.track_limit = float(desc.get("track_limit", 0.0))
    return d, keep


def plan(desc):
    """Host-only validation and packing plan (no GPU): dict or SgError."""
    lib = load_library()
    d, keep = make_c_desc(desc)
    info = SgPlanInfo()
    buf = ctypes.create_string_buffer(512)
    st = lib.sg_plan(ctypes.byref(d), ctypes.byref(info), buf, 512)
    if st != SG_OK:
        raise SgError(st, buf.value.decode())
    return dict(obs_dim=info.obs_dim, num_slots=info.num_slots, num_chains=info.num_chains,
                class_slots=list(info.class_slots))


def plan_packing(desc, packing):
    """Host-only warp order of a packing (no GPU): int32 array, entry w =
    the warp of the class-grouped order that position w holds."""
    import numpy as np
    lib = load_library()
    d, keep = make_c_desc(desc)
    info = SgPlanInfo()
    buf = ctypes.create_string_buffer(512)
    st = lib.sg_plan(ctypes.byref(d), ctypes.byref(info), buf, 512)
    if st != SG_OK:
        raise SgError(st, buf.value.decode())
    nw = info.num_slots // 32
    order = np.zeros(nw, dtype=np.int32)
    st = lib.sg_plan_packing(ctypes.byref(d), int(packing), order.ctypes.data_as(ctypes.c_void_p),
                             nw, buf, 512)
    if st != SG_OK:
        raise SgError(st, buf.value.decode())
    return order


def fp32_fma_rate(iters=4096, repeats=5, stream=None):
    """Measured FP32 FMA rate of the current device in TFLOP/s."""
    import torch
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    out = ctypes.c_float()
    st = lib.sg_measure_fp32_fma_rate(ctypes.c_void_p(s.cuda_stream), int(iters), int(repeats),
                                      ctypes.byref(out))
    if st != SG_OK:
        raise SgError(st, "sg_measure_fp32_fma_rate failed")
    return float(out.value)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def mlp_gemm(A, a_strides, B, b_strides, M, N, K, out, c_m, bias=None, elu=False, work=None,
             split=True, stream=None):
    """sg_mlp_gemm: out[m * c_m + n] = act(sum_k A(m, k) B(n, k) + bias[n]) with
    A(m, k) = A.flatten()[m * a_strides[0] + k * a_strides[1]] and
    B(n, k) = B.flatten()[n * b_strides[0] + k * b_strides[1]] (contraction of
    the PPO networks).  split: True / 1 three TF32 products (FP32-grade),
    False / 0 one TF32 product, 2 FP32-grade with narrow products as FP32
    FMA loops on the CUDA cores."""
    import torch
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib.sg_mlp_gemm(ctypes.c_void_p(s.cuda_stream), _ptr(A), int(a_strides[0]),
                         int(a_strides[1]), _ptr(B), int(b_strides[0]), int(b_strides[1]),
                         _ptr(bias), 1 if elu else 0, int(M), int(N), int(K), _ptr(out), int(c_m),
                         _ptr(work), int(work.numel()) if work is not None else 0,
                         int(split))
    if st != SG_OK:
        raise SgError(st, "sg_mlp_gemm failed")
    return out


class Env:
    """A batch of environments on the current CUDA device.

    ``desc`` is an ``sg_desc`` dictionary (see ``workloads.make_desc``).
    Tensors passed in must be contiguous CUDA tensors of the documented
    dtype and shape; outputs are allocated with torch and returned.
    """

    def __init__(self, desc, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA GPU is required (no CPU fallback)")
        self._torch = torch
        self.lib = load_library()
        d, keep = make_c_desc(desc)
        s = stream if stream is not None else torch.cuda.current_stream()
        self._stream = s
        ctx = ctypes.c_void_p()
        st = self.lib.sg_create(ctypes.byref(d), ctypes.c_void_p(s.cuda_stream), ctypes.byref(ctx))
        if st != SG_OK:
            raise SgError(st, self.lib.sg_last_error(None).decode())
        self.ctx = ctx
        self.num_envs = self.lib.sg_num_envs(ctx)
        self.max_joints = self.lib.sg_max_joints(ctx)
        self.obs_dim = self.lib.sg_obs_dim(ctx)
        self.device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.sg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ----------------------------------------------------------
    def _check(self, st):
        if st != SG_OK:
            raise SgError(st, self.lib.sg_last_error(self.ctx).decode())

    def _sync_stream(self):
        cur = self._torch.cuda.current_stream()
        if cur.cuda_stream != self._stream.cuda_stream:
            self._stream = cur
            self._check(self.lib.sg_set_stream(self.ctx, ctypes.c_void_p(cur.cuda_stream)))

    def _want(self, t, dtype, shape, name):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != dtype \
                or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError("%s must be a contiguous cuda %s tensor of shape %s" % (name, dtype, shape))
        return t

    def empty_outputs(self, T=None):
        torch = self._torch
        lead = () if T is None else (T,)
        E, D = self.num_envs, self.obs_dim
        return (torch.empty(lead + (E, D), dtype=torch.float32, device=self.device),
                torch.empty(lead + (E,), dtype=torch.float32, device=self.device),
                torch.empty(lead + (E,), dtype=torch.uint8, device=self.device))

    # -- API ----------------------------------------------------------------
    def reset(self, mask=None):
        self._sync_stream()
        if mask is not None:
            self._want(mask, self._torch.uint8, (self.num_envs,), "mask")
        self._check(self.lib.sg_reset(self.ctx, _ptr(mask)))

    def step(self, actions, dt, substeps, out=None):
        self._sync_stream()
        torch = self._torch
        self._want(actions, torch.float32, (self.num_envs, self.max_joints), "actions")
        obs, rew, done = out if out is not None else self.empty_outputs()
        self._check(self.lib.sg_step(self.ctx, _ptr(actions), float(dt), int(substeps),
                                     _ptr(obs), _ptr(rew), _ptr(done)))
        return obs, rew, done

    def observe(self, targets, mask=None, out=None):
        """Observation of the current state (no time advance): rows of the
        envs in ``mask`` (uint8 [E], None = all) are written to ``out``."""
        self._sync_stream()
        torch = self._torch
        self._want(targets, torch.float32, (self.num_envs, self.max_joints), "targets")
        if mask is not None:
            self._want(mask, torch.uint8, (self.num_envs,), "mask")
        if out is None:
            out = torch.zeros(self.num_envs, self.obs_dim, dtype=torch.float32, device=self.device)
        self._check(self.lib.sg_observe(self.ctx, _ptr(targets), _ptr(mask), _ptr(out)))
        return out

    def rollout(self, actions, dt, substeps, out=None):
        """T steps in one call: actions [T, E, J] -> obs [T, E, D], reward
        [T, E], done [T, E] (captured CUDA graph, see sg_rollout)."""
        self._sync_stream()
        torch = self._torch
        T = int(actions.shape[0])
        self._want(actions, torch.float32, (T, self.num_envs, self.max_joints), "actions")
        obs, rew, done = out if out is not None else self.empty_outputs(T)
        self._check(self.lib.sg_rollout(self.ctx, _ptr(actions), T, float(dt), int(substeps),
                                        _ptr(obs), _ptr(rew), _ptr(done)))
        return obs, rew, done

    def rollout_host(self, actions, dt, substeps, out):
        """Rollout on host tensors (ideally pinned): actions [T, E, J] float32
        and preallocated host outputs (obs, reward, done); asynchronous on the
        context's stream."""
        self._sync_stream()
        obs, rew, done = out
        for t in (actions, obs, rew, done):
            if t.device.type != "cpu" or not t.is_contiguous():
                raise ValueError("rollout_host takes contiguous host tensors")
        T = int(actions.shape[0])
        self._check(self.lib.sg_rollout_host(self.ctx, _ptr(actions), T, float(dt), int(substeps),
                                             _ptr(obs), _ptr(rew), _ptr(done)))

    def set_host_io(self, mode):
        """HOST_IO_AUTO (pipelined copies), HOST_IO_STAGED (serial copies) or
        HOST_IO_DIRECT (the kernel accesses page-locked host buffers)."""
        self._check(self.lib.sg_set_host_io(self.ctx, int(mode)))

    def set_launch(self, threads_per_block, mode, chain_split=1):
        self._check(self.lib.sg_set_launch(self.ctx, int(threads_per_block), int(mode),
                                           int(chain_split)))

    def get_launch(self):
        """(threads_per_block, rollout mode, chain split)"""
        t, m, sp = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.sg_get_launch(self.ctx, ctypes.byref(t), ctypes.byref(m),
                                           ctypes.byref(sp)))
        return t.value, m.value, sp.value

    def set_packing(self, packing):
        """PACK_CLASS (warps grouped by chain class) or PACK_INTERLEAVE
        (classes interleaved in proportion); results are bit-identical."""
        self._sync_stream()
        self._check(self.lib.sg_set_packing(self.ctx, int(packing)))

    @property
    def packing(self):
        return int(self.lib.sg_get_packing(self.ctx))

    def autotune(self, actions, dt, substeps, out=None, repeats=3):
        """Pick the fastest launch plan (and packing, see `packing`) for this
        rollout shape; returns (threads_per_block, mode, chain split, ms per
        rollout).  State is preserved."""
        self._sync_stream()
        torch = self._torch
        T = int(actions.shape[0])
        self._want(actions, torch.float32, (T, self.num_envs, self.max_joints), "actions")
        obs, rew, done = out if out is not None else self.empty_outputs(T)
        ms = ctypes.c_float()
        self._check(self.lib.sg_autotune(self.ctx, _ptr(actions), T, float(dt), int(substeps),
                                         _ptr(obs), _ptr(rew), _ptr(done), int(repeats),
                                         ctypes.byref(ms)))
        t, m, sp = self.get_launch()
        return t, m, sp, ms.value

    # -- differentiation -----------------------------------------------------
    def set_link_mass(self, mass):
        """Link masses [E, J] (inertias scale with them)."""
        self._sync_stream()
        self._want(mass, self._torch.float32, (self.num_envs, self.max_joints), "mass")
        self._check(self.lib.sg_set_link_mass(self.ctx, _ptr(mass)))

    def diff_forward(self, actions, dt, substeps, ckpt_every=8):
        """Tool-tip trajectory [T, E, 4, 3] from the current state (state
        unchanged); checkpoints kept for diff_backward."""
        self._sync_stream()
        torch = self._torch
        T = int(actions.shape[0])
        self._want(actions, torch.float32, (T, self.num_envs, self.max_joints), "actions")
        ee = torch.empty(T, self.num_envs, MAX_CHAINS, 3, dtype=torch.float32, device=self.device)
        self._check(self.lib.sg_diff_forward(self.ctx, _ptr(actions), T, float(dt), int(substeps),
                                             int(ckpt_every), _ptr(ee)))
        return ee

    def diff_backward(self, actions, dl_dee, initial_state=False):
        """Gradients for the last diff_forward: (dactions [T, E, J],
        dmass [E, J]) and, with initial_state, (dq0, dqd0) [E, J]."""
        self._sync_stream()
        torch = self._torch
        T = int(actions.shape[0])
        self._want(actions, torch.float32, (T, self.num_envs, self.max_joints), "actions")
        self._want(dl_dee, torch.float32, (T, self.num_envs, MAX_CHAINS, 3), "dl_dee")
        da = torch.empty_like(actions)
        dm = torch.empty(self.num_envs, self.max_joints, dtype=torch.float32, device=self.device)
        dq0 = torch.empty_like(dm) if initial_state else None
        dqd0 = torch.empty_like(dm) if initial_state else None
        self._check(self.lib.sg_diff_backward(self.ctx, _ptr(actions), _ptr(dl_dee), _ptr(da),
                                              _ptr(dm), _ptr(dq0), _ptr(dqd0)))
        return (da, dm, dq0, dqd0) if initial_state else (da, dm)

    def get_goal_state(self):
        """Tracking task: (goal offset, goal velocity) [E, 4, 3]."""
        self._sync_stream()
        torch = self._torch
        off = torch.empty(self.num_envs, MAX_CHAINS, 3, dtype=torch.float32, device=self.device)
        vel = torch.empty_like(off)
        self._check(self.lib.sg_get_goal_state(self.ctx, _ptr(off), _ptr(vel)))
        return off, vel

    def set_goal_state(self, offset=None, velocity=None):
        self._sync_stream()
        shape = (self.num_envs, MAX_CHAINS, 3)
        for t, name in ((offset, "offset"), (velocity, "velocity")):
            if t is not None:
                self._want(t, self._torch.float32, shape, name)
        self._check(self.lib.sg_set_goal_state(self.ctx, _ptr(offset), _ptr(velocity)))

    def set_paths(self, ctrl, mask=None):
        """Path task: rebuild the waypoint tables of the envs in ``mask``
        (uint8 [E], None = all) from control points ctrl [E, K, 3]."""
        self._sync_stream()
        if ctrl.dim() != 3:
            raise ValueError("ctrl must be [E, K, 3]")
        self._want(ctrl, self._torch.float32, (self.num_envs, int(ctrl.shape[1]), 3), "ctrl")
        if mask is not None:
            self._want(mask, self._torch.uint8, (self.num_envs,), "mask")
        self._check(self.lib.sg_set_paths(self.ctx, _ptr(ctrl), int(ctrl.shape[1]), _ptr(mask)))

    def get_paths(self, path_len):
        """Path task: the waypoint tables [E, path_len, 3]."""
        self._sync_stream()
        out = self._torch.empty(self.num_envs, int(path_len), 3, dtype=self._torch.float32,
                                device=self.device)
        self._check(self.lib.sg_get_paths(self.ctx, _ptr(out)))
        return out

    def get_state(self):
        self._sync_stream()
        torch = self._torch
        E, J = self.num_envs, self.max_joints
        q = torch.empty(E, J, dtype=torch.float32, device=self.device)
        qd = torch.empty_like(q)
        sc = torch.empty(E, dtype=torch.int32, device=self.device)
        self._check(self.lib.sg_get_state(self.ctx, _ptr(q), _ptr(qd), _ptr(sc)))
        return q, qd, sc

    def set_state(self, q=None, qd=None, step_count=None):
        self._sync_stream()
        torch = self._torch
        E, J = self.num_envs, self.max_joints
        if q is not None:
            self._want(q, torch.float32, (E, J), "q")
        if qd is not None:
            self._want(qd, torch.float32, (E, J), "qd")
        if step_count is not None:
            self._want(step_count, torch.int32, (E,), "step_count")
        self._check(self.lib.sg_set_state(self.ctx, _ptr(q), _ptr(qd), _ptr(step_count)))

    def sync_status(self):
        """Synchronise and return the device status code (raises nothing)."""
        return self.lib.sg_sync_status(self.ctx)

    @property
    def cuda_device(self):
        """The CUDA device the context belongs to."""
        return self.lib.sg_device(self.ctx)

    def debug_set_fault(self, mode, wait_limit_ns=0):
        """Test hook: FAULT_SKIP_PARAM_COPY / FAULT_SKIP_PARTNER make the
        step kernels' bounded waits run out (after ``wait_limit_ns``); see
        sg_debug_set_fault in include/sg.h."""
        self._check(self.lib.sg_debug_set_fault(self.ctx, int(mode), int(wait_limit_ns)))


class PPO:
    """GPU-resident PPO loop over the envs of ``env`` (see include/sg_ppo.h).

    Keyword arguments override ``PPO_DEFAULTS``."""

    def __init__(self, env, **cfg):
        import torch
        self._torch = torch
        self.env = env
        self.lib = env.lib
        c = dict(PPO_DEFAULTS, **cfg)
        self.cfg = c
        conf = SgPpoConfig(**{k: c[k] for k, _ in SgPpoConfig._fields_})
        h = ctypes.c_void_p()
        env._sync_stream()
        st = self.lib.sg_ppo_create(env.ctx, ctypes.byref(conf), ctypes.byref(h))
        if st != SG_OK:
            raise SgError(st, self.lib.sg_last_error(env.ctx).decode())
        self.h = h
        self.num_params = int(self.lib.sg_ppo_num_params(h))
        self.E, self.D, self.A = env.num_envs, env.obs_dim, env.max_joints
        self.n = c["n_steps"]
        self.B = self.E * self.n

    def close(self):
        if getattr(self, "h", None):
            self.lib.sg_ppo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        self.env._check(st)

    def set_params(self, flat):
        self.env._sync_stream()
        self.env._want(flat, self._torch.float32, (self.num_params,), "params")
        self._check(self.lib.sg_ppo_set_params(self.h, _ptr(flat)))

    def get_params(self):
        self.env._sync_stream()
        out = self._torch.empty(self.num_params, dtype=self._torch.float32, device=self.env.device)
        self._check(self.lib.sg_ppo_get_params(self.h, _ptr(out)))
        return out

    def reset(self, step0=0):
        self.env._sync_stream()
        self._check(self.lib.sg_ppo_reset(self.h, int(step0)))

    def collect(self):
        self.env._sync_stream()
        self._check(self.lib.sg_ppo_collect(self.h))

    def update(self, perms, stats=True):
        """perms: int32 [epochs][B] device tensor; returns per-minibatch
        (surrogate, value loss, entropy, grad norm) as a [epochs*mb][4] tensor."""
        torch = self._torch
        self.env._sync_stream()
        self.env._want(perms, torch.int32, (self.cfg["epochs"], self.B), "perms")
        out = None
        if stats:
            out = torch.empty(self.cfg["epochs"] * self.cfg["minibatches"], 4,
                              dtype=torch.float32, device=self.env.device)
        self._check(self.lib.sg_ppo_update(self.h, _ptr(perms), _ptr(out)))
        return out

    def _shape(self, which):
        n, E, D, A = self.n, self.E, self.D, self.A
        torch = self._torch
        return {PPO_OBS: ((n + 1, E, D), torch.float32), PPO_ACTIONS: ((n, E, A), torch.float32),
                PPO_LOGP: ((n, E), torch.float32), PPO_VALUES: ((n + 1, E), torch.float32),
                PPO_REWARDS: ((n, E), torch.float32), PPO_DONES: ((n, E), torch.uint8),
                PPO_ADVANTAGES: ((n, E), torch.float32), PPO_RETURNS: ((n, E), torch.float32),
                PPO_GRAD: ((self.num_params,), torch.float32)}[which]

    def get_buffer(self, which):
        self.env._sync_stream()
        shape, dt = self._shape(which)
        out = self._torch.empty(shape, dtype=dt, device=self.env.device)
        self._check(self.lib.sg_ppo_get_buffer(self.h, int(which), _ptr(out)))
        return out

    def set_buffer(self, which, src):
        self.env._sync_stream()
        shape, dt = self._shape(which)
        self.env._want(src, dt, shape, "buffer")
        self._check(self.lib.sg_ppo_set_buffer(self.h, int(which), _ptr(src)))

    def debug_set_fault(self, mode, wait_limit_ns=0):
        """Test hook: FAULT_SKIP_WEIGHT_COPY makes the tensor-core
        contraction's wait for its first weight chunk run out (bounded by
        wait_limit_ns, 0 = 2 s); see sg_ppo_debug_set_fault in
        include/sg_ppo.h."""
        self.env._sync_stream()
        self._check(self.lib.sg_ppo_debug_set_fault(self.h, int(mode), int(wait_limit_ns)))


def _autograd_function():
    import torch

    class TipRollout(torch.autograd.Function):
        """Differentiable tool-tip rollout through the library's adjoint
        kernel: forward(env, actions [T,E,J], mass [E,J] or None, dt,
        substeps, ckpt_every) -> ee [T,E,4,3]."""

        @staticmethod
        def forward(ctx, env, actions, mass, dt, substeps, ckpt_every):
            if mass is not None:
                env.set_link_mass(mass.detach().contiguous())
            a = actions.detach().contiguous()
            ee = env.diff_forward(a, dt, substeps, ckpt_every)
            ctx.env = env
            ctx.save_for_backward(a)
            ctx.has_mass = mass is not None
            return ee

        @staticmethod
        def backward(ctx, g):
            (a,) = ctx.saved_tensors
            da, dm = ctx.env.diff_backward(a, g.contiguous())
            return None, da, (dm if ctx.has_mass else None), None, None, None

    return TipRollout


_TIP_ROLLOUT = None


def tip_rollout(env, actions, dt, substeps, mass=None, ckpt_every=8):
    """Tool-tip positions [T, E, 4, 3] as a differentiable function of the
    actions (and optionally the link masses) -- backward runs the adjoint
    kernel with checkpointing every ``ckpt_every`` steps.  One outstanding
    forward per Env: a second call before backward overwrites the
    checkpoints."""
    global _TIP_ROLLOUT
    if _TIP_ROLLOUT is None:
        _TIP_ROLLOUT = _autograd_function()
    return _TIP_ROLLOUT.apply(env, actions, mass, dt, substeps, ckpt_every)
