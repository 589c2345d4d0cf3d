#!/usr/bin/env python
"""Benchmark of the batched articulated-arm step on one GB300 (or N replicas).

Default workload: 16384 heterogeneous environments -- 25% 4-DOF revolute
arms, 40% 7-DOF revolute, 20% 7-DOF with a prismatic insertion joint, 15%
14-DOF two-arm robots -- reach task, dt = 1/60 s, 2 substeps.  One bench
step is one 32-step rollout of every env (32 x 16384 env-steps), issued as
the autotuned persistent kernel captured in a CUDA graph.  The same rollout
on the same inputs from the same state is also timed as 32 single-step
kernels replayed from a CUDA graph and as 32 sg_step calls (the plain
one-kernel-per-step launch); all three produce identical bits.

Metric: env-steps/s (aggregate over all ranks).  Timing: CUDA events on the
launching stream, W warm-up steps, K timed steps, L2 flushed (a 256 MiB
write, outside the events) before every timed step, max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config C1|C2|C3|C4|C5|P1] [--envs E ...] [--launch T,M,S]

--config selects one of the other workloads (C1: 64 envs, latency; C2: 8192
envs path following, with the rebuild time of the path tables; C4: adjoint
of a 64-step rollout of 2048 envs; C5: the limit-spring 7-DOF sweep over
--envs sizes plus the 4096-env, 128-step adjoint; P1: the PPO loop with
learning, 16384 envs); each prints one line per workload.  --launch fixes
the launch plan (threads per block, rollout mode, chain split) instead of
running the autotuner, to profile one plan.
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s at 16k mixed-DOF envs, batched vs plain; % FP32 roofline; grad err"
ROLLOUT_T = {"C1": 50, "C2": 50, "C3": 32, "C5": 50}

# Algorithmic FP32 operations of the step's formulation (an FMA counts 2),
# counted by running the chain code on a counting scalar type
# (paper_2310_04676_gb300/flops; tests/test_flop_counts.py keeps these
# constants equal to its output): per substep of one chain, and per step for
# the tool-tip kinematics of one chain.
# Operations the compiler folds (a literal 0 operand, a factor of +-1, two
# literals) are not counted; ncu's executed FFMA x 2 + FADD + FMUL of the
# default workload agrees with this count to 2%.
FLOP_SUBSTEP = {"4R": 581, "7R": 1424, "7P": 1296}
FLOP_TIP = {"4R": 55, "7R": 127, "7P": 115}
FLOP_REWARD = 9          # distance to the goal (per chain)
FLOP_QUAT = 30           # tip quaternion (path task)
W_HIDDEN = (256, 128, 64)   # hidden widths of the PPO networks
# Adjoint pieces (same counting): one substep's adjoint (forward substep with
# its factorisation recomputed, the solve with the factor, the reverse RNEA)
# and the tool-tip Jacobian-transpose product.
FLOP_SUBSTEP_ADJ = {"4R": 1460, "7R": 3278, "7P": 3070}
FLOP_TIP_VJP = {"4R": 112, "7R": 238, "7P": 210}
# the replay part of a substep adjoint (recomputed substep with its factor,
# then the inverse-dynamics sweeps): with replay buffers, the forward kernel
# does it for the last segment instead of the backward kernel
FLOP_SUBSTEP_REPLAY = {"4R": 832, "7R": 1954, "7P": 1797}


def env_step_flops(kinds, substeps, task=0):
    tot = 0
    for k in kinds:
        for c in (["7R", "7R"] if k == "14B" else [k]):
            tot += substeps * FLOP_SUBSTEP[c] + FLOP_TIP[c] + FLOP_REWARD
            if task == 1:
                tot += FLOP_QUAT
    return tot


def adjoint_flops(kinds, substeps, T, every, replay=True):
    """Algorithmic FLOPs of one differentiable rollout: (forward kernel,
    backward kernel).  The pipelined backward (replay buffers) recomputes
    every substep once, in a replay warp, with its inverse-dynamics sweeps
    (FLOP_SUBSTEP_ADJ counts the recomputed forward substep with its
    factorisation, the sweeps and their reverse), plus one tip product per
    step -- except for the last segment, whose replay part
    (FLOP_SUBSTEP_REPLAY) the forward kernel does in place of its own
    substeps; the one-warp backward also recomputes each segment from its
    checkpoint and each step's substep start states."""
    fwd = bwd = 0
    seg_steps = [min(every, T - t0) for t0 in range(0, T, every)]
    last = seg_steps[-1]
    for k in kinds:
        for c in (["7R", "7R"] if k == "14B" else [k]):
            sub = FLOP_SUBSTEP[c]
            fwd += T * (substeps * sub + FLOP_TIP[c])
            bwd += T * (FLOP_TIP_VJP[c] + substeps * FLOP_SUBSTEP_ADJ[c])
            if replay:
                rep = FLOP_SUBSTEP_REPLAY[c]
                fwd += last * substeps * (rep - sub)
                bwd -= last * substeps * rep
            else:
                bwd += sum(L - 1 for L in seg_steps) * substeps * sub
                bwd += T * (substeps - 1) * sub
    return fwd, bwd


def env_step_bytes(desc, obs_dim):
    """Algorithmic HBM bytes of one env-step of the persistent rollout: the
    action row read, observation row, reward and done written (waypoint
    reads of the path task add 4 x 12 bytes)."""
    E = desc["num_envs"]
    dof = desc["chain_num_joints"].sum(1)
    extra = 48 * E if int(desc["task"]) == 1 else 0
    return int(4 * dof.sum() + E * (4 * obs_dim + 4 + 1) + extra)


KERNEL_SOURCES = {
    "step_kernel": ("sg_internal.h", "sg_kernels.h", "sg_rng.cuh", "sg_chain.cuh",
                    "sg_device.cuh", "sg_kernels.cu"),
    "step_kernel_pair": ("sg_internal.h", "sg_kernels.h", "sg_rng.cuh", "sg_chain.cuh",
                         "sg_device.cuh", "sg_pair.cuh", "sg_pair.cu"),
    "diff_backward_pipe_kernel": ("sg_internal.h", "sg_chain.cuh", "sg_device.cuh",
                                  "sg_adjoint.cuh", "sg_pair.cuh", "sg_diff.h", "sg_diff.cu"),
}
# committed ncu summary holding each kernel's counters (default workload of its config)
KERNEL_PROFILES = {"step_kernel": "step_kernel_c3.md", "step_kernel_pair": "step_kernel_c3.md",
                   "diff_backward_pipe_kernel": "diff_backward_c4.md"}


def kernel_source_hash(kernel):
    """Hash of the sources a step kernel is compiled from; a profile summary
    names the hash per kernel, and its counters are used only if it matches."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2310_04676_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_counter(kernel, name):
    """A per-launch counter (`traffic_bytes_per_launch`,
    `executed_flops_per_launch`) of `kernel` on the default workload, from the
    committed ncu summary, if it was taken from the current sources."""
    if kernel not in KERNEL_SOURCES:
        return None
    p = os.path.join(ROOT, "profiles", KERNEL_PROFILES[kernel])
    if not os.path.exists(p):
        return None
    text = open(p).read()
    m = re.search(r"source_hash\[%s\]:\s*([0-9a-f]+)" % re.escape(kernel), text)
    if not m or m.group(1) != kernel_source_hash(kernel):
        return None
    m = re.search(r"%s\[%s\]:\s*([0-9]+)" % (re.escape(name), re.escape(kernel)), text)
    return int(m.group(1)) if m else None


def profiled_traffic(kernel):
    return profiled_counter(kernel, "traffic_bytes_per_launch")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, path, device):
        self.path, self.device, self.proc = path, device, None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        rows = [[x.strip() for x in line.split(",")] for line in open(self.path)]
        rows = [r for r in rows if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        num = lambda s: s.replace(".", "", 1).isdigit()
        sm = sorted(float(r[1]) for r in rows if num(r[1]))
        mx = max((float(r[2]) for r in rows if num(r[2])), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ---- ranks (one process per GPU, independent replicas) ---------------------
def dist_setup():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(x, world, device=None):
    """Maximum of a float over all ranks (identity for one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, seconds_per_rank, world, device=None):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    return world * units_per_rank / reduce_max(seconds_per_rank, world, device)


def replica_desc(wl, rank):
    """Rank 0 runs the workload as stated; rank r > 0 an independent replica
    with its own seeded link parameters and goals."""
    from paper_2310_04676_gb300 import workloads as W
    if rank == 0:
        return wl.desc
    d = wl.desc
    return W.make_desc(wl.kinds, seed_params=1 + 1000 * rank, seed_goals=3 + 1000 * rank,
                       shared_params=False, k_limit=float(d["k_limit"].max()),
                       episode_len=int(d["episode_len"]), task=int(d["task"]),
                       path_len=int(d["path_len"] or 0))


# ---- CPU baseline (the FP64 oracle as it stands) ----------------------------
def cpu_baseline(wl, seconds=12.0, max_envs=2048):
    """The oracle on this host's cores, on a bounded sample of the workload
    (the first `max_envs` envs, as many steps as fit in `seconds`)."""
    import torch
    from oracle.env import OracleEnv
    from paper_2310_04676_gb300 import workloads as W
    E = wl.desc["num_envs"]
    n = min(E, max_envs)
    sub = {k: (v[:n] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
           for k, v in wl.desc.items()}
    sub["num_envs"] = n
    env = OracleEnv(sub)
    acts = W.joint_targets(sub, 64)
    env.step(acts[0], wl.dt, wl.substeps)        # first step excluded (timing starts after it)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds and steps < 63:
        env.step(acts[1 + steps], wl.dt, wl.substeps)
        steps += 1
    el = time.perf_counter() - t0
    return {"value": n * steps / el, "unit": "env-steps/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": "%d of %d envs (same kind mix), %d steps, FP64 PyTorch CPU, %.1f s"
                      % (n, E, steps, el)}


def sample_by_kind(kinds, per_kind, seed=12):
    """`per_kind` env indices drawn at random from each kind of the batch."""
    rng = np.random.default_rng(seed)
    kinds = np.asarray(kinds)
    pick = [rng.choice(np.flatnonzero(kinds == k), min(per_kind, int((kinds == k).sum())),
                       replace=False) for k in sorted(set(kinds.tolist()))]
    return np.sort(np.concatenate(pick))


def sub_desc(desc, pick):
    E = desc["num_envs"]
    sub = {k: (v[pick] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
           for k, v in desc.items()}
    sub["num_envs"] = len(pick)
    return sub


def equal_accuracy(wl, launch, per_kind=64, steps=100):
    """The whole batch for `steps` control steps from the reset state, in the
    measured launch plan, as one persistent rollout and as one sg_step call
    per step; joint positions of `per_kind` envs drawn at random from each
    kind against the FP64 oracle: max over the sampled envs of
    ||q_gpu - q_ref|| / max(||q_ref||, 1e-3) (tolerance 1e-3, as in the
    parity tests)."""
    import torch
    from oracle.env import OracleEnv
    from paper_2310_04676_gb300 import sg, workloads as W
    desc = dict(wl.desc)
    E = desc["num_envs"]
    desc["episode_len"] = max(int(desc["episode_len"]), steps + 1)
    pick = sample_by_kind(wl.kinds, per_kind)
    acts = W.joint_targets(desc, steps)
    ref = OracleEnv(sub_desc(desc, pick))
    for t in range(steps):
        ref.step(acts[t][pick], wl.dt, wl.substeps)
    threads, mode, split = launch
    a = torch.as_tensor(acts, device="cuda")
    out = {}
    for form in ("rollout", "plain"):
        env = sg.Env(desc)
        env.set_launch(threads, mode, split)
        if form == "rollout":
            env.rollout(a, wl.dt, wl.substeps)
        else:
            for t in range(steps):
                env.step(a[t], wl.dt, wl.substeps)
        q = env.get_state()[0].cpu().numpy().astype(np.float64)[pick]
        err = np.linalg.norm(q - ref.q, axis=1) / np.maximum(np.linalg.norm(ref.q, axis=1), 1e-3)
        out[form] = float(err.max())
        env.close()
    return {"q_rel_err_max": out, "tolerance": 1e-3, "within": max(out.values()) <= 1e-3,
            "sample": "%d envs drawn at random across the %d kinds (%d each) of the whole "
                      "%d-env batch, %d steps from the reset state, measured launch plan; "
                      "FP64 oracle" % (len(pick), len(set(wl.kinds)), per_kind, E, steps)}


def cpu_baseline_single_core(wl, seconds=6.0, max_envs=256):
    """The same oracle restricted to one host thread, on a smaller sample."""
    import torch
    prev = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        r = cpu_baseline(wl, seconds=seconds, max_envs=max_envs)
    finally:
        torch.set_num_threads(prev)
    return r


def grad_error(wl, acts_np, tg_np, da, dm, n_envs=16):
    """Adjoint gradients of the first `n_envs` envs against the oracle's
    reverse mode (FP64 autograd through its rollout): max per-env relative
    error of dL/d(actions) and dL/d(mass)."""
    import torch
    from oracle.env import ee_rollout
    desc = wl.desc
    idx = np.arange(n_envs)
    n = int(desc["chain_num_joints"][0, 0])
    A = torch.tensor(acts_np[:, idx, :n], dtype=torch.float64, requires_grad=True)
    m = torch.tensor(desc["link_mass"][idx, :n], dtype=torch.float64, requires_grad=True)
    ee = ee_rollout(desc, A, wl.dt, wl.substeps, mass=m, env_idx=idx)
    L = ((ee - torch.tensor(tg_np[:, idx, :1], dtype=torch.float64)) ** 2).sum()
    ga, gm = torch.autograd.grad(L, [A, m])
    rel = lambda x, y: np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-12)
    ea = max(rel(da[:, e, :n], ga[:, e].numpy()) for e in range(n_envs))
    em = max(rel(dm[e, :n], gm[e].numpy()) for e in range(n_envs))
    return ea, em


# ---- GPU measurements -------------------------------------------------------
class Ctx:
    def __init__(self, args, world, rank, local):
        import torch
        self.torch = torch
        self.args, self.world, self.rank, self.local = args, world, rank, local
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.current_stream()
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=self.dev)
        self.out_dir = args.out_dir or os.path.join(tempfile.gettempdir(), "sg_bench")
        os.makedirs(self.out_dir, exist_ok=True)

    def barrier(self):
        if self.world > 1:
            self.torch.distributed.barrier()
        self.torch.cuda.synchronize()

    def timed(self, fn, steps, sampler=None):
        """Per-step device times (ms) of fn, L2 flushed before each step."""
        torch = self.torch
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        self.barrier()
        if sampler:
            sampler.start()
        for k in range(steps):
            self.flush.zero_()
            evs[k][0].record(self.stream)
            fn()
            evs[k][1].record(self.stream)
        self.barrier()
        if sampler:
            sampler.stop()
        return [a.elapsed_time(b) for a, b in evs]


def measure_rollout(cx, wl, desc, T, with_e2e=True):
    """Autotuned persistent rollout vs the per-step forms on one workload."""
    torch = cx.torch
    from paper_2310_04676_gb300 import sg, workloads as W
    args = cx.args
    E, S, dt = desc["num_envs"], wl.substeps, wl.dt
    acts = torch.as_tensor(W.joint_targets(desc, T, seed=2 + 1000 * cx.rank), device=cx.dev)
    env = sg.Env(desc)
    out = env.empty_outputs(T)
    if args.launch:
        threads, mode, split = args.launch
        env.set_launch(threads, mode, split)
    else:
        threads, mode, split, _ = env.autotune(acts, dt, S, out=out, repeats=3)
    packing = env.packing
    sgraph, plain = sg.Env(desc), sg.Env(desc)
    sgraph.set_launch(threads, sg.ROLLOUT_STEP_GRAPH, split)
    plain.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    for e in (sgraph, plain):
        e.set_packing(packing)
    out_g, out_p = sgraph.empty_outputs(T), plain.empty_outputs(T)

    def plain_rollout():
        o, r, d = out_p
        for t in range(T):
            plain.step(acts[t], dt, S, out=(o[t], r[t], d[t]))

    forms = {"ours": lambda: env.rollout(acts, dt, S, out=out),
             "step_graph": lambda: sgraph.rollout(acts, dt, S, out=out_g),
             "plain": plain_rollout}
    for _ in range(args.warmup):
        for f in forms.values():
            f()
    cx.barrier()
    clk = ClockSampler(os.path.join(cx.out_dir, "clocks_r%d.csv" % cx.rank), cx.local)
    ms = {"ours": cx.timed(forms["ours"], args.steps, clk)}
    for k in ("step_graph", "plain"):
        ms[k] = cx.timed(forms[k], args.steps)
    same = True
    qa, qda, _ = env.get_state()
    for other, o2 in ((sgraph, out_g), (plain, out_p)):
        qb, qdb, _ = other.get_state()
        same = same and bool(torch.equal(qa, qb) and torch.equal(qda, qdb)
                             and torch.equal(out[0], o2[0]))
    res = {"T": T, "E": E, "ms": ms, "launch": (threads, mode, split), "packing": packing,
           "same_bits": same,
           "status": sg.STATUS_NAMES.get(env.sync_status()), "clocks": clk.summary(),
           "obs_dim": env.obs_dim}
    if with_e2e:
        env_h = sg.Env(desc)
        env_h.set_launch(threads, mode, split)
        env_h.set_packing(packing)
        a_h = acts.cpu().pin_memory()
        o_h = (torch.empty(T, E, env_h.obs_dim).pin_memory(), torch.empty(T, E).pin_memory(),
               torch.empty(T, E, dtype=torch.uint8).pin_memory())
        for _ in range(args.warmup):
            env_h.rollout_host(a_h, dt, S, o_h)
        res["ms_e2e"] = cx.timed(lambda: env_h.rollout_host(a_h, dt, S, o_h), args.steps)
        for mode, key in ((sg.HOST_IO_STAGED, "ms_e2e_staged"), (sg.HOST_IO_DIRECT, "ms_e2e_direct")):
            env_h.set_host_io(mode)
            for _ in range(args.warmup):
                env_h.rollout_host(a_h, dt, S, o_h)
            res[key] = cx.timed(lambda: env_h.rollout_host(a_h, dt, S, o_h), args.steps)
        res["h2d"] = T * E * env_h.max_joints * 4
        res["d2h"] = T * E * (env_h.obs_dim * 4 + 4 + 1)
        res["link"] = host_link_floor(cx, res["h2d"], res["d2h"])
    return res


def measure_path_build(cx, desc, repeats=20):
    """sg_set_paths over every env: device time per rebuild of all tables."""
    torch = cx.torch
    from paper_2310_04676_gb300 import sg
    env = sg.Env(desc)
    ctrl = torch.as_tensor(desc["path_ctrl"], device=cx.dev)
    for _ in range(3):
        env.set_paths(ctrl)
    ms = cx.timed(lambda: env.set_paths(ctrl), repeats)
    E, K, W_ = desc["num_envs"], int(desc["path_ctrl_len"]), int(desc["path_len"])
    us = 1e3 * sum(ms) / len(ms)
    nbytes = E * (K + W_) * 12                  # control points in, waypoint table out
    return {"us_per_rebuild": us, "envs": E, "ctrl_points": K, "waypoints": W_,
            "algorithmic_bytes": nbytes, "achieved_gbs": nbytes / (us * 1e-6) / 1e9,
            "form": "sg_set_paths, all envs, one launch", "gpu_launches": 1}


def host_link_floor(cx, h2d_bytes, d2h_bytes, repeats=10):
    """The host link's floor for one end-to-end step: plain pinned-memory
    copies of the same byte counts, both directions in flight on two
    streams (CUDA events, best of `repeats`)."""
    torch = cx.torch
    hi = torch.empty(h2d_bytes // 4).pin_memory()
    di = torch.empty(h2d_bytes // 4, device=cx.dev)
    ho = torch.empty(d2h_bytes // 4).pin_memory()
    do = torch.empty(d2h_bytes // 4, device=cx.dev)
    s1, s2 = torch.cuda.Stream(cx.dev), torch.cuda.Stream(cx.dev)

    def copies(which):
        cur = torch.cuda.current_stream(cx.dev)
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        if which in ("in", "both"):
            with torch.cuda.stream(s1):
                di.copy_(hi, non_blocking=True)
        if which in ("out", "both"):
            with torch.cuda.stream(s2):
                ho.copy_(do, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    out = {}
    for which in ("in", "out", "both"):
        best = None
        for _ in range(repeats + 2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            copies(which)
            b.record()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[which] = best
    return {"h2d_gbs": h2d_bytes / (out["in"] * 1e-3) / 1e9,
            "d2h_gbs": d2h_bytes / (out["out"] * 1e-3) / 1e9,
            "floor_ms_per_step": out["both"],
            "how": "pinned-memory copies of the step's bytes, both directions on two streams"}


def measure_adjoint(cx, wl, desc, T, every=8):
    """Differentiable rollout: checkpointed forward + adjoint, per rollout."""
    torch = cx.torch
    from paper_2310_04676_gb300 import sg, workloads as W
    S, dt = wl.substeps, wl.dt
    acts_np = W.joint_targets(desc, T, resample_every=8)
    tg_np = W.loss_targets(desc, T)
    acts = torch.as_tensor(acts_np, device=cx.dev)
    tg = torch.as_tensor(tg_np, device=cx.dev)
    env = sg.Env(desc)
    nc = torch.as_tensor(desc["env_num_chains"], device=cx.dev)
    mask = (torch.arange(4, device=cx.dev)[None, :] < nc[:, None]).float()[None, :, :, None]
    res = {}

    kev = []            # per timed rollout: events around the backward kernel

    def fwd_bwd():
        ee = env.diff_forward(acts, dt, S, every)
        g = (2.0 * (ee - tg) * mask).contiguous()
        if res.get("timing"):
            ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            ev[0].record(cx.stream)
            res["grads"] = env.diff_backward(acts, g)
            ev[1].record(cx.stream)
            kev.append(ev)
        else:
            res["grads"] = env.diff_backward(acts, g)

    for _ in range(cx.args.warmup):
        fwd_bwd()
    res["timing"] = True
    clk = ClockSampler(os.path.join(cx.out_dir, "clocks_adj_r%d.csv" % cx.rank), cx.local)
    ms = cx.timed(fwd_bwd, cx.args.steps, clk)
    res["timing"] = False
    ms_bwd = [a.elapsed_time(b) for a, b in kev]
    da, dm = (x.cpu().numpy() for x in res["grads"])
    return {"ms": ms, "ms_bwd": ms_bwd, "T": T, "E": desc["num_envs"], "da": da, "dm": dm,
            "acts": acts_np, "tg": tg_np, "every": every, "clocks": clk.summary()}


def executed_rate(kernel, seconds):
    """Executed FP32 TFLOP/s (ncu's FFMA x 2 + FADD + FMUL of the default
    workload's launch over this launch time), when the committed profile
    matches the sources and this is the default workload's launch."""
    f = profiled_counter(kernel, "executed_flops_per_launch")
    return f / seconds / 1e12 if f else None


_FMA_RATE = {}


def measured_fma_rate():
    """FP32 FMA rate of this GPU from the library's probe (TFLOP/s), once."""
    if "v" not in _FMA_RATE:
        from paper_2310_04676_gb300 import sg
        _FMA_RATE["v"] = sg.fp32_fma_rate(iters=1024, repeats=3)
    return _FMA_RATE["v"]


def roofline(kernel_name, flops_launch, bytes_launch, ms_per_launch, props, peaks, peak_src,
             profiled=False):
    """`profiled`: this is the launch the committed ncu summary was taken
    from (the default workload), so its DRAM traffic and executed FLOPs apply."""
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    s = ms_per_launch / 1e3
    achieved = flops_launch / s / 1e12
    fma = measured_fma_rate()
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": profiled_traffic(kernel_name) if profiled else None,
            # bytes the kernel wrote into L2 (ncu lts__t_sectors_op_write x 32):
            # DRAM writes undercount them when written lines are still in L2
            # as the kernel ends
            "l2_write_bytes": (profiled_counter(kernel_name, "l2_write_bytes_per_launch")
                               if profiled else None),
            "fma_probe_tflops": fma, "frac_of_fma_probe": achieved / fma,
            "kernel": kernel_name,
            "peak_source": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (%s max SM clock)"
                           % (props.multi_processor_count, sm_max, peak_src),
            "flops_per_launch": flops_launch, "algorithmic_bytes_per_launch": bytes_launch,
            "executed_tflops": executed_rate(kernel_name, s) if profiled else None,
            "hbm_gbs": bytes_launch / s / 1e9 if bytes_launch else None,
            "hbm_frac": (bytes_launch / s / 1e9 / float(peaks.get("hbm_gbs", 6800.0))
                         if bytes_launch else None)}


def stats(ms):
    """Median and interquartile range of per-step device times (ms)."""
    q1, med, q3 = np.percentile(np.asarray(ms, np.float64), [25, 50, 75])
    return {"median_ms": float(med), "iqr_ms": float(q3 - q1), "n": len(ms)}


def base_line(args, world, value, ms_step, config):
    return {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config}


def run_rollout_config(cx, name, E=None):
    from paper_2310_04676_gb300 import workloads as W
    torch = cx.torch
    wl = W.config(name, num_envs=E)
    desc = replica_desc(wl, cx.rank)
    T = ROLLOUT_T[name]
    r = measure_rollout(cx, wl, desc, T, with_e2e=(name == "C3"))
    args, world = cx.args, cx.world
    units = r["E"] * T * args.steps
    t = {k: sum(v) / 1e3 for k, v in r["ms"].items()}
    value = aggregate_rate(units, t["ours"], world, cx.dev)
    peaks, src = load_peaks()
    props = torch.cuda.get_device_properties(cx.dev)
    threads, mode, split = r["launch"]
    kname = "step_kernel_pair" if split == 2 else "step_kernel"
    flops = env_step_flops(wl.kinds, wl.substeps, int(desc["task"])) * T
    nbytes = env_step_bytes(desc, r["obs_dim"]) * T
    ms_launch = sum(r["ms"]["ours"]) / len(r["ms"]["ours"])
    cfg = {"workload": wl.name, "envs_per_gpu": r["E"], "rollout_steps": T,
           "substeps": wl.substeps, "dt": wl.dt,
           "l2": "flushed (256 MiB write) before every timed step"}
    line = base_line(args, world, value, 1e3 * t["ours"] / args.steps, cfg)
    line["form"] = "persistent kernel in a CUDA graph"
    line["launch"] = {"threads_per_block": threads, "mode": ["persistent", "step_graph"][mode],
                      "chain_split": split,
                      "packing": ["class-grouped", "interleaved"][r["packing"]]}
    line["us_per_control_step"] = 1e6 * t["ours"] / args.steps / T
    line["step_time_stats"] = stats(r["ms"]["ours"])
    for k, label in (("step_graph", "%d single-step kernels replayed from a CUDA graph" % T),
                     ("plain", "one sg_step call (one kernel launch) per control step")):
        line[k] = {"value": aggregate_rate(units, t[k], world, cx.dev), "unit": "env-steps/s",
                   "ms_per_step": 1e3 * t[k] / args.steps, "form": label,
                   "gpu_launches": T * args.steps}
    line["batched_over_plain"] = t["plain"] / t["ours"]
    line["batched_over_step_graph"] = t["step_graph"] / t["ours"]
    line["bitwise_equal_forms"] = r["same_bits"]
    line["status"] = r["status"]
    line["roofline"] = roofline(kname, flops, nbytes, ms_launch, props, peaks, src,
                                profiled=(name == "C3" and E is None and args.gpus == 1))
    if "ms_e2e" in r:
        te = sum(r["ms_e2e"]) / 1e3
        ts = sum(r["ms_e2e_staged"]) / 1e3
        td = sum(r["ms_e2e_direct"]) / 1e3
        line["e2e"] = {"value": aggregate_rate(units, te, world, cx.dev), "unit": "env-steps/s",
                       "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"],
                       "path": "sg_rollout_host on pinned host buffers, pipelined: the 32 steps "
                               "run as 8 chunks whose copy-in, rollout kernel and copy-out "
                               "overlap on separate streams",
                       "direct": {"value": aggregate_rate(units, td, world, cx.dev),
                                  "path": "the rollout kernel reads and writes the pinned "
                                          "host buffers itself (NVLink-C2C)"},
                       "link": dict(r["link"], frac=r["link"]["floor_ms_per_step"] /
                                    (1e3 * te / args.steps)),
                       "staged": {"value": aggregate_rate(units, ts, world, cx.dev),
                                  "path": "copy in, device rollout, copy out"}}
    line["gpu_launches"] = args.steps
    line["clocks"] = r["clocks"]
    if int(desc["task"]) == 1 and desc.get("path_ctrl") is not None:
        line["path_build"] = measure_path_build(cx, desc)
    return line, wl


def run_adjoint_config(cx, with_error, name="C4", E=None, T=None, err_envs=16):
    from paper_2310_04676_gb300 import workloads as W
    wl = W.config(name, num_envs=E)
    desc = replica_desc(wl, cx.rank)
    a = measure_adjoint(cx, wl, desc, T or wl.steps, every=8)
    t = sum(a["ms"]) / 1e3
    units = a["E"] * a["T"] * cx.args.steps
    out = {"workload": "%s, T=%d, S=%d, checkpoints every %d steps"
                       % (wl.name, a["T"], wl.substeps, a["every"]),
           "value": aggregate_rate(units, t, cx.world, cx.dev),
           "unit": "env-steps/s (forward with checkpoints + adjoint)",
           "ms_per_rollout": 1e3 * t / cx.args.steps,
           "rollout_time_stats": stats(a["ms"]),
           "gpu_launches": 2 * cx.args.steps}
    f_fwd, f_bwd = adjoint_flops(wl.kinds, wl.substeps, a["T"], a["every"])
    peaks, src = load_peaks()
    props = cx.torch.cuda.get_device_properties(cx.dev)
    ms_b = sum(a["ms_bwd"]) / len(a["ms_bwd"])
    # the committed profile's counters belong to the C4 launch at its default size
    profiled = name == "C4" and E is None and T is None and cx.args.gpus == 1
    rf = roofline("diff_backward_pipe_kernel", f_bwd, None, ms_b, props, peaks, src,
                  profiled=profiled)
    rf.pop("hbm_gbs", None), rf.pop("hbm_frac", None), rf.pop("algorithmic_bytes_per_launch", None)
    out["roofline"] = rf
    out["flops_per_rollout"] = {"forward": f_fwd, "backward": f_bwd}
    out["ms_backward_kernel"] = ms_b
    out["rollout_tflops"] = (f_fwd + f_bwd) / (t / cx.args.steps) / 1e12
    out["clocks"] = a["clocks"]
    if with_error:
        ea, em = grad_error(wl, a["acts"], a["tg"], a["da"], a["dm"], n_envs=err_envs)
        out["rel_err_actions"] = ea
        out["rel_err_mass"] = em
        out["error_vs"] = ("FP64 oracle reverse mode, %d envs, max per-env relative L2 error"
                           % err_envs)
    return out


def ppo_flops(D, A, E, n, epochs):
    """Algorithmic FLOPs of one PPO iteration's dense layers (an FMA counts
    2): the forward of both networks per env and step plus the last values,
    and per update row the forward, the weight gradients and the input
    gradients of every layer but the first."""
    dims = (D,) + W_HIDDEN
    fw = lambda out: 2 * sum(a * b for a, b in zip(dims, dims[1:] + (out,)))
    fwd = fw(A) + fw(1)
    bwd = 2 * fwd - 2 * D * W_HIDDEN[0] * 2          # dW of all layers + dX of layers 2..4
    collect = (n * E + E) * fwd - E * fw(A)
    update = epochs * n * E * (fwd + bwd)
    return collect, update


def measure_ppo(cx, wl, desc, tf32):
    """Iteration times (collect + update) of the PPO loop in one GEMM mode."""
    torch = cx.torch
    from paper_2310_04676_gb300 import sg, workloads as W
    args = cx.args
    env = sg.Env(desc)
    ppo = sg.PPO(env, n_steps=wl.steps, epochs=5, minibatches=4, dt=wl.dt, substeps=wl.substeps,
                 seed=1 + cx.rank, tf32=tf32)
    D, A = env.obs_dim, env.max_joints
    ppo.set_params(torch.as_tensor(W.ppo_init_params(D, A), device=cx.dev))
    ppo.reset(0)
    perms_h = torch.as_tensor(W.ppo_perms(ppo.B, 5)).pin_memory()
    perms = perms_h.to(cx.dev)
    stats_h = torch.empty(20, 4).pin_memory()
    ev = []

    def iteration(e2e=False):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        if e2e:
            perms.copy_(perms_h, non_blocking=True)
        a.record(cx.stream)
        ppo.collect()
        b.record(cx.stream)
        st = ppo.update(perms)
        if e2e:
            stats_h.copy_(st, non_blocking=True)
        ev.append((a, b))

    for _ in range(args.warmup):
        iteration()
    ev.clear()
    clk = ClockSampler(os.path.join(cx.out_dir, "clocks_ppo_r%d.csv" % cx.rank), cx.local)
    ms = cx.timed(iteration, args.steps, clk)
    ms_collect = [a.elapsed_time(b) for a, b in ev]
    ev.clear()
    ms_e2e = cx.timed(lambda: iteration(True), args.steps)
    return {"ms": ms, "ms_collect": ms_collect, "ms_e2e": ms_e2e, "clocks": clk.summary(),
            "status": sg.STATUS_NAMES.get(env.sync_status()), "D": D, "A": A,
            "E": env.num_envs, "B": ppo.B, "h2d": int(perms_h.numel() * 4),
            "d2h": int(stats_h.numel() * 4)}


def mlp_layer_times(cx, rows, D, A, repeats=10):
    """Per-layer time of the networks' products at one minibatch of `rows`
    rows, through sg_mlp_gemm with the PPO update's operand roles (forward
    X W^T + b with ELU on hidden layers and input gradient dY W: weights
    pre-split in a work buffer; weight gradient dY^T X: rows split over
    CTAs), in the update's mode: FP32-grade 3xTF32 on the tensor cores, the
    narrow products (28 inputs, 8-wide outputs) as FP32 FMA loops; CUDA
    events, L2 flushed before each run, median of `repeats`.  The update's
    input gradient also applies the ELU derivative and sums bias gradients in
    its epilogue; this plain product leaves those out, and each call here
    splits its weights itself (the update splits all layers' weights in one
    launch per minibatch)."""
    torch = cx.torch
    from paper_2310_04676_gb300 import sg
    dims = (D,) + W_HIDDEN
    layers = [(dims[i], dims[i + 1] if i < 3 else A, i < 3) for i in range(4)]
    work = torch.empty(2 * 152 * 256 * 128, device=cx.dev)
    g = torch.Generator(device=cx.dev).manual_seed(5)
    rnd = lambda *shape: torch.rand(*shape, device=cx.dev, generator=g) * 2 - 1
    out = []
    for i, (inp, o, elu) in enumerate(layers):
        X, dY = rnd(rows, inp), rnd(rows, o)
        Wt, b = rnd(o, inp) * 0.1, rnd(o)
        Y, dX, dW = (torch.empty(rows, o, device=cx.dev), torch.empty(rows, inp, device=cx.dev),
                     torch.empty(o, inp, device=cx.dev))
        calls = {"forward": (lambda: sg.mlp_gemm(X, (inp, 1), Wt, (inp, 1), rows, o, inp, Y, o,
                                                  bias=b, elu=elu, work=work, split=2),
                             rows, o, inp),
                 "weight_grad": (lambda: sg.mlp_gemm(dY, (1, o), X, (1, inp), o, inp, rows, dW,
                                                      inp, work=work, split=2), o, inp, rows)}
        if i > 0:
            calls["input_grad"] = (lambda: sg.mlp_gemm(dY, (o, 1), Wt, (1, inp), rows, inp, o,
                                                        dX, inp, work=work, split=2),
                                   rows, inp, o)
        for kind, (f, M, N, K) in calls.items():
            for _ in range(3):
                f()
            ts = []
            for _ in range(repeats):
                cx.flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                a.record()
                f()
                e.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(e))
            ms = float(np.median(ts))
            out.append({"layer": "%d->%d" % (inp, o), "product": kind, "M": M, "N": N, "K": K,
                        "ms": ms, "tflops": 2.0 * M * N * K / ms / 1e9})
        del X, dY, Y, dX, dW
    return out


def run_ppo_config(cx, name="P1", E=None):
    """The with-learning workload: collect + update per iteration, with FP32
    GEMMs (the line's value) and with TF32 tensor-core GEMMs (beside it)."""
    torch = cx.torch
    from paper_2310_04676_gb300 import workloads as W
    args = cx.args
    wl = W.ppo_config(name, num_envs=E)
    desc = replica_desc(wl, cx.rank)
    peaks, src = load_peaks()
    props = torch.cuda.get_device_properties(cx.dev)
    fp32_peak = props.multi_processor_count * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) \
        * 1e6 / 1e12
    tf32_peak = float(peaks.get("bf16_tflops", 1900.0)) * (1.1 / 2.25)
    runs = {m: measure_ppo(cx, wl, desc, m) for m in (0, 1)}
    r = runs[0]
    D, A, En = r["D"], r["A"], r["E"]
    frames = En * wl.steps * args.steps
    f_col, f_upd = ppo_flops(D, A, En, wl.steps, 5)

    def summary(rr, peak):
        t = sum(rr["ms"]) / 1e3
        it = t / args.steps
        return {"value": aggregate_rate(frames, t, world=cx.world, device=cx.dev),
                "ms_per_iteration": 1e3 * it, "ms_collect": float(np.mean(rr["ms_collect"])),
                "ms_update": 1e3 * it - float(np.mean(rr["ms_collect"])),
                "achieved_tflops": (f_col + f_upd) / it / 1e12,
                "frac": (f_col + f_upd) / it / 1e12 / peak}

    s32, stf = summary(r, fp32_peak), summary(runs[1], tf32_peak)
    cfg = {"workload": wl.name, "envs_per_gpu": En, "n_steps": wl.steps, "epochs": 5,
           "minibatches": 4, "minibatch_rows": r["B"] // 4, "substeps": wl.substeps, "dt": wl.dt,
           "networks": "actor and critic MLP %d-256-128-64-{%d,1}, ELU" % (D, A),
           "gemm": "this library's tcgen05 contraction, FP32-grade split precision (3xTF32), "
                   "weights split once per update",
           "l2": "flushed (256 MiB write) before every timed iteration"}
    line = base_line(args, cx.world, s32["value"], s32["ms_per_iteration"], cfg)
    line["metric"] = "with-learning frames/s (collect + PPO update), context for the step metric"
    line["unit"] = "frames/s"
    line["dtype"] = "f32"
    line["iteration_time_stats"] = stats(r["ms"])
    line["ms_collect"] = s32["ms_collect"]
    line["ms_update"] = s32["ms_update"]
    line["roofline"] = {"bound": "alu", "achieved": s32["achieved_tflops"], "peak": fp32_peak,
                        "unit": "TFLOP/s", "frac": s32["frac"], "traffic": None,
                        "kernel": "whole iteration (dense layers' FLOPs / iteration time)",
                        "peak_source": "SMs x 128 FP32 lanes x 2 x max SM clock",
                        "flops_per_iteration": {"collect": f_col, "update": f_upd}}
    # the actor's products at one minibatch (inputs padded to 4 columns, as
    # inside the library), outside the timed region
    line["layers"] = {"rows": r["B"] // 4,
                      "products": mlp_layer_times(cx, r["B"] // 4, (D + 3) // 4 * 4,
                                                  (A + 3) // 4 * 4)}
    line["tf32"] = dict(stf, dtype="tf32", gemm="this library's tcgen05 contraction, one TF32 product",
                        peak=tf32_peak, peak_source="measured bf16 burst x 1.1/2.25 (%s)" % src,
                        note="reduced-precision GEMM inputs (10-bit mantissa): context only")
    line["e2e"] = {"value": aggregate_rate(frames, sum(r["ms_e2e"]) / 1e3, world=cx.world,
                                           device=cx.dev),
                   "unit": "frames/s", "h2d_bytes_per_step": r["h2d"],
                   "d2h_bytes_per_step": r["d2h"]}
    # kernels of this library per iteration: the weights' TF32 split, then per
    # collect step 8 layer products (bias + ELU fused), pad, sampling, the env
    # step, bootstrap, reset, observe; then pad, 4 critic layers (last values),
    # GAE, 2 moments, step counter; per minibatch gather, the weights' TF32
    # split, 8 forward layers, 2 loss-head, per network 4 weight gradients
    # (product + fixed-order sum of the row splits), the output bias column
    # sums, 3 input gradients with the ELU backward and the hidden bias sums,
    # one launch finishing the four bias gradients; then 2 norm, Adam
    n_mb = 5 * 4
    line["gpu_launches"] = (1 + wl.steps * 14 + 9 + n_mb * 41) * args.steps
    line["library_launches"] = 0
    line["clocks"] = r["clocks"]
    line["status"] = r["status"]
    line["paper_context"] = ("Table II: 6.8 s per 1M timesteps with learning (147,059 frames/s), "
                             "20,000 envs on one 8 GB Quadro RTX 4000 (different engine and task)")
    return line


def _compact_rollout(line):
    """The figures of one rollout workload's line that the default line's
    `configs` object carries."""
    rf = line["roofline"]
    out = {"workload": line["config"]["workload"], "envs": line["config"]["envs_per_gpu"],
           "value": line["value"], "unit": line["unit"],
           "ms_per_rollout": line["ms_per_step"],
           "rollout_steps": line["config"]["rollout_steps"],
           "substeps": line["config"]["substeps"],
           "us_per_control_step": line["us_per_control_step"],
           "step_time_stats": line["step_time_stats"],
           "plain": {"value": line["plain"]["value"], "ms_per_rollout": line["plain"]["ms_per_step"]},
           "step_graph": {"value": line["step_graph"]["value"]},
           "batched_over_plain": line["batched_over_plain"],
           "bitwise_equal_forms": line["bitwise_equal_forms"], "status": line["status"],
           "roofline": {k: rf[k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                           "frac_of_fma_probe", "kernel", "flops_per_launch",
                                           "algorithmic_bytes_per_launch", "hbm_gbs",
                                           "hbm_frac")},
           "launch": line["launch"], "gpu_launches": line["gpu_launches"],
           "clocks": line["clocks"]}
    if "path_build" in line:
        out["path_build"] = line["path_build"]
    return out


def _compact_adjoint(g):
    keep = ("workload", "value", "unit", "ms_per_rollout", "rollout_time_stats",
            "ms_backward_kernel", "flops_per_rollout", "rollout_tflops", "gpu_launches",
            "clocks", "rel_err_actions", "rel_err_mass", "error_vs")
    out = {k: g[k] for k in keep if k in g}
    out["roofline"] = {k: g["roofline"][k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                     "frac_of_fma_probe", "kernel",
                                                     "flops_per_launch", "traffic",
                                                     "l2_write_bytes")}
    return out


def _compact_ppo(line):
    keep = ("value", "unit", "ms_per_step", "iteration_time_stats", "ms_collect", "ms_update",
            "roofline", "tf32", "gpu_launches", "library_launches", "clocks", "status", "e2e",
            "layers")
    out = {k: line[k] for k in keep if k in line}
    out["workload"] = line["config"]["workload"]
    out["config"] = line["config"]
    return out


def run_all_configs(cx, with_error):
    """Every other workload of the benchmark set at its stated size, each
    timed like the headline (W >= 3 warm-up steps, L2 flushed before every
    timed step, CUDA events, its own clock record), with fewer timed steps:
    C1 (64 envs, latency), C2 (8192 envs, path following, with the path
    table rebuild), the C5 sweep (1024 .. 262144 envs, limit springs, 8
    substeps) with its 4096-env, 128-step adjoint, and P1 (PPO with
    learning)."""
    args = cx.args
    saved = (args.steps, args.warmup)
    args.steps, args.warmup = min(args.steps, 10), 3
    out = {"timed_steps_per_workload": args.steps, "warmup": args.warmup}
    try:
        line, _ = run_rollout_config(cx, "C1")
        out["C1"] = _compact_rollout(line)
        line, _ = run_rollout_config(cx, "C2")
        out["C2"] = _compact_rollout(line)
        out["C5"] = {"sweep": [_compact_rollout(run_rollout_config(cx, "C5", E)[0])
                               for E in (1024, 4096, 16384, 65536, 262144)]}
        out["C5"]["adjoint"] = _compact_adjoint(
            run_adjoint_config(cx, with_error=with_error, name="C5", E=4096, T=128, err_envs=4))
        out["P1"] = _compact_ppo(run_ppo_config(cx))
    finally:
        args.steps, args.warmup = saved
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores,
    on the default workload.  Every step is one bounded sample of the
    workload (the first envs of the batch, as many control steps as fit in
    its time slice); `value` is env-steps per second of the timed samples and
    `ms_per_step` the measured wall time of one sample (not an extrapolation
    to the whole batch)."""
    world, rank, local = dist_setup()
    if rank != 0:
        return
    from paper_2310_04676_gb300 import workloads as W
    wl = W.config("C3")
    per = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    runs = []
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = cpu_baseline(wl, seconds=per)
        r["wall_s"] = time.perf_counter() - t0
        runs.append(r)
    timed = runs[args.warmup:]
    v = float(np.median([r["value"] for r in timed]))
    cb = dict(timed[-1])
    cb["value"] = v
    wall = [r["wall_s"] for r in timed]
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * float(np.median(wall)),
            "step_is": "one bounded sample of the workload (%s)" % cb["sample"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl.name, "envs_per_gpu": wl.desc["num_envs"],
                       "rollout_steps": ROLLOUT_T["C3"], "substeps": wl.substeps, "dt": wl.dt,
                       "l2": "not applicable (host run)"},
            "form": "FP64 oracle (batched PyTorch, CPU) on the host cores",
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="C3", choices=["C1", "C2", "C3", "C4", "C5", "P1"])
    ap.add_argument("--envs", type=int, nargs="*", default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="default workload only (leave out the other workloads' `configs`)")
    ap.add_argument("--out-dir", default=None,
                    help="where the nvidia-smi clock samples go (default: a temporary directory)")
    ap.add_argument("--launch", default=None,
                    help="threads,mode,split: fixed launch plan instead of the autotuner "
                         "(used to profile one plan)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.launch:
        args.launch = tuple(int(x) for x in args.launch.split(","))
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    cx = Ctx(args, world, rank, local)
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline

    if args.config == "P1":
        line = run_ppo_config(cx)
        if rank == 0:
            print(json.dumps(line))
    elif args.config == "C4":
        g = run_adjoint_config(cx, with_error=want_cpu)
        if rank == 0:
            line = base_line(args, world, g["value"], g["ms_per_rollout"],
                             {"workload": g["workload"]})
            line["unit"] = g["unit"]
            line["grad"] = g
            line["roofline"] = g["roofline"]
            line["gpu_launches"] = g["gpu_launches"]
            line["clocks"] = g["clocks"]
            print(json.dumps(line))
    elif args.config == "C5" or args.envs:
        for E in (args.envs or [1024, 4096, 16384, 65536, 262144]):
            line, _ = run_rollout_config(cx, args.config, E)
            if rank == 0:
                print(json.dumps(line))
        if args.config == "C5" and not args.envs:
            # the sweep's adjoint runs: 4096 envs, horizon 128, limit springs, 8 substeps
            g = run_adjoint_config(cx, with_error=want_cpu, name="C5", E=4096, T=128, err_envs=4)
            if rank == 0:
                line = base_line(args, world, g["value"], g["ms_per_rollout"],
                                 {"workload": g["workload"]})
                line["unit"] = g["unit"]
                line["grad"] = g
                line["roofline"] = g["roofline"]
                line["gpu_launches"] = g["gpu_launches"]
                line["clocks"] = g["clocks"]
                print(json.dumps(line))
    else:
        line, wl = run_rollout_config(cx, args.config)
        if args.config == "C3":
            line["grad"] = run_adjoint_config(cx, with_error=want_cpu)
            if not args.headline_only:
                line["configs"] = run_all_configs(cx, with_error=want_cpu)
        if rank == 0:
            line["cpu_baseline"] = cpu_baseline(wl) if want_cpu else None
            if want_cpu:
                line["cpu_baseline"]["single_core"] = cpu_baseline_single_core(wl)
                launch = line["launch"]
                line["equal_accuracy"] = equal_accuracy(
                    wl, (launch["threads_per_block"],
                         {"persistent": 0, "step_graph": 1}[launch["mode"]],
                         launch["chain_split"]))
            print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
