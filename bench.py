#!/usr/bin/env python
"""Benchmark of the batched articulated-arm step on one GB300 (or N replicas).

Workload (default): 16384 heterogeneous environments -- 25% 4-DOF revolute
arms, 40% 7-DOF revolute, 20% 7-DOF with a prismatic insertion joint, 15%
14-DOF two-arm robots -- reach task, dt = 1/60 s, 2 substeps.  One bench
step is one 32-step rollout of every env (32 x 16384 env-steps), issued as
the autotuned persistent kernel captured in a CUDA graph.  The plain
one-kernel-per-step launch runs the same rollout on the same inputs from
the same state and is reported beside it; both produce identical bits.

Metric: env-steps/s (aggregate over all ranks).  Timing: CUDA events on the
launching stream, W warm-up steps, K timed steps, L2 flushed (a 256 MiB
write) before every timed step, max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s at 16k mixed-DOF envs, batched vs plain; % FP32 roofline; grad err"
T_ROLLOUT = 32

# Algorithmic FP32 operations of the step's formulation (an FMA counts 2),
# counted by a counting-scalar run of the chain code: per substep of one
# chain, and per step for the tool-tip kinematics of one chain.
FLOP_SUBSTEP = {"4R": 774, "7R": 1697, "7P": 1580}
FLOP_TIP = {"4R": 96, "7R": 168, "7P": 156}
FLOP_REWARD = 9        # distance to the goal (per chain)


def env_step_flops(kinds, substeps):
    tot = 0
    for k in kinds:
        chains = ["7R", "7R"] if k == "14B" else [k]
        for c in chains:
            tot += substeps * FLOP_SUBSTEP[c] + FLOP_TIP[c] + FLOP_REWARD
    return tot


def env_step_bytes(desc, obs_dim):
    """Algorithmic HBM bytes of one env-step in the persistent rollout:
    action row read, observation row, reward and done written."""
    E = desc["num_envs"]
    dof = desc["chain_num_joints"].sum(1)
    return int(4 * dof.sum() + E * (4 * obs_dim + 4 + 1))


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

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
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
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_baseline(wl, seconds=12.0):
    """The FP64 oracle as it stands on this host's cores, on a bounded sample
    of the workload (a fixed subset of envs, as many steps as fit)."""
    import torch
    from oracle.env import OracleEnv
    from paper_2310_04676_gb300 import workloads as W
    E = wl.desc["num_envs"]
    n_sample = min(E, 2048)
    pick = np.arange(n_sample)
    sub = {k: (v[pick] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
           for k, v in wl.desc.items()}
    sub["num_envs"] = n_sample
    env = OracleEnv(sub)
    acts = W.joint_targets(sub, 64)
    env.step(acts[0], wl.dt, wl.substeps)        # first step excluded, as the paper times
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds and steps < 63:
        env.step(acts[1 + steps], wl.dt, wl.substeps)
        steps += 1
    el = time.perf_counter() - t0
    return {"value": n_sample * steps / el, "unit": "env-steps/s", "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": "%d of %d envs (same kind mix), %d steps, FP64 PyTorch CPU, %.1f s"
                      % (n_sample, E, steps, el)}


def run_reference(args):
    world, rank, local = dist_setup()
    if rank != 0:
        return
    from paper_2310_04676_gb300 import workloads as W
    wl = W.config("C3")
    vals = []
    samples = []
    per = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(wl, seconds=per)
        if i >= args.warmup:
            vals.append(cb["value"])
            samples.append(cb)
    v = float(np.median(vals))
    cb = dict(samples[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * T_ROLLOUT * wl.desc["num_envs"] / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl.name, "rollout_steps": T_ROLLOUT,
                                            "substeps": wl.substeps, "dt": wl.dt},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2310_04676_gb300 import sg, workloads as W

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    wl = W.config("C3")
    desc = wl.desc
    if rank:
        # independent replica per rank: its own link parameters and goals
        desc = W.make_desc(wl.kinds, seed_params=1 + 1000 * rank, seed_goals=3 + 1000 * rank,
                           episode_len=1000)
    E = desc["num_envs"]
    T, S, dt = T_ROLLOUT, wl.substeps, wl.dt
    acts = torch.as_tensor(W.joint_targets(desc, T, seed=2 + 1000 * rank), device=dev)
    stream = torch.cuda.current_stream()

    env = sg.Env(desc)                 # persistent kernel in a CUDA graph (autotuned)
    sgraph = sg.Env(desc)              # T single-step kernels replayed from a CUDA graph
    plain = sg.Env(desc)               # T sg_step calls from the host
    out = env.empty_outputs(T)
    out_g = sgraph.empty_outputs(T)
    out_p = plain.empty_outputs(T)
    threads, mode, split, tune_ms = env.autotune(acts, dt, S, out=out, repeats=3)
    sgraph.set_launch(threads, sg.ROLLOUT_STEP_GRAPH, split)
    plain.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def plain_rollout():
        o, r, d = out_p
        for t in range(T):
            plain.step(acts[t], dt, S, out=(o[t], r[t], d[t]))

    forms = {
        "ours": lambda: env.rollout(acts, dt, S, out=out),
        "step_graph": lambda: sgraph.rollout(acts, dt, S, out=out_g),
        "plain": plain_rollout,
    }
    for _ in range(args.warmup):
        for f in forms.values():
            f()
    barrier()

    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
    clk = ClockSampler(os.path.join(ROOT, "gpurun_out", "clocks_r%d.csv" % rank), local)

    def timed(fn, sampler=None):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        barrier()
        if sampler:
            sampler.__enter__()
        for k in range(args.steps):
            flush.zero_()                       # L2 flush, outside the timed events
            evs[k][0].record(stream)
            fn()
            evs[k][1].record(stream)
        barrier()
        if sampler:
            sampler.__exit__(None, None, None)
        return [a.elapsed_time(b) for a, b in evs]

    ms = timed(forms["ours"], clk)
    ms_g = timed(forms["step_graph"])
    ms_p = timed(forms["plain"])
    t_ours, t_graph, t_plain = sum(ms) / 1e3, sum(ms_g) / 1e3, sum(ms_p) / 1e3

    # identical arithmetic: all forms ran the same rollouts from the same state
    qa, qda, _ = env.get_state()
    same_bits = True
    for other, o2 in ((sgraph, out_g), (plain, out_p)):
        qb, qdb, _ = other.get_state()
        same_bits = same_bits and bool(torch.equal(qa, qb) and torch.equal(qda, qdb)
                                       and torch.equal(out[0], o2[0]))
    status = env.sync_status()

    # ---- end to end through the C ABI with host buffers
    env_h = sg.Env(desc)
    env_h.set_launch(threads, mode, split)
    a_h = acts.cpu().pin_memory()
    o_h = (torch.empty(T, E, env_h.obs_dim).pin_memory(), torch.empty(T, E).pin_memory(),
           torch.empty(T, E, dtype=torch.uint8).pin_memory())
    for _ in range(args.warmup):
        env_h.rollout_host(a_h, dt, S, o_h)
    barrier()
    eve = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        eve[k][0].record(stream)
        env_h.rollout_host(a_h, dt, S, o_h)
        eve[k][1].record(stream)
    barrier()
    t_e2e = sum(a.elapsed_time(b) for a, b in eve) / 1e3
    h2d = T * E * env_h.max_joints * 4
    d2h = T * E * (env_h.obs_dim * 4 + 4 + 1)

    # ---- aggregate over ranks (max time)
    def rmax(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    t_ours, t_graph, t_plain, t_e2e = rmax(t_ours), rmax(t_graph), rmax(t_plain), rmax(t_e2e)
    units = world * E * T * args.steps
    value = units / t_ours

    peaks, peak_src = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12
    flops_launch = env_step_flops(wl.kinds if rank == 0 else wl.kinds, S) * T
    kernel_s = (sum(ms) / len(ms)) / 1e3
    achieved = flops_launch / kernel_s / 1e12
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if os.path.exists(tfile):
        with open(tfile) as f:
            tj = json.load(f)
        if tj.get("kernel_source_hash") == _source_hash():
            traffic = tj.get("bytes_per_launch")

    if rank == 0:
        cb = None if (args.no_cpu_baseline or world > 1) else cpu_baseline(wl)
        line = {
            "metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_ours / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": wl.name, "envs_per_gpu": E, "rollout_steps": T,
                       "substeps": S, "dt": dt, "form": "persistent kernel in a CUDA graph",
                       "launch": {"threads_per_block": threads,
                                  "mode": ["persistent", "step_graph"][mode],
                                  "chain_split": split},
                       "l2": "flushed (256 MiB write) before every timed step"},
            "plain": {"value": world * E * T * args.steps / t_plain, "unit": "env-steps/s",
                      "ms_per_step": 1e3 * t_plain / args.steps,
                      "form": "one sg_step call (one kernel launch) per control step",
                      "gpu_launches": T * args.steps},
            "step_graph": {"value": world * E * T * args.steps / t_graph, "unit": "env-steps/s",
                           "ms_per_step": 1e3 * t_graph / args.steps,
                           "form": "32 single-step kernels replayed from a CUDA graph",
                           "gpu_launches": T * args.steps},
            "batched_over_plain": t_plain / t_ours,
            "batched_over_step_graph": t_graph / t_ours,
            "bitwise_equal_forms": same_bits,
            "status": sg.STATUS_NAMES.get(status, status),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_tflops,
                         "unit": "TFLOP/s", "frac": achieved / peak_tflops, "traffic": traffic,
                         "kernel": "%s (persistent, T=32)" % (
                             "step_kernel_pair" if split == 2 else "step_kernel"),
                         "peak_source": "SMs x 128 FP32 lanes x 2 x %.0f MHz (%s max clock)"
                                        % (sm_max, peak_src),
                         "flops_per_launch": flops_launch,
                         "hbm_gbs": env_step_bytes(desc, env.obs_dim) * T / kernel_s / 1e9},
            "e2e": {"value": units / t_e2e, "unit": "env-steps/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cb,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def _source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("sg_chain.cuh", "sg_kernels.cu"):
        with open(os.path.join(ROOT, "paper_2310_04676_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
