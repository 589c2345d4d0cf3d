"""Seeded synthetic robot workloads for the batched articulated-arm step.

The paper's robots (dVRK PSM/ECM, STAR) are described by asset files that
are not available, so a seeded family of serial arms stands in for them
(Methods, "Robot Descriptions": PSM/ECM joint order RRPRRR, STAR all
revolute; Results, "Multi-Tool Target Reaching": two-arm variants).

This module only builds *inputs*: per-environment robot descriptions
(link lengths, masses, box inertias, joint axes and limits, drive gains),
goals, path control points and joint-target action sequences.
It holds none of the dynamics.  Both the CUDA path and the FP64 oracle
consume exactly the arrays produced here.

Every array follows the layout of ``sg_desc`` in ``include/sg.h``:
per-joint arrays are ``[E][J]`` row-major with the joints of chain 0
first, then the joints of chain 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BOX_WIDTH = 0.05          # side of the square link cross-section [m]
GRAVITY = 9.81

# Joint structure of the four arm kinds.  Axis codes: 0=x, 1=y, 2=z;
# type codes: 0=revolute, 1=prismatic (along local z).
_AXES7 = [2, 1, 2, 1, 2, 1, 2]
KINDS = {
    "4R": dict(chains=[(4, [0] * 4, _AXES7[:4])]),
    "7R": dict(chains=[(7, [0] * 7, _AXES7)]),
    "7P": dict(chains=[(7, [0, 0, 1, 0, 0, 0, 0], _AXES7)]),
    "14B": dict(chains=[(7, [0] * 7, _AXES7), (7, [0] * 7, _AXES7)]),
    # three-arm (two instrument arms and a camera arm, all with the
    # RRP... insertion structure of the paper's PSM / ECM)
    "21T": dict(chains=[(7, [0, 0, 1, 0, 0, 0, 0], _AXES7)] * 3),
}
MAX_CHAINS = 4
BIMANUAL_BASE_Y = 0.25
TRIMANUAL_BASES = [(0.0, 0.3, 0.0), (0.0, -0.3, 0.0), (-0.2, 0.0, 0.0)]


def kind_dof(kind: str) -> int:
    return sum(c[0] for c in KINDS[kind]["chains"])


@dataclass
class Workload:
    """A batch description plus the run settings of one workload."""
    desc: dict            # sg_desc fields as numpy arrays / scalars
    kinds: list           # arm kind per env
    dt: float
    substeps: int
    steps: int
    name: str


def _box_inertia(m, L, w=BOX_WIDTH):
    ixx = m * (L * L + w * w) / 12.0
    izz = m * (w * w) / 12.0
    return ixx, ixx, izz


def make_desc(kinds, *, seed_params=1, seed_goals=3, shared_params=False,
              k_limit=0.0, kp=50.0, kd=5.0, damping=0.1, episode_len=1000,
              task=0, path_len=0, alpha=1.0, max_joints=None, drive=None, seed=7,
              track_sigma=0.01, track_limit=0.2):
    """Build an ``sg_desc`` dictionary for a list of arm kinds (one per env).

    ``drive`` selects the joint command type (0 position target, 1 velocity
    target, 2 torque): None (all position), an int, or an [E][J] array.

    Link lengths ~ U[0.05, 0.4] m and masses ~ U[0.1, 1.0] kg per link,
    solid-box inertias of width BOX_WIDTH, COM at mid-length, revolute
    limits +-pi/2 and prismatic range [0, 0.2] m.  With ``shared_params``
    every env uses the first env's link draw.
    """
    E = len(kinds)
    J = max_joints or max(kind_dof(k) for k in kinds)
    rp = np.random.default_rng(seed_params)
    rg = np.random.default_rng(seed_goals)

    f32 = np.float32
    d = dict(num_envs=E, max_joints=J, episode_len=int(episode_len), task=int(task),
             alpha=float(alpha), seed=int(seed), track_sigma=float(track_sigma),
             track_limit=float(track_limit))
    d["env_num_chains"] = np.zeros(E, np.int32)
    d["chain_num_joints"] = np.zeros((E, MAX_CHAINS), np.int32)
    for name in ("joint_type", "joint_axis"):
        d[name] = np.zeros((E, J), np.int32)
    for name in ("link_len", "link_mass", "link_com", "q_lo", "q_hi", "kp", "kd",
                 "damping", "k_limit", "q0"):
        d[name] = np.zeros((E, J), f32)
    d["link_inertia"] = np.zeros((E, J, 3), f32)
    d["base_offset"] = np.zeros((E, MAX_CHAINS, 3), f32)
    d["goal"] = np.zeros((E, MAX_CHAINS, 3), f32)

    shared_L = rp.uniform(0.05, 0.4, size=7 * MAX_CHAINS)
    shared_m = rp.uniform(0.1, 1.0, size=7 * MAX_CHAINS)
    for e, kind in enumerate(kinds):
        chains = KINDS[kind]["chains"]
        d["env_num_chains"][e] = len(chains)
        if shared_params:
            Ls, ms = shared_L, shared_m
        elif len(chains) <= 2:
            # (draw size kept for one- and two-arm envs: their seeded inputs
            # are unchanged by the wider arrays)
            Ls = rp.uniform(0.05, 0.4, size=14)
            ms = rp.uniform(0.1, 1.0, size=14)
        else:
            Ls = rp.uniform(0.05, 0.4, size=7 * MAX_CHAINS)
            ms = rp.uniform(0.1, 1.0, size=7 * MAX_CHAINS)
        j0 = 0
        for c, (n, types, axes) in enumerate(chains):
            d["chain_num_joints"][e, c] = n
            if len(chains) == 2:
                d["base_offset"][e, c] = (0.0, BIMANUAL_BASE_Y if c == 0 else -BIMANUAL_BASE_Y, 0.0)
            elif len(chains) == 3:
                d["base_offset"][e, c] = TRIMANUAL_BASES[c]
            reach = 0.0
            for i in range(n):
                j = j0 + i
                L = float(Ls[(7 * c + i) if not shared_params else i])
                m = float(ms[(7 * c + i) if not shared_params else i])
                reach += L
                d["joint_type"][e, j] = types[i]
                d["joint_axis"][e, j] = axes[i]
                d["link_len"][e, j] = L
                d["link_mass"][e, j] = m
                d["link_com"][e, j] = L / 2.0
                d["link_inertia"][e, j] = _box_inertia(m, L)
                if types[i] == 1:
                    d["q_lo"][e, j], d["q_hi"][e, j] = 0.0, 0.2
                else:
                    d["q_lo"][e, j], d["q_hi"][e, j] = -math.pi / 2, math.pi / 2
                d["kp"][e, j] = kp
                d["kd"][e, j] = kd
                d["damping"][e, j] = damping
                d["k_limit"][e, j] = k_limit
            # goal: uniform in a 0.3 m cube centred at (0.3R, 0, 0.5R) from the chain base
            centre = np.array([0.3 * reach, 0.0, 0.5 * reach]) + d["base_offset"][e, c]
            d["goal"][e, c] = centre + rg.uniform(-0.15, 0.15, size=3)
            j0 += n
    if drive is not None:
        # joint command type: one code for all joints, or an [E][J] array
        d["joint_drive"] = np.broadcast_to(np.asarray(drive, np.int32), (E, J)).copy()
    if task == 1:
        if any(len(KINDS[k]["chains"]) != 1 for k in kinds):
            raise ValueError("path following is defined for single-chain arms")
        d["path_len"] = int(path_len)          # waypoints the library builds per env
        d["path_ctrl"] = make_path_ctrl(d, rg)
        d["path_ctrl_len"] = d["path_ctrl"].shape[1]
        d["path"] = None
    else:
        d["path_len"] = 0
        d["path"] = None
    return d


def make_path_ctrl(d, rng, npts=16):
    """Control points [E][npts][3] of each env's path: uniform in a 0.3 m cube
    centred at (0.3R, 0, 0.5R), R the arm's reach (the library builds the
    spline and the waypoint table from them)."""
    E = d["num_envs"]
    ctrl = np.zeros((E, npts, 3), np.float32)
    for e in range(E):
        reach = float(d["link_len"][e, : d["chain_num_joints"][e, 0]].sum())
        centre = np.array([0.3 * reach, 0.0, 0.5 * reach])
        ctrl[e] = centre + rng.uniform(-0.15, 0.15, size=(npts, 3))
    return ctrl


def joint_targets(desc, T, *, seed=2, resample_every=50, t0=0):
    """Joint-target actions [T][E][J] drawn U[q_lo, q_hi] per joint,
    redrawn every ``resample_every`` steps (counted from ``t0``).

    The paper's benchmark drives the simulator with random actions
    (Results, "Simulator Performance Comparison"); here they are PD
    position targets within the joint limits.
    """
    E, J = desc["num_envs"], desc["max_joints"]
    lo = desc["q_lo"].astype(np.float64)
    hi = desc["q_hi"].astype(np.float64)
    out = np.zeros((T, E, J), np.float32)
    cache = {}
    for t in range(T):
        blk = (t0 + t) // resample_every
        if blk not in cache:
            r = np.random.default_rng([seed, blk])
            u = r.random((E, J))
            cache[blk] = (lo + u * (hi - lo)).astype(np.float32)
        out[t] = cache[blk]
    # padding joints beyond each env's DOF stay zero
    return out


def mixed_kinds(E, fractions, seed=4):
    """Env kinds for a heterogeneous batch: counts by largest-remainder
    rounding (ties in listed order), then a seeded permutation so that the
    kinds are interleaved in caller env order."""
    names = list(fractions)
    raw = np.array([fractions[k] * E for k in names])
    cnt = np.floor(raw).astype(int)
    rem = raw - cnt
    order = sorted(range(len(names)), key=lambda i: (-rem[i], i))
    for i in order[: E - cnt.sum()]:
        cnt[i] += 1
    kinds = []
    for k, c in zip(names, cnt):
        kinds += [k] * int(c)
    perm = np.random.default_rng(seed).permutation(E)
    return [kinds[i] for i in perm]


C3_FRACTIONS = {"4R": 0.25, "7R": 0.40, "7P": 0.20, "14B": 0.15}


def config(name, num_envs=None):
    """The five benchmark workloads (C1..C5) with their stated sizes."""
    if name == "C1":
        E = num_envs or 64
        d = make_desc(["7R"] * E, shared_params=True, episode_len=1000)
        return Workload(d, ["7R"] * E, 1.0 / 60.0, 2, 1000, "C1 reach 7R x%d" % E)
    if name == "C2":
        E = num_envs or 8192
        d = make_desc(["7R"] * E, task=1, path_len=500 + 3, episode_len=500)
        return Workload(d, ["7R"] * E, 1.0 / 60.0, 4, 500, "C2 path-follow 7R x%d" % E)
    if name == "C3":
        E = num_envs or 16384
        kinds = mixed_kinds(E, C3_FRACTIONS)
        d = make_desc(kinds, episode_len=1000)
        return Workload(d, kinds, 1.0 / 60.0, 2, 32, "C3 mixed 4R/7R/7P/14B x%d" % E)
    if name == "C4":
        E = num_envs or 2048
        d = make_desc(["7R"] * E, episode_len=1000)
        return Workload(d, ["7R"] * E, 1.0 / 60.0, 2, 64, "C4 adjoint 7R x%d" % E)
    if name == "C5":
        E = num_envs or 16384
        d = make_desc(["7R"] * E, k_limit=1e3, episode_len=1000)
        return Workload(d, ["7R"] * E, 1.0 / 60.0, 8, 1000, "C5 limits 7R x%d" % E)
    raise KeyError(name)


def loss_targets(desc, T, seed=5):
    """Per-env, per-chain EE targets [T][E][4][3], constant over the horizon
    (seeded; a draw in the same cube as the reaching goals)."""
    E = desc["num_envs"]
    r = np.random.default_rng(seed)
    g = desc["goal"].astype(np.float64) + r.uniform(-0.05, 0.05, size=(E, MAX_CHAINS, 3))
    return np.broadcast_to(g.astype(np.float32), (T, E, MAX_CHAINS, 3)).copy()


# ---- PPO inputs: initial network parameters and minibatch permutations ------
PPO_HIDDEN = (256, 128, 64)


def ppo_param_sizes(D, A):
    """Sizes of the flat parameter vector's pieces in order (actor W, b per
    layer, log_std, critic W, b per layer) with their fan-in (0: log_std)."""
    dims = (D,) + PPO_HIDDEN
    out = []
    for net_out in (A, 1):
        for i in range(4):
            fan_in, fan_out = dims[i], (dims[i + 1] if i < 3 else net_out)
            out += [(fan_out * fan_in, fan_in), (fan_out, fan_in)]
        if net_out == A:
            out.append((A, 0))
    return out


def ppo_init_params(D, A, seed=11):
    """Seeded initial parameters: weights and biases U(-1/sqrt(fan_in),
    1/sqrt(fan_in)) (the common default for linear layers), log_std = 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for n, fan_in in ppo_param_sizes(D, A):
        if fan_in == 0:
            parts.append(np.zeros(n))
        else:
            k = 1.0 / math.sqrt(fan_in)
            parts.append(rng.uniform(-k, k, size=n))
    return np.concatenate(parts).astype(np.float32)


def ppo_perms(B, epochs, seed=13, iteration=0):
    """Minibatch permutations [epochs][B] (int32) of one update."""
    rng = np.random.default_rng([seed, iteration])
    return np.stack([rng.permutation(B) for _ in range(epochs)]).astype(np.int32)


def ppo_config(name="P1", num_envs=None):
    """The with-learning workload: PPO on a reaching batch of 7-DOF
    insertion-joint arms (the PSM stand-in), 24 steps per env per update,
    5 epochs of 4 minibatches."""
    if name != "P1":
        raise KeyError(name)
    E = num_envs or 16384
    d = make_desc(["7P"] * E, episode_len=250)
    return Workload(d, ["7P"] * E, 1.0 / 60.0, 2, 24, "P1 PPO reach 7P x%d" % E)
