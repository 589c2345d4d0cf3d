"""Environment-level oracle: observation, reward, done, reset and step.

Follows the paper's task definitions (Results, "Environments"):

* base observation = concat(joint positions, joint velocities, tool-tip
  position, current PD targets) (Methods, "Observation Space"), plus the
  goal for the goal tasks;
* Target Reaching reward  r = rho * ||eta_t - g|| with rho = -1 (the sign
  is a reading: the paper leaves rho's sign open);
* Multi-Tool Target Reaching reward r = rho * sum_i ||eta_i - g_i||;
* Path Following reward r = -alpha * ||eta_t - P(t)||, observation
  [q, qd, tip position, tip quaternion, next three waypoints];
* Active Tracking: reaching with goals that move every step,
  g = g0 + d, d <- clamp(d + v, +-limit), v <- v + sigma N(0, 1) (the
  paper's random walk of the goal position and velocity with a maximum
  offset; its noise variance "1^{-4}" is read as 1e-4, i.e. sigma = 0.01);
* time-outs are reported apart from terminations (Methods, "Policy
  learning and control").

Observation layouts (n = total DOF, nc = number of chains):
  reach, tracking: [q(n), qd(n), tip_c(3) for each chain, q*(n), goal_c(3) for each chain]
  path:  [q(n), qd(n), tip(3), quat(4) as (x, y, z, w) with w >= 0,
          waypoint[t+1], waypoint[t+2], waypoint[t+3]]
padded with zeros to the widest env of the batch.  Done bits: bit0 =
terminated (reserved, never set), bit1 = time-out (step count reached the
episode length), bit2 = non-finite state.
"""
import numpy as np
import torch

from . import dynamics as dyn
from . import path as path_mod
from .model import PRISMATIC, groups, make_params
from .rng import goal_noise
from .spatial import DT


def obs_dim_of(desc, e):
    nc = int(desc["env_num_chains"][e])
    n = int(desc["chain_num_joints"][e, :nc].sum())
    if int(desc["task"]) == 1:
        return 2 * n + 16
    return 3 * n + 6 * nc


def obs_dim(desc):
    return max(obs_dim_of(desc, e) for e in range(int(desc["num_envs"])))


def tip_quaternion(tree, q):
    """World orientation of each chain's tip link as the Hamilton product of
    the per-joint axis-angle quaternions (independent of the rotation
    matrices of ``dynamics.fk``), returned as (x, y, z, w) with w >= 0."""
    E = q.shape[0]
    out = []
    for tip in tree.tips:
        chain = tree.chain_of[tip]
        Q = torch.zeros(E, 4, dtype=DT)
        Q[:, 0] = 1.0                                  # (w, x, y, z)
        for i in range(tree.n):
            if tree.chain_of[i] != chain or tree.jtype[i] == PRISMATIC:
                continue
            half = 0.5 * q[:, i]
            r = torch.zeros(E, 4, dtype=DT)
            r[:, 0] = torch.cos(half)
            r[:, 1 + tree.axis[i]] = torch.sin(half)
            w1, x1, y1, z1 = Q.unbind(-1)
            w2, x2, y2, z2 = r.unbind(-1)
            Q = torch.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                             w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                             w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                             w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], -1)
        sign = torch.where(Q[:, 0] < 0, -1.0, 1.0).to(DT)
        Q = Q * sign[:, None]
        out.append(torch.stack([Q[:, 1], Q[:, 2], Q[:, 3], Q[:, 0]], -1))
    return torch.stack(out, 1)


class OracleEnv:
    """Batched reference environment with FP64 state."""

    def __init__(self, desc):
        self.desc = desc
        self.E = int(desc["num_envs"])
        self.J = int(desc["max_joints"])
        self.task = int(desc["task"])
        self.D = obs_dim(desc)
        self.groups = []
        for idx, tree in groups(desc):
            self.groups.append((idx, tree, make_params(tree, desc, idx)))
        self.q = np.zeros((self.E, self.J))
        self.qd = np.zeros((self.E, self.J))
        self.step_count = np.zeros(self.E, np.int64)
        self.goal_off = np.zeros((self.E, 4, 3))     # tracking task: goal offset, velocity
        self.goal_vel = np.zeros((self.E, 4, 3))
        self.path = None                             # path task: waypoint tables [E, W, 3]
        if self.task == 1:
            W = int(desc["path_len"])
            if desc.get("path") is not None:
                self.path = np.asarray(desc["path"], np.float64).reshape(self.E, W, 3).copy()
            else:
                self.path = path_mod.waypoints(desc["path_ctrl"], W)
        self.reset()

    def set_paths(self, ctrl, mask=None):
        """New waypoint tables for the envs in ``mask`` from control points [E, K, 3]."""
        m = np.ones(self.E, bool) if mask is None else np.asarray(mask).astype(bool)
        if m.any():
            self.path[m] = path_mod.waypoints(np.asarray(ctrl)[m], self.path.shape[1])

    # -- state -------------------------------------------------------------
    def reset(self, mask=None):
        m = np.ones(self.E, bool) if mask is None else np.asarray(mask).astype(bool)
        self.q[m] = np.asarray(self.desc["q0"], np.float64)[m]
        self.qd[m] = 0.0
        self.step_count[m] = 0
        self.goal_off[m] = 0.0
        self.goal_vel[m] = 0.0

    def set_state(self, q, qd, step_count=None):
        self.q = np.array(q, np.float64, copy=True)
        self.qd = np.array(qd, np.float64, copy=True)
        if step_count is not None:
            self.step_count = np.array(step_count, np.int64, copy=True)

    # -- one control step --------------------------------------------------
    def step(self, actions, dt, substeps):
        """Advance every env by one control step of ``substeps`` substeps.
        Returns (obs [E][D], reward [E], done [E] uint8)."""
        actions = np.asarray(actions, np.float64)
        h = dt / substeps
        obs = np.zeros((self.E, self.D))
        reward = np.zeros(self.E)
        done = np.zeros(self.E, np.uint8)
        self.step_count += 1
        if self.task == 2:
            self._move_goals()
        for idx, tree, P in self.groups:
            n = tree.n
            q = torch.as_tensor(self.q[idx, :n])
            qd = torch.as_tensor(self.qd[idx, :n])
            qs = torch.as_tensor(actions[idx, :n])
            for _ in range(substeps):
                q, qd, _ = dyn.substep(tree, P, q, qd, qs, h)
            self.q[idx, :n] = q.numpy()
            self.qd[idx, :n] = qd.numpy()
            o, r = self._obs_reward(idx, tree, P, q, qd, qs)
            obs[idx, : o.shape[1]] = o
            reward[idx] = r
        done[self.step_count >= int(self.desc["episode_len"])] |= 2
        bad = ~np.isfinite(self.q).all(1) | ~np.isfinite(self.qd).all(1)
        done[bad] |= 4
        return obs, reward, done

    def observe(self, targets, mask=None):
        """Observation rows [E][D] of the current state with ``targets`` as the
        current commands, without advancing time (rows outside ``mask`` are
        returned as NaN)."""
        targets = np.asarray(targets, np.float64)
        m = np.ones(self.E, bool) if mask is None else np.asarray(mask).astype(bool)
        obs = np.full((self.E, self.D), np.nan)
        for idx, tree, P in self.groups:
            n = tree.n
            o, _ = self._obs_reward(idx, tree, P, torch.as_tensor(self.q[idx, :n]),
                                    torch.as_tensor(self.qd[idx, :n]),
                                    torch.as_tensor(targets[idx, :n]))
            rows = np.zeros((len(idx), self.D))
            rows[:, : o.shape[1]] = o
            sel = m[idx]
            obs[idx[sel]] = rows[sel]
        return obs

    def _move_goals(self):
        """One random-walk step of every chain's goal (tracking task)."""
        nc = np.asarray(self.desc["env_num_chains"])
        lim = float(self.desc["track_limit"])
        sig = float(self.desc["track_sigma"])
        env = np.arange(self.E)[:, None]
        chain = np.arange(4)[None, :]
        z = goal_noise(int(self.desc["seed"]), env, chain, self.step_count[:, None])
        has = (chain < nc[:, None])[..., None]
        self.goal_off = np.where(has, np.clip(self.goal_off + self.goal_vel, -lim, lim), 0.0)
        self.goal_vel = np.where(has, self.goal_vel + sig * z, 0.0)

    def goals(self, idx, nc):
        g = np.asarray(self.desc["goal"], np.float64)[idx][:, :nc]
        if self.task == 2:
            g = g + self.goal_off[idx][:, :nc]
        return g

    def _obs_reward(self, idx, tree, P, q, qd, qs):
        ee, _ = dyn.end_effectors(tree, P, q)                    # [E, nc, 3]
        nc = tree.n_chains
        if self.task == 1:
            W = int(self.desc["path_len"])
            path = self.path[idx]                                  # [E, W, 3]
            t = self.step_count[idx]
            wp = lambda k: torch.as_tensor(path[np.arange(len(idx)), np.minimum(t + k, W - 1)])
            quat = tip_quaternion(tree, q)[:, 0]
            o = torch.cat([q, qd, ee[:, 0], quat, wp(1), wp(2), wp(3)], -1)
            r = -float(self.desc["alpha"]) * torch.linalg.norm(ee[:, 0] - wp(0), dim=-1)
        else:
            goal = torch.as_tensor(self.goals(idx, nc))
            o = torch.cat([q, qd, ee.reshape(len(idx), -1), qs, goal.reshape(len(idx), -1)], -1)
            r = -torch.linalg.norm(ee - goal, dim=-1).sum(-1)
        return o.numpy(), r.numpy()


def ee_rollout(desc, actions, dt, substeps, q0=None, qd0=None, mass=None, env_idx=None):
    """Differentiable FP64 rollout of single-structure envs: returns the
    tool-tip positions after every control step, [T, E, nc, 3].

    ``actions`` is a float64 tensor [T, E, n] (may require grad); ``mass`` an
    optional float64 tensor [E, n] (may require grad) that replaces the link
    masses (inertias scale with it).  All envs of ``env_idx`` (default: all)
    must share one structure.
    """
    gs = groups(desc)
    if env_idx is None:
        assert len(gs) == 1, "ee_rollout needs envs of a single structure"
        env_idx, tree = gs[0]
    else:
        env_idx = np.asarray(env_idx)
        tree = [t for idx, t in gs if np.isin(env_idx, idx).all()][0]
    P = make_params(tree, desc, env_idx, mass=mass)
    n = tree.n
    E = len(env_idx)
    q = torch.zeros(E, n, dtype=DT) if q0 is None else torch.as_tensor(q0, dtype=DT)
    qd = torch.zeros(E, n, dtype=DT) if qd0 is None else torch.as_tensor(qd0, dtype=DT)
    h = dt / substeps
    out = []
    for t in range(actions.shape[0]):
        for _ in range(substeps):
            q, qd, _ = dyn.substep(tree, P, q, qd, actions[t], h)
        out.append(dyn.end_effectors(tree, P, q)[0])
    return torch.stack(out, 0)


__all__ = ["OracleEnv", "obs_dim", "obs_dim_of", "tip_quaternion", "ee_rollout"]
