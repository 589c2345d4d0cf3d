"""Pins of the oracle's observation, reward, done and reset semantics."""
import numpy as np
import torch

from oracle import dynamics as dyn
from oracle.env import OracleEnv, obs_dim
from paper_2310_04676_gb300 import workloads as W


def test_obs_layout_and_reach_reward():
    d = W.make_desc(["7R", "4R", "14B", "7P"])
    env = OracleEnv(d)
    assert obs_dim(d) == 54
    acts = W.joint_targets(d, 1)[0]
    obs, rew, done = env.step(acts, 1 / 60, 2)
    for e, kind in enumerate(["7R", "4R", "14B", "7P"]):
        nc = int(d["env_num_chains"][e])
        n = W.kind_dof(kind)
        o = obs[e]
        assert np.allclose(o[:n], env.q[e, :n]) and np.allclose(o[n:2 * n], env.qd[e, :n])
        ee = o[2 * n:2 * n + 3 * nc].reshape(nc, 3)
        assert np.allclose(o[2 * n + 3 * nc:3 * n + 3 * nc], acts[e, :n])
        goal = o[3 * n + 3 * nc:3 * n + 6 * nc].reshape(nc, 3)
        assert np.allclose(goal, d["goal"][e, :nc])
        assert np.all(o[3 * n + 6 * nc:] == 0)
        assert np.isclose(rew[e], -np.linalg.norm(ee - goal, axis=1).sum())
    assert (done == 0).all()


def test_timeout_bit_and_reset():
    d = W.make_desc(["7R"] * 3, episode_len=3)
    env = OracleEnv(d)
    acts = W.joint_targets(d, 4)
    for t in range(3):
        _, _, done = env.step(acts[t], 1 / 60, 2)
    assert (done == 2).all()
    q_before = env.q.copy()
    env.reset(np.array([0, 1, 0], np.uint8))
    assert (env.q[1] == d["q0"][1]).all() and (env.qd[1] == 0).all()
    assert (env.q[[0, 2]] == q_before[[0, 2]]).all()
    assert env.step_count.tolist() == [3, 0, 3]
    _, _, done = env.step(acts[3], 1 / 60, 2)
    assert done.tolist() == [2, 0, 2]


def test_nonfinite_bit():
    d = W.make_desc(["4R"] * 2)
    env = OracleEnv(d)
    acts = np.zeros((2, 4), np.float32)
    acts[1, 0] = np.nan
    _, _, done = env.step(acts, 1 / 60, 2)
    assert done.tolist() == [0, 4]


def test_path_following_obs_and_reward():
    W_ = 12
    d = W.make_desc(["7R"] * 3, task=1, path_len=W_, episode_len=10)
    env = OracleEnv(d)
    assert env.D == 30
    acts = W.joint_targets(d, 11)
    for t in range(11):
        obs, rew, _ = env.step(acts[t], 1 / 60, 4)
        k = t + 1
        path = env.path
        for e in range(3):
            o = obs[e]
            ee = o[14:17]
            quat = o[17:21]
            assert quat[3] >= 0 and np.isclose(np.linalg.norm(quat), 1.0)
            for j in range(3):
                assert np.allclose(o[21 + 3 * j:24 + 3 * j], path[e, min(k + 1 + j, W_ - 1)])
            assert np.isclose(rew[e], -np.linalg.norm(ee - path[e, min(k, W_ - 1)]))


def test_step_is_batch_and_permutation_invariant():
    kinds = ["7R", "4R", "14B", "7P", "7R"]
    d = W.make_desc(kinds)
    perm = np.array([3, 0, 4, 2, 1])
    dp = {k: (v[perm] if isinstance(v, np.ndarray) and v.shape[:1] == (5,) else v)
          for k, v in d.items()}
    a = W.joint_targets(d, 2)
    e1, e2 = OracleEnv(d), OracleEnv(dp)
    for t in range(2):
        o1, r1, _ = e1.step(a[t], 1 / 60, 2)
        o2, r2, _ = e2.step(a[t][perm], 1 / 60, 2)
    assert np.array_equal(o1[perm], o2) and np.array_equal(r1[perm], r2)
