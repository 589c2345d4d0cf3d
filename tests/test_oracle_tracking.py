"""Pins of the tracking task's generator and goal random walk (no GPU)."""
import numpy as np

from oracle.env import OracleEnv
from oracle.rng import goal_noise, mix64, splitmix64_next
from paper_2310_04676_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    """SplitMix64 from state 0 (Steele, Lea and Flood 2014; the published
    reference generator): first outputs."""
    s = np.uint64(0)
    outs = []
    for _ in range(3):
        s, o = splitmix64_next(s)
        outs.append(int(o))
    assert outs[0] == 0xE220A8397B1DCDAF
    assert outs[1] == 0x6E789E6AA1B965F4
    assert outs[2] == 0x06C45D188009454F


def test_goal_noise_is_standard_normal_and_counter_based():
    env = np.arange(20000)
    z = goal_noise(11, env[:, None], np.arange(3)[None, :], 5)     # [E, 3, 3]
    flat = z.reshape(-1)
    assert abs(flat.mean()) < 0.02 and abs(flat.std() - 1.0) < 0.02
    # same counters, same draws; any other counter, different draws
    assert np.array_equal(goal_noise(11, 7, 1, 5), goal_noise(11, 7, 1, 5))
    for other in (goal_noise(12, 7, 1, 5), goal_noise(11, 8, 1, 5), goal_noise(11, 7, 2, 5),
                  goal_noise(11, 7, 1, 6)):
        assert not np.allclose(other, goal_noise(11, 7, 1, 5))


def test_goal_random_walk_order_clamp_and_reset():
    d = W.make_desc(["7R", "14B"], task=2, track_sigma=0.05, track_limit=0.1)
    env = OracleEnv(d)
    acts = W.joint_targets(d, 60)
    off, vel = np.zeros((2, 4, 3)), np.zeros((2, 4, 3))
    for t in range(60):
        obs, rew, _ = env.step(acts[t], 1 / 60, 2)
        z = goal_noise(d["seed"], np.arange(2)[:, None], np.arange(4)[None, :], t + 1)
        off = np.clip(off + vel, -0.1, 0.1)             # position first, with the old velocity
        vel = vel + 0.05 * z
        off[0, 1:] = vel[0, 1:] = 0.0
        off[1, 2:] = vel[1, 2:] = 0.0
        assert np.allclose(env.goal_off, off) and np.allclose(env.goal_vel, vel)
    assert np.abs(env.goal_off).max() <= 0.1 + 1e-15 and np.abs(env.goal_off).max() > 0.09
    # the observation carries the moved goal; the reward uses it
    g0 = d["goal"][0, 0] + env.goal_off[0, 0]
    assert np.allclose(obs[0, 24:27], g0)
    assert np.isclose(rew[0], -np.linalg.norm(obs[0, 14:17] - g0))
    env.reset(np.array([1, 0], np.uint8))
    assert (env.goal_off[0] == 0).all() and (env.goal_vel[0] == 0).all()
    assert (env.goal_off[1] != 0).any()
