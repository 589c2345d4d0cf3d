"""Path-following waypoint tables built on the device (sg_create from
control points, sg_set_paths) against the FP64 oracle of the spline and
the equal-arc-length resampling.

Tolerance: the device evaluates the spline and the chord lengths in FP32
and sums arc length in FP64; positions of about 0.5 m carry FP32 rounding
of about 6e-8 m per operation, so the tables must agree with the oracle to
2e-6 m per coordinate.  Envs outside a mask must keep their table bit for
bit."""
import numpy as np
import pytest
import torch

from oracle import path as OP
from oracle.env import OracleEnv
from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu

TOL = 2e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def _ctrl(E, K, seed):
    rng = np.random.default_rng(seed)
    centre = np.array([0.3, 0.0, 0.5])
    return (centre + rng.uniform(-0.15, 0.15, size=(E, K, 3))).astype(np.float32)


@pytest.mark.parametrize("E,K,W_", [(37, 16, 503), (5, 2, 4), (9, 3, 40), (6, 64, 1000), (130, 16, 77)])
def test_device_tables_match_oracle(E, K, W_):
    desc = W.make_desc(["7R"] * E, task=1, path_len=W_)
    desc["path_ctrl"] = _ctrl(E, K, seed=K + E)
    desc["path_ctrl_len"] = K
    env = sg.Env(desc)
    got = env.get_paths(W_).cpu().numpy().astype(np.float64)
    ref = OP.waypoints(desc["path_ctrl"], W_)
    assert np.abs(got - ref).max() <= TOL
    # end points are the first and last control points
    assert np.abs(got[:, 0] - desc["path_ctrl"][:, 0]).max() <= TOL
    assert np.abs(got[:, -1] - desc["path_ctrl"][:, -1]).max() <= TOL


def test_set_paths_masked_rebuild():
    E, Wn = 45, 120
    desc = W.make_desc(["7R"] * E, task=1, path_len=Wn)
    env = sg.Env(desc)
    before = env.get_paths(Wn).cpu().numpy()
    new = _ctrl(E, 11, seed=99)
    mask = np.zeros(E, np.uint8)
    mask[[0, 3, 4, 17, 31, 32, 44]] = 1
    env.set_paths(torch.as_tensor(new, device="cuda"), torch.as_tensor(mask, device="cuda"))
    after = env.get_paths(Wn).cpu().numpy()
    m = mask.astype(bool)
    assert np.array_equal(after[~m], before[~m])
    assert np.abs(after[m].astype(np.float64) - OP.waypoints(new[m], Wn)).max() <= TOL
    # all envs, a different K
    new2 = _ctrl(E, 64, seed=7)
    env.set_paths(torch.as_tensor(new2, device="cuda"))
    assert np.abs(env.get_paths(Wn).cpu().numpy() - OP.waypoints(new2, Wn)).max() <= TOL


def test_set_paths_argument_errors():
    desc = W.make_desc(["7R"] * 4, task=1, path_len=10)
    env = sg.Env(desc)
    for K in (1, 65):
        bad = torch.zeros(4, K, 3, device="cuda")
        with pytest.raises(sg.SgError) as ei:
            env.set_paths(bad)
        assert ei.value.status == sg.SG_ERR_INVALID_ARG
    reach = sg.Env(W.make_desc(["7R"] * 4))
    with pytest.raises(sg.SgError):
        reach.set_paths(torch.zeros(4, 8, 3, device="cuda"))
    with pytest.raises(sg.SgError):
        reach.get_paths(10)


def test_episode_with_new_paths_matches_oracle():
    """Reset + new paths mid-run: observations (next waypoints) and rewards
    of the following steps follow the rebuilt tables."""
    E, T = 24, 12
    desc = W.make_desc(["7R"] * E, task=1, path_len=T + 3, episode_len=T)
    env, ref = sg.Env(desc), OracleEnv(desc)
    acts = W.joint_targets(desc, 2 * T)
    for t in range(5):
        env.step(torch.as_tensor(acts[t], device="cuda"), 1 / 60, 4)
        ref.step(acts[t], 1 / 60, 4)
    mask = (np.arange(E) % 3 == 0).astype(np.uint8)
    new = _ctrl(E, 16, seed=5)
    env.set_paths(torch.as_tensor(new, device="cuda"), torch.as_tensor(mask, device="cuda"))
    env.reset(torch.as_tensor(mask, device="cuda"))
    ref.set_paths(new, mask)
    ref.reset(mask)
    for t in range(5, 10):
        obs, rew, _ = env.step(torch.as_tensor(acts[t], device="cuda"), 1 / 60, 4)
        o_ref, r_ref, _ = ref.step(acts[t], 1 / 60, 4)
        obs = obs.cpu().numpy()
        # waypoint part of the observation: exact table entries, compared to the oracle's tables
        assert np.abs(obs[:, 21:30] - o_ref[:, 21:30]).max() <= TOL
        assert np.abs(rew.cpu().numpy() - r_ref).max() <= 1e-3
