"""Persistent / graph rollout and the autotuner against per-step launches."""
import numpy as np
import pytest
import torch

from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("mode", [sg.ROLLOUT_PERSISTENT, sg.ROLLOUT_STEP_GRAPH])
@pytest.mark.parametrize("threads", [32, 128, 256])
def test_rollout_equals_steps_bitwise(mode, threads):
    kinds = W.mixed_kinds(777, W.C3_FRACTIONS)
    desc = W.make_desc(kinds, episode_len=20)
    T = 32
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    B.set_launch(threads, mode)
    steps = [A.step(acts[t], DT, 2) for t in range(T)]
    obs, rew, done = B.rollout(acts, DT, 2)
    for t in range(T):
        assert torch.equal(steps[t][0], obs[t])
        assert torch.equal(steps[t][1], rew[t])
        assert torch.equal(steps[t][2], done[t])
    qa, qda, sca = A.get_state()
    qb, qdb, scb = B.get_state()
    assert torch.equal(qa, qb) and torch.equal(qda, qdb) and torch.equal(sca, scb)
    # a second replay of the captured graph continues the trajectory
    obs2, _, _ = B.rollout(acts, DT, 2)
    s2 = [A.step(acts[t], DT, 2) for t in range(T)]
    assert torch.equal(obs2[-1], s2[-1][0])


def test_host_rollout_matches_device_rollout():
    desc = W.make_desc(W.mixed_kinds(300, W.C3_FRACTIONS))
    T = 8
    acts_np = W.joint_targets(desc, T)
    A, B = sg.Env(desc), sg.Env(desc)
    obs, rew, done = A.rollout(cuda(acts_np), DT, 2)
    a_h = torch.from_numpy(acts_np).pin_memory()
    out = (torch.empty(T, B.num_envs, B.obs_dim).pin_memory(),
           torch.empty(T, B.num_envs).pin_memory(),
           torch.empty(T, B.num_envs, dtype=torch.uint8).pin_memory())
    B.rollout_host(a_h, DT, 2, out)
    assert B.sync_status() == sg.SG_OK
    assert torch.equal(out[0], obs.cpu()) and torch.equal(out[1], rew.cpu())
    assert torch.equal(out[2], done.cpu())


def test_autotune_keeps_state_and_picks_a_plan():
    desc = W.make_desc(W.mixed_kinds(2000, W.C3_FRACTIONS))
    T = 16
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    th, mode, ms = B.autotune(acts, DT, 2, repeats=2)
    assert th in (32, 64, 128, 256) and mode in (0, 1) and ms > 0
    qa, qda, sca = A.get_state()
    qb, qdb, scb = B.get_state()
    assert torch.equal(qa, qb) and torch.equal(qda, qdb) and torch.equal(sca, scb)
    oa, _, _ = A.rollout(acts, DT, 2)
    ob, _, _ = B.rollout(acts, DT, 2)
    assert torch.equal(oa, ob)


def test_rollout_argument_errors():
    env = sg.Env(W.make_desc(["7R"] * 8))
    with pytest.raises(sg.SgError):
        env.set_launch(48, 0)
    with pytest.raises(sg.SgError):
        env.set_launch(64, 5)
    with pytest.raises(ValueError):
        env.rollout(torch.zeros(4, 8, 6, device="cuda"), DT, 2)
