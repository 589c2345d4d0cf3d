"""Adjoint of the step (differentiable rollout) against the FP64 oracle:
reverse mode (autograd through the oracle rollout) and central finite
differences (h = 1e-6).  Bar: <= 1e-3 relative per env,
||g_gpu - g_ref|| / ||g_ref||, for the action and link-mass gradients of
L = sum_t ||tip_t - target||^2."""
import numpy as np
import pytest
import torch

from oracle.env import ee_rollout
from oracle.model import groups
from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0
D64 = torch.float64


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def gpu_grads(desc, acts, targets, S, every, env=None):
    env = env or sg.Env(desc)
    a = cuda(acts)
    ee = env.diff_forward(a, DT, S, every)
    tg = cuda(targets)
    nc = torch.as_tensor(desc["env_num_chains"], device="cuda")
    chain_mask = (torch.arange(4, device="cuda")[None, :] < nc[:, None]).float()[None, :, :, None]
    g = 2.0 * (ee - tg) * chain_mask
    da, dm = env.diff_backward(a, g.contiguous())
    return ee.cpu().numpy(), da.cpu().numpy(), dm.cpu().numpy()


def oracle_grads(desc, acts, targets, S, idx):
    """Autograd of the FP64 oracle rollout for envs `idx` (one structure)."""
    (gi, tree), = [(i, t) for i, t in groups(desc) if np.isin(idx, i).all()]
    n, nc = tree.n, tree.n_chains
    A = torch.tensor(acts[:, idx, :n], dtype=D64, requires_grad=True)
    m = torch.tensor(desc["link_mass"][idx, :n], dtype=D64, requires_grad=True)
    ee = ee_rollout(desc, A, DT, S, mass=m, env_idx=idx)           # [T, E, nc, 3]
    tg = torch.tensor(targets[:, idx, :nc], dtype=D64)
    L = ((ee - tg) ** 2).sum()
    ga, gm = torch.autograd.grad(L, [A, m])
    return ee.detach().numpy(), ga.numpy(), gm.numpy(), n


def rel_env(x, y):
    """per-env relative error over all remaining axes; x, y [..., E, ...] with env axis 1 for
    actions [T, E, n] and axis 0 for masses [E, n]"""
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-12)


@pytest.mark.parametrize("kind", ["7R", "7P", "4R", "14B", "21T"])
def test_adjoint_matches_oracle_reverse_mode(kind):
    E, T, S = 48, 16, 2
    desc = W.make_desc([kind] * E)
    acts = W.joint_targets(desc, T, resample_every=5)
    tg = W.loss_targets(desc, T)
    ee_g, da, dm = gpu_grads(desc, acts, tg, S, 8)
    idx = np.arange(E)
    ee_r, ga, gm, n = oracle_grads(desc, acts, tg, S, idx)
    assert np.abs(ee_g[:, :, :ee_r.shape[2]] - ee_r).max() < 1e-4
    worst_a = max(rel_env(da[:, e, :n], ga[:, e]) for e in range(E))
    worst_m = max(rel_env(dm[e, :n], gm[e]) for e in range(E))
    assert worst_a <= 1e-3, worst_a
    assert worst_m <= 1e-3, worst_m
    assert (da[:, :, n:] == 0).all() and (dm[:, n:] == 0).all()


def test_adjoint_with_limit_springs_and_mixed_batch():
    kinds = ["7R", "4R", "7P", "14B"] * 12
    desc = W.make_desc(kinds, k_limit=1e3)
    T, S = 12, 4
    acts = W.joint_targets(desc, T, resample_every=3)
    tg = W.loss_targets(desc, T)
    _, da, dm = gpu_grads(desc, acts, tg, S, 5)
    for idx, tree in groups(desc):
        _, ga, gm, n = oracle_grads(desc, acts, tg, S, idx)
        for k, e in enumerate(idx):
            assert rel_env(da[:, e, :n], ga[:, k]) <= 1e-3
            assert rel_env(dm[e, :n], gm[k]) <= 1e-3


def test_checkpoint_interval_does_not_change_gradients():
    """Recomputing from checkpoints reproduces the forward trajectory to
    rounding (the backward kernel is compiled apart from the forward kernel),
    so gradients agree across intervals to 1e-5 relative."""
    desc = W.make_desc(["7R", "14B"] * 40)
    T, S = 13, 2
    acts = W.joint_targets(desc, T)
    tg = W.loss_targets(desc, T)
    env = sg.Env(desc)
    ref = None
    for every in (1, 4, 8, 13, 32):
        _, da, dm = gpu_grads(desc, acts, tg, S, every, env=env)
        if ref is None:
            ref = (da, dm)
        else:
            assert rel_env(da, ref[0]) <= 1e-5 and rel_env(dm, ref[1]) <= 1e-5


@pytest.mark.parametrize("T,every", [(16, 8), (13, 4), (5, 8)])
def test_second_backward_after_one_forward(T, every):
    """The first reverse pass after a forward starts from the last segment's
    substep records written by the forward kernel; a second reverse pass
    (which overwrote them) recomputes that segment from its checkpoint.  Both
    give the same gradients to rounding (1e-5 relative: the forward and
    backward kernels are compiled apart), for a last segment that is full,
    partial, or the only one."""
    desc = W.make_desc(["7R", "7P", "4R", "14B"] * 20)
    S = 2
    acts = W.joint_targets(desc, T)
    tg = W.loss_targets(desc, T)
    env = sg.Env(desc)
    a = cuda(acts)
    ee = env.diff_forward(a, DT, S, every)
    nc = torch.as_tensor(desc["env_num_chains"], device="cuda")
    chain_mask = (torch.arange(4, device="cuda")[None, :] < nc[:, None]).float()[None, :, :, None]
    g = (2.0 * (ee - cuda(tg)) * chain_mask).contiguous()
    da1, dm1 = [x.cpu().numpy() for x in env.diff_backward(a, g)]
    da2, dm2 = [x.cpu().numpy() for x in env.diff_backward(a, g)]
    assert np.isfinite(da1).all() and np.isfinite(dm1).all()
    assert rel_env(da2, da1) <= 1e-5 and rel_env(dm2, dm1) <= 1e-5


def test_diff_forward_leaves_state_and_matches_rollout():
    desc = W.make_desc(W.mixed_kinds(300, W.C3_FRACTIONS))
    T = 9
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    s0 = [x.clone() for x in B.get_state()]
    ee = B.diff_forward(acts, DT, 2, 4)
    for x, y in zip(s0, B.get_state()):
        assert torch.equal(x, y)
    obs, _, _ = A.rollout(acts, DT, 2)
    # reach observation holds the tip of chain c at 2 n + 3 c
    dof = torch.as_tensor(desc["chain_num_joints"].sum(1), device="cuda").long()
    for c in range(2):
        has = torch.as_tensor(desc["env_num_chains"] > c, device="cuda")
        cols = (2 * dof + 3 * c)[:, None] + torch.arange(3, device="cuda")[None]
        tip_obs = torch.gather(obs, 2, cols[None].expand(T, -1, -1))
        # small batches run the forward as warp pairs (sg_pair.cuh), so it
        # agrees with the one-thread rollout to rounding, not bit for bit
        assert torch.allclose(ee[:, has, c], tip_obs[:, has], atol=1e-5)


def test_full_size_adjoint_sampled_against_oracle_and_central_differences():
    """The 2048-env, 64-step, 2-substep workload with checkpoints every 8
    steps: 16 envs against the oracle's reverse mode, and a sample of
    action coordinates plus all masses against FP64 central differences."""
    wl = W.config("C4")
    desc = wl.desc
    T, S = wl.steps, wl.substeps
    acts = W.joint_targets(desc, T, resample_every=8)
    tg = W.loss_targets(desc, T)
    _, da, dm = gpu_grads(desc, acts, tg, S, 8)
    idx = np.arange(16)
    _, ga, gm, n = oracle_grads(desc, acts, tg, S, idx)
    for k in range(16):
        assert rel_env(da[:, k, :n], ga[:, k]) <= 1e-3
        assert rel_env(dm[k, :n], gm[k]) <= 1e-3
    # central differences on 4 envs: 6 action coordinates and all 7 masses
    rng = np.random.default_rng(0)
    coords = [(int(rng.integers(T)), int(rng.integers(n))) for _ in range(6)]
    envs = np.arange(4)
    h = 1e-6
    reps = 2 * (len(coords) + n)
    A = torch.tensor(np.tile(acts[:, envs, :n], (1, reps, 1)), dtype=D64)
    M = torch.tensor(np.tile(desc["link_mass"][envs, :n], (reps, 1)), dtype=D64)
    k = 0
    for (t, j) in coords:
        for s in (1, -1):
            A[t, k * 4:(k + 1) * 4, j] += s * h
            k += 1
    for j in range(n):
        for s in (1, -1):
            M[k * 4:(k + 1) * 4, j] += s * h
            k += 1
    with torch.no_grad():
        ee = ee_rollout(desc, A, DT, S, mass=M, env_idx=np.tile(envs, reps))
        L = ((ee - torch.tensor(np.tile(tg[:, envs, :1], (1, reps, 1, 1)), dtype=D64)) ** 2)
        L = L.sum((0, 2, 3)).reshape(reps, 4)
    fd = ((L[0::2] - L[1::2]) / (2 * h)).numpy()       # [coords + n, 4]
    for ci, (t, j) in enumerate(coords):
        got = da[t, envs, j]
        assert np.abs(got - fd[ci]).max() <= 1e-3 * max(np.abs(ga[:, :4]).max(), 1e-6)
    fdm = fd[len(coords):].T
    for e in range(4):
        assert rel_env(dm[e, :n], fdm[e]) <= 1e-3


def test_autograd_function_and_set_link_mass():
    desc = W.make_desc(["7R"] * 64)
    T, S = 10, 2
    acts = cuda(W.joint_targets(desc, T)).requires_grad_(True)
    mass = cuda(desc["link_mass"] * 1.3).requires_grad_(True)
    tg = cuda(W.loss_targets(desc, T))
    env = sg.Env(desc)
    ee = sg.tip_rollout(env, acts, DT, S, mass=mass)
    loss = ((ee[:, :, :1] - tg[:, :, :1]) ** 2).sum()
    loss.backward()
    d2 = dict(desc)
    d2["link_mass"] = desc["link_mass"] * np.float32(1.3)
    d2["link_inertia"] = desc["link_inertia"] * np.float32(1.3)
    _, ga, gm, n = oracle_grads(d2, W.joint_targets(desc, T), W.loss_targets(desc, T), S,
                                np.arange(64))
    assert rel_env(acts.grad.cpu().numpy(), ga) <= 1e-3
    assert rel_env(mass.grad.cpu().numpy(), gm) <= 1e-3


@pytest.mark.parametrize("mode", [1, 2])
def test_adjoint_velocity_and_torque_commands(mode):
    E, T, S = 32, 10, 2
    desc = W.make_desc(["7R"] * E, drive=mode)
    acts = W.joint_targets(desc, T, resample_every=4)
    tg = W.loss_targets(desc, T)
    _, da, dm = gpu_grads(desc, acts, tg, S, 4)
    _, ga, gm, n = oracle_grads(desc, acts, tg, S, np.arange(E))
    assert max(rel_env(da[:, e, :n], ga[:, e]) for e in range(E)) <= 1e-3
    assert max(rel_env(dm[e, :n], gm[e]) for e in range(E)) <= 1e-3
