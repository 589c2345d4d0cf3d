"""GPU PPO loop (include/sg_ppo.h) against the FP64 oracle (oracle/ppo.py).

Tolerances, from the arithmetic: the collect loop runs the FP32 env and
FP32 networks against FP64 ones over a few steps, so observations, actions,
values and log-probabilities agree to ~1e-5 relative and are checked at
1e-3 (absolute, quantities of order 1-10); done bits are exact (step
counts).  The update is checked piece by piece on the GPU's own batch: the
minibatch loss gradient (FP32 GEMMs and reductions vs FP64 autograd) to
1e-4 in relative L2 norm per layer, one Adam step from that gradient to
1e-6 relative, the per-minibatch losses to 1e-4, and the parameters after
a full update (2 epochs x 2 minibatches) to 1e-2 of their change in L2
norm (Adam divides by |g|, which turns rounding in near-zero gradient
components into visible but bounded steps).  TF32 GEMMs (10-bit mantissa)
are checked at 2e-2."""
import numpy as np
import pytest
import torch

from oracle import ppo as P
from oracle.env import OracleEnv
from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu

CFG = dict(n_steps=6, epochs=2, minibatches=2, gamma=0.99, lam=0.95, clip=0.2, value_coef=1.0,
           entropy_coef=0.01, lr=1e-3, max_grad_norm=1.0, dt=1.0 / 60.0, substeps=2, seed=21,
           tf32=0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def _setup(kinds, episode_len=4, **over):
    cfg = dict(CFG, **over)
    desc = W.make_desc(kinds, episode_len=episode_len)
    env = sg.Env(desc)
    ppo = sg.PPO(env, **cfg)
    flat = W.ppo_init_params(env.obs_dim, env.max_joints, seed=3)
    ppo.set_params(torch.as_tensor(flat, device="cuda"))
    ppo.reset(step0=100)
    return desc, env, ppo, flat, cfg


def _np(t):
    return t.cpu().numpy().astype(np.float64)


def test_collect_matches_oracle_including_time_outs():
    kinds = (["7R", "14B", "4R", "7P", "21T"] * 5)[:23]
    desc, env, ppo, flat, cfg = _setup(kinds)
    ppo.collect()
    ref_env = OracleEnv(desc)
    E, A = len(kinds), desc["max_joints"]
    obs0 = ref_env.observe(np.zeros((E, A)))
    buf = P.collect(ref_env, flat.astype(np.float64), cfg, obs0, 100)
    assert np.array_equal(ppo.get_buffer(sg.PPO_DONES).cpu().numpy(), buf["dones"])
    assert (buf["dones"][3] == 2).all()                    # every env timed out at step 4
    for which, key in ((sg.PPO_OBS, "obs"), (sg.PPO_ACTIONS, "actions"), (sg.PPO_LOGP, "logp"),
                       (sg.PPO_REWARDS, "rewards"), (sg.PPO_ADVANTAGES, "advantages"),
                       (sg.PPO_RETURNS, "returns")):
        got = _np(ppo.get_buffer(which))
        assert np.abs(got - buf[key]).max() <= 1e-3, key
    vals = _np(ppo.get_buffer(sg.PPO_VALUES))
    assert np.abs(vals[:-1] - buf["values"]).max() <= 1e-3
    assert np.abs(vals[-1] - buf["last_values"]).max() <= 1e-3


def test_second_collect_replays_the_graph_and_continues():
    kinds = ["7R", "4R"] * 8
    desc, env, ppo, flat, cfg = _setup(kinds, episode_len=5)
    ref_env = OracleEnv(desc)
    E, A = len(kinds), desc["max_joints"]
    obs = ref_env.observe(np.zeros((E, A)))
    for it in range(2):
        ppo.collect()
        buf = P.collect(ref_env, flat.astype(np.float64), cfg, obs, 100 + it * cfg["n_steps"])
        obs = buf["obs"][-1]
        assert np.array_equal(ppo.get_buffer(sg.PPO_DONES).cpu().numpy(), buf["dones"])
        assert np.abs(_np(ppo.get_buffer(sg.PPO_ACTIONS)) - buf["actions"]).max() <= 1e-3
        assert np.abs(_np(ppo.get_buffer(sg.PPO_RETURNS)) - buf["returns"]).max() <= 1e-3


def _gpu_batch(ppo, n, E):
    g = lambda w: _np(ppo.get_buffer(w))
    vals = g(sg.PPO_VALUES)
    return dict(obs=g(sg.PPO_OBS), actions=g(sg.PPO_ACTIONS), logp=g(sg.PPO_LOGP),
                values=vals[:n], advantages=g(sg.PPO_ADVANTAGES), returns=g(sg.PPO_RETURNS),
                rewards=g(sg.PPO_REWARDS))


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_minibatch_gradient_and_adam_step_match_oracle():
    kinds = ["7R", "14B", "4R", "7P"] * 6
    desc, env, ppo, flat, cfg = _setup(kinds, epochs=1, minibatches=1)
    ppo.collect()
    n, E = cfg["n_steps"], len(kinds)
    batch = _gpu_batch(ppo, n, E)
    perms = W.ppo_perms(n * E, 1)
    stats = ppo.update(torch.as_tensor(perms, device="cuda"))
    grad = _np(ppo.get_buffer(sg.PPO_GRAD))
    new = _np(ppo.get_params())
    # oracle gradient of the same minibatch (the whole batch here)
    D, A = env.obs_dim, env.max_joints
    B = n * E
    mask = np.broadcast_to(P.joint_mask(desc)[None], (n, E, A)).reshape(B, A)
    t = lambda x: torch.as_tensor(np.ascontiguousarray(x))
    idx = perms[0]
    args = (t(batch["obs"][:n].reshape(B, D)[idx]), t(batch["actions"].reshape(B, A)[idx]),
            t(batch["logp"].reshape(B)[idx]), t(batch["values"].reshape(B)[idx]),
            t(P.normalise(batch["advantages"]).reshape(B)[idx]),
            t(batch["returns"].reshape(B)[idx]), t(mask[idx]))
    pt = torch.tensor(flat.astype(np.float64), requires_grad=True)
    total, surr, vloss, ent = P.loss_terms(pt, D, A, *args, cfg)
    (g_ref,) = torch.autograd.grad(total, [pt])
    g_ref = g_ref.numpy()
    k = 0
    for shp in P.param_shapes(D, A):
        m = int(np.prod(shp))
        assert _rel(grad[k:k + m], g_ref[k:k + m]) <= 1e-4, (k, shp)
        k += m
    st = stats.cpu().numpy()[0]
    assert np.allclose(st[:3], [surr.item(), vloss.item(), ent.item()], rtol=1e-4, atol=1e-6)
    assert np.isclose(st[3], np.linalg.norm(g_ref), rtol=1e-4)
    # Adam from the GPU's own gradient
    gn = np.linalg.norm(grad)
    gc = grad * min(1.0, cfg["max_grad_norm"] / (gn + 1e-6))
    p1, _, _ = P.adam_step(flat.astype(np.float64), gc, np.zeros_like(gc), np.zeros_like(gc), 1,
                           cfg["lr"])
    assert _rel(new - flat, p1 - flat) <= 1e-5


@pytest.mark.parametrize("tf32,tol", [(0, 1e-2), (1, 5e-2)])
def test_full_update_matches_oracle(tf32, tol):
    kinds = ["7R", "4R", "14B"] * 8
    desc, env, ppo, flat, cfg = _setup(kinds, tf32=tf32)
    ppo.collect()
    n, E = cfg["n_steps"], len(kinds)
    batch = _gpu_batch(ppo, n, E)
    perms = W.ppo_perms(n * E, cfg["epochs"])
    stats = ppo.update(torch.as_tensor(perms, device="cuda")).cpu().numpy()
    new = _np(ppo.get_params())
    p_ref, _, st_ref = P.update(flat.astype(np.float64), (np.zeros(len(flat)), np.zeros(len(flat)), 0),
                                batch, perms, desc, cfg)
    loss_tol = 1e-4 if tf32 == 0 else 2e-2
    assert np.allclose(stats[:, :3], st_ref[:, :3], rtol=loss_tol, atol=1e-5)
    assert _rel(new - flat, p_ref - flat) <= tol


def test_update_of_a_batch_set_by_the_caller():
    """sg_ppo_set_buffer: an update on caller-provided buffers equals the
    update on the same buffers collected by the loop."""
    kinds = ["7R"] * 16
    desc, env, ppo, flat, cfg = _setup(kinds)
    ppo.collect()
    bufs = {w: ppo.get_buffer(w) for w in (sg.PPO_OBS, sg.PPO_ACTIONS, sg.PPO_LOGP, sg.PPO_VALUES,
                                            sg.PPO_ADVANTAGES, sg.PPO_RETURNS)}
    perms = torch.as_tensor(W.ppo_perms(cfg["n_steps"] * 16, cfg["epochs"]), device="cuda")
    s1 = ppo.update(perms)
    p1 = ppo.get_params()
    desc2, env2, ppo2, _, _ = _setup(kinds)
    for w, b in bufs.items():
        ppo2.set_buffer(w, b)
    s2 = ppo2.update(perms)
    assert torch.equal(s1, s2) and torch.equal(p1, ppo2.get_params())


def test_two_handles_give_identical_bits_at_scale():
    """Every kernel of the loop is deterministic (fixed-order sums, no
    atomics on values) and the actor, the critic and each network's weight
    gradients run on separate streams joined by events: two handles fed the
    same inputs must agree bit for bit over two full iterations at a size
    with hundreds of row tiles per product."""
    kinds = ["7P"] * 4096
    cfg = dict(CFG, n_steps=24, epochs=2, minibatches=4)
    out = []
    for _ in range(2):
        desc = W.make_desc(kinds, episode_len=50)
        env = sg.Env(desc)
        ppo = sg.PPO(env, **cfg)
        ppo.set_params(torch.as_tensor(W.ppo_init_params(env.obs_dim, env.max_joints, seed=3),
                                       device="cuda"))
        ppo.reset(step0=0)
        perms = torch.as_tensor(W.ppo_perms(ppo.B, cfg["epochs"]), device="cuda")
        stats = []
        for _ in range(2):
            ppo.collect()
            stats.append(ppo.update(perms).clone())
        torch.cuda.synchronize()
        assert env.sync_status() == sg.SG_OK
        out.append((torch.stack(stats), ppo.get_params(), ppo.get_buffer(sg.PPO_VALUES)))
    for a, b in zip(*out):
        assert torch.equal(a, b)


def test_configuration_errors():
    desc = W.make_desc(["7R"] * 10)
    env = sg.Env(desc)
    for bad in (dict(minibatches=7), dict(n_steps=0), dict(gamma=1.5), dict(lr=0.0), dict(substeps=0)):
        with pytest.raises(sg.SgError) as ei:
            sg.PPO(env, **dict(CFG, **bad))
        assert ei.value.status == sg.SG_ERR_INVALID_ARG
