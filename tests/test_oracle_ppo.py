"""Pins of the PPO oracle (no GPU): the exploration-noise generator, the
network's layout and activation, the Gaussian policy's density and entropy
against scipy, GAE against closed forms, time-out bootstrapping and resets
against a separately stepped env, the clipped losses at special points,
autograd gradients against central differences, and Adam against the
library optimiser."""
import math

import numpy as np
import pytest
import torch

from oracle import ppo as P
from oracle.env import OracleEnv
from oracle.rng import action_noise
from paper_2310_04676_gb300 import workloads as W

CFG = dict(n_steps=4, epochs=2, minibatches=2, gamma=0.99, lam=0.95, clip=0.2, value_coef=1.0,
           entropy_coef=0.01, lr=1e-3, max_grad_norm=1.0, dt=1 / 60, substeps=2, seed=5)


def _params(D, A, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    out = []
    for shp in P.param_shapes(D, A):
        fan_in = shp[1] if len(shp) == 2 else 64
        out.append(rng.uniform(-1, 1, size=shp).ravel() * scale / math.sqrt(fan_in))
    return np.concatenate(out)


def test_action_noise_is_standard_normal_and_counter_based():
    z = action_noise(9, np.arange(20000)[:, None], np.arange(2)[None, :], 3).reshape(-1)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02
    zz = action_noise(9, np.arange(20000), 0, 3)
    assert abs(np.corrcoef(zz[:, 0], zz[:, 1])[0, 1]) < 0.03        # the two halves of a pair
    assert abs(np.corrcoef(zz[:, 1], zz[:, 3])[0, 1]) < 0.03
    assert np.array_equal(action_noise(9, 4, 1, 3), action_noise(9, 4, 1, 3))
    for other in (action_noise(8, 4, 1, 3), action_noise(9, 5, 1, 3), action_noise(9, 4, 2, 3),
                  action_noise(9, 4, 1, 4)):
        assert not np.allclose(other, action_noise(9, 4, 1, 3))
    e = P.noise(9, 3, 7, 3)                          # joint j -> block j // 4, component j % 4
    assert np.array_equal(e[2, 5], action_noise(9, 2, 1, 3)[1])


def test_parameter_count_closed_form():
    D, A = 27, 7
    actor = D * 256 + 256 + 256 * 128 + 128 + 128 * 64 + 64 + 64 * A + A + A
    critic = D * 256 + 256 + 256 * 128 + 128 + 128 * 64 + 64 + 64 + 1
    assert P.num_params(D, A) == actor + critic
    a, ls, c = P.unflatten(np.arange(P.num_params(D, A), dtype=float), D, A)
    assert a[0][0].shape == (256, D) and a[3][0].shape == (A, 64) and ls.shape == (A,)
    assert c[3][0].shape == (1, 64) and c[0][0][0, 0] == actor   # critic starts after log_std


def test_elu_values():
    x = torch.tensor([-50.0, -1.0, 0.0, 2.0], dtype=torch.float64)
    assert torch.allclose(P.elu(x), torch.tensor([-1.0, math.exp(-1) - 1, 0.0, 2.0], dtype=torch.float64))


def test_mlp_is_the_matrix_product_where_all_preactivations_are_positive():
    """Non-negative weights, biases and inputs keep every hidden unit in
    ELU's identity branch: the network is then the affine composition."""
    rng = np.random.default_rng(1)
    dims = [5, 256, 128, 64, 3]
    layers = [(rng.uniform(0, 0.1, (dims[i + 1], dims[i])), rng.uniform(0, 0.1, dims[i + 1]))
              for i in range(4)]
    x = rng.uniform(0, 1, (4, 5))
    y = x
    for W_, b in layers:
        y = y @ W_.T + b
    got = P.mlp([(torch.as_tensor(W_), torch.as_tensor(b)) for W_, b in layers], torch.as_tensor(x))
    assert np.allclose(got.numpy(), y, rtol=1e-12)


def test_gaussian_logp_and_entropy_match_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(2)
    mu, a = rng.normal(size=(6, 7)), rng.normal(size=(6, 7))
    log_std = rng.normal(scale=0.3, size=7)
    mask = (np.arange(7)[None, :] < np.array([7, 4, 7, 2, 7, 7])[:, None]).astype(float)
    lp = P.gaussian_logp(torch.as_tensor(a), torch.as_tensor(mu), torch.as_tensor(log_std),
                         torch.as_tensor(mask)).numpy()
    ref = (stats.norm.logpdf(a, mu, np.exp(log_std)) * mask).sum(1)
    assert np.allclose(lp, ref, rtol=1e-12)
    ent = P.gaussian_entropy(torch.as_tensor(log_std), torch.as_tensor(mask)).numpy()
    assert np.allclose(ent, (stats.norm.entropy(scale=np.exp(log_std))[None] * mask).sum(1))


def test_gae_closed_forms():
    rng = np.random.default_rng(3)
    n, E = 6, 5
    r, v = rng.normal(size=(n, E)), rng.normal(size=(n + 1, E))
    none = np.zeros((n, E), np.uint8)
    adv, ret = P.gae(r, v, none, 0.0, 0.95)              # gamma = 0: one-step advantage
    assert np.allclose(adv, r - v[:n]) and np.allclose(ret, r)
    g = 0.9
    adv, _ = P.gae(r, v, none, g, 1.0)                    # lambda = 1: discounted return - value
    for t in range(n):
        G = sum(g ** k * r[t + k] for k in range(n - t)) + g ** (n - t) * v[n]
        assert np.allclose(adv[t], G - v[t])
    d = none.copy()
    d[2, 1] = 2                                           # a done step ends the recursion
    adv, _ = P.gae(r, v, d, g, 0.7)
    assert np.isclose(adv[2, 1], r[2, 1] - v[2, 1])
    d1 = r[1, 1] + g * v[2, 1] - v[1, 1]
    assert np.isclose(adv[1, 1], d1 + g * 0.7 * adv[2, 1])


def test_collect_bootstraps_time_outs_and_resets():
    desc = W.make_desc(["7R", "14B", "4R"], episode_len=3)
    E, A = 3, desc["max_joints"]
    env = OracleEnv(desc)
    D = env.D
    flat = _params(D, A)
    obs0 = env.observe(np.zeros((E, A)))
    cfg = dict(CFG, n_steps=5)
    buf = P.collect(env, flat, cfg, obs0, step0=10)
    # a second env stepped with the recorded actions gives the raw rewards
    twin = OracleEnv(desc)
    for t in range(5):
        o, r, d = twin.step(buf["actions"][t], cfg["dt"], cfg["substeps"])
        assert np.array_equal(d, buf["dones"][t])
        boot = cfg["gamma"] * buf["values"][t] * ((d & 2) != 0)
        assert np.allclose(buf["rewards"][t], r + boot, rtol=1e-12)
        if d.any():
            twin.reset(d != 0)
            o = np.where((d != 0)[:, None], twin.observe(buf["actions"][t], d != 0), o)
        assert np.allclose(buf["obs"][t + 1], o, rtol=1e-12)
    assert (buf["dones"][2] == 2).all() and (buf["dones"][4] == 0).all()
    # actions: mean + std * counter noise of global steps 10..14
    actor, log_std, _ = P.unflatten(torch.as_tensor(flat), D, A)
    mu = P.mlp(actor, torch.as_tensor(buf["obs"][1])).numpy()
    assert np.allclose(buf["actions"][1], mu + np.exp(log_std.numpy()) * P.noise(5, E, A, 11))


def _minibatch(seed=4):
    desc = W.make_desc(["7R", "4R"] * 3)
    env = OracleEnv(desc)
    E, A, D = 6, desc["max_joints"], env.D
    flat = _params(D, A, seed)
    buf = P.collect(env, flat, CFG, env.observe(np.zeros((E, A))), 0)
    n = CFG["n_steps"]
    B = n * E
    t = lambda x: torch.as_tensor(np.ascontiguousarray(x))
    mask = np.broadcast_to(P.joint_mask(desc)[None], (n, E, A)).reshape(B, A)
    args = (t(buf["obs"][:n].reshape(B, D)), t(buf["actions"].reshape(B, A)),
            t(buf["logp"].reshape(B)), t(buf["values"].reshape(B)),
            t(P.normalise(buf["advantages"]).reshape(B)), t(buf["returns"].reshape(B)), t(mask))
    return desc, flat, buf, D, A, args


def test_losses_at_the_behaviour_policy():
    """With the parameters that collected the batch: ratio 1, surrogate =
    -mean(A) (0 after normalisation), value loss = mean((V - R)^2)."""
    desc, flat, buf, D, A, args = _minibatch()
    total, surr, vloss, ent = P.loss_terms(torch.as_tensor(flat), D, A, *args, CFG)
    adv = args[4].numpy()
    assert np.isclose(float(surr), -adv.mean(), atol=1e-12) and abs(adv.mean()) < 1e-12
    assert np.isclose(float(vloss), ((args[3] - args[5]) ** 2).mean().item(), rtol=1e-10)
    _, log_std, _ = P.unflatten(flat, D, A)
    per_env = (0.5 + 0.5 * math.log(2 * math.pi) + log_std) @ args[6].numpy().T
    assert np.isclose(float(ent), per_env.mean(), rtol=1e-12)


def test_clipped_samples_contribute_no_policy_gradient():
    """A sample whose ratio is above 1 + clip with a positive advantage sits
    on the flat part of the clipped objective."""
    desc, flat, buf, D, A, args = _minibatch()
    x, a, lp, v, adv, ret, mask = (z[:1].clone() for z in args)
    adv[:] = 1.0
    lp = lp - math.log(1.5)                              # ratio = 1.5 > 1.2
    pt = torch.tensor(flat, requires_grad=True)
    _, surr, _, _ = P.loss_terms(pt, D, A, x, a, lp, v, adv, ret, mask, CFG)
    (g,) = torch.autograd.grad(surr, [pt])
    assert torch.count_nonzero(g) == 0
    assert np.isclose(surr.item(), -1.2)


def test_autograd_gradient_matches_central_differences():
    desc, flat, buf, D, A, args = _minibatch(seed=7)
    pt = torch.tensor(flat, requires_grad=True)
    total, *_ = P.loss_terms(pt, D, A, *args, CFG)
    (g,) = torch.autograd.grad(total, [pt])
    rng = np.random.default_rng(0)
    n_actor = sum(int(np.prod(s)) for s in P.param_shapes(D, A)[:9])
    picks = list(rng.choice(len(flat), 12, replace=False)) + [n_actor - 1, n_actor - 3, len(flat) - 1]
    h = 1e-6
    for k in picks:
        fp, fm = flat.copy(), flat.copy()
        fp[k] += h
        fm[k] -= h
        with torch.no_grad():
            fd = (P.loss_terms(torch.as_tensor(fp), D, A, *args, CFG)[0]
                  - P.loss_terms(torch.as_tensor(fm), D, A, *args, CFG)[0]) / (2 * h)
        assert abs(g[k].item() - fd.item()) <= 1e-6 * max(1.0, abs(fd.item())), k


def test_adam_matches_library_optimiser_and_clip():
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=50)
    pt = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([pt], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for t in range(1, 5):
        g = rng.normal(size=50)
        opt.zero_grad()
        pt.grad = torch.tensor(g.copy())
        opt.step()
        p, m, v = P.adam_step(p, g, m, v, t, 3e-3)
    assert np.allclose(p, pt.detach().numpy(), rtol=1e-12, atol=1e-15)
    # first step from zero moments moves every coordinate by lr * sign(g) (up to eps)
    g = rng.normal(size=50)
    p1, _, _ = P.adam_step(np.zeros(50), g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(p1, -1e-3 * np.sign(g), rtol=1e-6)


def test_update_clips_the_global_norm_and_matches_a_hand_loop():
    desc, flat, buf, D, A, args = _minibatch(seed=9)
    B = CFG["n_steps"] * 6
    perms = [np.random.default_rng(k).permutation(B) for k in range(CFG["epochs"])]
    cfg = dict(CFG, max_grad_norm=1e-3)                  # every step clipped
    p, (m, v, t), stats = P.update(flat, (np.zeros_like(flat), np.zeros_like(flat), 0), buf, perms,
                                   desc, cfg)
    assert t == 4 and stats.shape == (4, 4) and (stats[:, 3] > 1e-3).all()
    # first minibatch by hand: clipped gradient has norm max_grad_norm
    idx = perms[0][: B // 2]
    sub = tuple(z[idx] for z in args)
    pt = torch.tensor(flat, requires_grad=True)
    (g,) = torch.autograd.grad(P.loss_terms(pt, D, A, *sub, cfg)[0], [pt])
    g = g.numpy() * (1e-3 / (np.linalg.norm(g.numpy()) + 1e-6))
    assert np.isclose(np.linalg.norm(g), 1e-3, rtol=1e-5)
    p1, _, _ = P.adam_step(flat, g, np.zeros_like(flat), np.zeros_like(flat), 1, cfg["lr"])
    # one epoch of one minibatch (the first half of the permutation) is the hand step
    p_first, _, _ = P.update(flat, (np.zeros_like(flat), np.zeros_like(flat), 0), buf,
                             [perms[0][: B // 2]], desc, dict(cfg, epochs=1, minibatches=1))
    assert np.allclose(p_first, p1, rtol=1e-12, atol=1e-15)
