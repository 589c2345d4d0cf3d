"""FP64 oracle of the GPU-resident PPO loop (Methods, "Policy learning and
control"; Results, "Simulator Performance Comparison", Table II).

TEST INFRASTRUCTURE ONLY (see the package header).

What the paper fixes: PPO (Schulman et al. 2017) with batch B = n_robots x
n_steps split into large minibatches, generalized advantage estimation
(Schulman et al. 2016), time-outs told apart from terminations and handled
by adding the critic's value prediction to the reward ("bootstrapping"), and
a policy network with hidden layers 256, 128, 64 and ELU activations.
Readings where it is silent:

* actor and critic are separate MLPs D -> 256 -> 128 -> 64 -> out with ELU
  after every hidden layer; the policy is a diagonal Gaussian with a
  state-independent log standard deviation per action;
* the action of a joint is its drive command (a position target for the
  default drive); joints an env does not have are sampled but ignored by the
  env and left out of log-probabilities and entropy;
* bootstrapping: on a time-out step r_t <- r_t + gamma V(o_t), V evaluated
  on the observation the action was taken from (the value the critic
  predicted for the continuing episode); any done bit ends the GAE recursion;
* after a done step the env is reset and its next observation is that of
  the reset state (with the last command as the current targets);
* advantages are normalised over the whole batch (mean 0, unbiased std 1,
  + 1e-8); the loss is the clipped surrogate plus value_coef times the
  clipped value loss minus entropy_coef times the entropy; gradients are
  clipped to a global norm; Adam updates the parameters.

The exploration noise is the counter-based generator of ``rng.action_noise``
keyed by (seed, env, joint block, global step); minibatch permutations are
inputs.  Everything here is plain PyTorch in float64; gradients come from
autograd (a library primitive, pinned against central differences in
tests/test_oracle_ppo.py).
"""
import math

import numpy as np
import torch

from .rng import action_noise

HIDDEN = (256, 128, 64)
DT = torch.float64


def param_shapes(D, A):
    """Shapes of the flat parameter vector, in order: actor layers (W, b) x 4,
    log_std, critic layers (W, b) x 4.  W is [out][in]."""
    shapes = []
    dims = (D,) + HIDDEN
    for net_out in (A, 1):
        layer = []
        for i in range(3):
            layer += [(dims[i + 1], dims[i]), (dims[i + 1],)]
        layer += [(net_out, HIDDEN[-1]), (net_out,)]
        shapes += layer
        if net_out == A:
            shapes.append((A,))                     # log_std
    return shapes


def unflatten(flat, D, A):
    """Split a flat vector into (actor [(W, b)] x 4, log_std, critic [(W, b)] x 4)."""
    out, k = [], 0
    for shp in param_shapes(D, A):
        n = int(np.prod(shp))
        out.append(flat[k:k + n].reshape(shp))
        k += n
    actor = [(out[2 * i], out[2 * i + 1]) for i in range(4)]
    log_std = out[8]
    critic = [(out[9 + 2 * i], out[10 + 2 * i]) for i in range(4)]
    return actor, log_std, critic


def num_params(D, A):
    return sum(int(np.prod(s)) for s in param_shapes(D, A))


def elu(x):
    """ELU with alpha = 1 (Clevert et al. 2016)."""
    return torch.where(x > 0, x, torch.expm1(x))


def mlp(layers, x):
    for i, (W, b) in enumerate(layers):
        x = x @ W.T + b
        if i < len(layers) - 1:
            x = elu(x)
    return x


def gaussian_logp(a, mu, log_std, mask):
    """Sum over the active joints of the diagonal Gaussian log-density."""
    z = (a - mu) / torch.exp(log_std)
    lp = -0.5 * z * z - log_std - 0.5 * math.log(2 * math.pi)
    return (lp * mask).sum(-1)


def gaussian_entropy(log_std, mask):
    return ((0.5 + 0.5 * math.log(2 * math.pi) + log_std) * mask).sum(-1)


def joint_mask(desc):
    """[E][A] 1.0 for the joints each env has."""
    E, A = int(desc["num_envs"]), int(desc["max_joints"])
    dof = np.asarray(desc["chain_num_joints"]).sum(1)
    return (np.arange(A)[None, :] < dof[:, None]).astype(np.float64)


def noise(seed, E, A, step):
    """Exploration noise eps [E][A] of global step `step`."""
    blocks = (A + 3) // 4
    z = action_noise(seed, np.arange(E)[:, None], np.arange(blocks)[None, :], step)   # [E, blocks, 4]
    return z.reshape(E, 4 * blocks)[:, :A]


def collect(env, flat, cfg, obs0, step0):
    """n_steps of acting and stepping from observations obs0 [E][D].

    Returns the rollout buffers (obs [n+1][E][D], actions, logp, values,
    rewards (bootstrapped), dones [n][E]) and the GAE advantages and returns.
    `env` is an OracleEnv whose state matches obs0."""
    E, D = obs0.shape
    A = int(env.J)
    actor, log_std, critic = unflatten(torch.as_tensor(flat, dtype=DT), D, A)
    mask = torch.as_tensor(joint_mask(env.desc))
    n, gamma = cfg["n_steps"], cfg["gamma"]
    obs = np.zeros((n + 1, E, D))
    obs[0] = obs0
    acts = np.zeros((n, E, A))
    logp = np.zeros((n, E))
    vals = np.zeros((n + 1, E))
    rews = np.zeros((n, E))
    dones = np.zeros((n, E), np.uint8)
    for t in range(n):
        x = torch.as_tensor(obs[t])
        mu = mlp(actor, x)
        v = mlp(critic, x)[:, 0]
        eps = torch.as_tensor(noise(cfg["seed"], E, A, step0 + t))
        a = mu + torch.exp(log_std) * eps
        acts[t] = a.numpy()
        logp[t] = gaussian_logp(a, mu, log_std, mask).numpy()
        vals[t] = v.numpy()
        o, r, d = env.step(acts[t], cfg["dt"], cfg["substeps"])
        timeout = (d & 2) != 0
        rews[t] = r + gamma * vals[t] * timeout
        dones[t] = d
        reset = d != 0
        if reset.any():
            env.reset(reset)
            o = np.where(reset[:, None], env.observe(acts[t], reset), o)
        obs[t + 1] = o
    vals[n] = mlp(critic, torch.as_tensor(obs[n]))[:, 0].numpy()
    adv, ret = gae(rews, vals, dones, gamma, cfg["lam"])
    return dict(obs=obs, actions=acts, logp=logp, values=vals[:n], last_values=vals[n],
                rewards=rews, dones=dones, advantages=adv, returns=ret)


def gae(rewards, values, dones, gamma, lam):
    """Generalized advantage estimation (Schulman et al. 2016) with a done
    step ending the recursion.  values is [n+1][E] (the last row: the value
    of the observation after the last step)."""
    n = rewards.shape[0]
    adv = np.zeros_like(rewards)
    nxt = np.zeros(rewards.shape[1])
    for t in range(n - 1, -1, -1):
        keep = 1.0 - (dones[t] != 0)
        delta = rewards[t] + gamma * values[t + 1] * keep - values[t]
        nxt = delta + gamma * lam * keep * nxt
        adv[t] = nxt
    return adv, adv + values[:n]


def normalise(adv):
    a = adv.reshape(-1)
    return (adv - a.mean()) / (a.std(ddof=1) + 1e-8)


def loss_terms(flat_t, D, A, x, a, logp_old, v_old, adv, ret, mask, cfg):
    """(total loss, surrogate, value loss, entropy) of one minibatch."""
    actor, log_std, critic = unflatten(flat_t, D, A)
    mu = mlp(actor, x)
    v = mlp(critic, x)[:, 0]
    logp = gaussian_logp(a, mu, log_std, mask)
    ratio = torch.exp(logp - logp_old)
    eps = cfg["clip"]
    surr = torch.maximum(-adv * ratio, -adv * torch.clamp(ratio, 1 - eps, 1 + eps)).mean()
    v_clip = v_old + torch.clamp(v - v_old, -eps, eps)
    vloss = torch.maximum((v - ret) ** 2, (v_clip - ret) ** 2).mean()
    ent = gaussian_entropy(log_std, mask).mean()
    total = surr + cfg["value_coef"] * vloss - cfg["entropy_coef"] * ent
    return total, surr, vloss, ent


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) with bias correction; t counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def update(flat, adam, buf, perms, desc, cfg):
    """PPO epochs over the rollout buffers.  perms [epochs][B] permute the
    flattened batch index t * E + e.  adam = (m, v, t).  Returns the new
    parameters, Adam state and per-minibatch stats [epochs * mb][4] =
    (surrogate, value loss, entropy, gradient norm before clipping)."""
    n, E = buf["rewards"].shape
    D = buf["obs"].shape[2]
    A = buf["actions"].shape[2]
    B = n * E
    mb = cfg["minibatches"]
    size = B // mb
    X = buf["obs"][:n].reshape(B, D)
    Acts = buf["actions"].reshape(B, A)
    LP = buf["logp"].reshape(B)
    V = buf["values"].reshape(B)
    ADV = normalise(buf["advantages"]).reshape(B)
    RET = buf["returns"].reshape(B)
    maskE = joint_mask(desc)
    MASK = np.broadcast_to(maskE[None], (n, E, A)).reshape(B, A)
    p = np.array(flat, np.float64)
    m, v, t = (np.array(adam[0], np.float64), np.array(adam[1], np.float64), int(adam[2]))
    stats = []
    for ep in range(cfg["epochs"]):
        for k in range(mb):
            idx = np.asarray(perms[ep][k * size:(k + 1) * size])
            pt = torch.tensor(p, dtype=DT, requires_grad=True)
            total, surr, vloss, ent = loss_terms(
                pt, D, A, torch.as_tensor(X[idx]), torch.as_tensor(Acts[idx]),
                torch.as_tensor(LP[idx]), torch.as_tensor(V[idx]), torch.as_tensor(ADV[idx]),
                torch.as_tensor(RET[idx]), torch.as_tensor(MASK[idx]), cfg)
            (g,) = torch.autograd.grad(total, [pt])
            g = g.numpy()
            norm = float(np.sqrt((g * g).sum()))
            coef = cfg["max_grad_norm"] / (norm + 1e-6)
            if coef < 1.0:
                g = g * coef
            t += 1
            p, m, v = adam_step(p, g, m, v, t, cfg["lr"])
            stats.append([surr.item(), vloss.item(), ent.item(), norm])
    return p, (m, v, t), np.array(stats)
