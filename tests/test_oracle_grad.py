"""The oracle's reverse-mode gradient (autograd through the FP64 rollout)
against FP64 central finite differences (h = 1e-6) of the same rollout."""
import numpy as np
import torch

from oracle.env import ee_rollout
from paper_2310_04676_gb300 import workloads as W

D = torch.float64


def _loss(desc, acts, mass, targets, env_idx, T, S):
    ee = ee_rollout(desc, acts, 1 / 60, S, mass=mass, env_idx=env_idx)
    return ((ee - targets) ** 2).sum((0, 2, 3))      # per env


def test_reverse_mode_matches_central_differences():
    E, T, S, n = 4, 3, 2, 7
    d = W.make_desc(["7R"] * E)
    acts = torch.as_tensor(W.joint_targets(d, T)[:, :, :n], dtype=D)
    tg = torch.as_tensor(W.loss_targets(d, T)[:, :, :1], dtype=D)
    mass = torch.as_tensor(d["link_mass"][:, :n], dtype=D)
    a = acts.clone().requires_grad_(True)
    m = mass.clone().requires_grad_(True)
    L = _loss(d, a, m, tg, np.arange(E), T, S)
    ga, gm = torch.autograd.grad(L.sum(), [a, m])

    # central differences, all perturbations batched as replicated envs
    h = 1e-6
    nA = T * n
    reps = 2 * (nA + n)
    idx = np.tile(np.arange(E), reps)
    A = acts.repeat(1, reps, 1)
    Mm = mass.repeat(reps, 1)
    k = 0
    for t in range(T):
        for j in range(n):
            for s in (+1, -1):
                A[t, k * E:(k + 1) * E, j] += s * h
                k += 1
    for j in range(n):
        for s in (+1, -1):
            Mm[k * E:(k + 1) * E, j] += s * h
            k += 1
    with torch.no_grad():
        Lf = _loss(d, A, Mm, tg.repeat(1, reps, 1, 1), idx, T, S).reshape(reps, E)
    fd = (Lf[0::2] - Lf[1::2]) / (2 * h)                        # [nA + n, E]
    fd_a = fd[:nA].reshape(T, n, E).permute(0, 2, 1)
    fd_m = fd[nA:].T
    rel = lambda x, y: ((x - y).abs().max() / y.abs().max()).item()
    assert rel(ga, fd_a) < 1e-6
    assert rel(gm, fd_m) < 1e-6


def test_reverse_mode_matches_central_differences_velocity_and_torque_commands():
    E, T, S, n = 2, 3, 2, 7
    for mode in (1, 2):
        d = W.make_desc(["7R"] * E, drive=mode)
        acts = torch.as_tensor(W.joint_targets(d, T)[:, :, :n], dtype=D)
        tg = torch.as_tensor(W.loss_targets(d, T)[:, :, :1], dtype=D)
        a = acts.clone().requires_grad_(True)
        L = _loss(d, a, None, tg, np.arange(E), T, S)
        ga, = torch.autograd.grad(L.sum(), [a])
        h = 1e-6
        for (t, j) in [(0, 0), (1, 3), (2, 6), (0, 5)]:
            ap, am = acts.clone(), acts.clone()
            ap[t, :, j] += h
            am[t, :, j] -= h
            with torch.no_grad():
                fd = (_loss(d, ap, None, tg, np.arange(E), T, S)
                      - _loss(d, am, None, tg, np.arange(E), T, S)) / (2 * h)
            assert torch.allclose(ga[t, :, j], fd, rtol=1e-6, atol=1e-9)
