"""Pins of the FP64 oracle's kinematics and dynamics against closed forms,
invariants and an independent Lagrangian derivation (no GPU)."""
import math

import numpy as np
import pytest
import torch

from oracle import dynamics as dyn
from oracle import lagrangian as lag
from oracle.env import tip_quaternion
from oracle.model import groups, make_params
from tests.helpers import chain_desc

G = 9.81
D = torch.float64


def single(desc):
    (idx, tree), = groups(desc)
    return tree, make_params(tree, desc, idx)


def rand(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.rand(shape, dtype=D, generator=g) * 2 - 1) * scale


# ---------------------------------------------------------------- kinematics
def test_fk_two_link_planar_closed_form():
    d = chain_desc([([0, 0], [1, 1])], E=5, seed=3)
    tree, P = single(d)
    q = rand((5, 2), 1, 2.0)
    ee, _ = dyn.end_effectors(tree, P, q)
    l1, l2 = P.L[:, 0], P.L[:, 1]
    s1, c1 = torch.sin(q[:, 0]), torch.cos(q[:, 0])
    s12, c12 = torch.sin(q.sum(1)), torch.cos(q.sum(1))
    want = torch.stack([l1 * s1 + l2 * s12, torch.zeros(5, dtype=D), l1 * c1 + l2 * c12], -1)
    assert torch.allclose(ee[:, 0], want, atol=1e-14)


def test_fk_straight_pose_and_z_rotations():
    d = chain_desc([([0] * 7, [2, 1, 2, 1, 2, 1, 2])], E=3, seed=4,
                   base=[(0.1, -0.2, 0.3)])
    tree, P = single(d)
    q0 = torch.zeros(3, 7, dtype=D)
    ee0, _ = dyn.end_effectors(tree, P, q0)
    want = torch.tensor([0.1, -0.2, 0.3], dtype=D) + torch.stack(
        [torch.zeros(3, dtype=D), torch.zeros(3, dtype=D), P.L.sum(1)], -1)
    assert torch.allclose(ee0[:, 0], want, atol=1e-14)
    # rotating the z joints of a straight arm leaves the tip where it is
    qz = q0.clone()
    qz[:, [0, 2, 4, 6]] = rand((3, 4), 2, 3.0)
    eez, _ = dyn.end_effectors(tree, P, qz)
    assert torch.allclose(eez, ee0, atol=1e-14)


def test_fk_prismatic_extends_along_z():
    d = chain_desc([([0, 0, 1, 0], [2, 1, 2, 1])], E=2, seed=5)
    tree, P = single(d)
    q = torch.zeros(2, 4, dtype=D)
    e0, _ = dyn.end_effectors(tree, P, q)
    q[:, 2] = torch.tensor([0.05, 0.17], dtype=D)
    e1, _ = dyn.end_effectors(tree, P, q)
    assert torch.allclose(e1[:, 0, 2] - e0[:, 0, 2], q[:, 2], atol=1e-15)
    assert torch.allclose(e1[:, 0, :2], e0[:, 0, :2], atol=1e-15)


def test_quaternion_matches_fk_rotation():
    d = chain_desc([([0, 0, 1, 0, 0, 0, 0], [2, 1, 2, 1, 2, 0, 2])], E=16, seed=6)
    tree, P = single(d)
    q = rand((16, 7), 7, 3.0)
    _, Rt = dyn.end_effectors(tree, P, q)
    x, y, z, w = tip_quaternion(tree, q)[:, 0].unbind(-1)
    assert (w >= 0).all()
    assert torch.allclose(x * x + y * y + z * z + w * w, torch.ones(16, dtype=D), atol=1e-14)
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        torch.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        torch.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], -2)
    assert torch.allclose(R, Rt[:, 0], atol=1e-13)


# ---------------------------------------------------------------- dynamics
def test_single_pendulum():
    """Link upright at q = 0 rotating about y: I_p qdd = tau + m g c sin q."""
    d = chain_desc([([0], [1])], E=4, seed=8)
    tree, P = single(d)
    q = rand((4, 1), 9, 3.0)
    qdd = rand((4, 1), 10, 5.0)
    m, c, Iyy = P.m[:, 0], P.c[:, 0], P.Ic[:, 0, 1]
    Ip = Iyy + m * c * c
    tau = dyn.rnea(tree, P, q, rand((4, 1), 11), qdd)[:, 0]
    assert torch.allclose(tau, Ip * qdd[:, 0] - m * G * c * torch.sin(q[:, 0]), rtol=1e-13, atol=1e-13)
    # forward dynamics agrees with the same closed form
    qdd_free = dyn.aba(tree, P, q, torch.zeros_like(q), torch.zeros_like(q))[:, 0]
    assert torch.allclose(qdd_free, m * G * c * torch.sin(q[:, 0]) / Ip, rtol=1e-13)


def test_vertical_prismatic_slider():
    """Distal mass on a vertical slider: (sum m) qdd = tau - (sum m) g."""
    d = chain_desc([([1, 0, 0], [2, 2, 2])], E=3, seed=12)
    tree, P = single(d)
    q = torch.zeros(3, 3, dtype=D)
    q[:, 0] = torch.tensor([0.0, 0.1, 0.2], dtype=D)
    q[:, 1:] = rand((3, 2), 13, 3.0)           # z rotations keep the arm vertical
    qdd = rand((3, 3), 14)
    qdd[:, 1:] = 0
    tau = dyn.rnea(tree, P, q, torch.zeros_like(q), qdd)
    msum = P.m.sum(1)
    assert torch.allclose(tau[:, 0], msum * (qdd[:, 0] + G), rtol=1e-13)
    M = dyn.crba(tree, P, q)
    assert torch.allclose(M[:, 0, 0], msum, rtol=1e-14)


def test_two_link_planar_lagrangian_closed_form():
    d = chain_desc([([0, 0], [1, 1])], E=6, seed=15)
    tree, P = single(d)
    q, qd = rand((6, 2), 16, 3.0), rand((6, 2), 17, 2.0)
    m1, m2 = P.m[:, 0], P.m[:, 1]
    l1, c1, c2 = P.L[:, 0], P.c[:, 0], P.c[:, 1]
    I1, I2 = P.Ic[:, 0, 1], P.Ic[:, 1, 1]
    cq2, sq2 = torch.cos(q[:, 1]), torch.sin(q[:, 1])
    M11 = I1 + I2 + m1 * c1 ** 2 + m2 * (l1 ** 2 + c2 ** 2 + 2 * l1 * c2 * cq2)
    M12 = I2 + m2 * (c2 ** 2 + l1 * c2 * cq2)
    M22 = I2 + m2 * c2 ** 2
    M = dyn.crba(tree, P, q)
    assert torch.allclose(M[:, 0, 0], M11, rtol=1e-13)
    assert torch.allclose(M[:, 0, 1], M12, rtol=1e-13)
    assert torch.allclose(M[:, 1, 0], M12, rtol=1e-13)
    assert torch.allclose(M[:, 1, 1], M22, rtol=1e-13)
    hq = -m2 * l1 * c2 * sq2
    Cqd = torch.stack([hq * (2 * qd[:, 0] * qd[:, 1] + qd[:, 1] ** 2), -hq * qd[:, 0] ** 2], -1)
    s1, s12 = torch.sin(q[:, 0]), torch.sin(q.sum(1))
    Gv = torch.stack([-G * ((m1 * c1 + m2 * l1) * s1 + m2 * c2 * s12), -G * m2 * c2 * s12], -1)
    bias = dyn.rnea(tree, P, q, qd, torch.zeros_like(q))
    assert torch.allclose(bias, Cqd + Gv, rtol=1e-12, atol=1e-12)


CHAINS_SMALL = [
    [([0, 0, 0], [2, 1, 0])],
    [([0, 1, 0, 0], [1, 2, 1, 2])],
    [([0, 0, 0, 0], [2, 1, 2, 1])],
]


@pytest.mark.parametrize("chains", CHAINS_SMALL)
def test_lagrangian_fd_matches_rnea_crba(chains):
    d = chain_desc(chains, E=4, seed=18)
    tree, P = single(d)
    n = tree.n
    q, qd, qdd = rand((4, n), 19, 2.0), rand((4, n), 20, 2.0), rand((4, n), 21, 2.0)
    M_l = lag.mass_matrix(tree, P, q)
    M = dyn.crba(tree, P, q)
    assert ((M_l - M).abs().max() / M.abs().max()) < 1e-7
    tau_l = lag.inverse_dynamics(tree, P, q, qd, qdd)
    tau = dyn.rnea(tree, P, q, qd, qdd)
    assert ((tau_l - tau).abs().max() / tau.abs().max()) < 1e-7


@pytest.mark.parametrize("chains", [
    [([0] * 7, [2, 1, 2, 1, 2, 1, 2])],
    [([0, 0, 1, 0, 0, 0, 0], [2, 1, 2, 1, 2, 1, 2])],
    [([0] * 4, [2, 1, 2, 1])],
])
def test_mass_matrix_spd_and_columns(chains):
    d = chain_desc(chains, E=8, seed=22)
    tree, P = single(d)
    n = tree.n
    q = rand((8, n), 23, 3.0)
    M = dyn.crba(tree, P, q)
    assert torch.allclose(M, M.transpose(-1, -2), atol=0)
    assert (torch.linalg.eigvalsh(M)[:, 0] > 0).all()
    zero = torch.zeros_like(q)
    g0 = dyn.rnea(tree, P, q, zero, zero)
    for j in range(n):
        e = torch.zeros_like(q)
        e[:, j] = 1.0
        col = dyn.rnea(tree, P, q, zero, e) - g0
        assert torch.allclose(col, M[:, :, j], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("chains", [
    [([0] * 7, [2, 1, 2, 1, 2, 1, 2])],
    [([0, 0, 1, 0, 0, 0, 0], [2, 1, 2, 1, 2, 1, 2])],
    [([0] * 7, [2, 1, 2, 1, 2, 1, 2]), ([0] * 7, [2, 1, 2, 1, 2, 1, 2])],
])
def test_rnea_of_aba_is_identity(chains):
    d = chain_desc(chains, E=6, seed=24, base=[(0, 0.25, 0), (0, -0.25, 0)])
    tree, P = single(d)
    n = tree.n
    q, qd, tau = rand((6, n), 25, 2.0), rand((6, n), 26, 2.0), rand((6, n), 27, 5.0)
    qdd = dyn.aba(tree, P, q, qd, tau)
    back = dyn.rnea(tree, P, q, qd, qdd)
    assert (back - tau).abs().max() < 1e-10
    # with armature: (M + diag(a)) qdd = tau - c
    arm = rand((6, n), 28).abs() + 0.01
    qdd_a = dyn.aba(tree, P, q, qd, tau, armature=arm)
    M = dyn.crba(tree, P, q)
    c = dyn.rnea(tree, P, q, qd, torch.zeros_like(q))
    lhs = ((M + torch.diag_embed(arm)) @ qdd_a[..., None])[..., 0]
    assert (lhs - (tau - c)).abs().max() < 1e-10


def test_bimanual_mass_matrix_is_block_diagonal():
    arm = ([0] * 7, [2, 1, 2, 1, 2, 1, 2])
    L = list(np.linspace(0.1, 0.3, 7)) * 2
    m = list(np.linspace(0.2, 0.9, 7)) * 2
    d2 = chain_desc([arm, arm], E=4, seed=29, base=[(0, 0.25, 0), (0, -0.25, 0)], L=L, m=m)
    d1 = chain_desc([arm], E=4, seed=29, L=L[:7], m=m[:7])
    t2, P2 = single(d2)
    t1, P1 = single(d1)
    q = rand((4, 14), 30, 2.0)
    M = dyn.crba(t2, P2, q)
    assert M[:, :7, 7:].abs().max() == 0 and M[:, 7:, :7].abs().max() == 0
    for k in range(2):
        Mk = dyn.crba(t1, P1, q[:, 7 * k:7 * k + 7])
        assert torch.allclose(M[:, 7 * k:7 * k + 7, 7 * k:7 * k + 7], Mk, rtol=1e-13)
