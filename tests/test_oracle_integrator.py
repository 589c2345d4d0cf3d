"""Pins of the oracle's implicit-drive substep and of energy conservation."""
import numpy as np
import torch

from oracle import dynamics as dyn
from oracle.model import groups, make_params
from tests.helpers import chain_desc

D = torch.float64
G = 9.81


def single(desc):
    (idx, tree), = groups(desc)
    return tree, make_params(tree, desc, idx)


def rand(shape, seed, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.rand(shape, dtype=D, generator=g) * 2 - 1) * scale


def test_zero_gains_reduce_to_symplectic_euler_pendulum():
    """kp = kd = b = k_lim = 0: qd' = qd + h qdd(q, qd), q' = q + h qd'
    with the pendulum's closed-form acceleration m g c sin(q) / I_p."""
    d = chain_desc([([0], [1])], E=3, seed=1)
    tree, P = single(d)
    q, qd = rand((3, 1), 2, 2.0), rand((3, 1), 3, 2.0)
    h = 1.0 / 240
    q1, qd1, qdd = dyn.substep(tree, P, q, qd, torch.zeros_like(q), h)
    m, c, Iyy = P.m[:, 0], P.c[:, 0], P.Ic[:, 0, 1]
    acc = m * G * c * torch.sin(q[:, 0]) / (Iyy + m * c * c)
    assert torch.allclose(qd1[:, 0], qd[:, 0] + h * acc, rtol=1e-13)
    assert torch.allclose(q1[:, 0], q[:, 0] + h * qd1[:, 0], rtol=1e-13)
    assert torch.allclose(qdd[:, 0], acc, rtol=1e-12)


def test_implicit_drive_residual():
    """The substep satisfies M (qd'-qd)/h + c(q, qd) = kp (q* - q - h qd')
    - d qd' + tau_lim(q) - h k_lim[active] qd'."""
    d = chain_desc([([0, 0, 1, 0, 0, 0, 0], [2, 1, 2, 1, 2, 1, 2])], E=8, seed=4,
                   kp=50.0, kd=5.0, damping=0.1, k_limit=1e3)
    tree, P = single(d)
    q = rand((8, 7), 5, 2.2)
    q[:, 2] = rand((8,), 6, 0.3) + 0.1
    qd, qs = rand((8, 7), 7, 2.0), rand((8, 7), 8, 1.5)
    h = 1.0 / 120
    q1, qd1, _ = dyn.substep(tree, P, q, qd, qs, h)
    M = dyn.crba(tree, P, q)
    c = dyn.rnea(tree, P, q, qd, torch.zeros_like(q))
    tau_lim, active = dyn.limit_state(P, q)
    assert active.any() and (~active).any()
    dd = P.kd + P.b
    lhs = (M @ ((qd1 - qd) / h)[..., None])[..., 0] + c
    rhs = (P.kp * (qs - q - h * qd1) - dd * qd1 + tau_lim
           - h * P.klim * active.to(D) * qd1)
    assert ((lhs - rhs).abs().max() / rhs.abs().max()) < 1e-11
    # the implicit solve is ABA with armature h d + h^2 k_s
    ks = P.kp + P.klim * active.to(D)
    tau_eff = P.kp * (qs - q) - dd * qd + tau_lim - h * ks * qd
    qdd = dyn.aba(tree, P, q, qd, tau_eff, armature=h * dd + h * h * ks)
    assert torch.allclose(qdd, (qd1 - qd) / h, rtol=1e-9, atol=1e-9)


def test_pd_drive_converges_to_target_without_gravity():
    d = chain_desc([([0] * 4, [2, 1, 2, 1])], E=4, seed=9, kp=50.0, kd=5.0, damping=0.1)
    tree, P = single(d)
    q, qd = torch.zeros(4, 4, dtype=D), torch.zeros(4, 4, dtype=D)
    qs = rand((4, 4), 10, 1.2)
    for _ in range(3000):
        q, qd, _ = dyn.substep(tree, P, q, qd, qs, 1.0 / 120, gravity=0.0)
    assert torch.allclose(q, qs, atol=1e-8)
    assert qd.abs().max() < 1e-8


def _energy_drift_rk4(gravity):
    d = chain_desc([([0, 0, 0], [2, 1, 1])], E=3, seed=11)
    tree, P = single(d)
    q, qd = rand((3, 3), 12, 1.0), rand((3, 3), 13, 2.0)
    T0, V0 = dyn.energy(tree, P, q, qd, gravity)
    E0 = T0 + V0
    for _ in range(1000):
        q, qd = dyn.rk4_step(tree, P, q, qd, 1e-4, gravity)
    T1, V1 = dyn.energy(tree, P, q, qd, gravity)
    scale = T0.abs() + V0.abs()
    return ((T1 + V1 - E0).abs() / scale.abs()).max().item()


def test_energy_conserved_rk4_gravity_off():
    assert _energy_drift_rk4(0.0) < 1e-6


def test_energy_conserved_rk4_gravity_on():
    d = _energy_drift_rk4(G)
    assert d < 1e-6


def _semi_implicit_energy_error(chains, gravity, h, seconds=1000 / 120):
    d = chain_desc(chains, E=4, seed=14)
    tree, P = single(d)
    n = tree.n
    q, qd = rand((4, n), 15, 1.0), rand((4, n), 16, 1.0)
    T0, V0 = dyn.energy(tree, P, q, qd, gravity)
    steps = int(round(seconds / h))
    first, second = 0.0, 0.0
    for k in range(steps):
        q, qd, _ = dyn.substep(tree, P, q, qd, torch.zeros_like(q), h, gravity=gravity)
        if k % 5 == 0:
            T, V = dyn.energy(tree, P, q, qd, gravity)
            err = ((T + V - T0 - V0).abs() / (T0.abs() + V0.abs())).max().item()
            if k < steps // 2:
                first = max(first, err)
            else:
                second = max(second, err)
    return first, second


def test_semi_implicit_energy_bounded_first_order():
    """Zero gains: the substep is symplectic Euler.  Over 1000 steps at
    h = 1/120 the energy error stays small and halves when h halves (first
    order).  For the pendulum (constant inertia, exactly symplectic) it
    also shows no secular growth: the second half of the run is no worse
    than the first."""
    f1, s1 = _semi_implicit_energy_error([([0], [1])], 9.81, 1 / 120)
    f2, s2 = _semi_implicit_energy_error([([0], [1])], 9.81, 1 / 240)
    assert max(f1, s1) < 5e-2 and s1 <= 1.1 * f1
    assert 0.45 < max(f2, s2) / max(f1, s1) < 0.55
    f1, s1 = _semi_implicit_energy_error([([0, 0], [1, 1])], 0.0, 1 / 120)
    f2, s2 = _semi_implicit_energy_error([([0, 0], [1, 1])], 0.0, 1 / 240)
    assert max(f1, s1) < 1e-2
    assert 0.45 < max(f2, s2) / max(f1, s1) < 0.55


def test_limit_spring_pushes_back():
    d = chain_desc([([0], [2])], E=2, seed=17, k_limit=1e3)
    tree, P = single(d)
    q = torch.tensor([[2.0], [-2.0]], dtype=D)
    tau, active = dyn.limit_state(P, q)
    assert active.all()
    assert tau[0, 0] < 0 and tau[1, 0] > 0
    assert np.isclose(tau[0, 0].item(), -1e3 * (2.0 - P.q_hi[0, 0].item()))


def test_torque_command_pendulum_closed_form():
    """Torque commands (no damping): qd' = qd + h (a + m g c sin q) / I_p."""
    d = chain_desc([([0], [1])], E=3, seed=21, drive=2, kp=50.0, kd=5.0)
    tree, P = single(d)
    q, qd, a = rand((3, 1), 22, 1.5), rand((3, 1), 23, 1.0), rand((3, 1), 24, 2.0)
    h = 1.0 / 240
    q1, qd1, _ = dyn.substep(tree, P, q, qd, a, h)
    m, c, Iyy = P.m[:, 0], P.c[:, 0], P.Ic[:, 0, 1]
    acc = (a[:, 0] + m * G * c * torch.sin(q[:, 0])) / (Iyy + m * c * c)
    assert torch.allclose(qd1[:, 0], qd[:, 0] + h * acc, rtol=1e-13)


def test_velocity_command_converges_to_damped_target_speed():
    """A free joint about the vertical axis under a velocity target v*:
    I qdd = kd (v* - qd) - b qd, so qd -> kd v* / (kd + b)."""
    d = chain_desc([([0], [2])], E=2, seed=25, drive=1, kp=50.0, kd=5.0, damping=0.4)
    tree, P = single(d)
    q, qd = torch.zeros(2, 1, dtype=D), torch.zeros(2, 1, dtype=D)
    v = torch.tensor([[1.5], [-0.7]], dtype=D)
    for _ in range(2000):
        q, qd, _ = dyn.substep(tree, P, q, qd, v, 1.0 / 120)
    assert torch.allclose(qd, v * 5.0 / 5.4, rtol=1e-9)


def test_command_types_residual():
    """Every command type satisfies its implicit-drive equation
    M (qd' - qd)/h + c = tau(q, qd', a) with stiffness at q + h qd'."""
    for mode in (1, 2):
        d = chain_desc([([0, 0, 1, 0], [2, 1, 2, 1])], E=6, seed=26 + mode, kp=50.0, kd=5.0,
                       damping=0.1, k_limit=1e3, drive=mode)
        tree, P = single(d)
        q = rand((6, 4), 27, 2.2)
        q[:, 2] = rand((6,), 28, 0.3) + 0.1
        qd, a = rand((6, 4), 29, 2.0), rand((6, 4), 30, 1.5)
        h = 1.0 / 120
        q1, qd1, _ = dyn.substep(tree, P, q, qd, a, h)
        M = dyn.crba(tree, P, q)
        c = dyn.rnea(tree, P, q, qd, torch.zeros_like(q))
        tau_lim, active = dyn.limit_state(P, q)
        drive = (P.kd * (a - qd1) - P.b * qd1) if mode == 1 else (a - P.b * qd1)
        rhs = drive + tau_lim - h * P.klim * active.to(D) * qd1
        lhs = (M @ ((qd1 - qd) / h)[..., None])[..., 0] + c
        assert ((lhs - rhs).abs().max() / rhs.abs().max()) < 1e-11
