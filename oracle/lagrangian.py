"""Equations of motion from the Lagrangian, independent of RNEA/CRBA.

For a tree with link centre-of-mass positions c_i(q) and orientations
R_i(q) from plain 4x4 forward kinematics (written again here, dtype
generic, so that complex arguments work):

    T(q, qd) = 1/2 sum_i ( m_i |d c_i/dt|^2 + w_i^T Ic_i w_i ),
    V(q)     = sum_i m_i g z(c_i),
    w_i      = body-frame angular velocity, skew(w_i) = R_i^T dR_i/dt,

and the Euler-Lagrange equation M(q) qdd + C(q, qd) qd + G(q) = tau with

    M = d^2 T / d qd^2                (polarisation of the quadratic T),
    C(q, qd) qd = Mdot qd - 1/2 d/dq (qd^T M qd),
    G = dV/dq.

Position Jacobians come from the complex-step derivative (Squire and
Trapp 1998: f'(x) = Im f(x + i h) / h, exact to rounding for analytic f);
the q-derivatives of M are central finite differences.
"""
import torch

from .model import PRISMATIC

GRAVITY = 9.81
CSTEP = 1e-30


def _rot(axis, q):
    c, s = torch.cos(q), torch.sin(q)
    o, i = torch.zeros_like(q), torch.ones_like(q)
    if axis == 0:
        rows = [[i, o, o], [o, c, -s], [o, s, c]]
    elif axis == 1:
        rows = [[c, o, s], [o, i, o], [-s, o, c]]
    else:
        rows = [[c, -s, o], [s, c, o], [o, o, i]]
    return torch.stack([torch.stack(r, -1) for r in rows], -2)


def link_poses(tree, P, q):
    """Centres of mass [E, n, 3] and rotations [E, n, 3, 3], in q's dtype."""
    E = q.shape[0]
    dt = q.dtype
    L, c = P.L.to(dt), P.c.to(dt)
    base = P.base.to(dt)
    Rs, ps, coms = [None] * tree.n, [None] * tree.n, [None] * tree.n
    eye = torch.eye(3, dtype=dt).expand(E, 3, 3)
    for i in range(tree.n):
        par = tree.parent[i]
        if par < 0:
            Rp, pp = eye, base[:, tree.chain_of[i]]
        else:
            Rp = Rs[par]
            pp = ps[par] + Rp[:, :, 2] * L[:, par, None]
        if tree.jtype[i] == PRISMATIC:
            Rs[i] = Rp
            ps[i] = pp + Rp[:, :, 2] * q[:, i, None]
        else:
            Rs[i] = Rp @ _rot(tree.axis[i], q[:, i])
            ps[i] = pp
        coms[i] = ps[i] + Rs[i][:, :, 2] * c[:, i, None]
    return torch.stack(coms, 1), torch.stack(Rs, 1)


def jacobians(tree, P, q):
    """d com / d q_j and d R / d q_j by complex step: [E, n, 3, n], [E, n, 3, 3, n]."""
    E, n = q.shape
    Jc, JR = [], []
    for j in range(n):
        qc = q.to(torch.complex128).clone()
        qc[:, j] = qc[:, j] + 1j * CSTEP
        com, R = link_poses(tree, P, qc)
        Jc.append(com.imag / CSTEP)
        JR.append(R.imag / CSTEP)
    return torch.stack(Jc, -1), torch.stack(JR, -1)


def kinetic(tree, P, q, qd):
    Jc, JR = jacobians(tree, P, q)
    _, R = link_poses(tree, P, q)
    v = (Jc * qd[:, None, None, :]).sum(-1)                    # [E, n, 3]
    Rdot = (JR * qd[:, None, None, None, :]).sum(-1)           # [E, n, 3, 3]
    Wb = R.transpose(-1, -2) @ Rdot                            # skew(w_body)
    wb = torch.stack([Wb[..., 2, 1], Wb[..., 0, 2], Wb[..., 1, 0]], -1)
    T = 0.5 * (P.m[..., None] * v * v).sum((-1, -2)) + 0.5 * (P.Ic * wb * wb).sum((-1, -2))
    return T


def potential(tree, P, q):
    com, _ = link_poses(tree, P, q)
    return (P.m * GRAVITY * com[..., 2]).sum(-1)


def mass_matrix(tree, P, q):
    """M_ii = 2 T(e_i), M_ij = T(e_i + e_j) - T(e_i) - T(e_j)."""
    E, n = q.shape
    eye = torch.eye(n, dtype=q.dtype)
    Ti = [kinetic(tree, P, q, eye[i].expand(E, n)) for i in range(n)]
    M = torch.zeros(E, n, n, dtype=q.dtype)
    for i in range(n):
        M[:, i, i] = 2.0 * Ti[i]
        for j in range(i + 1, n):
            Tij = kinetic(tree, P, q, (eye[i] + eye[j]).expand(E, n))
            M[:, i, j] = M[:, j, i] = Tij - Ti[i] - Ti[j]
    return M


def gravity_vector(tree, P, q):
    """G = dV/dq by complex step."""
    E, n = q.shape
    G = []
    for j in range(n):
        qc = q.to(torch.complex128).clone()
        qc[:, j] = qc[:, j] + 1j * CSTEP
        G.append(potential(tree, P, qc).imag / CSTEP)
    return torch.stack(G, -1)


def coriolis(tree, P, q, qd, h=1e-5):
    """C(q, qd) qd = sum_k dM/dq_k qd_k qd - 1/2 [qd^T dM/dq_k qd]_k with
    dM/dq_k by central differences of step h."""
    E, n = q.shape
    dM = []
    for k in range(n):
        e = torch.zeros(n, dtype=q.dtype)
        e[k] = h
        dM.append((mass_matrix(tree, P, q + e) - mass_matrix(tree, P, q - e)) / (2 * h))
    dM = torch.stack(dM, 1)                                     # [E, k, n, n]
    Mdot = (dM * qd[:, :, None, None]).sum(1)
    term1 = (Mdot @ qd[..., None])[..., 0]
    term2 = 0.5 * torch.einsum("ekij,ei,ej->ek", dM, qd, qd)
    return term1 - term2


def inverse_dynamics(tree, P, q, qd, qdd):
    M = mass_matrix(tree, P, q)
    return (M @ qdd[..., None])[..., 0] + coriolis(tree, P, q, qd) + gravity_vector(tree, P, q)


__all__ = ["link_poses", "jacobians", "kinetic", "potential", "mass_matrix",
           "gravity_vector", "coriolis", "inverse_dynamics"]
