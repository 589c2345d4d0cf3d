"""Kinematics and dynamics of the oracle (float64, batched over envs).

* ``fk``          forward kinematics by 4x4 homogeneous transforms.
* ``rnea``        recursive Newton-Euler inverse dynamics, tau = ID(q, qd, qdd)
                  (Featherstone 2008, Table 5.1), gravity by base
                  acceleration.
* ``crba``        composite-rigid-body joint-space inertia H(q)
                  (Featherstone 2008, Table 6.2).
* ``aba``         articulated-body forward dynamics with optional joint
                  armature (Featherstone 2008, Table 7.1).
* ``substep``     one implicit-drive semi-implicit Euler substep: the PD
                  drive, joint damping and active limit springs are taken
                  implicitly at the end-of-substep velocity, everything
                  else (gravity, Coriolis, centrifugal) explicitly.  The
                  paper's engine sub-steps each control step (Methods,
                  "Simulation Setup"); the drive formula is the PD joint
                  drive named there; the implicit treatment is a reading
                  (the paper gives no integrator formula).
* ``rk4_step``    classical Runge-Kutta 4 of the continuous dynamics, used
                  only for conservation tests.
"""
import torch

from .model import PRISMATIC
from .spatial import DT, crf, crm, plucker, rot_active

GRAVITY = 9.81


def jcalc(jtype, axis, q):
    """Joint transform X_J(q) and motion subspace S for a batch of angles."""
    E = q.shape[0]
    eye = torch.eye(3, dtype=DT).expand(E, 3, 3)
    S = torch.zeros(E, 6, dtype=DT)
    if jtype == PRISMATIC:
        r = torch.stack([torch.zeros_like(q), torch.zeros_like(q), q], -1)
        S[:, 5] = 1.0
        return plucker(eye, r), S
    S[:, axis] = 1.0
    return plucker(rot_active(axis, q).transpose(-1, -2), torch.zeros(E, 3, dtype=DT)), S


def fk(tree, P, q):
    """World rotation R_i and origin p_i of every link frame (lists)."""
    E = q.shape[0]
    R, p = [None] * tree.n, [None] * tree.n
    for i in range(tree.n):
        par = tree.parent[i]
        if par < 0:
            Rp = torch.eye(3, dtype=DT).expand(E, 3, 3)
            pp = P.base[:, tree.chain_of[i]]
        else:
            Rp = R[par]
            pp = p[par] + Rp[:, :, 2] * P.L[:, par, None]
        if tree.jtype[i] == PRISMATIC:
            R[i] = Rp
            p[i] = pp + Rp[:, :, 2] * q[:, i, None]
        else:
            R[i] = Rp @ rot_active(tree.axis[i], q[:, i])
            p[i] = pp
    return R, p


def end_effectors(tree, P, q):
    """Tool-tip position of every chain: [E, n_chains, 3], and the tip link
    rotations [E, n_chains, 3, 3]."""
    R, p = fk(tree, P, q)
    ee = [p[k] + R[k][:, :, 2] * P.L[:, k, None] for k in tree.tips]
    return torch.stack(ee, 1), torch.stack([R[k] for k in tree.tips], 1)


def rnea(tree, P, q, qd, qdd, gravity=GRAVITY):
    E = q.shape[0]
    n = tree.n
    a0 = torch.zeros(E, 6, dtype=DT)
    a0[:, 5] = gravity                      # base acceleration = -g
    Xup, S, v, a, f = [None] * n, [None] * n, [None] * n, [None] * n, [None] * n
    for i in range(n):
        XJ, S[i] = jcalc(tree.jtype[i], tree.axis[i], q[:, i])
        Xup[i] = XJ @ P.XT[i]
        vJ = S[i] * qd[:, i, None]
        par = tree.parent[i]
        if par < 0:
            v[i] = vJ
            a[i] = (Xup[i] @ a0[..., None])[..., 0] + S[i] * qdd[:, i, None]
        else:
            v[i] = (Xup[i] @ v[par][..., None])[..., 0] + vJ
            a[i] = ((Xup[i] @ a[par][..., None])[..., 0] + S[i] * qdd[:, i, None]
                    + (crm(v[i]) @ vJ[..., None])[..., 0])
        Iv = (P.I[i] @ v[i][..., None])[..., 0]
        f[i] = (P.I[i] @ a[i][..., None])[..., 0] + (crf(v[i]) @ Iv[..., None])[..., 0]
    tau = [None] * n
    for i in reversed(range(n)):
        tau[i] = (S[i] * f[i]).sum(-1)
        par = tree.parent[i]
        if par >= 0:
            f[par] = f[par] + (Xup[i].transpose(-1, -2) @ f[i][..., None])[..., 0]
    return torch.stack(tau, -1)


def crba(tree, P, q):
    E = q.shape[0]
    n = tree.n
    Xup, S = [None] * n, [None] * n
    for i in range(n):
        XJ, S[i] = jcalc(tree.jtype[i], tree.axis[i], q[:, i])
        Xup[i] = XJ @ P.XT[i]
    IC = list(P.I)
    for i in reversed(range(n)):
        par = tree.parent[i]
        if par >= 0:
            IC[par] = IC[par] + Xup[i].transpose(-1, -2) @ IC[i] @ Xup[i]
    H = [[None] * n for _ in range(n)]
    zero = torch.zeros(E, dtype=DT)
    for i in range(n):
        F = (IC[i] @ S[i][..., None])[..., 0]
        H[i][i] = (S[i] * F).sum(-1)
        j = i
        while tree.parent[j] >= 0:
            F = (Xup[j].transpose(-1, -2) @ F[..., None])[..., 0]
            j = tree.parent[j]
            H[i][j] = H[j][i] = (S[j] * F).sum(-1)
    rows = [torch.stack([H[i][j] if H[i][j] is not None else zero for j in range(n)], -1)
            for i in range(n)]
    return torch.stack(rows, -2)


def aba(tree, P, q, qd, tau, armature=None, gravity=GRAVITY):
    """qdd = FD(q, qd, tau) with an optional joint armature [E, n] added to
    each joint's articulated inertia (D_i = S^T U_i + armature_i)."""
    E = q.shape[0]
    n = tree.n
    a0 = torch.zeros(E, 6, dtype=DT)
    a0[:, 5] = gravity
    Xup, S, v, c, IA, pA = [[None] * n for _ in range(6)]
    for i in range(n):
        XJ, S[i] = jcalc(tree.jtype[i], tree.axis[i], q[:, i])
        Xup[i] = XJ @ P.XT[i]
        vJ = S[i] * qd[:, i, None]
        par = tree.parent[i]
        if par < 0:
            v[i] = vJ
            c[i] = torch.zeros(E, 6, dtype=DT)
        else:
            v[i] = (Xup[i] @ v[par][..., None])[..., 0] + vJ
            c[i] = (crm(v[i]) @ vJ[..., None])[..., 0]
        IA[i] = P.I[i]
        pA[i] = (crf(v[i]) @ (P.I[i] @ v[i][..., None]))[..., 0]
    U, d, u = [None] * n, [None] * n, [None] * n
    for i in reversed(range(n)):
        U[i] = (IA[i] @ S[i][..., None])[..., 0]
        d[i] = (S[i] * U[i]).sum(-1)
        if armature is not None:
            d[i] = d[i] + armature[:, i]
        u[i] = tau[:, i] - (S[i] * pA[i]).sum(-1)
        par = tree.parent[i]
        if par >= 0:
            Ia = IA[i] - U[i][..., :, None] * U[i][..., None, :] / d[i][:, None, None]
            pa = (pA[i] + (Ia @ c[i][..., None])[..., 0]
                  + U[i] * (u[i] / d[i])[:, None])
            XtT = Xup[i].transpose(-1, -2)
            IA[par] = IA[par] + XtT @ Ia @ Xup[i]
            pA[par] = pA[par] + (XtT @ pa[..., None])[..., 0]
    a = [None] * n
    qdd = [None] * n
    for i in range(n):
        par = tree.parent[i]
        ap = a0 if par < 0 else a[par]
        ai = (Xup[i] @ ap[..., None])[..., 0] + c[i]
        qdd[i] = (u[i] - (U[i] * ai).sum(-1)) / d[i]
        a[i] = ai + S[i] * qdd[i][:, None]
    return torch.stack(qdd, -1)


def limit_state(P, q):
    """Limit-spring torque tau_lim(q) and activity mask at q: a spring of
    stiffness k_limit pushes back beyond q_hi / below q_lo, zero inside."""
    hi = q > P.q_hi
    lo = q < P.q_lo
    tau_lim = torch.where(hi, -P.klim * (q - P.q_hi),
                          torch.where(lo, -P.klim * (q - P.q_lo), torch.zeros_like(q)))
    return tau_lim, (hi | lo)


def drive_law(P, q, qd, a):
    """Joint torque of the drive and its implicit coefficients, per joint
    command type (Methods, "Simulation Setup": position or velocity PD
    targets, or torques):
        position: tau = kp (a - q) - (kd + b) qd + tau_lim,  k_s = kp + k_lim[act], d = kd + b
        velocity: tau = kd (a - qd) - b qd + tau_lim,        k_s = k_lim[act],      d = kd + b
        torque:   tau = a - b qd + tau_lim,                  k_s = k_lim[act],      d = b
    Returns (tau, k_s, d)."""
    tau_lim, active = limit_state(P, q)
    klim = P.klim * active.to(DT)
    pos, vel = P.drive == 0, P.drive == 1
    tau = torch.where(pos, P.kp * (a - q) - (P.kd + P.b) * qd,
                      torch.where(vel, P.kd * (a - qd) - P.b * qd, a - P.b * qd)) + tau_lim
    ks = torch.where(pos, P.kp + klim, klim)
    d = torch.where(pos | vel, P.kd + P.b, P.b)
    return tau, ks, d


def substep(tree, P, q, qd, qstar, h, gravity=GRAVITY):
    """One implicit-drive semi-implicit Euler substep of length h.

    With the drive torque tau_d, stiffness k_s and damping d of
    ``drive_law`` (all taken at the substep start), the velocity change solves
        (M(q) + h d I + h^2 k_s I) dqd = h (tau_d - h k_s qd - c(q, qd)),
    i.e. stiffness and damping act at the end-of-substep state; then
    qd' = qd + dqd and q' = q + h qd'.  Returns (q', qd', dqd/h).
    """
    tau_d, ks, d = drive_law(P, q, qd, qstar)
    c = rnea(tree, P, q, qd, torch.zeros_like(q), gravity)
    M = crba(tree, P, q)
    A = M + torch.diag_embed(h * d + h * h * ks)
    rhs = h * (tau_d - h * ks * qd - c)
    # cholesky_ex: a non-finite state yields NaN (flagged by the caller)
    # instead of an exception
    Lc, _ = torch.linalg.cholesky_ex(A)
    dqd = torch.cholesky_solve(rhs[..., None], Lc)[..., 0]
    qd1 = qd + dqd
    q1 = q + h * qd1
    return q1, qd1, dqd / h


def free_accel(tree, P, q, qd, gravity=GRAVITY):
    """Continuous dynamics with drives, damping and limits off."""
    return aba(tree, P, q, qd, torch.zeros_like(q), gravity=gravity)


def rk4_step(tree, P, q, qd, h, gravity=GRAVITY):
    def f(x, v):
        return v, free_accel(tree, P, x, v, gravity)
    k1q, k1v = f(q, qd)
    k2q, k2v = f(q + 0.5 * h * k1q, qd + 0.5 * h * k1v)
    k3q, k3v = f(q + 0.5 * h * k2q, qd + 0.5 * h * k2v)
    k4q, k4v = f(q + h * k3q, qd + h * k3v)
    q1 = q + h / 6.0 * (k1q + 2 * k2q + 2 * k3q + k4q)
    qd1 = qd + h / 6.0 * (k1v + 2 * k2v + 2 * k3v + k4v)
    return q1, qd1


def energy(tree, P, q, qd, gravity=GRAVITY):
    """Kinetic energy from the link spatial velocities plus potential energy
    of the link centres of mass (height times weight)."""
    E = q.shape[0]
    n = tree.n
    Xup, v = [None] * n, [None] * n
    T = torch.zeros(E, dtype=DT)
    for i in range(n):
        XJ, S = jcalc(tree.jtype[i], tree.axis[i], q[:, i])
        Xup[i] = XJ @ P.XT[i]
        vJ = S * qd[:, i, None]
        par = tree.parent[i]
        v[i] = vJ if par < 0 else (Xup[i] @ v[par][..., None])[..., 0] + vJ
        T = T + 0.5 * (v[i] * (P.I[i] @ v[i][..., None])[..., 0]).sum(-1)
    R, p = fk(tree, P, q)
    V = torch.zeros(E, dtype=DT)
    for i in range(n):
        com = p[i] + R[i][:, :, 2] * P.c[:, i, None]
        V = V + P.m[:, i] * gravity * com[:, 2]
    return T, V
