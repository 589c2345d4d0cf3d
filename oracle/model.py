"""Robot trees for the oracle, built from an ``sg_desc`` dictionary.

An environment is one or two serial chains on a fixed base (Methods,
"Simulation Setup": actors of rigid bodies joined by revolute/prismatic
joints; Results, "Multi-Tool Target Reaching": several arms in one
environment).  The oracle treats the whole environment as one kinematic
tree with parent indices, so a two-arm environment is a single tree whose
two roots hang off the fixed base.

Geometry of joint i (0-based within its chain): its frame sits at
(0, 0, L_{i-1}) in the parent link's frame (at the chain's base offset for
i = 0); a revolute joint then rotates about its local x/y/z axis, a
prismatic joint translates along local z.  Link i extends along its local
+z; its centre of mass is at (0, 0, c_i) with diagonal rotational inertia
about the centre of mass.
"""
from dataclasses import dataclass

import numpy as np
import torch

from .spatial import DT, mcI, plucker

REVOLUTE, PRISMATIC = 0, 1


@dataclass(frozen=True)
class Tree:
    n: int
    parent: tuple
    jtype: tuple
    axis: tuple
    chain_of: tuple
    tips: tuple          # last joint of each chain
    n_chains: int


@dataclass
class Params:
    """Per-env link parameters of one structure group (float64, [E, n])."""
    L: torch.Tensor
    c: torch.Tensor
    m: torch.Tensor
    Ic: torch.Tensor       # [E, n, 3] diagonal inertia about the COM
    base: torch.Tensor     # [E, n_chains, 3]
    q_lo: torch.Tensor
    q_hi: torch.Tensor
    kp: torch.Tensor
    kd: torch.Tensor
    b: torch.Tensor
    klim: torch.Tensor
    drive: torch.Tensor    # [E, n] 0 position, 1 velocity, 2 torque command
    XT: list               # n x [E, 6, 6] fixed parent->joint transforms
    I: list                # n x [E, 6, 6] spatial inertias about link origins


def structure_key(desc, e):
    nc = int(desc["env_num_chains"][e])
    key, j0 = [], 0
    for c in range(nc):
        n = int(desc["chain_num_joints"][e, c])
        key.append((n, tuple(int(t) for t in desc["joint_type"][e, j0:j0 + n]),
                    tuple(int(a) for a in desc["joint_axis"][e, j0:j0 + n])))
        j0 += n
    return tuple(key)


def tree_from_key(key):
    parent, jtype, axis, chain_of, tips = [], [], [], [], []
    j0 = 0
    for c, (n, types, axes) in enumerate(key):
        for i in range(n):
            parent.append(-1 if i == 0 else j0 + i - 1)
            jtype.append(types[i])
            axis.append(axes[i])
            chain_of.append(c)
        tips.append(j0 + n - 1)
        j0 += n
    return Tree(j0, tuple(parent), tuple(jtype), tuple(axis), tuple(chain_of),
                tuple(tips), len(key))


def make_params(tree, desc, env_idx, mass=None):
    """Float64 parameters of the envs ``env_idx``.  If ``mass`` ([E, n]
    float64 tensor, possibly requiring grad) is given it replaces the link
    masses and the rotational inertias scale with it (fixed box size)."""
    n = tree.n
    t = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64)[env_idx][:, :n])
    L, c, m0 = t(desc["link_len"]), t(desc["link_com"]), t(desc["link_mass"])
    Ic0 = torch.as_tensor(np.asarray(desc["link_inertia"], np.float64)[env_idx][:, :n])
    m = m0 if mass is None else mass
    Ic = Ic0 if mass is None else Ic0 * (mass / m0)[..., None]
    base = torch.as_tensor(np.asarray(desc["base_offset"], np.float64)[env_idx][:, :tree.n_chains])
    E = len(env_idx)
    eye = torch.eye(3, dtype=DT).expand(E, 3, 3)
    XT, I = [], []
    for i in range(n):
        p = tree.parent[i]
        if p < 0:
            r = base[:, tree.chain_of[i]]
        else:
            r = torch.stack([torch.zeros(E, dtype=DT), torch.zeros(E, dtype=DT), L[:, p]], -1)
        XT.append(plucker(eye, r))
        com = torch.stack([torch.zeros(E, dtype=DT), torch.zeros(E, dtype=DT), c[:, i]], -1)
        I.append(mcI(m[:, i], com, torch.diag_embed(Ic[:, i])))
    jd = desc.get("joint_drive")
    drive = (torch.zeros(E, n, dtype=torch.long) if jd is None
             else torch.as_tensor(np.asarray(jd, dtype=np.int64)[env_idx][:, :n]))
    return Params(L, c, m, Ic, base, t(desc["q_lo"]), t(desc["q_hi"]), t(desc["kp"]),
                  t(desc["kd"]), t(desc["damping"]), t(desc["k_limit"]), drive, XT, I)


def groups(desc):
    """Split the envs of ``desc`` by structure: [(env_idx, Tree)]."""
    by = {}
    for e in range(int(desc["num_envs"])):
        by.setdefault(structure_key(desc, e), []).append(e)
    return [(np.array(idx), tree_from_key(k)) for k, idx in by.items()]
