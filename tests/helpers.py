"""Small hand-built robot descriptions for the oracle and parity tests."""
import numpy as np


def chain_desc(chains, E=1, *, kp=0.0, kd=0.0, damping=0.0, k_limit=0.0,
               q_lo=-1.5707963, q_hi=1.5707963, base=None, episode_len=100, seed=0,
               width=0.05, L=None, m=None, drive=None):
    """``chains`` = list of (types, axes) per chain.  Link lengths/masses are
    drawn U[0.05, 0.4] / U[0.1, 1.0] unless given; inertias are solid boxes of
    side ``width`` (given to the oracle as plain inputs)."""
    rng = np.random.default_rng(seed)
    J = sum(len(t) for t, _ in chains)
    f32 = np.float32
    d = dict(num_envs=E, max_joints=J, episode_len=episode_len, task=0, alpha=1.0,
             path=None, path_len=0)
    d["env_num_chains"] = np.full(E, len(chains), np.int32)
    d["chain_num_joints"] = np.zeros((E, 4), np.int32)
    d["joint_type"] = np.zeros((E, J), np.int32)
    d["joint_axis"] = np.zeros((E, J), np.int32)
    for k in ("link_len", "link_mass", "link_com", "q_lo", "q_hi", "kp", "kd", "damping",
              "k_limit", "q0"):
        d[k] = np.zeros((E, J), f32)
    d["link_inertia"] = np.zeros((E, J, 3), f32)
    d["base_offset"] = np.zeros((E, 4, 3), f32)
    d["goal"] = np.zeros((E, 4, 3), f32)
    for e in range(E):
        j = 0
        for c, (types, axes) in enumerate(chains):
            d["chain_num_joints"][e, c] = len(types)
            if base is not None:
                d["base_offset"][e, c] = base[c]
            for i, (t, a) in enumerate(zip(types, axes)):
                Lj = rng.uniform(0.05, 0.4) if L is None else L[j]
                mj = rng.uniform(0.1, 1.0) if m is None else m[j]
                d["joint_type"][e, j] = t
                d["joint_axis"][e, j] = a
                d["link_len"][e, j] = Lj
                d["link_mass"][e, j] = mj
                d["link_com"][e, j] = Lj / 2
                ix = mj * (Lj * Lj + width * width) / 12
                d["link_inertia"][e, j] = (ix, ix, mj * width * width / 12)
                d["q_lo"][e, j], d["q_hi"][e, j] = (0.0, 0.2) if t == 1 else (q_lo, q_hi)
                d["kp"][e, j], d["kd"][e, j], d["damping"][e, j] = kp, kd, damping
                d["k_limit"][e, j] = k_limit
                j += 1
    if drive is not None:
        d["joint_drive"] = np.broadcast_to(np.asarray(drive, np.int32), (E, J)).copy()
    return d
