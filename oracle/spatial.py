"""Spatial vector algebra (Featherstone 2008, ch. 2), batched, float64.

Motion vectors are [angular; linear], force vectors [moment; force].
A Pluecker transform ``X = rot(E) @ xlt(r)`` maps motion vectors from
frame A coordinates to frame B coordinates, where B's origin sits at ``r``
(A coordinates) and ``E`` maps A coordinates of a free vector to B
coordinates.  Forces transform with ``X^{-T}``; the transpose ``X^T`` maps
B-forces back to A.
"""
import torch

DT = torch.float64


def skew(v):
    """[..., 3] -> [..., 3, 3] with skew(a) @ b = a x b."""
    x, y, z = v.unbind(-1)
    o = torch.zeros_like(x)
    return torch.stack([torch.stack([o, -z, y], -1),
                        torch.stack([z, o, -x], -1),
                        torch.stack([-y, x, o], -1)], -2)


def rot_active(axis, q):
    """Active rotation matrix Rot(axis, q) (axis 0/1/2 = x/y/z), [..., 3, 3]."""
    c, s = torch.cos(q), torch.sin(q)
    o, i = torch.zeros_like(q), torch.ones_like(q)
    if axis == 0:
        rows = [[i, o, o], [o, c, -s], [o, s, c]]
    elif axis == 1:
        rows = [[c, o, s], [o, i, o], [-s, o, c]]
    else:
        rows = [[c, -s, o], [s, c, o], [o, o, i]]
    return torch.stack([torch.stack(r, -1) for r in rows], -2)


def plucker(E, r):
    """X = [[E, 0], [-E skew(r), E]] (motion transform)."""
    Z = torch.zeros_like(E)
    top = torch.cat([E, Z], -1)
    bot = torch.cat([-E @ skew(r), E], -1)
    return torch.cat([top, bot], -2)


def crm(v):
    """Motion cross-product operator v x (.)."""
    w, u = v[..., :3], v[..., 3:]
    W, U = skew(w), skew(u)
    Z = torch.zeros_like(W)
    return torch.cat([torch.cat([W, Z], -1), torch.cat([U, W], -1)], -2)


def crf(v):
    """Force cross-product operator v x* (.) = -crm(v)^T."""
    return -crm(v).transpose(-1, -2)


def mcI(m, c, Ic):
    """Spatial inertia about a frame origin of a body with mass m, centre of
    mass c and rotational inertia Ic about the centre of mass."""
    C = skew(c)
    mm = m[..., None, None]
    top = torch.cat([Ic + mm * (C @ C.transpose(-1, -2)), mm * C], -1)
    eye = torch.eye(3, dtype=m.dtype).expand(C.shape)
    bot = torch.cat([mm * C.transpose(-1, -2), mm * eye], -1)
    return torch.cat([top, bot], -2)
