"""The device chain code, compiled for the host in double precision, against
the FP64 oracle (no GPU).

tests/host_chain/driver.cpp runs sg_chain.cuh / sg_adjoint.cuh / sg_rng.cuh
with `float` replaced by `double` on parameter records made by the library's
own packer, one chain at a time.  In double precision the device algorithm (body-frame
RNEA, composite-rigid-body mass matrix, in-register Cholesky, the adjoint's
inverse-dynamics sweeps and their reverse) and the oracle's (spatial-algebra
RNEA/CRBA, library Cholesky, autograd) differ only by rounding and by the
packer's float32 sum kd + b (relative 6e-8), so one substep's state and its
vector-Jacobian product must agree to 1e-6 relative (measured: 1e-9 to
3e-8) -- a check of the device formulas a hundred times tighter than the
FP32 parity tests, run on every CPU test pass.  The tool-tip pose, the
tip quaternion and the tip Jacobian-transpose product involve no packed sums
and agree to 1e-12, as do the counter-based noise draws (exact integer
key arithmetic, double-precision Box-Muller); the adjoint's inverse-dynamics
sweeps give the oracle's RNEA torques to 1e-10, and the warp pair's split
of a substep (bias-only and mass-only sweeps, shared solve) equals the
fused substep.  A sign flipped in the
Coriolis term, in the adjoint's prismatic-offset term or a dropped moment
term in the mass cotangent moves the result by 1e-4 to 0.5.
"""
import ctypes
import os
import re
import shutil
import subprocess

import numpy as np
import pytest
import torch

from oracle import dynamics as dyn
from oracle.env import tip_quaternion
from oracle.model import groups, make_params
from oracle.rng import action_noise, goal_noise
from paper_2310_04676_gb300 import sg, workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2310_04676_gb300", "csrc")
D64 = torch.float64
H = 1.0 / 120.0
TOL = 1e-6


def _host_copy(src, dst, drop):
    text = open(src).read()
    for inc in drop:
        text = text.replace(inc, "")
    with open(dst, "w") as f:
        f.write(re.sub(r"\bfloat\b", "double", text))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("needs a host C++ compiler")
    tmp = str(tmp_path_factory.mktemp("host_chain"))
    _host_copy(os.path.join(CSRC, "sg_chain.cuh"), os.path.join(tmp, "chain_host.h"),
               ["#include <cuda_runtime.h>"])
    _host_copy(os.path.join(CSRC, "sg_adjoint.cuh"), os.path.join(tmp, "adjoint_host.h"),
               ['#include "sg_chain.cuh"'])
    _host_copy(os.path.join(CSRC, "sg_rng.cuh"), os.path.join(tmp, "rng_host.h"), [])
    so = os.path.join(tmp, "libhostchain.so")
    cmd = [cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I" + tmp, "-I" + CSRC,
           "-I" + os.path.join(ROOT, "include"), os.path.join(HERE, "host_chain", "driver.cpp"),
           os.path.join(CSRC, "sg_pack.cpp"), "-o", so]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    L = ctypes.CDLL(so)
    dp = ctypes.POINTER(ctypes.c_double)
    L.host_plan.argtypes = [ctypes.c_void_p]
    L.host_substep.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp, dp]
    L.host_substep_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double,
                                       dp, dp, dp, dp]
    L.host_tip.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
    L.host_tip_vjp.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp]
    L.host_inverse_dynamics.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
    L.host_substep_split.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double, dp,
                                     dp]
    L.host_goal_noise.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
    L.host_action_noise.argtypes = [ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_longlong,
                                    dp]
    return L


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _desc(kinds, variant):
    """Six envs of `kinds`: position drives; position drives with limit
    springs (k = 1e3); or the three command types mixed over the joints."""
    desc = W.make_desc((kinds * 6)[:6], k_limit=1e3 if variant == "limits" else 0.0)
    if variant == "drives":
        E, J = desc["num_envs"], desc["max_joints"]
        desc["joint_drive"] = ((np.arange(J)[None] + np.arange(E)[:, None]) % 3).astype(np.int32)
    return desc


def _plan(lib, desc):
    cdesc, keep = sg.make_c_desc(desc)
    n = lib.host_plan(ctypes.byref(cdesc))
    assert n > 0
    return keep


def _state(desc, seed):
    """Random joint positions inside (and, for limit springs, a little
    beyond) the limits, velocities and commands, [E][J]."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(desc["q_lo"], np.float64), np.asarray(desc["q_hi"], np.float64)
    span = hi - lo
    q = lo - 0.1 * span + 1.2 * span * rng.random(lo.shape)
    qd = rng.normal(0.0, 1.0, lo.shape)
    qs = lo + span * rng.random(lo.shape)
    return q, qd, qs


def _chains(desc, e):
    """(chain index, first joint, joints) of env e."""
    out, jo = [], 0
    for c in range(int(desc["env_num_chains"][e])):
        n = int(desc["chain_num_joints"][e][c])
        out.append((c, jo, n))
        jo += n
    return out


KINDS = [["7R"], ["7P"], ["4R"], ["14B"], ["21T"], ["7R", "4R", "7P", "14B", "21T"]]


@pytest.mark.parametrize("kinds", KINDS, ids=lambda k: "+".join(k))
@pytest.mark.parametrize("variant", ["position", "limits", "drives"])
def test_substep_matches_oracle(lib, kinds, variant):
    desc = _desc(kinds, variant)
    keep = _plan(lib, desc)
    q, qd, qs = _state(desc, 1)
    for idx, tree in groups(desc):
        n = tree.n
        P = make_params(tree, desc, idx)
        t = lambda a: torch.as_tensor(a[idx, :n])
        q1, qd1, _ = dyn.substep(tree, P, t(q), t(qd), t(qs), H)
        for k, e in enumerate(idx):
            for c, jo, nc in _chains(desc, e):
                qo, qdo = np.zeros(7), np.zeros(7)
                args = [np.ascontiguousarray(a[e, jo:jo + nc]) for a in (q, qd, qs)]
                assert lib.host_substep(int(e), c, *map(_p, args), H, _p(qo), _p(qdo)) == nc
                for got, ref in ((qo[:nc], q1[k, jo:jo + nc]), (qdo[:nc], qd1[k, jo:jo + nc])):
                    ref = ref.numpy()
                    assert np.linalg.norm(got - ref) <= TOL * max(np.linalg.norm(ref), 1.0), \
                        (variant, kinds, e, c)
    del keep


@pytest.mark.parametrize("kinds", KINDS, ids=lambda k: "+".join(k))
@pytest.mark.parametrize("variant", ["position", "limits", "drives"])
def test_substep_adjoint_matches_oracle_autograd(lib, kinds, variant):
    """Cotangents of (q, qd), the commands and the link masses of one
    substep's output functional lq.q' + lqd.qd', against autograd through
    the oracle's substep."""
    desc = _desc(kinds, variant)
    keep = _plan(lib, desc)
    q, qd, qs = _state(desc, 2)
    rng = np.random.default_rng(3)
    lq, lqd = rng.normal(size=q.shape), rng.normal(size=q.shape)
    mass = np.asarray(desc["link_mass"], np.float64)
    for idx, tree in groups(desc):
        n = tree.n
        t = lambda a: torch.tensor(a[idx, :n], dtype=D64, requires_grad=True)
        Q, QD, QS, M = t(q), t(qd), t(qs), t(mass)
        P = make_params(tree, desc, idx, mass=M)
        q1, qd1, _ = dyn.substep(tree, P, Q, QD, QS, H)
        L = (torch.as_tensor(lq[idx, :n]) * q1).sum() + (torch.as_tensor(lqd[idx, :n]) * qd1).sum()
        gq, gqd, gqs, gm = torch.autograd.grad(L, [Q, QD, QS, M])
        for k, e in enumerate(idx):
            for c, jo, nc in _chains(desc, e):
                sl = slice(jo, jo + nc)
                a_q, a_qd = np.ascontiguousarray(lq[e, sl]), np.ascontiguousarray(lqd[e, sl])
                lqs, lm = np.zeros(nc), np.zeros(nc)
                args = [np.ascontiguousarray(a[e, sl]) for a in (q, qd, qs)]
                assert lib.host_substep_adjoint(int(e), c, *map(_p, args), H, _p(a_q), _p(a_qd),
                                                _p(lqs), _p(lm)) == nc
                for got, ref in ((a_q, gq), (a_qd, gqd), (lqs, gqs), (lm, gm)):
                    ref = ref[k, sl].numpy()
                    assert np.linalg.norm(got - ref) <= TOL * max(np.linalg.norm(ref), 1.0), \
                        (variant, kinds, e, c)
    del keep


@pytest.mark.parametrize("kinds", KINDS, ids=lambda k: "+".join(k))
def test_tip_pose_and_jacobian_transpose_match_oracle(lib, kinds):
    """Tool-tip position, tip quaternion (Shepperd on the device rotation,
    against the oracle's product of joint quaternions, both with w >= 0) and
    J_tip^T g (against autograd of g . tip) of every chain."""
    desc = _desc(kinds, "position")
    keep = _plan(lib, desc)
    q, _, _ = _state(desc, 4)
    rng = np.random.default_rng(5)
    for idx, tree in groups(desc):
        n = tree.n
        P = make_params(tree, desc, idx)
        Q = torch.tensor(q[idx, :n], dtype=D64, requires_grad=True)
        tips, _ = dyn.end_effectors(tree, P, Q)
        quats = tip_quaternion(tree, Q.detach())
        g = torch.as_tensor(rng.normal(size=tips.shape))
        (gq,) = torch.autograd.grad((g * tips).sum(), [Q])
        for k, e in enumerate(idx):
            for c, jo, nc in _chains(desc, e):
                qa = np.ascontiguousarray(q[e, jo:jo + nc])
                tip, quat, jt = np.zeros(3), np.zeros(4), np.zeros(nc)
                assert lib.host_tip(int(e), c, _p(qa), _p(tip), _p(quat)) == nc
                gb = np.ascontiguousarray(g[k, c].numpy())
                assert lib.host_tip_vjp(int(e), c, _p(qa), _p(gb), _p(jt)) == nc
                assert np.abs(tip - tips[k, c].detach().numpy()).max() <= 1e-12
                assert np.abs(quat - quats[k, c].numpy()).max() <= 1e-12
                ref = gq[k, jo:jo + nc].numpy()
                assert np.abs(jt - ref).max() <= 1e-12 * max(np.abs(ref).max(), 1.0)
    del keep


def test_counter_based_noise_matches_oracle(lib):
    """The device's key arithmetic (seed, env, chain or joint block, step;
    shifts, masks, 64-bit step counts) and Box-Muller draw the oracle's
    deviates: in double precision they agree to 1e-12."""
    rng = np.random.default_rng(6)
    for _ in range(200):
        seed = int(rng.integers(0, 2**32))
        env, c, blk = int(rng.integers(0, 2**20)), int(rng.integers(0, 4)), int(rng.integers(0, 7))
        step = int(rng.integers(0, 2**28))
        big = int(rng.integers(0, 2**50))
        z3, z4 = np.zeros(3), np.zeros(4)
        lib.host_goal_noise(seed, env, c, step, _p(z3))
        assert np.abs(z3 - goal_noise(seed, env, c, step)).max() <= 1e-12
        lib.host_action_noise(seed, env, blk, big, _p(z4))
        assert np.abs(z4 - action_noise(seed, env, blk, big)).max() <= 1e-12


@pytest.mark.parametrize("kinds", KINDS, ids=lambda k: "+".join(k))
def test_inverse_dynamics_sweeps_match_oracle_rnea(lib, kinds):
    """The adjoint's inverse-dynamics sweeps (body-frame recursion, link
    wrenches) give the oracle's spatial-algebra RNEA torques."""
    desc = _desc(kinds, "position")
    keep = _plan(lib, desc)
    q, qd, _ = _state(desc, 7)
    qdd = np.random.default_rng(8).normal(0.0, 3.0, q.shape)
    for idx, tree in groups(desc):
        n = tree.n
        P = make_params(tree, desc, idx)
        t = lambda a: torch.as_tensor(a[idx, :n])
        tau = dyn.rnea(tree, P, t(q), t(qd), t(qdd)).numpy()
        for k, e in enumerate(idx):
            for c, jo, nc in _chains(desc, e):
                args = [np.ascontiguousarray(a[e, jo:jo + nc]) for a in (q, qd, qdd)]
                out = np.zeros(nc)
                assert lib.host_inverse_dynamics(int(e), c, *map(_p, args), _p(out)) == nc
                ref = tau[k, jo:jo + nc]
                assert np.linalg.norm(out - ref) <= 1e-10 * max(np.linalg.norm(ref), 1.0)
    del keep


@pytest.mark.parametrize("kinds", KINDS, ids=lambda k: "+".join(k))
@pytest.mark.parametrize("variant", ["position", "limits", "drives"])
def test_warp_pair_split_equals_the_fused_substep(lib, kinds, variant):
    """The warp pair's decomposition of a substep (bias-only and mass-only
    backward sweeps in two roles, then the shared solve) computes the fused
    one-thread substep."""
    desc = _desc(kinds, variant)
    keep = _plan(lib, desc)
    q, qd, qs = _state(desc, 9)
    for e in range(desc["num_envs"]):
        for c, jo, nc in _chains(desc, e):
            args = [np.ascontiguousarray(a[e, jo:jo + nc]) for a in (q, qd, qs)]
            a1, b1, a2, b2 = np.zeros(7), np.zeros(7), np.zeros(7), np.zeros(7)
            assert lib.host_substep(e, c, *map(_p, args), H, _p(a1), _p(b1)) == nc
            assert lib.host_substep_split(e, c, *map(_p, args), H, _p(a2), _p(b2)) == nc
            assert np.abs(a1 - a2).max() <= 1e-13 and np.abs(b1 - b2).max() <= 1e-11
    del keep
