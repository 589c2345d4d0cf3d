"""sg_diff_track_noalloc: the allocation-free tracking-loss gradient.

Callers that cannot allocate device memory when they need gradients (a loop
inside a host program that owns all device memory through its own pool, or
one that must not stall on cudaMalloc/cudaFree) use this entry point; its
scratch lives in a static device array.  It must agree with the allocating
path (sg_diff_forward + sg_diff_backward with dL/d(ee) = 2 (ee - target))
to the tolerance the gradient tests use, on two calls in a row (the shared
array keeps the first call's contents).  This file is collected last so
that a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _rel(x, y):
    return (x - y).norm().item() / max(y.norm().item(), 1e-12)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def _reference(env, desc, acts, tgt, S, every):
    ee = env.diff_forward(acts, DT, S, every)
    nc = torch.as_tensor(desc["env_num_chains"], device="cuda")
    mask = (torch.arange(4, device="cuda")[None, :] < nc[:, None]).float()[None, :, :, None]
    diff = (ee - tgt) * mask
    da, dm = env.diff_backward(acts, (2.0 * diff).contiguous())
    return ee, (diff ** 2).sum((0, 2, 3)), da, dm


def test_noalloc_matches_allocating_path_twice():
    lib = sg.load_library()
    kinds = W.mixed_kinds(600, W.C3_FRACTIONS)
    desc = W.make_desc(kinds)
    env = sg.Env(desc)
    E, J = env.num_envs, env.max_joints
    for call, (T, S, every, seed) in enumerate([(24, 2, 8, 2), (17, 3, 5, 7)]):
        acts = torch.as_tensor(W.joint_targets(desc, T, seed=seed), device="cuda")
        tgt = torch.as_tensor(W.loss_targets(desc, T, seed=seed + 1), device="cuda")
        ee = torch.empty(T, E, 4, 3, device="cuda")
        loss = torch.empty(E, device="cuda")
        da = torch.empty(T, E, J, device="cuda")
        dm = torch.empty(E, J, device="cuda")
        st = lib.sg_diff_track_noalloc(env.ctx, _ptr(acts), T, ctypes.c_float(DT), S, every,
                                       _ptr(tgt), _ptr(ee), _ptr(loss), _ptr(da), _ptr(dm))
        assert st == sg.SG_OK, lib.sg_last_error(env.ctx)
        torch.cuda.synchronize()
        ee_r, loss_r, da_r, dm_r = _reference(env, desc, acts, tgt, S, every)
        torch.cuda.synchronize()
        nc = torch.as_tensor(desc["env_num_chains"], device="cuda")
        has = (torch.arange(4, device="cuda")[None, :] < nc[:, None])
        assert _rel(ee[:, has], ee_r[:, has]) <= 1e-5, call
        assert _rel(loss, loss_r) <= 1e-5, call
        assert _rel(da, da_r) <= 1e-5, call
        assert _rel(dm, dm_r) <= 1e-5, call
        assert env.sync_status() == sg.SG_OK


def test_noalloc_rejects_requests_beyond_the_static_scratch():
    lib = sg.load_library()
    desc = W.make_desc(["7R"] * 4096)
    env = sg.Env(desc)
    T = 4096                                # 6 * T * E floats alone exceed 32 MiB
    dummy = torch.zeros(1, device="cuda")
    st = lib.sg_diff_track_noalloc(env.ctx, _ptr(dummy), T, ctypes.c_float(DT), 2, 32,
                                   _ptr(dummy), _ptr(dummy), _ptr(dummy), _ptr(dummy), _ptr(dummy))
    assert st == sg.SG_ERR_INVALID_ARG
    assert b"32 MiB" in lib.sg_last_error(env.ctx)
