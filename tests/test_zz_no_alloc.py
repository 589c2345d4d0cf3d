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


def _noalloc(lib, env, acts, tgt, S, every):
    T, E, J = acts.shape
    out = (torch.empty(T, E, 4, 3, device="cuda"), torch.empty(E, device="cuda"),
           torch.empty(T, E, J, device="cuda"), torch.empty(E, J, device="cuda"))
    st = lib.sg_diff_track_noalloc(env.ctx, _ptr(acts), T, ctypes.c_float(DT), S, every,
                                   _ptr(tgt), *(_ptr(x) for x in out))
    return st, out


def test_noalloc_between_forward_and_backward_leaves_them_alone():
    """sg_diff_forward, then this call, then sg_diff_backward: the gradients
    equal those of a forward + backward pair with nothing in between (the
    call touches neither the context's checkpoints nor the forward's replay
    records)."""
    lib = sg.load_library()
    desc = W.make_desc(W.mixed_kinds(300, W.C3_FRACTIONS))
    env = sg.Env(desc)
    T, S, every = 24, 2, 8
    acts = torch.as_tensor(W.joint_targets(desc, T, seed=3), device="cuda")
    tgt = torch.as_tensor(W.loss_targets(desc, T, seed=4), device="cuda")
    ee, _, da, dm = _reference(env, desc, acts, tgt, S, every)
    # the same pair with a no-allocation call of another shape in between
    ee2 = env.diff_forward(acts, DT, S, every)
    acts_b = torch.as_tensor(W.joint_targets(desc, 13, seed=5), device="cuda")
    tgt_b = torch.as_tensor(W.loss_targets(desc, 13, seed=6), device="cuda")
    st, _ = _noalloc(lib, env, acts_b, tgt_b, 3, 5)
    assert st == sg.SG_OK, lib.sg_last_error(env.ctx)
    nc = torch.as_tensor(desc["env_num_chains"], device="cuda")
    mask = (torch.arange(4, device="cuda")[None, :] < nc[:, None]).float()[None, :, :, None]
    da2, dm2 = env.diff_backward(acts, (2.0 * (ee2 - tgt) * mask).contiguous())
    assert torch.equal(ee, ee2)
    assert torch.equal(da, da2) and torch.equal(dm, dm2)
    assert env.sync_status() == sg.SG_OK


def test_noalloc_allocates_no_device_memory():
    """After a first call, a second call of the same shape leaves the free
    device memory exactly unchanged."""
    lib = sg.load_library()
    desc = W.make_desc(["7R", "14B"] * 100)
    env = sg.Env(desc)
    T, S, every = 32, 2, 8
    acts = torch.as_tensor(W.joint_targets(desc, T, seed=8), device="cuda")
    tgt = torch.as_tensor(W.loss_targets(desc, T, seed=9), device="cuda")
    st, out = _noalloc(lib, env, acts, tgt, S, every)
    assert st == sg.SG_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = lib.sg_diff_track_noalloc(env.ctx, _ptr(acts), T, ctypes.c_float(DT), S, every,
                                   _ptr(tgt), *(_ptr(x) for x in out))
    assert st == sg.SG_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert env.sync_status() == sg.SG_OK


def test_noalloc_limit_is_exact():
    """(ceil(T / k) + 1) * 14 * num_slots + 12 * T * E <= 8388608 floats:
    512 7-DOF envs (512 slots) with k = 24 reach the limit exactly at
    T = 1300, which is accepted; T = 1301 is rejected."""
    lib = sg.load_library()
    desc = W.make_desc(["7R"] * 512)
    assert sg.plan(desc)["num_slots"] == 512
    E, k, T = 512, 24, 1300
    assert (-(-T // k) + 1) * 14 * E + 12 * T * E == 8388608
    assert (-(-(T + 1) // k) + 1) * 14 * E + 12 * (T + 1) * E > 8388608
    env = sg.Env(desc)
    acts = torch.as_tensor(W.joint_targets(desc, T + 1, seed=10), device="cuda")
    tgt = torch.as_tensor(W.loss_targets(desc, T + 1, seed=11), device="cuda")
    st, out = _noalloc(lib, env, acts[:T].contiguous(), tgt[:T].contiguous(), 1, k)
    assert st == sg.SG_OK, lib.sg_last_error(env.ctx)
    assert env.sync_status() == sg.SG_OK
    assert torch.isfinite(out[2]).all() and torch.isfinite(out[3]).all()
    st, _ = _noalloc(lib, env, acts, tgt, 1, k)
    assert st == sg.SG_ERR_INVALID_ARG
    assert b"32 MiB" in lib.sg_last_error(env.ctx)
