"""Bounded device-side waits run out instead of hanging (test hook
sg_debug_set_fault; no GPU fault is made).

The step kernels wait on mbarriers for the bulk copy of each warp's
parameter record and, in the warp-pair kernel, for the partner warp at
every substep's exchange.  Every such wait is bounded in wall-clock time.
The hook makes a wait's completion impossible on a small case -- no copy is
started (one-thread kernel) or the partner leaves out its first arrival
(warp-pair kernel) -- with the bound shortened to a few milliseconds, and
the tests check that the call returns, that sg_sync_status reports
SG_ERR_TIMEOUT, that the context's state is unchanged, and that the same
context then steps normally, bit-identical to a fresh one.
"""
import time

import numpy as np
import pytest
import torch

from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu

DT = 1.0 / 60.0
LIMIT_NS = 2_000_000          # 2 ms per wait


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


CASES = [(sg.FAULT_SKIP_PARAM_COPY, 1, 32), (sg.FAULT_SKIP_PARAM_COPY, 1, 128),
         (sg.FAULT_SKIP_PARTNER, 2, 64), (sg.FAULT_SKIP_PARTNER, 2, 256)]


@pytest.mark.parametrize("mode,split,threads", CASES,
                         ids=["copy-32", "copy-128", "partner-64", "partner-256"])
@pytest.mark.parametrize("form", ["step", "rollout"])
def test_wait_runs_out_and_reports_timeout(mode, split, threads, form):
    desc = W.make_desc(["7R", "14B", "4R"] * 11)        # 3 chain classes, a few warps
    acts = torch.as_tensor(W.joint_targets(desc, 4), device="cuda")
    env = sg.Env(desc)
    env.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    q0, qd0, sc0 = (x.clone() for x in env.get_state())
    assert env.sync_status() == sg.SG_OK
    env.debug_set_fault(mode, LIMIT_NS)
    t0 = time.perf_counter()
    if form == "step":
        env.step(acts[0], DT, 2)
    else:
        env.rollout(acts, DT, 2)
    st = env.sync_status()
    elapsed = time.perf_counter() - t0
    assert st == sg.SG_ERR_TIMEOUT, sg.STATUS_NAMES.get(st)
    assert elapsed < 2.0, elapsed                       # bounded: a few waits of 2 ms
    q1, qd1, sc1 = env.get_state()
    assert torch.equal(q0, q1) and torch.equal(qd0, qd1) and torch.equal(sc0, sc1)
    assert env.sync_status() == sg.SG_OK                # flags were cleared by the read
    # the context is intact: with the hook off it steps like a fresh context
    env.debug_set_fault(sg.FAULT_NONE, 0)
    ref = sg.Env(desc)
    ref.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    if form == "step":
        out, out_ref = env.step(acts[1], DT, 2), ref.step(acts[1], DT, 2)
    else:
        out, out_ref = env.rollout(acts, DT, 2), ref.rollout(acts, DT, 2)
    assert env.sync_status() == sg.SG_OK and ref.sync_status() == sg.SG_OK
    for a, b in zip(out, out_ref):
        assert torch.equal(a, b)
    assert all(torch.equal(a, b) for a, b in zip(env.get_state(), ref.get_state()))


def test_hook_validates_its_arguments():
    env = sg.Env(W.make_desc(["7R"] * 4))
    with pytest.raises(sg.SgError):
        env.debug_set_fault(7, 0)
    with pytest.raises(sg.SgError):
        env.debug_set_fault(sg.FAULT_NONE, 3_000_000_000)
    with pytest.raises(sg.SgError):
        env.debug_set_fault(sg.FAULT_NONE, -1)
    env.debug_set_fault(sg.FAULT_NONE, 0)
    assert env.cuda_device == torch.cuda.current_device()


def _ppo_run(env, ppo, perms):
    ppo.set_params(torch.as_tensor(W.ppo_init_params(env.obs_dim, env.max_joints, seed=5),
                                   device="cuda"))
    ppo.reset(step0=0)
    ppo.collect()
    stats = ppo.update(perms)
    return stats


def test_contraction_wait_runs_out_and_ppo_recovers():
    """The tensor-core contraction's bounded waits (hook
    sg_ppo_debug_set_fault): with the copy of each CTA's first weight chunk
    left out, every product with pre-split weights gives up after the bound
    (its CTAs wait, bounded, for their copies in flight and release their
    tensor memory), the collect and the update return, and the env context
    reports SG_ERR_TIMEOUT.  With the hook off the same handles collect and
    update bit-identically to fresh ones."""
    cfg = dict(n_steps=4, epochs=2, minibatches=2, gamma=0.99, lam=0.95, clip=0.2,
               value_coef=1.0, entropy_coef=0.0, lr=3e-4, max_grad_norm=1.0, dt=DT, substeps=2)
    desc = W.make_desc(["7P"] * 300, episode_len=50)     # 1200 collect rows: 10 row tiles
    env = sg.Env(desc)
    ppo = sg.PPO(env, **cfg)
    perms = torch.as_tensor(W.ppo_perms(ppo.B, cfg["epochs"]), device="cuda")
    assert env.sync_status() == sg.SG_OK
    ppo.debug_set_fault(sg.FAULT_SKIP_WEIGHT_COPY, LIMIT_NS)
    t0 = time.perf_counter()
    ppo.set_params(torch.as_tensor(W.ppo_init_params(env.obs_dim, env.max_joints, seed=5),
                                   device="cuda"))
    ppo.reset(step0=0)
    ppo.collect()
    st = env.sync_status()
    assert st == sg.SG_ERR_TIMEOUT, sg.STATUS_NAMES.get(st)
    ppo.update(perms)
    st = env.sync_status()
    assert st == sg.SG_ERR_TIMEOUT, sg.STATUS_NAMES.get(st)
    elapsed = time.perf_counter() - t0
    # about 60 products, each a few waits of 2 ms (all CTAs wait together)
    assert elapsed < 10.0, elapsed
    # hook off: the same handles work like fresh ones
    ppo.debug_set_fault(sg.FAULT_NONE, 0)
    stats = _ppo_run(env, ppo, perms)
    ref_env = sg.Env(desc)
    ref = sg.PPO(ref_env, **cfg)
    ref_stats = _ppo_run(ref_env, ref, perms)
    assert env.sync_status() == sg.SG_OK and ref_env.sync_status() == sg.SG_OK
    assert torch.equal(stats, ref_stats)
    assert torch.equal(ppo.get_params(), ref.get_params())
    assert torch.equal(ppo.get_buffer(sg.PPO_VALUES), ref.get_buffer(sg.PPO_VALUES))
    with pytest.raises(sg.SgError):
        ppo.debug_set_fault(1, 0)                      # a step-kernel mode: not this hook's
    with pytest.raises(sg.SgError):
        ppo.debug_set_fault(sg.FAULT_SKIP_WEIGHT_COPY, 3_000_000_000)
