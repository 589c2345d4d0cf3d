"""Persistent / graph rollout and the autotuner against per-step launches."""
import numpy as np
import pytest
import torch

from paper_2310_04676_gb300 import sg, workloads as W

pytestmark = pytest.mark.gpu
DT = 1.0 / 60.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


@pytest.mark.parametrize("mode", [sg.ROLLOUT_PERSISTENT, sg.ROLLOUT_STEP_GRAPH])
@pytest.mark.parametrize("threads,split", [(32, 1), (128, 1), (256, 1), (64, 2), (256, 2)])
def test_rollout_equals_steps_bitwise(mode, threads, split):
    kinds = W.mixed_kinds(777, W.C3_FRACTIONS) + ["21T"] * 23
    desc = W.make_desc(kinds, episode_len=20)
    T = 32
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    A.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)   # sg_step uses the same kernel
    B.set_launch(threads, mode, split)
    steps = [A.step(acts[t], DT, 2) for t in range(T)]
    obs, rew, done = B.rollout(acts, DT, 2)
    for t in range(T):
        assert torch.equal(steps[t][0], obs[t])
        assert torch.equal(steps[t][1], rew[t])
        assert torch.equal(steps[t][2], done[t])
    qa, qda, sca = A.get_state()
    qb, qdb, scb = B.get_state()
    assert torch.equal(qa, qb) and torch.equal(qda, qdb) and torch.equal(sca, scb)
    # a second replay of the captured graph continues the trajectory
    obs2, _, _ = B.rollout(acts, DT, 2)
    s2 = [A.step(acts[t], DT, 2) for t in range(T)]
    assert torch.equal(obs2[-1], s2[-1][0])


def _close(x, y, tol):
    return (x - y).abs().max().item() <= tol * max(1.0, y.abs().max().item())


@pytest.mark.parametrize("kinds", [["7R"], ["14B"], ["4R", "7P"], ["7R", "4R", "7P", "14B"],
                                   ["21T", "7R"]],
                         ids=lambda k: "+".join(k))
@pytest.mark.parametrize("pair_threads", [128, 256])
def test_warp_pair_kernel_matches_single_thread_kernel(kinds, pair_threads):
    """Chain split 2 (two cooperating warps per chain block) agrees with one
    thread per chain to rounding (1e-5 of the largest entry over 6 steps),
    with identical done flags, for every chain class and with two or four
    pairs per block."""
    desc = W.make_desc((kinds * 200)[:200])
    T = 6
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    A.set_launch(128, sg.ROLLOUT_PERSISTENT, 1)
    B.set_launch(pair_threads, sg.ROLLOUT_PERSISTENT, 2)
    oa, ra, da = A.rollout(acts, DT, 2)
    ob, rb, db = B.rollout(acts, DT, 2)
    assert _close(ob, oa, 1e-5) and _close(rb, ra, 1e-5) and torch.equal(da, db)
    qa, qda, sca = A.get_state()
    qb, qdb, scb = B.get_state()
    assert _close(qb, qa, 1e-5) and _close(qdb, qda, 1e-4) and torch.equal(sca, scb)


def test_warp_pair_path_task():
    desc = W.make_desc(["7R"] * 100, task=1, path_len=20, episode_len=10)
    acts = cuda(W.joint_targets(desc, 12))
    A, B = sg.Env(desc), sg.Env(desc)
    B.set_launch(64, sg.ROLLOUT_STEP_GRAPH, 2)
    oa, ra, da = A.rollout(acts, DT, 4)
    ob, rb, db = B.rollout(acts, DT, 4)
    assert _close(ob, oa, 1e-5) and _close(rb, ra, 1e-5) and torch.equal(da, db)


def test_host_rollout_matches_device_rollout():
    desc = W.make_desc(W.mixed_kinds(300, W.C3_FRACTIONS))
    T = 8
    acts_np = W.joint_targets(desc, T)
    A, B = sg.Env(desc), sg.Env(desc)
    obs, rew, done = A.rollout(cuda(acts_np), DT, 2)
    a_h = torch.from_numpy(acts_np).pin_memory()
    out = (torch.empty(T, B.num_envs, B.obs_dim).pin_memory(),
           torch.empty(T, B.num_envs).pin_memory(),
           torch.empty(T, B.num_envs, dtype=torch.uint8).pin_memory())
    B.rollout_host(a_h, DT, 2, out)              # default: pipelined chunks
    assert B.sync_status() == sg.SG_OK
    assert torch.equal(out[0], obs.cpu()) and torch.equal(out[1], rew.cpu())
    assert torch.equal(out[2], done.cpu())
    # serial copies, direct host access and pageable memory give the same bits
    for mode, pin in ((sg.HOST_IO_STAGED, True), (sg.HOST_IO_DIRECT, True),
                      (sg.HOST_IO_AUTO, False), (sg.HOST_IO_DIRECT, False)):
        C = sg.Env(desc)
        C.set_host_io(mode)
        mk = (lambda t: t.pin_memory()) if pin else (lambda t: t)
        a2 = mk(torch.from_numpy(acts_np.copy()))
        o2 = (mk(torch.empty(T, C.num_envs, C.obs_dim)), mk(torch.empty(T, C.num_envs)),
              mk(torch.empty(T, C.num_envs, dtype=torch.uint8)))
        C.rollout_host(a2, DT, 2, o2)
        assert C.sync_status() == sg.SG_OK
        assert torch.equal(o2[0], out[0]) and torch.equal(o2[1], out[1])
        assert torch.equal(o2[2], out[2])
    with pytest.raises(sg.SgError):
        B.set_host_io(5)


def test_autotune_keeps_state_and_picks_a_plan():
    desc = W.make_desc(W.mixed_kinds(2000, W.C3_FRACTIONS))
    T = 16
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    th, mode, split, ms = B.autotune(acts, DT, 2, repeats=2)
    assert th in (32, 64, 128, 256) and mode in (0, 1) and split in (1, 2) and ms > 0
    A.set_launch(th, mode, split)
    qa, qda, sca = A.get_state()
    qb, qdb, scb = B.get_state()
    assert torch.equal(qa, qb) and torch.equal(qda, qdb) and torch.equal(sca, scb)
    oa, _, _ = A.rollout(acts, DT, 2)
    ob, _, _ = B.rollout(acts, DT, 2)
    assert torch.equal(oa, ob)


@pytest.mark.parametrize("task", [0, 2])
@pytest.mark.parametrize("threads,split", [(128, 1), (256, 1), (128, 2)])
def test_packings_give_identical_bits(task, threads, split):
    """The interleaved packing reorders whole warps: every env's outputs and
    state are the same bits as with the class-grouped packing, for both
    chain splits, the reach and the tracking task (per-slot goal state), and
    after a masked reset and a change of link masses; switching back restores
    the class-grouped order."""
    kinds = W.mixed_kinds(3000, W.C3_FRACTIONS) + ["21T"] * 40
    desc = W.make_desc(kinds, episode_len=12, task=task)
    T = 16
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    for env in (A, B):
        env.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    B.set_packing(sg.PACK_INTERLEAVE)
    assert B.packing == sg.PACK_INTERLEAVE and A.packing == sg.PACK_CLASS
    mass = cuda(np.asarray(desc["link_mass"], dtype=np.float32).reshape(A.num_envs, -1) * 1.3)
    mask = cuda((np.arange(A.num_envs) % 3 == 0).astype(np.uint8))
    for env in (A, B):
        env.rollout(acts, DT, 2)
        env.set_link_mass(mass)
        env.reset(mask)
    outs = [env.rollout(acts, DT, 2) for env in (A, B)]
    for x, y in zip(*outs):
        assert torch.equal(x, y)
    for x, y in zip(A.get_state(), B.get_state()):
        assert torch.equal(x, y)
    if task == 2:
        for x, y in zip(A.get_goal_state(), B.get_goal_state()):
            assert torch.equal(x, y)
    B.set_packing(sg.PACK_CLASS)
    oa = A.rollout(acts, DT, 2)[0]
    ob = B.rollout(acts, DT, 2)[0]
    assert torch.equal(oa, ob)


def test_packing_change_discards_a_pending_gradient_forward():
    desc = W.make_desc(W.mixed_kinds(500, W.C3_FRACTIONS))
    env = sg.Env(desc)
    acts = cuda(W.joint_targets(desc, 8))
    env.diff_forward(acts, DT, 2, ckpt_every=4)
    env.set_packing(sg.PACK_INTERLEAVE)
    with pytest.raises(sg.SgError) as e:
        env.diff_backward(acts, torch.zeros(8, env.num_envs, 4, 3, device="cuda"))
    assert e.value.status == sg.SG_ERR_INVALID_ARG
    with pytest.raises(sg.SgError):
        env.set_packing(9)


def test_autotune_searches_the_packing():
    """A mixed batch has two distinct packings; the autotuner leaves the
    fastest in place and the results stay those of the class-grouped order."""
    desc = W.make_desc(W.mixed_kinds(6000, W.C3_FRACTIONS))
    T = 16
    acts = cuda(W.joint_targets(desc, T))
    A, B = sg.Env(desc), sg.Env(desc)
    th, mode, split, ms = B.autotune(acts, DT, 2, repeats=2)
    assert B.packing in (sg.PACK_CLASS, sg.PACK_INTERLEAVE) and ms > 0
    A.set_launch(th, mode, split)
    oa, _, _ = A.rollout(acts, DT, 2)
    ob, _, _ = B.rollout(acts, DT, 2)
    assert torch.equal(oa, ob)


def test_rollout_argument_errors():
    env = sg.Env(W.make_desc(["7R"] * 8))
    with pytest.raises(sg.SgError):
        env.set_launch(48, 0)
    with pytest.raises(sg.SgError):
        env.set_launch(64, 5)
    with pytest.raises(sg.SgError):
        env.set_launch(32, 0, 2)
    with pytest.raises(ValueError):
        env.rollout(torch.zeros(4, 8, 6, device="cuda"), DT, 2)


@pytest.mark.parametrize("kind,E", [("7R", 100), ("7P", 64), ("4R", 96), ("14B", 70), ("21T", 40)])
@pytest.mark.parametrize("split", [1, 2])
def test_block_and_row_writes_agree(kind, E, split):
    """Observation rows of a warp whose envs are consecutive are written as
    one contiguous block, other warps' rows one by one.  The same envs in
    caller order (block writes; the ragged last warp row by row) and
    permuted (row by row) give the same rows, bit for bit, for odd and even
    row widths, in the per-step and persistent forms."""
    desc = W.make_desc([kind] * E)
    perm = np.random.default_rng(5).permutation(E)
    dp = {k: (v[perm] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
          for k, v in desc.items()}
    acts = W.joint_targets(desc, 5)
    a = torch.as_tensor(acts, device="cuda")
    ap = torch.as_tensor(np.ascontiguousarray(acts[:, perm]), device="cuda")
    threads = 64 * split
    A, B = sg.Env(desc), sg.Env(dp)
    A.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    B.set_launch(threads, sg.ROLLOUT_PERSISTENT, split)
    oa, ra, da = A.rollout(a, DT, 2)
    ob, rb, db = B.rollout(ap, DT, 2)
    assert torch.equal(oa[:, perm], ob) and torch.equal(ra[:, perm], rb)
    assert torch.equal(da[:, perm], db)
    o1, r1, d1 = A.step(a[0], DT, 2)
    o2, r2, d2 = B.step(ap[0], DT, 2)
    assert torch.equal(o1[perm], o2) and torch.equal(r1[perm], r2)
    # observe: all rows (block writes) and a masked subset (row by row)
    full = A.observe(a[0])
    mask = torch.zeros(E, dtype=torch.uint8, device="cuda")
    mask[::3] = 1
    part = torch.full_like(full, -7.0)
    A.observe(a[0], mask, out=part)
    m = mask.bool()
    assert torch.equal(part[m], full[m]) and bool((part[~m] == -7.0).all())
    assert A.sync_status() == sg.SG_OK and B.sync_status() == sg.SG_OK
