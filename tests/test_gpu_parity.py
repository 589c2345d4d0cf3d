"""CUDA step vs the FP64 oracle, element by element, through the C ABI.

Tolerances (from the step's arithmetic): the FP32 step must reproduce the
oracle's per-step acceleration to 1e-4 relative,
    ||qdd_gpu - qdd_ref|| / max(||qdd_ref||, 1e-3) <= 1e-4  per env,
from the same FP32 state, and the joint positions after 100 damped steps
to 1e-3 relative, ||q_gpu - q_ref|| / max(||q_ref||, 1e-3).  Observation
and reward formulas are checked on the GPU's own resulting state to 1e-5.
Reset, indexing and batching are bit-exact.
"""
import numpy as np
import pytest
import torch

from oracle.env import OracleEnv
from paper_2310_04676_gb300 import sg, workloads as W
from tests.helpers import chain_desc

pytestmark = pytest.mark.gpu

DT = 1.0 / 60.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def random_state(desc, seed, qd_scale=2.0):
    rng = np.random.default_rng(seed)
    E, J = desc["num_envs"], desc["max_joints"]
    lo, hi = desc["q_lo"].astype(np.float64), desc["q_hi"].astype(np.float64)
    span = hi - lo
    q = (lo - 0.1 * span + rng.random((E, J)) * 1.2 * span).astype(np.float32)
    qd = rng.uniform(-qd_scale, qd_scale, (E, J)).astype(np.float32)
    ndof = desc["chain_num_joints"].sum(1)
    for e in range(E):
        q[e, ndof[e]:] = 0
        qd[e, ndof[e]:] = 0
    return q, qd


def cuda(x):
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda")


def rel_rows(a, b, floor=1e-3):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), floor)


def one_step_accel(desc, substeps, seed=0, split=1):
    env = sg.Env(desc)
    env.set_launch(64 * split, sg.ROLLOUT_PERSISTENT, split)
    ref = OracleEnv(desc)
    q, qd = random_state(desc, seed)
    env.set_state(cuda(q), cuda(qd))
    ref.set_state(q, qd)
    acts = W.joint_targets(desc, 1, seed=seed + 7)[0]
    obs, rew, done = env.step(cuda(acts), DT, substeps)
    ref.step(acts, DT, substeps)
    q1, qd1, sc = env.get_state()
    torch.cuda.synchronize()
    acc_gpu = (qd1.cpu().numpy().astype(np.float64) - qd) / DT
    acc_ref = (ref.qd - qd) / DT
    return rel_rows(acc_gpu, acc_ref), env, obs, rew, done


KINDS = [["7R"], ["7P"], ["4R"], ["14B"], ["7R", "4R", "7P", "14B"]]


@pytest.mark.parametrize("kinds", KINDS, ids=lambda k: "+".join(k))
@pytest.mark.parametrize("substeps", [1, 2])
@pytest.mark.parametrize("split", [1, 2])
def test_step_acceleration_matches_oracle(kinds, substeps, split):
    E = 197                                   # several warps and a ragged tail
    desc = W.make_desc((kinds * E)[:E])
    rel, env, *_ = one_step_accel(desc, substeps, split=split)
    assert rel.max() <= 1e-4, rel.max()
    assert env.sync_status() == sg.SG_OK


@pytest.mark.parametrize("chains", [
    [([0, 1, 0, 0], [0, 2, 1, 0])],
    [([1, 0, 0], [2, 0, 1])],
    [([0] * 6, [1, 0, 2, 2, 1, 0])],
    [([0, 0, 0, 0], [2, 1, 2, 1]), ([0, 0, 1, 0, 0], [0, 1, 2, 2, 0])],
], ids=["x-axes", "prismatic-root", "six", "mixed-pair"])
@pytest.mark.parametrize("split", [1, 2])
def test_generic_chains_match_oracle(chains, split):
    desc = chain_desc(chains, E=70, seed=5, kp=50.0, kd=5.0, damping=0.1,
                      base=[(0, 0.25, 0), (0, -0.25, 0)])
    rel, env, *_ = one_step_accel(desc, 2, split=split)
    assert rel.max() <= 1e-4, rel.max()


@pytest.mark.parametrize("split", [1, 2])
def test_largest_and_smallest_envs_match_oracle(split):
    """The widest env the description allows (four 7-joint chains, 28 DOF,
    108-wide observation rows) and envs of single-joint chains."""
    seven_r = ([0] * 7, [2, 1, 2, 1, 2, 1, 2])
    seven_p = ([0, 0, 1, 0, 0, 0, 0], [2, 1, 2, 1, 2, 1, 2])
    mixed = ([0, 1, 0, 0, 0, 0, 0], [0, 2, 1, 2, 0, 1, 2])
    desc = chain_desc([seven_r, seven_p, mixed, seven_r], E=37, seed=9, kp=50.0, kd=5.0,
                      damping=0.1, base=[(0, 0.3, 0), (0, -0.3, 0), (-0.2, 0, 0), (0.2, 0, 0)])
    rel, env, obs, *_ = one_step_accel(desc, 2, split=split)
    assert env.max_joints == 28 and env.obs_dim == 3 * 28 + 6 * 4
    assert rel.max() <= 1e-4, rel.max()
    desc = chain_desc([([0], [2]), ([1], [2])], E=45, seed=3, kp=50.0, kd=5.0, damping=0.1,
                      base=[(0, 0.2, 0), (0, -0.2, 0)])
    rel, env, *_ = one_step_accel(desc, 2, split=split)
    assert rel.max() <= 1e-4, rel.max()


@pytest.mark.parametrize("split", [1, 2])
def test_limit_springs_match_oracle(split):
    desc = W.make_desc(["7R"] * 150 + ["7P"] * 40, k_limit=1e3)
    rel, *_ = one_step_accel(desc, 8, split=split)
    assert rel.max() <= 1e-4, rel.max()


@pytest.mark.parametrize("kinds,S", [(["7R"], 2), (["7R", "4R", "7P", "14B"], 2)],
                         ids=["7R", "mixed"])
def test_q_after_100_damped_steps(kinds, S):
    E = 64
    desc = W.make_desc((kinds * E)[:E], shared_params=(kinds == ["7R"]))
    env, ref = sg.Env(desc), OracleEnv(desc)
    acts = W.joint_targets(desc, 100)
    for t in range(100):
        env.step(cuda(acts[t]), DT, S)
        ref.step(acts[t], DT, S)
    q, qd, sc = env.get_state()
    rel = rel_rows(q.cpu().numpy().astype(np.float64), ref.q)
    assert rel.max() <= 1e-3, rel.max()
    assert (sc.cpu().numpy() == 100).all()


def test_obs_reward_done_formulas_on_gpu_state():
    """Reach task: obs/reward/done of the GPU equal the oracle's formulas
    evaluated on the GPU's own post-step state."""
    kinds = ["7R", "4R", "7P", "14B"] * 20
    desc = W.make_desc(kinds, episode_len=3)
    env = sg.Env(desc)
    acts = W.joint_targets(desc, 3)
    for t in range(3):
        q0, qd0, sc0 = env.get_state()
        obs, rew, done = env.step(cuda(acts[t]), DT, 2)
        q1, qd1, sc1 = env.get_state()
        ref = OracleEnv(desc)
        ref.set_state(q0.cpu().numpy(), qd0.cpu().numpy(), sc0.cpu().numpy())
        ref.step(acts[t], DT, 2)
        # evaluate the oracle's observation on the GPU state
        ref.set_state(q1.cpu().numpy(), qd1.cpu().numpy(), sc1.cpu().numpy())
        o_ref = np.zeros((len(kinds), env.obs_dim))
        r_ref = np.zeros(len(kinds))
        for idx, tree, P in ref.groups:
            n = tree.n
            o, r = ref._obs_reward(idx, tree, P, torch.as_tensor(ref.q[idx, :n]),
                                   torch.as_tensor(ref.qd[idx, :n]), torch.as_tensor(
                                       acts[t][idx, :n].astype(np.float64)))
            o_ref[idx, :o.shape[1]] = o
            r_ref[idx] = r
        o_g = obs.cpu().numpy()
        assert np.abs(o_g - o_ref).max() <= 1e-5 * max(1.0, np.abs(o_ref).max())
        assert np.abs(rew.cpu().numpy() - r_ref).max() <= 1e-5
        want_done = np.full(len(kinds), 2 if t == 2 else 0, np.uint8)
        assert (done.cpu().numpy() == want_done).all()


def test_path_following_matches_oracle():
    E, T = 96, 12
    desc = W.make_desc(["7R"] * E, task=1, path_len=T + 3, episode_len=T)
    env, ref = sg.Env(desc), OracleEnv(desc)
    assert env.obs_dim == 30
    acts = W.joint_targets(desc, T)
    table = env.get_paths(T + 3).cpu().numpy()            # built on the device at create
    assert np.abs(table - ref.path).max() <= 2e-6
    for t in range(T):
        q0, qd0, sc0 = env.get_state()
        obs, rew, done = env.step(cuda(acts[t]), DT, 4)
        q1, qd1, sc1 = env.get_state()
        ref.set_state(q1.cpu().numpy(), qd1.cpu().numpy(), sc1.cpu().numpy())
        (idx, tree, P), = ref.groups
        o, r = ref._obs_reward(idx, tree, P, torch.as_tensor(ref.q[idx, :7]),
                               torch.as_tensor(ref.qd[idx, :7]), None)
        o_g = obs.cpu().numpy()
        qg, qr = o_g[:, 17:21], o[:, 17:21]
        sgn = np.where((qg * qr).sum(1, keepdims=True) < 0, -1.0, 1.0)
        assert np.abs(qg * sgn - qr).max() <= 1e-5
        assert np.abs(o_g[:, :17] - o[:, :17]).max() <= 1e-5
        k = np.minimum(t + 1 + np.arange(1, 4), T + 2)
        assert np.array_equal(o_g[:, 21:30], table[:, k].reshape(E, 9))   # waypoints copied
        assert np.abs(o_g[:, 21:] - o[:, 21:]).max() <= 2e-6
        assert np.abs(rew.cpu().numpy() - r).max() <= 1e-5
    assert (done.cpu().numpy() == 2).all()


def test_reset_is_bit_exact_and_masked():
    kinds = ["7R", "4R", "7P", "14B"] * 25
    desc = W.make_desc(kinds)
    a, b = sg.Env(desc), sg.Env(desc)
    acts = W.joint_targets(desc, 6)
    for t in range(3):
        a.step(cuda(acts[t]), DT, 2)
        b.step(cuda(acts[t]), DT, 2)
    mask = np.zeros(len(kinds), np.uint8)
    mask[::3] = 1
    a.reset(cuda(mask))
    qa, qda, sca = (x.cpu().numpy() for x in a.get_state())
    qb, qdb, scb = (x.cpu().numpy() for x in b.get_state())
    m = mask.astype(bool)
    assert np.array_equal(qa[m], desc["q0"][m]) and (qda[m] == 0).all() and (sca[m] == 0).all()
    assert np.array_equal(qa[~m], qb[~m]) and np.array_equal(qda[~m], qdb[~m])
    for t in range(3, 6):
        oa, ra, da = a.step(cuda(acts[t]), DT, 2)
        ob, rb, db = b.step(cuda(acts[t]), DT, 2)
    oa, ob = oa.cpu().numpy(), ob.cpu().numpy()
    assert np.array_equal(oa[~m], ob[~m])


def test_permutation_and_batching_are_bit_exact():
    kinds = ["7R", "4R", "7P", "14B", "7R", "4R"] * 20
    E = len(kinds)
    desc = W.make_desc(kinds)
    perm = np.random.default_rng(3).permutation(E)
    dp = {k: (v[perm] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
          for k, v in desc.items()}
    A, B = sg.Env(desc), sg.Env(dp)
    acts = W.joint_targets(desc, 4)
    for t in range(4):
        oa, ra, da = A.step(cuda(acts[t]), DT, 2)
        ob, rb, db = B.step(cuda(acts[t][perm]), DT, 2)
    assert np.array_equal(oa.cpu().numpy()[perm], ob.cpu().numpy())
    assert np.array_equal(ra.cpu().numpy()[perm], rb.cpu().numpy())
    # an env alone gives the same bits as inside the mixed batch
    for e in (0, 3):
        de = {k: (v[[e]] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
              for k, v in desc.items()}
        de["num_envs"] = 1
        C = sg.Env(de)
        for t in range(4):
            oc, rc, dc = C.step(cuda(acts[t][[e]]), DT, 2)
        oc_row = oc.cpu().numpy()[0]
        oa_row = oa.cpu().numpy()[e]
        assert np.array_equal(oc_row, oa_row[:oc_row.size])
        assert (oa_row[oc_row.size:] == 0).all()
        assert np.array_equal(rc.cpu().numpy()[0], ra.cpu().numpy()[e])


def test_nonfinite_action_sets_done_bit_and_status():
    desc = W.make_desc(["7R"] * 40)
    env = sg.Env(desc)
    acts = W.joint_targets(desc, 1)[0].copy()
    acts[5, 3] = np.nan
    obs, rew, done = env.step(cuda(acts), DT, 2)
    d = done.cpu().numpy()
    assert d[5] & sg.DONE_NONFINITE and (np.delete(d, 5) == 0).all()
    assert env.sync_status() == sg.SG_ERR_NONFINITE
    assert env.sync_status() == sg.SG_OK          # flags clear after being read


def test_argument_errors():
    desc = W.make_desc(["7R"] * 4)
    env = sg.Env(desc)
    a = torch.zeros(4, 7, device="cuda")
    with pytest.raises(sg.SgError) as ei:
        env.step(a, -1.0, 2)
    assert ei.value.status == sg.SG_ERR_INVALID_ARG
    with pytest.raises(sg.SgError):
        env.step(a, DT, 0)
    with pytest.raises(ValueError):
        env.step(torch.zeros(4, 6, device="cuda"), DT, 2)


def test_full_size_mixed_batch_sampled_parity():
    """The 16384-env mixed batch in the launch configuration of the
    benchmark: one step from a random state, 256 sampled envs vs the oracle."""
    wl = W.config("C3")
    desc = wl.desc
    env = sg.Env(desc)
    q, qd = random_state(desc, 11)
    env.set_state(cuda(q), cuda(qd))
    acts = W.joint_targets(desc, 1)[0]
    env.step(cuda(acts), wl.dt, wl.substeps)
    q1, qd1, _ = env.get_state()
    pick = np.random.default_rng(0).choice(desc["num_envs"], 256, replace=False)
    sub = {k: (v[pick] if isinstance(v, np.ndarray) and v.shape[:1] == (desc["num_envs"],) else v)
           for k, v in desc.items()}
    sub["num_envs"] = len(pick)
    ref = OracleEnv(sub)
    ref.set_state(q[pick], qd[pick])
    ref.step(acts[pick], wl.dt, wl.substeps)
    acc_gpu = (qd1.cpu().numpy()[pick].astype(np.float64) - qd[pick]) / wl.dt
    acc_ref = (ref.qd - qd[pick]) / wl.dt
    assert rel_rows(acc_gpu, acc_ref).max() <= 1e-4


def _sub_desc(desc, pick):
    E = desc["num_envs"]
    sub = {k: (v[pick] if isinstance(v, np.ndarray) and v.shape[:1] == (E,) else v)
           for k, v in desc.items()}
    sub["num_envs"] = len(pick)
    return sub


def _sample_by_kind(kinds, per_kind, seed):
    """`per_kind` envs drawn at random from each kind of a mixed batch."""
    rng = np.random.default_rng(seed)
    kinds = np.asarray(kinds)
    pick = [rng.choice(np.flatnonzero(kinds == k), per_kind, replace=False)
            for k in sorted(set(kinds.tolist()))]
    return np.sort(np.concatenate(pick))


def test_full_c3_batch_100_damped_steps_sampled_in_autotuned_plan():
    """The whole 16384-env mixed batch for 100 control steps in the launch
    plan the autotuner picks (one 100-step rollout), from the reset state:
    256 envs drawn at random across the four kinds (64 each) against the
    oracle -- joint positions to 1e-3 relative after 100 steps and the
    rewards of every step to 1e-3 relative."""
    wl = W.config("C3")
    desc = wl.desc
    E, steps = desc["num_envs"], 100
    acts = W.joint_targets(desc, steps)
    env = sg.Env(desc)
    a = cuda(acts)
    plan = env.autotune(a[:32], wl.dt, wl.substeps, repeats=1)
    obs, rew, done = env.rollout(a, wl.dt, wl.substeps)
    q = env.get_state()[0].cpu().numpy().astype(np.float64)
    assert env.sync_status() == sg.SG_OK
    pick = _sample_by_kind(wl.kinds, 64, seed=12)
    ref = OracleEnv(_sub_desc(desc, pick))
    r_ref = np.zeros((steps, len(pick)))
    for t in range(steps):
        _, r_ref[t], _ = ref.step(acts[t][pick], wl.dt, wl.substeps)
    rel_q = rel_rows(q[pick], ref.q)
    assert rel_q.max() <= 1e-3, (plan, rel_q.max())
    r_gpu = rew.cpu().numpy()[:, pick].astype(np.float64)
    rel_r = np.abs(r_gpu - r_ref) / np.maximum(np.abs(r_ref), 1e-3)
    assert rel_r.max() <= 1e-3, (plan, rel_r.max())


def test_c1_latency_workload_trajectory():
    """64 envs of one shared 7-DOF arm: 100 steps as two 50-step rollouts in
    the autotuned plan; positions within 1e-3 and rewards within 1e-3 of the
    oracle, time-out bit at the episode length."""
    wl = W.config("C1")
    desc = dict(wl.desc)
    desc["episode_len"] = 100
    env, ref = sg.Env(desc), OracleEnv(desc)
    acts = W.joint_targets(desc, 100)
    a = cuda(acts)
    env.autotune(a[:50], wl.dt, wl.substeps)
    for half in range(2):
        obs, rew, done = env.rollout(a[50 * half:50 * (half + 1)], wl.dt, wl.substeps)
    for t in range(100):
        _, r_ref, d_ref = ref.step(acts[t], wl.dt, wl.substeps)
    q, qd, sc = env.get_state()
    assert rel_rows(q.cpu().numpy().astype(np.float64), ref.q).max() <= 1e-3
    assert np.abs(rew[-1].cpu().numpy() - r_ref).max() <= 1e-3
    assert (done[-1].cpu().numpy() == d_ref).all() and (d_ref == 2).all()


def test_c2_path_following_full_size_sampled():
    """8192 envs path following, one 50-step rollout in the autotuned plan;
    64 sampled envs against the oracle (positions 1e-3, rewards 1e-3)."""
    wl = W.config("C2")
    desc = wl.desc
    env = sg.Env(desc)
    acts = W.joint_targets(desc, 50)
    a = cuda(acts)
    env.autotune(a, wl.dt, wl.substeps)
    obs, rew, done = env.rollout(a, wl.dt, wl.substeps)
    pick = np.random.default_rng(1).choice(desc["num_envs"], 64, replace=False)
    ref = OracleEnv(_sub_desc(desc, pick))
    for t in range(50):
        _, r_ref, _ = ref.step(acts[t][pick], wl.dt, wl.substeps)
    q, _, _ = env.get_state()
    assert rel_rows(q.cpu().numpy()[pick].astype(np.float64), ref.q).max() <= 1e-3
    assert np.abs(rew[-1].cpu().numpy()[pick] - r_ref).max() <= 1e-3


def test_c5_largest_sweep_point_sampled():
    """262144 envs with limit springs and 8 substeps (the largest sweep
    point) in the autotuned plan: one step from a random state, 128 sampled
    envs' accelerations within 1e-4 of the oracle."""
    wl = W.config("C5", num_envs=262144)
    desc = wl.desc
    env = sg.Env(desc)
    acts = W.joint_targets(desc, 2)
    env.autotune(cuda(acts[:1]), wl.dt, wl.substeps, repeats=1)
    q, qd = random_state(desc, 21)
    env.set_state(cuda(q), cuda(qd))
    env.rollout(cuda(acts[1:2]), wl.dt, wl.substeps)
    q1, qd1, _ = env.get_state()
    pick = np.random.default_rng(2).choice(desc["num_envs"], 128, replace=False)
    ref = OracleEnv(_sub_desc(desc, pick))
    ref.set_state(q[pick], qd[pick])
    ref.step(acts[1][pick], wl.dt, wl.substeps)
    acc_gpu = (qd1.cpu().numpy()[pick].astype(np.float64) - qd[pick]) / wl.dt
    acc_ref = (ref.qd - qd[pick]) / wl.dt
    assert rel_rows(acc_gpu, acc_ref).max() <= 1e-4


@pytest.mark.parametrize("split", [1, 2])
def test_velocity_and_torque_commands_match_oracle(split):
    """Per-joint mix of position targets, velocity targets and torques."""
    kinds = (["7R", "4R", "7P", "14B"] * 50)[:190]
    E = len(kinds)
    modes = np.random.default_rng(8).integers(0, 3, size=(E, 14)).astype(np.int32)
    desc = W.make_desc(kinds, drive=modes, k_limit=1e3)
    rel, env, *_ = one_step_accel(desc, 2, seed=3, split=split)
    assert rel.max() <= 1e-4, rel.max()


@pytest.mark.parametrize("split", [1, 2])
def test_three_arm_envs_match_oracle(split):
    """Three-arm envs (lane groups of four with one idle lane) mixed with
    one- and two-arm envs: accelerations, observation and reward."""
    kinds = (["21T", "7R", "14B", "21T", "4R", "7P"] * 30)[:160]
    desc = W.make_desc(kinds, k_limit=1e3)
    assert sg.plan(desc)["obs_dim"] == 81
    rel, env, obs, rew, done = one_step_accel(desc, 2, seed=4, split=split)
    assert rel.max() <= 1e-4, rel.max()
    # observation and reward formulas on the GPU state
    q1, qd1, sc1 = env.get_state()
    ref = OracleEnv(desc)
    ref.set_state(q1.cpu().numpy(), qd1.cpu().numpy(), sc1.cpu().numpy())
    acts = W.joint_targets(desc, 1, seed=11)[0]
    o_ref = np.zeros((len(kinds), env.obs_dim))
    r_ref = np.zeros(len(kinds))
    for idx, tree, P in ref.groups:
        n = tree.n
        o, r = ref._obs_reward(idx, tree, P, torch.as_tensor(ref.q[idx, :n]),
                               torch.as_tensor(ref.qd[idx, :n]),
                               torch.as_tensor(acts[idx, :n].astype(np.float64)))
        o_ref[idx, :o.shape[1]] = o
        r_ref[idx] = r
    assert np.abs(obs.cpu().numpy() - o_ref).max() <= 1e-5 * max(1.0, np.abs(o_ref).max())
    assert np.abs(rew.cpu().numpy() - r_ref).max() <= 1e-5


@pytest.mark.parametrize("split", [1, 2])
def test_tracking_task_matches_oracle(split):
    """Moving goals (counter-based noise drawn on both sides): goals in the
    observation, rewards and the goal state follow the oracle over 40 steps;
    masked reset clears the goal state."""
    kinds = (["7R", "14B", "21T", "4R"] * 40)[:150]
    desc = W.make_desc(kinds, task=2, track_sigma=0.02, track_limit=0.15, seed=99)
    E = len(kinds)
    env, ref = sg.Env(desc), OracleEnv(desc)
    env.set_launch(128, sg.ROLLOUT_PERSISTENT, split)
    acts = W.joint_targets(desc, 40)
    obs, rew, done = env.rollout(cuda(acts), DT, 2)
    for t in range(40):
        o_ref, r_ref, _ = ref.step(acts[t], DT, 2)
    off, vel = env.get_goal_state()
    assert np.abs(off.cpu().numpy() - ref.goal_off).max() <= 1e-5
    assert np.abs(vel.cpu().numpy() - ref.goal_vel).max() <= 1e-5
    assert np.abs(rew[-1].cpu().numpy() - r_ref).max() <= 1e-3
    dof = desc["chain_num_joints"].sum(1)
    nc = desc["env_num_chains"]
    for e in range(0, E, 7):
        n, c = dof[e], nc[e]
        g_obs = obs[-1, e].cpu().numpy()[3 * n + 3 * c:3 * n + 6 * c].reshape(c, 3)
        assert np.abs(g_obs - ref.goals([e], c)[0]).max() <= 1e-5
    mask = np.zeros(E, np.uint8)
    mask[::2] = 1
    env.reset(cuda(mask))
    off, vel = env.get_goal_state()
    assert (off.cpu().numpy()[::2] == 0).all() and (vel.cpu().numpy()[::2] == 0).all()
    assert (off.cpu().numpy()[1::2] != 0).any()


def test_tracking_rollout_equals_steps_and_state_roundtrip():
    desc = W.make_desc(["7R", "14B"] * 50, task=2)
    acts = cuda(W.joint_targets(desc, 16))
    A, B = sg.Env(desc), sg.Env(desc)
    o, r, d = A.rollout(acts, DT, 2)
    for t in range(16):
        ob, rb, db = B.step(acts[t], DT, 2)
    assert torch.equal(o[-1], ob) and torch.equal(r[-1], rb)
    off, vel = A.get_goal_state()
    C = sg.Env(desc)
    C.set_state(*A.get_state())
    C.set_goal_state(off, vel)
    oc, rc, _ = C.step(acts[0], DT, 2)
    oa, ra, _ = A.step(acts[0], DT, 2)
    assert torch.equal(oa, oc) and torch.equal(ra, rc)


@pytest.mark.parametrize("task", [0, 1, 2])
def test_observe_matches_step_rows_and_oracle(task):
    """sg_observe: with the last step's commands it reproduces that step's
    observation rows bit for bit; after a masked reset it writes exactly the
    masked rows, equal to the oracle's observation of the reset state."""
    kinds = ["7R"] * 40 if task == 1 else (["7R", "14B", "21T", "4R", "7P"] * 8)
    desc = W.make_desc(kinds, task=task, path_len=20 if task == 1 else 0, episode_len=50)
    E = len(kinds)
    env, ref = sg.Env(desc), OracleEnv(desc)
    acts = W.joint_targets(desc, 6)
    for t in range(6):
        obs, _, _ = env.step(cuda(acts[t]), DT, 2)
        ref.step(acts[t], DT, 2)
    again = env.observe(cuda(acts[5]))
    assert torch.equal(again, obs)
    mask = np.zeros(E, np.uint8)
    mask[::3] = 1
    env.reset(cuda(mask))
    ref.reset(mask)
    sentinel = torch.full_like(obs, 7.0)
    out = env.observe(cuda(acts[5]), cuda(mask), out=sentinel.clone())
    m = torch.as_tensor(mask.astype(bool), device="cuda")
    assert torch.equal(out[~m], sentinel[~m])
    o_ref = ref.observe(acts[5], mask)
    got = out.cpu().numpy()[mask.astype(bool)]
    assert np.abs(got - o_ref[mask.astype(bool)]).max() <= 1e-5
