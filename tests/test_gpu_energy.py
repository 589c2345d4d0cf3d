"""Energy behaviour of the FP32 CUDA step with the drives, damping and limit
springs off (kp = kd = b = k_lim = 0, gravity on): the implicit-drive
substep is then plain semi-implicit (symplectic) Euler.

Reading of the energy bar.  Symplectic Euler conserves a modified energy, so
the true energy oscillates with an amplitude of first order in the substep
h and shows no secular drift where the method is stable.  For the pendulum
family of the configs' link ranges (L ~ U[0.05, 0.4] m) at h = 1/120 the
FP64 oracle's own energy error reaches about 9% of |T0| + |V0| (a 1e-2
bound is out of reach of the integrator itself), and multi-link chains
without damping are unstable at that step in FP64 as well; the FP32 path is
therefore held to the FP64 oracle running the same integrator from the same
state:
  * the GPU energy follows the oracle's energy step by step to 2e-3 of
    |T0| + |V0| over 1000 steps, against an integrator error of up to 13%
    (pendulums that swing over the top amplify rounding into a small phase
    offset, measured 3e-4; FP32 rounding adds no drift);
  * its largest error is within 5% of the oracle's, and the second half of
    the run is no worse than the first (no secular drift);
  * halving h halves the error (first order), as the oracle's does.
Energies are the oracle's T(q, qd) + V(q) applied to the GPU states, read
from the observation rows (q, qd lead every reach-task row).
"""
import numpy as np
import pytest
import torch

from oracle import dynamics as dyn
from oracle.model import groups, make_params
from paper_2310_04676_gb300 import sg
from tests.helpers import chain_desc

pytestmark = pytest.mark.gpu

H = 1.0 / 120.0
STEPS = 1000


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    sg.load_library()


def _start(desc, seed):
    rng = np.random.default_rng(seed)
    E, J = desc["num_envs"], desc["max_joints"]
    q = rng.uniform(-1.0, 1.0, (E, J)).astype(np.float32)
    qd = rng.uniform(-1.0, 1.0, (E, J)).astype(np.float32)
    return q, qd


def _energy(tree, P, q, qd):
    T, V = dyn.energy(tree, P, torch.as_tensor(q, dtype=torch.float64),
                      torch.as_tensor(qd, dtype=torch.float64))
    return (T + V).numpy(), (T.abs() + V.abs()).numpy()


def _gpu_trajectory(desc, q, qd, substeps):
    """q, qd after every control step (dt = H, `substeps` substeps each)."""
    env = sg.Env(desc)
    env.set_state(torch.as_tensor(q, device="cuda"), torch.as_tensor(qd, device="cuda"))
    acts = torch.zeros(STEPS, desc["num_envs"], desc["max_joints"], device="cuda")
    obs, _, _ = env.rollout(acts, H, substeps)
    assert env.sync_status() == sg.SG_OK
    n = desc["max_joints"]
    o = obs.cpu().numpy().astype(np.float64)
    return o[:, :, :n], o[:, :, n:2 * n]


def _oracle_trajectory(tree, P, q, qd, substeps):
    h = H / substeps
    q = torch.as_tensor(q, dtype=torch.float64)
    qd = torch.as_tensor(qd, dtype=torch.float64)
    zero = torch.zeros_like(q)
    Q, QD = [], []
    for _ in range(STEPS):
        for _ in range(substeps):
            q, qd, _ = dyn.substep(tree, P, q, qd, zero, h)
        Q.append(q.numpy())
        QD.append(qd.numpy())
    return np.stack(Q), np.stack(QD)


def _errors(tree, P, E0, scale, Q, QD, every=5):
    """Relative energy error per checked step [k][E]."""
    return np.stack([np.abs(_energy(tree, P, Q[k], QD[k])[0] - E0) / scale
                     for k in range(0, STEPS, every)])


@pytest.mark.parametrize("L", [None, 2.0], ids=["config-links", "long-link"])
def test_pendulum_energy_follows_the_oracle(L):
    desc = chain_desc([([0], [1])], E=64, seed=14, L=None if L is None else [L],
                      episode_len=10 * STEPS)
    (idx, tree), = groups(desc)
    P = make_params(tree, desc, idx)
    q, qd = _start(desc, 21)
    E0, scale = _energy(tree, P, q, qd)
    res = {}
    for S in (1, 2):
        Qg, QDg = _gpu_trajectory(desc, q, qd, S)
        Qr, QDr = _oracle_trajectory(tree, P, q, qd, S)
        eg = _errors(tree, P, E0, scale, Qg, QDg)
        er = _errors(tree, P, E0, scale, Qr, QDr)
        # energy of the GPU states follows the oracle's (FP32 adds no drift)
        Eg = np.stack([_energy(tree, P, Qg[k], QDg[k])[0] for k in range(0, STEPS, 50)])
        Er = np.stack([_energy(tree, P, Qr[k], QDr[k])[0] for k in range(0, STEPS, 50)])
        assert (np.abs(Eg - Er) / scale).max() <= 2e-3
        half = eg.shape[0] // 2
        first, second = eg[:half].max(), eg[half:].max()
        assert eg.max() <= 1.05 * er.max() + 1e-5
        assert second <= 1.05 * first + 1e-5            # no secular drift
        res[S] = eg.max()
    # first order in h: halving the substep halves the error
    assert 0.4 < res[2] / res[1] < 0.6, res
    if L is not None:
        assert res[1] <= 3.5e-2, res   # a 2 m pendulum at h = 1/120: 3.0% (FP64 oracle)
