"""FP64 CPU oracle for the batched articulated-arm step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this
package: only the tests, the smoke check and the benchmark's CPU-baseline
leg may call it.  It shares no code with the CUDA path.

What it computes (plain PyTorch CPU ops in float64, batched over
environments of identical structure, loops over links in Python):

* ``spatial``     Featherstone spatial algebra (6x6 Pluecker transforms,
                  spatial inertias, cross-product operators).
* ``model``       robot trees built from an ``sg_desc`` dictionary.
* ``dynamics``    forward kinematics (4x4 homogeneous transforms), RNEA,
                  CRBA, ABA, the implicit-drive semi-implicit Euler substep
                  and an RK4 integrator for conservation tests.
* ``env``         the per-environment observation, reward, done, reset and
                  step of the reaching / path-following / two-arm tasks.
* ``path``        the path-following waypoints: natural cubic spline through
                  control points, resampled at equal arc length.
* ``ppo``         the GPU-resident PPO loop: actor/critic MLPs, rollout with
                  time-out bootstrapping and resets, GAE, clipped PPO update
                  with Adam.
* ``rng``         the counter-based normal deviates of the tracking task's
                  moving goals and of the policy's exploration noise
                  (SplitMix64 finaliser, Box-Muller).
* ``lagrangian``  an independent equation of motion from the Lagrangian
                  L = T - V of plain forward kinematics (complex-step
                  Jacobians, central finite differences).

The paper (Surgical Gym) specifies the joint types, PD drives, sub-stepping,
observation vector, rewards and time-out handling (Methods, Results) but no
dynamics formulas; the dynamics are textbook reduced-coordinate rigid-body
dynamics (Featherstone, "Rigid Body Dynamics Algorithms", 2008).

Parity pins: every function is checked in ``tests/test_oracle_*.py``
against closed forms, invariants and finite differences; none is
"parity unpinned".
"""
from . import spatial, model, dynamics, env, lagrangian, path, ppo, rng  # noqa: F401
