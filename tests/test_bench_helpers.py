"""The benchmark's bookkeeping (no GPU): FLOP and byte counts per workload,
timing statistics, replica seeding, the single-rank aggregation, and the
gate that attaches profiled counters only to the launch they came from."""
import sys

import numpy as np
import pytest

from paper_2310_04676_gb300 import workloads as W

sys.argv = ["bench"]
import bench  # noqa: E402


def test_env_step_flops_by_hand():
    S = 2
    sub, tip, rew = bench.FLOP_SUBSTEP, bench.FLOP_TIP, bench.FLOP_REWARD
    got = bench.env_step_flops(["7R", "4R", "14B", "7P"], S)
    want = (S * sub["7R"] + tip["7R"] + rew) * 3 + (S * sub["4R"] + tip["4R"] + rew) \
        + (S * sub["7P"] + tip["7P"] + rew)
    assert got == want
    # the path task adds the tip quaternion once per chain
    assert bench.env_step_flops(["7R"], S, task=1) - bench.env_step_flops(["7R"], S) == bench.FLOP_QUAT


def test_adjoint_flops_by_hand():
    T, S, k = 20, 3, 8                       # segments of 8, 8, 4 steps
    f, b = bench.adjoint_flops(["7R"], S, T, k)
    sub, adj = bench.FLOP_SUBSTEP["7R"], bench.FLOP_SUBSTEP_ADJ["7R"]
    rep = bench.FLOP_SUBSTEP_REPLAY["7R"]
    # the forward does the last segment's (4 steps) replay part instead of its substeps
    assert f == T * (S * sub + bench.FLOP_TIP["7R"]) + 4 * S * (rep - sub)
    assert b == T * (bench.FLOP_TIP_VJP["7R"] + S * adj) - 4 * S * rep
    # forward + backward together: every substep once forward, once as an adjoint
    assert f + b == T * (S * sub + bench.FLOP_TIP["7R"] + bench.FLOP_TIP_VJP["7R"] + S * adj) \
        - 4 * S * sub
    f1, b1 = bench.adjoint_flops(["7R"], S, T, k, replay=False)
    assert f1 == T * (S * sub + bench.FLOP_TIP["7R"])
    assert b1 == T * (bench.FLOP_TIP_VJP["7R"] + S * adj) + (7 + 7 + 3) * S * sub \
        + T * (S - 1) * sub
    # a two-arm env counts two chains
    assert bench.adjoint_flops(["14B"], S, T, k) == (2 * f, 2 * b)


def test_env_step_bytes():
    d = W.make_desc(["7R", "14B"])
    D = 54
    assert bench.env_step_bytes(d, D) == 4 * (7 + 14) + 2 * (4 * D + 4 + 1)
    dp = W.make_desc(["7R"] * 3, task=1, path_len=10)
    assert bench.env_step_bytes(dp, 30) == 4 * 21 + 3 * (4 * 30 + 5) + 48 * 3


def test_ppo_flops_closed_form():
    D, A, E, n, ep = 28, 8, 100, 4, 5
    h = (256, 128, 64)
    fw_a = 2 * (D * h[0] + h[0] * h[1] + h[1] * h[2] + h[2] * A)
    fw_c = 2 * (D * h[0] + h[0] * h[1] + h[1] * h[2] + h[2] * 1)
    col, upd = bench.ppo_flops(D, A, E, n, ep)
    assert col == n * E * (fw_a + fw_c) + E * fw_c
    assert upd == ep * n * E * (fw_a + fw_c + 2 * (fw_a + fw_c) - 4 * D * h[0])


def test_stats_median_and_iqr():
    st = bench.stats([1.0, 2.0, 3.0, 4.0, 100.0])
    assert st["median_ms"] == 3.0 and st["n"] == 5
    assert np.isclose(st["iqr_ms"], np.percentile([1, 2, 3, 4, 100], 75) - np.percentile([1, 2, 3, 4, 100], 25))


def test_single_rank_aggregation():
    assert bench.aggregate_rate(1000, 2.0, world=1) == 500.0


def test_replicas_draw_their_own_robots():
    wl = W.config("C3", num_envs=64)
    d0, d1 = bench.replica_desc(wl, 0), bench.replica_desc(wl, 1)
    assert d0 is wl.desc
    assert np.array_equal(d0["chain_num_joints"], d1["chain_num_joints"])   # same kinds
    assert not np.array_equal(d0["link_len"], d1["link_len"])               # own parameters


def test_profile_counters_only_for_the_profiled_launch():
    """The committed step-kernel summary's counters are attached to the
    default workload's launch only; elsewhere traffic is null."""
    class P:
        multi_processor_count = 152
    peaks = {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}
    bench._FMA_RATE["v"] = 78.0          # no GPU here: a stand-in for the probe
    r = bench.roofline("step_kernel", 1.5e9, 1.3e8, 0.12, P, peaks, "measured", profiled=False)
    assert r["traffic"] is None and r["executed_tflops"] is None and r["l2_write_bytes"] is None
    assert np.isclose(r["peak"], 152 * 128 * 2 * 2070e6 / 1e12)
    assert np.isclose(r["frac"], 1.5e9 / 0.12e-3 / 1e12 / r["peak"])
    r = bench.roofline("step_kernel", 1.5e9, 1.3e8, 0.12, P, peaks, "measured", profiled=True)
    if bench.profiled_traffic("step_kernel") is not None:      # summary matches the sources
        assert r["traffic"] == bench.profiled_traffic("step_kernel")
        assert r["executed_tflops"] > 0
        # the L2 write sectors: at least the DRAM writes, at most all L2 sector traffic
        assert r["l2_write_bytes"] == bench.profiled_counter("step_kernel",
                                                             "l2_write_bytes_per_launch")
        assert r["l2_write_bytes"] > 0
    bench._FMA_RATE.clear()
