"""Input generators: counts, ranges, path control points and action draws."""
import numpy as np

from paper_2310_04676_gb300 import workloads as W


def test_mixed_counts_largest_remainder():
    kinds = W.mixed_kinds(16384, W.C3_FRACTIONS)
    cnt = {k: kinds.count(k) for k in W.C3_FRACTIONS}
    assert cnt == {"4R": 4096, "7R": 6554, "7P": 3277, "14B": 2457}
    assert kinds[:8] != sorted(kinds[:8])          # interleaved by the permutation


def test_desc_ranges():
    d = W.make_desc(["7R", "7P", "14B", "4R"] * 4)
    nj = d["chain_num_joints"].sum(1)
    for e in range(16):
        n = nj[e]
        L, m = d["link_len"][e, :n], d["link_mass"][e, :n]
        assert (L >= 0.05).all() and (L <= 0.4).all() and (m >= 0.1).all() and (m <= 1.0).all()
        pris = d["joint_type"][e, :n] == 1
        assert np.allclose(d["q_hi"][e, :n][pris], 0.2)
        assert np.allclose(d["q_hi"][e, :n][~pris], np.pi / 2)


def test_path_control_points_in_goal_cube():
    d = W.make_desc(["7R"] * 6, task=1, path_len=40)
    assert d["path"] is None and d["path_len"] == 40
    ctrl = d["path_ctrl"]
    assert ctrl.shape == (6, d["path_ctrl_len"], 3) and ctrl.dtype == np.float32
    for e in range(6):
        R = d["link_len"][e, :7].sum()
        centre = np.array([0.3 * R, 0.0, 0.5 * R])
        assert (np.abs(ctrl[e] - centre) <= 0.15 + 1e-6).all()


def test_joint_targets_resampled_every_50_steps():
    d = W.make_desc(["7R", "4R"])
    a = W.joint_targets(d, 120)
    assert (a[0] == a[49]).all() and not (a[49] == a[50]).all() and (a[50] == a[99]).all()
    assert (a[:, 1, 4:] == 0).all()
    assert (a >= d["q_lo"][None]).all() and (a <= d["q_hi"][None]).all()
