"""Input generators: counts, ranges and the path spline (host-side inputs)."""
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


def test_natural_spline_interpolates_with_zero_end_curvature():
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1, 1, size=(16, 3))
    a, b, c, d = W.natural_cubic_spline(pts)
    assert np.allclose(d, pts[:-1])
    assert np.allclose(a[-1] + b[-1] + c[-1] + d[-1], pts[-1])
    assert np.allclose(b[0], 0)                        # S''(t_0) = 2b = 0
    assert np.allclose(6 * a[-1] + 2 * b[-1], 0)       # S''(t_end) = 0
    # C2 continuity at interior knots
    assert np.allclose(3 * a[:-1] + 2 * b[:-1] + c[:-1], c[1:])
    assert np.allclose(6 * a[:-1] + 2 * b[:-1], 2 * b[1:])


def test_waypoints_equally_spaced():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-0.15, 0.15, size=(16, 3))
    wp = W.resample_equal_arclength(*W.natural_cubic_spline(pts), 503)
    seg = np.linalg.norm(np.diff(wp, axis=0), axis=1)
    assert seg.std() / seg.mean() < 0.02
    assert np.allclose(wp[0], pts[0]) and np.allclose(wp[-1], pts[-1])


def test_joint_targets_resampled_every_50_steps():
    d = W.make_desc(["7R", "4R"])
    a = W.joint_targets(d, 120)
    assert (a[0] == a[49]).all() and not (a[49] == a[50]).all() and (a[50] == a[99]).all()
    assert (a[:, 1, 4:] == 0).all()
    assert (a >= d["q_lo"][None]).all() and (a <= d["q_hi"][None]).all()
