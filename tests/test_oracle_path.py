"""Pins of the path-following waypoint oracle (Results, "Path following":
cubic spline through the path points, waypoints at regular intervals of
distance along it).

The spline is checked against what a natural cubic spline is (interpolation,
C2 continuity, zero end curvature, a closed form for three points, the
library routine scipy.interpolate.CubicSpline), the resampling against a
brute-force walk along the polyline and a straight line, where the
waypoints are known in closed form."""
import numpy as np
import pytest

from oracle import path as OP


def _pts(seed, K=16):
    return np.random.default_rng(seed).uniform(-0.15, 0.15, size=(K, 3)) + [0.3, 0.0, 0.5]


def _eval(coef, t):
    a, b, c, d = coef
    i = np.minimum(np.floor(t).astype(int), a.shape[0] - 1)
    s = (t - i)[:, None]
    return ((a[i] * s + b[i]) * s + c[i]) * s + d[i]


def test_spline_interpolates_and_is_c2_with_natural_ends():
    P = _pts(0)
    a, b, c, d = OP.natural_spline_coeffs(P)
    assert np.allclose(d, P[:-1], atol=1e-14)
    assert np.allclose(a[-1] + b[-1] + c[-1] + d[-1], P[-1], atol=1e-14)
    assert np.allclose(b[0], 0.0)                                  # S''(t_0) = 2 b_0
    assert np.allclose(6 * a[-1] + 2 * b[-1], 0.0, atol=1e-12)     # S''(t_end)
    assert np.allclose(3 * a[:-1] + 2 * b[:-1] + c[:-1], c[1:], atol=1e-12)   # S'
    assert np.allclose(6 * a[:-1] + 2 * b[:-1], 2 * b[1:], atol=1e-12)        # S''


def test_three_point_closed_form():
    """K = 3: one interior unknown, 4 M_1 = 6 (P_2 - 2 P_1 + P_0)."""
    P = _pts(1, K=3)
    a, b, c, d = OP.natural_spline_coeffs(P)
    M1 = 1.5 * (P[2] - 2 * P[1] + P[0])
    assert np.allclose(a[0], M1 / 6) and np.allclose(a[1], -M1 / 6)
    assert np.allclose(b[1], M1 / 2)
    assert np.allclose(c[0], P[1] - P[0] - M1 / 6)


def test_two_points_is_the_segment():
    P = _pts(2, K=2)
    a, b, c, d = OP.natural_spline_coeffs(P)
    assert np.allclose(a, 0) and np.allclose(b, 0) and np.allclose(c[0], P[1] - P[0])


def test_matches_library_natural_spline():
    interp = pytest.importorskip("scipy.interpolate")
    for seed, K in ((3, 16), (4, 5), (5, 64)):
        P = _pts(seed, K)
        coef = OP.natural_spline_coeffs(P)
        cs = interp.CubicSpline(np.arange(K, dtype=np.float64), P, bc_type="natural")
        t = np.linspace(0, K - 1, 997)
        assert np.abs(_eval(coef, t) - cs(t)).max() < 1e-12


def test_dense_polyline_samples_the_spline():
    P = _pts(6, K=7)
    coef = OP.natural_spline_coeffs(P)
    D = OP.dense_polyline(*coef, dense=64)
    assert D.shape == (64 * 6 + 1, 3)
    t = np.arange(64 * 6 + 1) / 64.0
    assert np.abs(D - _eval(coef, t)).max() < 1e-13


def test_straight_line_waypoints_closed_form():
    """Collinear, equally spaced control points: the natural spline is the
    line itself and the waypoints divide it evenly."""
    p0, p1 = np.array([0.1, -0.2, 0.4]), np.array([0.5, 0.3, 0.2])
    P = p0 + np.linspace(0, 1, 9)[:, None] * (p1 - p0)
    wp = OP.waypoints(P[None], 41)[0]
    expect = p0 + np.linspace(0, 1, 41)[:, None] * (p1 - p0)
    assert np.abs(wp - expect).max() < 1e-12


def test_waypoints_at_equal_arc_length_brute_force():
    """Each waypoint lies on the dense polyline at arc length w L / (W - 1),
    found by walking the polyline segment by segment."""
    P = _pts(7)
    coef = OP.natural_spline_coeffs(P)
    D = OP.dense_polyline(*coef)
    W = 203
    wp = OP.resample_equal_arclength(*coef, W)
    seg = [float(np.sqrt(((D[k + 1] - D[k]) ** 2).sum())) for k in range(len(D) - 1)]
    L = sum(seg)
    for w in range(0, W, 7):
        target, k, acc = w * L / (W - 1), 0, 0.0
        while k < len(seg) - 1 and acc + seg[k] < target:
            acc += seg[k]
            k += 1
        f = (target - acc) / seg[k]
        assert np.abs(wp[w] - (D[k] + f * (D[k + 1] - D[k]))).max() < 1e-9
    assert np.allclose(wp[0], P[0]) and np.allclose(wp[-1], P[-1])


def test_batched_tables_match_per_env():
    ctrl = np.stack([_pts(s) for s in range(3)])
    tab = OP.waypoints(ctrl, 50)
    for e in range(3):
        assert np.array_equal(tab[e], OP.resample_equal_arclength(*OP.natural_spline_coeffs(ctrl[e]), 50))
