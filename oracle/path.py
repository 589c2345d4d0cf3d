"""Path-following waypoints (Results, "Path following"): a cubic spline
S(t) = a (t - t_i)^3 + b (t - t_i)^2 + c (t - t_i) + d through the control
points, sampled at regular intervals of distance along the curve.

Readings (the paper names neither): uniform knots t_i = i, natural end
conditions S'' = 0 at both ends, and distance measured along a dense
polyline of 64 samples per segment, inverted linearly.
"""
import numpy as np


def natural_spline_coeffs(P):
    """Coefficients (a, b, c, d) [K-1, 3] of the natural cubic spline through
    P [K, 3] at t_i = i.  With second derivatives M_i (M_0 = M_{K-1} = 0),
    M_{i-1} + 4 M_i + M_{i+1} = 6 (P_{i+1} - 2 P_i + P_{i-1}) for interior i."""
    P = np.asarray(P, np.float64)
    K = P.shape[0]
    M = np.zeros_like(P)
    if K > 2:
        A = 4.0 * np.eye(K - 2) + np.eye(K - 2, k=1) + np.eye(K - 2, k=-1)
        M[1:-1] = np.linalg.solve(A, 6.0 * (P[2:] - 2.0 * P[1:-1] + P[:-2]))
    a = (M[1:] - M[:-1]) / 6.0
    b = M[:-1] / 2.0
    c = (P[1:] - P[:-1]) - (2.0 * M[:-1] + M[1:]) / 6.0
    d = P[:-1]
    return a, b, c, d


def dense_polyline(a, b, c, d, dense=64):
    """Samples of every segment at s = j / dense, j < dense, plus the end point."""
    s = np.arange(dense, dtype=np.float64) / dense
    pts = [((a[i] * s[:, None] + b[i]) * s[:, None] + c[i]) * s[:, None] + d[i]
           for i in range(a.shape[0])]
    last = a[-1] + b[-1] + c[-1] + d[-1]
    return np.concatenate(pts + [last[None]], 0)


def resample_equal_arclength(a, b, c, d, W, dense=64):
    """W waypoints equally spaced in distance along the dense polyline."""
    P = dense_polyline(a, b, c, d, dense)
    cum = np.concatenate([[0.0], np.cumsum(np.linalg.norm(np.diff(P, axis=0), axis=1))])
    target = np.linspace(0.0, cum[-1], W)
    return np.stack([np.interp(target, cum, P[:, k]) for k in range(3)], -1)


def waypoints(ctrl, W, dense=64):
    """Waypoint tables [E, W, 3] from control points [E, K, 3]."""
    ctrl = np.asarray(ctrl, np.float64)
    return np.stack([resample_equal_arclength(*natural_spline_coeffs(P), W, dense) for P in ctrl])
