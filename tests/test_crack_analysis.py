"""The crack-geometry extraction on drawn phase fields with a known answer (CPU)."""
import math

import numpy as np

from paper_2602_15149_b300 import workloads as W
from paper_2602_15149_b300.crack import CrackTracker, image, runs


def _y_crack(case, x_b, half_angle_deg, x_end, width, tilt_lo=0.0):
    """s = 0 on a straight crack along the notch plane up to x_b, then on two straight branches at
    +half_angle and -(half_angle + tilt_lo) degrees up to x_end, each ``width`` thick; 1 elsewhere."""
    X = case.X0
    y0, xn = 0.02, 0.05
    s = np.ones(case.n)
    stem = (X[:, 0] > xn) & (X[:, 0] <= x_b) & (np.abs(X[:, 1] - y0) < width / 2)
    s[stem] = 0.0
    for sign, ang in ((1, half_angle_deg), (-1, half_angle_deg + tilt_lo)):
        k = math.tan(math.radians(ang))
        on = (X[:, 0] > x_b) & (X[:, 0] <= x_end) & (np.abs(X[:, 1] - (y0 + sign * k * (X[:, 0] - x_b))) < width / 2)
        s[on] = 0.0
    return s


def test_runs_and_image_round_trip():
    assert runs(np.array([0, 1, 1, 0, 1, 0, 0, 1], bool)) == [(1, 2), (4, 4), (7, 7)]
    case = W.notched_plate(nx=50, ny=20)
    s = np.arange(case.n, dtype=float)
    img = image(case.X0, s, case.dp)
    assert img.shape == (20, 50)
    i = np.rint(case.X0[:, 0] / case.dp - 0.5).astype(int)
    j = np.rint(case.X0[:, 1] / case.dp - 0.5).astype(int)
    assert np.array_equal(img[j, i], s) and np.unique(img).size == case.n


def test_recovers_branch_point_angle_and_symmetry():
    case = W.notched_plate(nx=500, ny=200)
    tr = CrackTracker(case.X0, case.dp, 0.02, 0.05)
    tr.add(1e-6, np.ones(case.n))
    assert tr.t_init is None
    tr.add(2e-6, _y_crack(case, 0.055, 30.0, 0.055, 1e-3))       # straight crack only
    assert tr.t_init == 2e-6 and tr.t_branch is None
    tr.add(3e-6, _y_crack(case, 0.06, 30.0, 0.08, 1e-3))
    assert tr.t_branch == 3e-6
    g = tr.geometry()
    assert abs(g["angle_deg"] - 60.0) < 4.0
    assert abs(g["angle_up_deg"] - g["angle_lo_deg"]) < 2.0
    assert 0.06 <= g["branch_x"] < 0.065
    assert g["asymmetry"] < 0.05
    tip = [x for _, x in tr.tip_x]
    assert math.isnan(tip[0]) and tip[-1] > 0.079


def test_asymmetric_pattern_is_reported():
    case = W.notched_plate(nx=500, ny=200)
    tr = CrackTracker(case.X0, case.dp, 0.02, 0.05)
    tr.add(1e-6, _y_crack(case, 0.06, 30.0, 0.08, 1e-3, tilt_lo=20.0))
    g = tr.geometry()
    assert g["asymmetry"] > 0.3
    assert g["angle_lo_deg"] - g["angle_up_deg"] > 12.0


def test_vectorised_branch_detection_equals_column_scan():
    """branched_columns against a plain per-column scan of the runs, on random patterns."""
    from paper_2602_15149_b300.crack import branched_columns
    rng = np.random.default_rng(0)
    for _ in range(200):
        ny, nx = rng.integers(10, 40), rng.integers(1, 20)
        c = rng.random((ny, nx)) < rng.uniform(0.05, 0.6)
        j0, gap = rng.uniform(2, ny - 3), int(rng.integers(0, 4))
        ref = {}
        for i in range(nx):
            rs = runs(c[:, i])
            up = [r for r in rs if r[0] >= j0 + gap]
            lo = [r for r in rs if r[1] <= j0 - gap]
            if up and lo:
                u, d = min(up, key=lambda r: r[0]), max(lo, key=lambda r: r[1])
                ref[i] = (0.5 * (u[0] + u[1]), 0.5 * (d[0] + d[1]))
        assert branched_columns(c, j0, gap) == ref
