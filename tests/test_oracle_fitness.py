"""Pins of the oracle's fitness (Eqs. path_fit, lenth, penalty; Sec. 3.3.2).

Length is checked against closed forms, the collision count Q against dense
point sampling and hand-built geometric cases, the penalty against hand values.
"""
import json
from pathlib import Path

import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300.inputs import SepsoConfig, random_circles

GOLDEN = Path(__file__).parent / "golden"


def _cfg(T, alpha=30.0, beta=4):
    return SepsoConfig(T=T, G=1, N=1, alpha=alpha, beta=beta)


def _row(xs, ys):
    return np.array(list(xs) + list(ys), dtype=np.float64)


def test_length_straight_line_is_distance():
    # Collinear, evenly spaced waypoints: the polyline length is |target - start|.
    T = 8
    s, t = np.array([20.0, 20.0]), np.array([380.0, 380.0])
    lam = np.arange(1, T + 1) / (T + 1)
    w = s[None, :] + lam[:, None] * (t - s)[None, :]
    F, Q, L = oracle.evaluate(_cfg(T), oracle.Scene(s, t, np.zeros((0, 3))), _row(w[:, 0], w[:, 1]))
    assert Q[0] == 0
    assert L[0] == pytest.approx(360.0 * np.sqrt(2.0), rel=1e-12)
    assert F[0] == L[0]


def test_hand_cases_from_golden():
    cases = json.loads((GOLDEN / "fitness_hand.json").read_text())["cases"]
    for c in cases:
        T = len(c["waypoints"])
        w = np.array(c["waypoints"], dtype=np.float64)
        sc = oracle.Scene(c["start"], c["target"], np.array(c["circles"], dtype=np.float64).reshape(-1, 3))
        F, Q, L = oracle.evaluate(_cfg(T, c["alpha"], c["beta"]), sc, _row(w[:, 0], w[:, 1]))
        assert Q[0] == c["Q"], c["name"]
        assert L[0] == pytest.approx(c["length"], rel=1e-12, abs=1e-12), c["name"]
        assert F[0] == pytest.approx(c["F"], rel=1e-12), c["name"]


def _dense_min_dist(a, b, c, n=20001):
    t = np.linspace(0.0, 1.0, n)
    pts = a[None, :] + t[:, None] * (b - a)[None, :]
    return np.sqrt(((pts - c[None, :]) ** 2).sum(1)).min()


def test_point_segment_distance_matches_dense_sampling():
    rng = np.random.default_rng(7)
    for _ in range(300):
        a, b, c = rng.uniform(0, 100, (3, 2))
        d = oracle.seg_point_dist(a, b, c)
        dense = _dense_min_dist(a, b, c)
        # dense sampling over-estimates by at most half the sampling step
        step = np.linalg.norm(b - a) / 20000
        assert d <= dense + 1e-12
        assert dense - d <= step / 2 + 1e-9


def test_point_segment_distance_zero_length_segment():
    assert oracle.seg_point_dist((3, 4), (3, 4), (0, 0)) == pytest.approx(5.0)


def test_collision_count_matches_dense_sampling():
    # Tiny random scenes, pairs near tangency excluded: Q from the oracle equals the
    # count of (segment, circle) pairs whose dense samples come within r.
    rng = np.random.default_rng(11)
    T = 3
    cfg = _cfg(T, alpha=1.0, beta=1)
    checked = 0
    for trial in range(40):
        circ = random_circles(rng, 5, lo=10, hi=90, r_lo=3, r_hi=15).astype(np.float64)
        s, t = rng.uniform(0, 100, 2), rng.uniform(0, 100, 2)
        w = rng.uniform(0, 100, (T, 2))
        sc = oracle.Scene(s, t, circ)
        _, Q, _ = oracle.evaluate(cfg, sc, _row(w[:, 0], w[:, 1]))
        pts = np.vstack([s, w, t])
        q, near = 0, False
        for j in range(T + 1):
            for o in range(circ.shape[0]):
                dd = _dense_min_dist(pts[j], pts[j + 1], circ[o, :2])
                if abs(dd - circ[o, 2]) < 0.05:
                    near = True
                q += int(dd < circ[o, 2])
        if near:
            continue
        checked += 1
        assert Q[0] == q
    assert checked >= 20


@pytest.mark.parametrize("name,a,b,expect", [
    ("through centre", (0, 50), (100, 50), 1),
    ("parallel just inside", (0, 59.99), (100, 59.99), 1),
    ("parallel just outside", (0, 60.01), (100, 60.01), 0),
    ("fully inside disk", (48, 49), (52, 51), 1),
    ("stops short of disk", (0, 50), (39.9, 50), 0),
    ("endpoint inside disk", (0, 50), (41, 50), 1),
    ("zero length inside", (45, 45), (45, 45), 1),
    ("zero length outside", (45, 65), (45, 65), 0),
])
def test_collision_analytic_cases(name, a, b, expect):
    # One circle at (50, 50) with r = 10; a path of one waypoint placed at b, with
    # start at a and target at b, so segment 0 is [a, b] and segment 1 has length 0.
    circ = np.array([[50.0, 50.0, 10.0]])
    sc = oracle.Scene(a, b, circ)
    F, Q, L = oracle.evaluate(_cfg(1, alpha=1.0, beta=1), sc, _row([b[0]], [b[1]]))
    # the zero-length second segment [b, b] is inside the disk exactly when b is
    inside_b = np.hypot(b[0] - 50, b[1] - 50) < 10
    assert Q[0] == expect + int(inside_b), name


def test_penalty_power_and_alpha():
    # Straight path crossing two disks: Q = 2, so penalty = 30 * 2^4 = 480.
    circ = np.array([[100.0, 50.0, 10.0], [200.0, 50.0, 10.0]])
    sc = oracle.Scene((0, 50), (300, 50), circ)
    F, Q, L = oracle.evaluate(_cfg(1, alpha=30.0, beta=4), sc, _row([150.0], [50.0]))
    assert Q[0] == 2
    assert L[0] == pytest.approx(300.0)
    assert F[0] == pytest.approx(300.0 + 480.0)
    F1, _, _ = oracle.evaluate(_cfg(1, alpha=1000.0, beta=1), sc, _row([150.0], [50.0]))
    assert F1[0] == pytest.approx(300.0 + 2000.0)
