"""The oracle's polygon-obstacle objective (Sec. 3.3.1 map model, Eq. penalty with Q
the number of crossings between path segments and obstacle edges), pinned without a
GPU: hand cases of the segment test, a parametric solver as an independent check,
the crossing counts of hand-made paths (Fig. path: a path through two boxes has Q = 4;
Fig. obstype: a path through the notch of a non-convex obstacle has Q = 0), and run
invariants of DTPSO on a polygon scene.
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300.inputs import (POLYGON_PATH, TABLE_HYPER8_PATH, BFConfig, polygon_edges,
                                           polygon_workload)


def test_segment_crossing_hand_cases():
    assert oracle.seg_cross((0, 0), (2, 2), (0, 2), (2, 0))           # an X
    assert not oracle.seg_cross((0, 0), (1, 1), (1, 1), (2, 0))       # shared endpoint
    assert not oracle.seg_cross((0, 0), (2, 0), (1, 0), (3, 0))       # collinear overlap
    assert not oracle.seg_cross((0, 0), (1, 0), (0, 1), (1, 1))       # parallel
    assert not oracle.seg_cross((0, 0), (2, 0), (1, 0), (1, 5))       # T-junction on the segment
    assert not oracle.seg_cross((0, 0), (1, 1), (2, 0), (3, -5))      # lines cross beyond the ends
    assert oracle.seg_cross((0, 0), (4, 1), (1, -3), (2, 3))


def _param_cross(a, b, c, d):
    """Independent check: solve a + t (b - a) = c + u (d - c); a proper crossing has
    0 < t < 1 and 0 < u < 1."""
    A = np.array([[b[0] - a[0], -(d[0] - c[0])], [b[1] - a[1], -(d[1] - c[1])]])
    det = np.linalg.det(A)
    if abs(det) < 1e-9:
        return None
    t, u = np.linalg.solve(A, np.array([c[0] - a[0], c[1] - a[1]]))
    if min(abs(t), abs(t - 1), abs(u), abs(u - 1)) < 1e-9:
        return None
    return bool(0 < t < 1 and 0 < u < 1)


def test_segment_crossing_matches_parametric_solver():
    rng = np.random.default_rng(3)
    n = 0
    for _ in range(4000):
        a, b, c, d = rng.uniform(0, 10, (4, 2))
        want = _param_cross(a, b, c, d)
        if want is None:
            continue
        assert oracle.seg_cross(a, b, c, d) == want
        n += want
    assert n > 300                                   # both outcomes exercised


def _eval(edges, start, target, waypoints, alpha=30.0, beta=4):
    T = len(waypoints)
    cfg = BFConfig(fn=POLYGON_PATH, D=2 * T, G=1, N=1, map_w=400.0, map_h=400.0, alpha=alpha,
                   beta=beta)
    sc = oracle.Scene(start, target, np.zeros((0, 3)), edges)
    w = np.asarray(waypoints, np.float64)
    x = np.concatenate([w[:, 0], w[:, 1]])
    F, Q = oracle.BFSwarm(cfg, TABLE_HYPER8_PATH[:1], sc).evaluate(x[None], with_q=True)
    return float(F[0]), int(Q[0])


BOX = [(100, 100), (200, 100), (200, 200), (100, 200)]
BOX2 = [(260, 100), (320, 100), (320, 200), (260, 200)]
U = [(100, 100), (200, 100), (200, 200), (170, 200), (170, 130), (130, 130), (130, 200), (100, 200)]


def test_crossing_counts_of_hand_paths():
    e1 = polygon_edges([BOX])
    line = [(50 + 37 * i, 150.0) for i in range(1, 8)]             # on y = 150, off every edge
    F, Q = _eval(e1, (40, 150), (390, 150), line)
    assert Q == 2                                                   # in and out of the box
    assert F == pytest.approx(350.0 + 30.0 * 2 ** 4, rel=1e-12)
    F, Q = _eval(polygon_edges([BOX, BOX2]), (40, 150), (390, 150), line)
    assert Q == 4                                                   # through two boxes
    below = [(50 + 37 * i, 60.0) for i in range(1, 8)]
    assert _eval(e1, (40, 60), (390, 60), below)[1] == 0            # around the box
    inside = [(120, 150), (180, 150)]
    assert _eval(e1, (110, 150), (190, 150), inside)[1] == 0        # wholly inside: no crossing


def test_non_convex_obstacle():
    eu = polygon_edges([U])
    # down into the notch and back out through its mouth: no edge crossed
    notch = [(150, 210), (150, 150), (150, 140), (150, 210)]
    assert _eval(eu, (150, 260), (150, 260), notch)[1] == 0
    # straight across both arms and the notch: four crossings
    across = [(60 + 43 * i, 170.0) for i in range(1, 7)]
    assert _eval(eu, (40, 170), (390, 170), across)[1] == 4
    # across the base of the U: two crossings
    base = [(60 + 43 * i, 115.0) for i in range(1, 7)]
    assert _eval(eu, (40, 115), (390, 115), base)[1] == 2


def test_workload_shape_and_run_invariants():
    cfg, start, target, polys, edges, hy = polygon_workload(0, N=12, iters=40)
    assert edges.shape == (12 * 4 + 4 * 8, 4)
    assert cfg.D == 16 and cfg.fn == POLYGON_PATH
    sc = oracle.Scene(start, target, np.zeros((0, 3)), edges)
    sw = oracle.BFSwarm(cfg, hy, sc)
    hist = sw.run(40)
    assert np.all(np.diff(hist) <= 0)
    F, Q = sw.evaluate(sw.s["Tb"][None], with_q=True)
    assert F[0] == pytest.approx(sw.s["Tfit"][0], rel=1e-12)
    X = sw.s["X"].reshape(-1, cfg.D)
    assert X.min() >= 0.0 and X.max() <= 400.0
    assert hist[-1] < hist[0]


def test_polygon_workload_shapes():
    # 12 convex boxes and 4 non-convex U outlines; every polygon closed, inside the map
    cfg, start, target, polys, edges, hy = polygon_workload(5)
    assert len(polys) == 16 and edges.shape == (80, 4)

    def turns(poly):
        v = np.asarray(poly, np.float64)
        d = np.roll(v, -1, axis=0) - v
        return np.sign(d[:, 0] * np.roll(d, -1, axis=0)[:, 1] - d[:, 1] * np.roll(d, -1, axis=0)[:, 0])

    for poly in polys[:12]:
        t = turns(poly)
        assert len(poly) == 4 and (np.all(t > 0) or np.all(t < 0))          # convex
    for poly in polys[12:]:
        t = turns(poly)
        assert len(poly) == 8 and np.any(t > 0) and np.any(t < 0)           # non-convex
    # consecutive edges join, and the last edge returns to the first vertex
    e = edges[:48].reshape(12, 4, 4)                     # the boxes' edges
    np.testing.assert_array_equal(e[:, 1:, :2], e[:, :-1, 2:])
    np.testing.assert_array_equal(e[:, 0, :2], e[:, -1, 2:])
    assert edges.min() >= 0.0 and edges.max() <= 400.0


# ---------------------------------------------------------------------------
# Moving polygons (the box obstacles of Sec. 4.3, moved as in the Fig. PP caption)
# ---------------------------------------------------------------------------

def _box(x0, y0, x1, y1):
    return [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]


def _adv(polys, vel, W=400.0, H=400.0, start=(20, 40), svel=(0, 3), target=(346, 326), tvel=(0, -8)):
    edges = polygon_edges(polys)
    off = np.concatenate([[0], np.cumsum([len(p) for p in polys])]).astype(np.int32)
    return oracle.advance_polygons(W, H, edges, off, np.asarray(vel, np.float64), start, svel, target, tvel)


def test_moving_boxes_hand_values():
    # left wall: [10,30]x[100,120] moving (-15, 2) -> [-5,15]x[102,122]; the box lies
    # past x = 0 moving left, so vx flips; vy does not
    e, v, *_ = _adv([_box(10, 100, 30, 120)], [(-15.0, 2.0)])
    np.testing.assert_array_equal(e, polygon_edges([_box(-5, 102, 15, 122)]))
    np.testing.assert_array_equal(v, [[15.0, 2.0]])
    # top-right corner: both components flip
    e, v, *_ = _adv([_box(380, 390, 395, 398)], [(8.0, 5.0)])
    np.testing.assert_array_equal(e, polygon_edges([_box(388, 395, 403, 403)]))
    np.testing.assert_array_equal(v, [[-8.0, -5.0]])
    # interior: plain translation
    e, v, *_ = _adv([_box(100, 100, 150, 130)], [(-2.5, 4.0)])
    np.testing.assert_array_equal(e, polygon_edges([_box(97.5, 104, 147.5, 134)]))
    np.testing.assert_array_equal(v, [[-2.5, 4.0]])
    # past the wall but already moving away: no flip
    e, v, *_ = _adv([_box(-10, 100, 5, 130)], [(3.0, 0.0)])
    np.testing.assert_array_equal(v, [[3.0, 0.0]])
    # touching exactly (box edge at x = 0 after the move) is not past it
    e, v, *_ = _adv([_box(2, 100, 22, 130)], [(-2.0, 0.0)])
    np.testing.assert_array_equal(v, [[-2.0, 0.0]])


def test_moving_polygons_keep_their_edges_and_bounce_alone():
    # two polygons: a U outline (8 edges) bouncing off the bottom wall through a
    # vertex that is not the first, and a box in the interior
    u = [(100, 5), (160, 5), (160, 65), (145, 65), (145, 20), (115, 20), (115, 65), (100, 65)]
    u = [(x, y + 1.0) for x, y in u]
    u[5] = (115, 1.5)   # lowest vertex of the outline is not the first one
    polys = [_box(200, 200, 240, 230), u]
    e, v, s, sv, t, tv = _adv(polys, [(1.0, 1.0), (0.0, -2.0)])
    e0 = polygon_edges(polys)
    np.testing.assert_allclose(e[:4], e0[:4] + np.array([1.0, 1.0, 1.0, 1.0]), rtol=0, atol=1e-12)
    np.testing.assert_allclose(e[4:], e0[4:] + np.array([0.0, -2.0, 0.0, -2.0]), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(v, [[1.0, 1.0], [0.0, 2.0]])   # only the U's vy flips (its y min is -0.5)
    # start and target move as with circles
    np.testing.assert_array_equal(s, [20, 43])
    np.testing.assert_array_equal(t, [346, 318])


def test_moving_box_follows_the_circle_rule():
    # a square of half-size r moves like a circle of radius r centred on it (both
    # bounce when centre -/+ r passes the border they move towards)
    rng = np.random.default_rng(8)
    for _ in range(50):
        r = rng.uniform(5, 30)
        c = rng.uniform(r, 400 - r, 2)
        vel = rng.uniform(-6, 6, 2)
        circ = np.array([[c[0], c[1], r]])
        cv = vel.reshape(1, 2)
        x0, y0, x1, y1 = c[0] - r, c[1] - r, c[0] + r, c[1] + r
        e = np.array([[x0, y0, x1, y0], [x1, y0, x1, y1], [x1, y1, x0, y1], [x0, y1, x0, y0]])
        off = np.array([0, 4], np.int32)
        bv = vel.reshape(1, 2)
        st, sv, tg, tv = (0, 0), (0, 0), (0, 0), (0, 0)
        for _ in range(120):
            circ, cv, *_ = oracle.advance_scene(400.0, 400.0, circ, cv, st, sv, tg, tv)
            e, bv, *_ = oracle.advance_polygons(400.0, 400.0, e, off, bv, st, sv, tg, tv)
        np.testing.assert_array_equal(cv, bv)
        np.testing.assert_allclose(e[0, :2], circ[0, :2] - r, rtol=0, atol=1e-9)


def test_planner_goes_around_a_box():
    # one box across the straight line: the optimum runs along the box, around a
    # corner pair; its length is |s - c1| + |c1 - c2| + |c2 - t| = 2 sqrt(100^2 + 50^2)
    # + 100 = 323.607 (touching a corner is not a crossing)
    from paper_2308_10169_gb300.inputs import SepsoConfig
    edges = polygon_edges([_box(150, 150, 250, 250)])
    cfg = SepsoConfig(T=8, G=8, N=40, alpha=30.0, beta=4, max_iters=200, obstacle_kind=1, seed=3,
                      max_obstacles=4)
    hy = np.ascontiguousarray(TABLE_HYPER8_PATH, np.float64)
    sw = oracle.Swarm(cfg, hy)
    r = sw.plan(oracle.Scene((50, 200), (350, 200), np.zeros((0, 3)), edges))
    best = 2 * np.hypot(100, 50) + 100
    assert r["Q"] == 0
    assert best - 1e-9 <= r["cost"] <= best * 1.02
    # the returned cost is the fitness of the returned path among the polygons
    F, Q, L = oracle.evaluate(cfg, oracle.Scene((50, 200), (350, 200), np.zeros((0, 3)), edges),
                              r["waypoints"].reshape(1, -1))
    assert Q[0] == 0 and abs(F[0] - r["cost"]) < 1e-9
