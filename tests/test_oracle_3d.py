"""The oracle's 3D path objective (the Conclusion's extension from 2D to 3D planning:
Eqs. path_fit, lenth, penalty with a third coordinate, spheres as obstacles and Q the
number of (segment, sphere) pairs closer than the radius), pinned without a GPU:

* the 3D segment-point distance against brute-force dense sampling and analytic
  cases (through the centre, parallel at r +- 0.01, inside the sphere, zero length,
  beyond either end);
* lengths by Pythagorean quadruples and collinear waypoints;
* a hand-worked path;
* the reduction to the pinned 2D circle objective when every z is 0;
* invariance under a permutation of the axes (a swapped or mis-indexed coordinate
  block fails it);
* DTPSO on the 3D box: per-axis initial and clipped ranges, Priori Initialization's
  count and interval, and the obstacle-free optimum |target - start|.
"""
import math

import numpy as np

import oracle
from paper_2308_10169_gb300.inputs import (SPHERE_PATH, TABLE_HYPER8_PATH, BFConfig, random_paths3,
                                           sphere_workload)


def _cfg(T, G=1, N=1, **kw):
    return BFConfig(fn=SPHERE_PATH, D=3 * T, G=G, N=N, map_w=400.0, map_h=400.0, map_d=400.0,
                    alpha=kw.pop("alpha", 30.0), beta=kw.pop("beta", 4), **kw)


def _row(waypoints):
    w = np.asarray(waypoints, np.float64).reshape(-1, 3)
    return np.concatenate([w[:, 0], w[:, 1], w[:, 2]])


def _eval(cfg, scene, X):
    sw = oracle.BFSwarm(cfg, TABLE_HYPER8_PATH[:cfg.G], scene)
    F, Q = sw.evaluate(np.atleast_2d(X), with_q=True)
    return F, Q


def _brute_dist(a, b, c, n=10001):
    t = np.linspace(0.0, 1.0, n)[:, None]
    pts = np.asarray(a)[None] + t * (np.asarray(b) - np.asarray(a))[None]
    return float(np.min(np.linalg.norm(pts - np.asarray(c)[None], axis=1)))


def test_distance_matches_dense_sampling():
    rng = np.random.default_rng(11)
    for _ in range(300):
        a, b, c = rng.uniform(-5, 5, (3, 3))
        d = oracle.seg_point_dist3(a, b, c)
        # sampling at 1e-4 of the segment overestimates by at most |ab| 1e-4 / 2
        assert d <= _brute_dist(a, b, c) + 1e-12
        assert d >= _brute_dist(a, b, c) - np.linalg.norm(b - a) * 1e-4


def test_distance_analytic_cases():
    a, b = np.array([1.0, 2.0, 3.0]), np.array([7.0, 2.0, 3.0])
    assert oracle.seg_point_dist3(a, b, (4.0, 2.0, 3.0)) == 0.0             # on the segment
    assert abs(oracle.seg_point_dist3(a, b, (4.0, 2.0, 8.0)) - 5.0) < 1e-12  # straight above
    assert abs(oracle.seg_point_dist3(a, b, (4.0, 5.0, 7.0)) - 5.0) < 1e-12  # 3-4-5 across y and z
    assert abs(oracle.seg_point_dist3(a, b, (10.0, 6.0, 3.0)) - 5.0) < 1e-12  # beyond b: distance to b
    assert abs(oracle.seg_point_dist3(a, b, (-2.0, 2.0, -1.0)) - 5.0) < 1e-12  # before a: distance to a
    p = np.array([2.0, -1.0, 4.0])
    assert abs(oracle.seg_point_dist3(p, p, (4.0, 2.0, 10.0)) - 7.0) < 1e-12  # zero length: 2-3-6-7
    # a slanted segment: the perpendicular distance from its parametrisation
    a, b = np.array([0.0, 0.0, 0.0]), np.array([4.0, 4.0, 2.0])
    n = np.array([1.0, -1.0, 0.0]) / math.sqrt(2.0)
    for off in (9.99, 10.01):
        c = 0.5 * (a + b) + off * n
        assert abs(oracle.seg_point_dist3(a, b, c) - off) < 1e-12


def test_q_counts_spheres_at_the_radius_boundary():
    T = 1
    cfg = _cfg(T)
    x = _row([(200.0, 200.0, 200.0)])
    start, target = (100.0, 200.0, 200.0), (300.0, 200.0, 200.0)   # both segments on the line y = z = 200
    for off, want in ((9.99, 1), (10.01, 0)):
        # one sphere of radius 10 above the first segment, one inside it at the second
        sc = oracle.Scene3(start, target, [(150.0, 200.0, 200.0 + off, 10.0), (250.0, 200.0, 200.0, 5.0)])
        F, Q = _eval(cfg, sc, x)
        assert Q[0] == want + 1
    # a segment wholly inside a sphere counts once
    sc = oracle.Scene3(start, target, [(200.0, 200.0, 200.0, 500.0)])
    assert _eval(cfg, sc, x)[1][0] == 2


def test_lengths_by_pythagorean_quadruples():
    cfg = _cfg(2, alpha=0.0)
    sc = oracle.Scene3((0.0, 0.0, 0.0), (3.0, 4.0, 14.0), np.zeros((0, 4)))
    # (0,0,0) -> (1,2,2): 3; -> (3,5,8): 7; -> (3,4,14)... (0,-1,6): sqrt(37)
    F, Q = _eval(cfg, sc, _row([(1.0, 2.0, 2.0), (3.0, 5.0, 8.0)]))
    assert Q[0] == 0 and abs(F[0] - (3.0 + 7.0 + math.sqrt(37.0))) < 1e-12
    # collinear waypoints: exactly the straight-line length
    s, t = np.array([20.0, 30.0, 40.0]), np.array([380.0, 250.0, 330.0])
    cfg = _cfg(5, alpha=0.0)
    w = [s + f * (t - s) for f in (0.1, 0.3, 0.35, 0.8, 0.9)]
    F, _ = _eval(cfg, oracle.Scene3(s, t, np.zeros((0, 4))), _row(w))
    assert abs(F[0] - np.linalg.norm(t - s)) < 1e-9


def test_hand_worked_path():
    cfg = _cfg(1, alpha=30.0, beta=4)
    sc = oracle.Scene3((0.0, 0.0, 0.0), (10.0, 10.0, 0.0), [(5.0, 0.0, 3.0, 4.0), (10.0, 5.0, 2.0, 1.5)])
    # segment 1 (0,0,0)-(10,0,0): sphere 1 at distance 3 < 4 (hit), sphere 2 at
    # (0, 5, 2) from (10,0,0): sqrt(29) (miss); segment 2 (10,0,0)-(10,10,0):
    # sphere 1 at distance sqrt(25 + 9) (miss), sphere 2 at distance 2 (miss, r = 1.5)
    F, Q = _eval(cfg, sc, _row([(10.0, 0.0, 0.0)]))
    assert Q[0] == 1 and abs(F[0] - (20.0 + 30.0)) < 1e-12
    sc = oracle.Scene3((0.0, 0.0, 0.0), (10.0, 10.0, 0.0), [(5.0, 0.0, 3.0, 4.0), (10.0, 5.0, 2.0, 2.5)])
    F, Q = _eval(cfg, sc, _row([(10.0, 0.0, 0.0)]))
    assert Q[0] == 2 and abs(F[0] - (20.0 + 30.0 * 16.0)) < 1e-12


def test_flat_scene_reduces_to_the_circle_objective():
    """Every z = 0: the 3D objective equals the (pinned) 2D circle objective."""
    from paper_2308_10169_gb300.inputs import SepsoConfig
    rng = np.random.default_rng(5)
    T, n = 8, 64
    circles = np.column_stack([rng.uniform(60, 340, (24, 2)), rng.uniform(10, 30, 24)])
    s2, t2 = (20.0, 20.0), (380.0, 380.0)
    X2 = rng.uniform(0, 400, (n, 2 * T))
    cfg2 = SepsoConfig(T=T, G=1, N=n, alpha=30.0, beta=4)
    F2, Q2, L2 = oracle.evaluate(cfg2, oracle.Scene(s2, t2, circles), X2)
    X3 = np.concatenate([X2, np.zeros((n, T))], axis=1)
    sph = np.column_stack([circles[:, :2], np.zeros(24), circles[:, 2]])
    F3, Q3 = _eval(_cfg(T, N=n), oracle.Scene3((*s2, 0.0), (*t2, 0.0), sph), X3)
    assert np.array_equal(Q3, Q2) and Q2.sum() > 20
    np.testing.assert_allclose(F3, F2, rtol=1e-12)


def test_invariant_under_axis_permutation():
    cfg, sc, _ = sphere_workload(0, T=6)
    X = random_paths3(2, 256, 6).astype(np.float64)
    base = oracle.Scene3(sc["start"], sc["target"], sc["spheres"])
    F, Q = _eval(cfg.with_(N=256, G=1), base, X)
    m = oracle.sphere_margin(cfg, base, X)
    keep = m > 1e-6
    T = 6
    for perm in ((1, 2, 0), (2, 0, 1), (0, 2, 1)):
        Xp = np.concatenate([X[:, a * T:(a + 1) * T] for a in perm], axis=1)
        sp = sc["spheres"].astype(np.float64)[:, list(perm) + [3]]
        scp = oracle.Scene3(sc["start"][list(perm)], sc["target"][list(perm)], sp)
        Fp, Qp = _eval(cfg.with_(N=256, G=1), scp, Xp)
        assert np.array_equal(Qp[keep], Q[keep]) and Q.sum() > 50
        np.testing.assert_allclose(Fp, F, rtol=1e-12)


def test_run_stays_in_the_box_and_reaches_the_straight_line():
    """Per-axis ranges (W, H, Z all different) at init and after clipping; no
    obstacles: the best cost approaches |target - start|."""
    cfg = BFConfig(fn=SPHERE_PATH, D=3 * 4, G=4, N=32, map_w=400.0, map_h=300.0, map_d=200.0, alpha=30.0,
                   beta=4, max_iters=300, seed=3)
    start, target = np.array([10.0, 20.0, 30.0]), np.array([390.0, 280.0, 170.0])
    sc = oracle.Scene3(start, target, np.zeros((0, 4)))
    sw = oracle.BFSwarm(cfg, TABLE_HYPER8_PATH[:4], sc)
    sw.init()
    T, box = 4, (400.0, 300.0, 200.0)
    X = sw.s["X"].reshape(-1, 3 * T)
    V = sw.s["V"].reshape(-1, 3 * T)
    vlim = np.repeat(TABLE_HYPER8_PATH[:4, 5], 32)[:, None]
    for a in range(3):
        xa, va = X[:, a * T:(a + 1) * T], V[:, a * T:(a + 1) * T]
        assert xa.min() >= 0.0 and xa.max() <= box[a] and xa.max() > 0.9 * box[a]
        assert np.all(np.abs(va) <= vlim * box[a] + 1e-9)
    for _ in range(300):
        sw.iteration()
    X = sw.s["X"].reshape(-1, 3 * T)
    for a in range(3):
        assert X[:, a * T:(a + 1) * T].min() >= 0.0 and X[:, a * T:(a + 1) * T].max() <= box[a]
    best = sw.s["Tfit"][0]
    assert best <= np.linalg.norm(target - start) * 1.005


def test_priori_initialization_in_3d():
    cfg, sc, hyper = sphere_workload(1, T=5, N=20)
    cfg = cfg.with_(G=2)
    scene = oracle.Scene3(sc["start"], sc["target"], sc["spheres"])
    sw = oracle.BFSwarm(cfg, hyper[:2], scene)
    prev = np.linspace(30.0, 370.0, 15)
    sw.set_previous(prev, cycle=4)
    sw.init()
    X = sw.s["X"].reshape(2, 20, 15)
    n_pi = math.ceil(float(np.float32(0.25)) * 20)
    assert n_pi == 5
    near = np.all(np.abs(X - prev[None, None]) <= 20.0 + 1e-9, axis=2)
    assert near[:, :n_pi].all() and not near[:, n_pi:].any()


def test_auto_truncation_stops_at_the_first_collision_free_tbest():
    """With a stall limit of 1 and an unreachable improvement tolerance, Auto
    Truncation (Sec. 3.3.4, stall reading) fires at the first iteration after the
    first (whose Tbest always improves on none) in which Tbest collides with nothing:
    the iteration found by stepping without AT and reading Q(Tbest) after each
    iteration.  The planned state is that iteration's: its bests, and the positions it
    evaluated (no particle moved after it)."""
    stopped = 0
    for seed in range(4):
        cfg, sc, hy = sphere_workload(seed, T=6, N=12, S=48, iters=40)
        cfg = cfg.with_(G=3, at_stall=1, stall_tol=1e30)
        scene = oracle.Scene3(sc["start"], sc["target"], sc["spheres"])
        ref = oracle.BFSwarm(cfg.with_(at_stall=0), hy[:3], scene)
        ref.init()
        want, X_eval, Tb = cfg.max_iters, None, None
        for k in range(1, cfg.max_iters + 1):
            Xk = ref.s["X"].copy()
            ref.iteration()
            if k >= 2 and ref.s["TQ"][0] == 0:
                want, X_eval, Tb = k, Xk, ref.s["Tb"].copy()
                break
        res = oracle.BFSwarm(cfg, hy[:3], scene).plan()
        assert res["iters"] == want
        if X_eval is not None:
            stopped += 1
            sw = oracle.BFSwarm(cfg, hy[:3], scene)
            res = sw.plan()
            assert res["Q"] == 0
            np.testing.assert_array_equal(sw.s["X"], X_eval)
            np.testing.assert_array_equal(sw.s["Tb"], Tb)
    assert stopped >= 2


def test_auto_truncation_needs_a_collision_free_tbest():
    """A scene whose target sits inside a sphere: every path collides, so the stall
    counter alone never stops a run and it reaches the cap."""
    cfg, sc, hy = sphere_workload(0, T=4, N=10, S=8, iters=25)
    cfg = cfg.with_(G=2, at_stall=2, stall_tol=1e30)
    sph = sc["spheres"].copy()
    sph[0] = (380.0, 380.0, 380.0, 15.0)
    res = oracle.BFSwarm(cfg, hy[:2], oracle.Scene3(sc["start"], sc["target"], sph)).plan()
    assert res["iters"] == cfg.max_iters and res["Q"] > 0
