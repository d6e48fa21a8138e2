"""Polygon scenes in the batched planner (sepso_batch_scene.obstacle_kind = 1: the
scene's obstacles are polygon edges, Q counts proper crossings of path segments and
edges, Sec. 3.3.1) beside circle scenes in one batch, vs the FP64 oracle through the
C ABI.

Tolerances as in test_gpu_batch: cost 1e-4 relative, Q exact, waypoints 1e-5
relative with a floor of 1e-5 x the map, for the first iterations, on the scenes whose
evaluated positions stay clear of flipping decisions (crossing decisions more than
1e-6 of the product of the lengths from a flip; circle pairs more than 1e-3 from
tangency).
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300 import BatchPlanner
from paper_2308_10169_gb300.inputs import BatchSceneSpec, box, polygon_edges, random_circles, sample_hyper

pytestmark = pytest.mark.gpu


def _mixed_batch(iters, seed=0):
    rng = np.random.default_rng(300 + seed)
    # (T, G, N, obstacles, polygon?)
    shapes = [(8, 2, 17, 6, True), (3, 3, 9, 10, False), (20, 2, 33, 3, True), (1, 1, 5, 1, True),
              (12, 4, 40, 12, True), (5, 2, 11, 30, False), (31, 1, 21, 8, True), (8, 8, 32, 0, True)]
    specs, hyper, obst = [], [], []
    for i, (T, G, N, k, poly) in enumerate(shapes):
        if poly:
            boxes = [box(*rng.uniform(60, 340, 2), *rng.uniform(10, 30, 2)) for _ in range(k)]
            o = polygon_edges(boxes) if boxes else np.zeros((0, 4), np.float32)
        else:
            o = random_circles(rng, k, lo=20, hi=380, r_lo=5, r_hi=30)
        specs.append(BatchSceneSpec(T=T, G=G, N=N, O=len(o), max_iters=iters, alpha=30.0, beta=4,
                                    seed=11 + seed, run_id=i, obstacle_kind=1 if poly else 0))
        h = sample_hyper(70 + i, G)
        h[:, 2] = (i % 2) * 0.7
        hyper.append(h)
        obst.append(o)
    points = np.tile(np.array([[20, 20, 380, 380]], np.float32), (len(specs), 1))
    return specs, hyper, points, obst


def _scene(spec, pts, o):
    if spec.obstacle_kind:
        return oracle.Scene(pts[:2], pts[2:], np.zeros((0, 3)), o)
    return oracle.Scene(pts[:2], pts[2:], o)


def _clear(spec, sc, X):
    cfg = spec.config()
    X = np.asarray(X, np.float64).reshape(-1, spec.D)
    if spec.obstacle_kind:
        return np.all(oracle.poly_margin(cfg, sc, X) > 1e-6)
    return np.all(oracle.tangency_margin(cfg, sc, X) > 1e-3)


def _oracle_plan(spec, hyper, sc):
    """The oracle's planning cycle, or None when an evaluated position came within
    the margin of a flipping decision."""
    sw = oracle.Swarm(spec.config(), hyper)
    sw.init()
    while True:
        if not _clear(spec, sc, sw.s["X"]):
            return None
        if sw.iteration(sc, check_stop=True):
            break
    return {"cost": float(sw.s["Tfit"][0]), "Q": int(sw.s["TQ"][0]), "iters": int(sw.s["k"][0]),
            "waypoints": sw.s["Tb"].copy()}


@pytest.mark.parametrize("iters", [1, 2, 3])
def test_mixed_batch_first_iterations_match_oracle(native, iters):
    specs, hyper, points, obst = _mixed_batch(iters)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, obst)
    res = bp.run(use_graph=False)
    checked = polys = 0
    for s, r in enumerate(res):
        o = _oracle_plan(specs[s], hyper[s], _scene(specs[s], points[s], obst[s]))
        if o is None:
            continue
        checked += 1
        polys += specs[s].obstacle_kind
        assert r["iters"] == o["iters"] == iters
        assert r["Q"] == o["Q"], s
        assert r["cost"] == pytest.approx(o["cost"], rel=1e-4), s
        np.testing.assert_allclose(r["waypoints"], o["waypoints"], rtol=1e-5, atol=4e-3)
    assert checked >= 6 and polys >= 4


def test_polygon_scene_alone_equals_scene_in_the_mix(native):
    specs, hyper, points, obst = _mixed_batch(15, seed=1)
    mix = BatchPlanner(specs)
    mix.set_inputs(hyper, points, obst)
    mix.autotune(trial_launches=3)
    rm = mix.run()
    for s in (0, 2, 4, 6):
        assert specs[s].obstacle_kind == 1
        alone = BatchPlanner([specs[s]])
        alone.set_inputs([hyper[s]], points[s:s + 1], [obst[s]])
        ra = alone.run()[0]
        assert ra["cost"] == rm[s]["cost"] and ra["Q"] == rm[s]["Q"]
        np.testing.assert_array_equal(ra["waypoints"], rm[s]["waypoints"])


def test_polygon_scene_rejects_bad_kind_and_edges(native):
    specs, hyper, points, obst = _mixed_batch(2, seed=2)
    bad = [BatchSceneSpec(**{**specs[0].__dict__, "obstacle_kind": 2})]
    with pytest.raises(RuntimeError, match="obstacle_kind"):
        BatchPlanner(bad)
    bp = BatchPlanner(specs[:1])
    e = obst[0].copy()
    e[0, 0] = np.nan
    with pytest.raises(RuntimeError, match="edge"):
        bp.set_inputs(hyper[:1], points[:1], [e])
