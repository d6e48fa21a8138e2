"""Batched planning of uneven scenes (sepso_batch_*) vs the FP64 oracle, through the C ABI.

Each scene of a batch is an independent run of Algorithm 1 (no PI, no AT), so the
oracle's single-scene plan with the same seed and run id is its reference.
Tolerances as in test_gpu_parity: cost 1e-4 relative, Q exact, waypoints 1e-5
relative with a floor of 1e-5 x the map extent, for the first iterations (FP32 and
FP64 trajectories separate later); medians over many scenes within 1% for full runs.
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300 import BatchPlanner
from paper_2308_10169_gb300.inputs import BatchSceneSpec, batch_workload, random_circles, sample_hyper

pytestmark = pytest.mark.gpu


def _small_batch(iters, seed=0):
    rng = np.random.default_rng(100 + seed)
    shapes = [(1, 1, 1, 0), (3, 2, 5, 4), (8, 3, 17, 20), (20, 2, 33, 64), (5, 1, 9, 1),
              (12, 4, 40, 7), (64, 1, 3, 30), (2, 8, 11, 13), (31, 2, 9, 100), (8, 8, 32, 16)]
    specs, hyper, circles = [], [], []
    for i, (T, G, N, O) in enumerate(shapes):
        specs.append(BatchSceneSpec(T=T, G=G, N=N, O=O, max_iters=iters, alpha=30.0, beta=4,
                                    seed=7 + seed, run_id=i))
        h = sample_hyper(50 + i, G)
        h[:, 2] = (i % 2) * 0.7          # C3 on for odd scenes
        h[:, 4] = h[:, 3] * 0.5          # a decreasing inertia
        hyper.append(h)
        circles.append(random_circles(rng, O, lo=20, hi=380, r_lo=5, r_hi=30))
    points = np.tile(np.array([[20, 20, 380, 380]], np.float32), (len(specs), 1))
    return specs, hyper, points, circles


def _oracle(spec, hyper, pts, circ):
    return oracle.Swarm(spec.config(), hyper).plan(oracle.Scene(pts[:2], pts[2:], circ))


@pytest.mark.parametrize("iters", [1, 2, 3])
def test_batch_first_iterations_match_oracle(native, iters):
    specs, hyper, points, circles = _small_batch(iters)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    res = bp.run(use_graph=False)
    for s, r in enumerate(res):
        o = _oracle(specs[s], hyper[s], points[s], circles[s])
        assert r["iters"] == o["iters"] == iters
        assert r["Q"] == o["Q"], s
        assert r["cost"] == pytest.approx(o["cost"], rel=1e-4), s
        np.testing.assert_allclose(r["waypoints"], o["waypoints"], rtol=1e-5, atol=4e-3)


def test_batch_graph_and_shapes_do_not_change_results(native):
    specs, hyper, points, circles = _small_batch(12, seed=1)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    ref = bp.run(use_graph=False)
    again = bp.run(use_graph=True)
    bp.set_shape(tile=8, threads=128)
    other = bp.run(use_graph=True)
    for a, b, c in zip(ref, again, other):
        assert a["cost"] == b["cost"] == c["cost"]
        np.testing.assert_array_equal(a["waypoints"], b["waypoints"])
        np.testing.assert_array_equal(a["waypoints"], c["waypoints"])


def test_scene_alone_equals_scene_in_the_mix(native):
    specs, hyper, points, circles = _small_batch(15, seed=2)
    mix = BatchPlanner(specs)
    mix.set_inputs(hyper, points, circles)
    mix.autotune(trial_launches=3)
    rm = mix.run()
    for s in (0, 3, 6, 9):
        alone = BatchPlanner([specs[s]])
        alone.set_inputs([hyper[s]], points[s:s + 1], [circles[s]])
        ra = alone.run()[0]
        assert ra["cost"] == rm[s]["cost"] and ra["Q"] == rm[s]["Q"]
        np.testing.assert_array_equal(ra["waypoints"], rm[s]["waypoints"])


def test_batch_median_cost_matches_oracle(native):
    specs, hyper, points, circles = batch_workload(seed=3, n=48, T_range=(4, 10), O_range=(4, 24),
                                                   N_range=(8, 24), G=4, max_iters=60)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    res = bp.run()
    gpu = [r["cost"] for r in res]
    ora = [_oracle(specs[s], hyper[s], points[s], circles[s])["cost"] for s in range(len(specs))]
    assert abs(np.median(gpu) - np.median(ora)) <= 0.01 * np.median(ora), (np.median(gpu), np.median(ora))


def test_full_size_batch_shapes_sampled_against_oracle(native):
    # Shapes of the batched workload (T up to 64, O up to 1024, N up to 512 per group),
    # two iterations, sampled scenes checked one by one.
    specs, hyper, points, circles = batch_workload(seed=4, n=96, max_iters=2)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    res = bp.run()
    cost = [sp.N * sp.G * (sp.T + 1) * sp.O for sp in specs]
    pick = {int(np.argmax(cost)), int(np.argmin(cost)), 17}
    for s in sorted(pick):
        o = _oracle(specs[s], hyper[s], points[s], circles[s])
        r = res[s]
        assert r["Q"] == o["Q"]
        assert r["cost"] == pytest.approx(o["cost"], rel=1e-4)
        np.testing.assert_allclose(r["waypoints"], o["waypoints"], rtol=1e-5, atol=4e-3)
    # every result is the fitness of its own waypoints
    for s in range(0, len(specs), 7):
        F, Q, L = oracle.evaluate(specs[s].config(), oracle.Scene(points[s, :2], points[s, 2:], circles[s]),
                                  res[s]["waypoints"])
        assert res[s]["Q"] == Q[0]
        assert res[s]["cost"] == pytest.approx(F[0], rel=1e-4)
