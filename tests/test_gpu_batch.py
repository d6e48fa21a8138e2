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


def _warm_batch(iters, seed=3, stall=0, tol=0.0):
    """The small batch with warm starts: PI for scenes with a previous path, and a
    learned-prior seed, half of the proposals close to the previous path."""
    specs, hyper, points, circles = _small_batch(iters, seed=seed)
    rng = np.random.default_rng(900 + seed)
    n = len(specs)
    for i, sp in enumerate(specs):
        sp.n_pi = (sp.N + 3) // 4
        sp.n_prior = [0, 1, (sp.N + 2) // 3][i % 3]
        sp.cycle = 3 + i
        sp.pi_halfwidth = 15.0
        sp.stall_iters = stall
        sp.stall_tol = tol
    Dmax = max(sp.D for sp in specs)
    prev = np.zeros((n, Dmax), np.float32)
    prior = np.zeros((n, Dmax), np.float32)
    for i, sp in enumerate(specs):
        T = sp.T
        line = np.concatenate([np.linspace(20, 380, T + 2)[1:-1], np.linspace(20, 380, T + 2)[1:-1]])
        prev[i, :sp.D] = np.clip(line + rng.normal(0, 40, sp.D), 0, 400)
        prior[i, :sp.D] = np.clip((prev[i, :sp.D] if i % 2 else line) + rng.normal(0, 10, sp.D), 0, 400)
    has_prev = np.array([0 if i % 4 == 1 else 1 for i in range(n)], np.int32)
    return specs, hyper, points, circles, prev, prior, has_prev


def _oracle_gate(sp, pts, circ, prev_row, prior_row, hp):
    """(use the proposal, ambiguous): fitness of the proposal below the previous path's."""
    if sp.n_prior == 0:
        return False, False
    if not (hp and sp.n_pi > 0):
        return True, False
    sc = oracle.Scene(pts[:2], pts[2:], circ)
    f, _, _ = oracle.evaluate(sp.config(), sc, np.stack([prior_row[:sp.D], prev_row[:sp.D]]))
    return bool(f[0] < f[1]), abs(f[0] - f[1]) <= 1e-3 * max(abs(f[1]), 1.0)


def _oracle_warm(sp, hyper, pts, circ, prev_row, prior_row, hp, use):
    sw = oracle.Swarm(sp.config(), hyper)
    st = {"has_prev": [hp], "prevT": prev_row[:sp.D], "cycle": [sp.cycle]}
    if use:
        st.update({"n_prior": [sp.n_prior], "priorT": prior_row[:sp.D]})
    sw.load(st)
    return sw.plan(oracle.Scene(pts[:2], pts[2:], circ))


@pytest.mark.parametrize("iters", [1, 2])
def test_batch_warm_starts_match_oracle(native, iters):
    import torch
    specs, hyper, points, circles, prev, prior, has_prev = _warm_batch(iters)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    bp.set_starts(prev=torch.from_numpy(prev).cuda(), prior=torch.from_numpy(prior).cuda(), has_prev=has_prev)
    res = bp.run(use_graph=False)
    n_use = 0
    for s, r in enumerate(res):
        use, ambiguous = _oracle_gate(specs[s], points[s], circles[s], prev[s], prior[s], has_prev[s])
        n_use += use
        if ambiguous:
            continue
        o = _oracle_warm(specs[s], hyper[s], points[s], circles[s], prev[s], prior[s], has_prev[s], use)
        assert r["iters"] == o["iters"] == iters
        assert r["Q"] == o["Q"], s
        assert r["cost"] == pytest.approx(o["cost"], rel=1e-4), s
        np.testing.assert_allclose(r["waypoints"], o["waypoints"], rtol=1e-5, atol=4e-3)
    assert bp.prior_used() == n_use
    assert 0 < n_use < len(specs)


def test_batch_stores_results_as_next_pi_centres(native):
    # set_starts without prev keeps the stored paths: each scene's last result
    import torch
    specs, hyper, points, circles, prev, prior, has_prev = _warm_batch(4, seed=4)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    bp.set_starts(prev=torch.from_numpy(prev).cuda(), has_prev=has_prev)
    first = bp.run(use_graph=True)
    bp.set_starts(has_prev=np.ones(len(specs), np.int32))
    second = bp.run(use_graph=True)
    for s, sp in enumerate(specs):
        o = _oracle_warm(sp, hyper[s], points[s], circles[s], first[s]["waypoints"], prior[s], 1, False)
        assert second[s]["Q"] == o["Q"], s
        assert second[s]["cost"] == pytest.approx(o["cost"], rel=1e-3), s


def test_batch_stall_truncation(native):
    # Auto Truncation by stall counter in the batch (Sec. 3.3.4): scenes stop early
    # once their best path is collision-free and stalls, and truncation does not
    # change the trajectory (the same scene run for exactly that many iterations
    # without AT gives the same result); median cost over 48 scenes within 2% of the
    # oracle's (FP32 and FP64 trajectories separate over many iterations).
    import torch
    rng = np.random.default_rng(77)
    n = 48
    specs, hyper, circles = [], [], []
    for i in range(n):
        specs.append(BatchSceneSpec(T=8, G=3, N=12, O=6, max_iters=150, alpha=30.0, beta=4, seed=5, run_id=i,
                                    stall_iters=10, stall_tol=1.0, n_pi=3, pi_halfwidth=20.0, cycle=1))
        hyper.append(sample_hyper(300 + i, 3))
        circles.append(random_circles(rng, 6, lo=20, hi=380, r_lo=5, r_hi=25))
    points = np.tile(np.array([[20, 20, 380, 380]], np.float32), (n, 1))
    prev = np.clip(np.linspace(40, 360, 16)[None, :] + rng.normal(0, 30, (n, 16)), 0, 400).astype(np.float32)
    prev[:, 8:] = prev[:, :8]
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    bp.set_starts(prev=torch.from_numpy(prev).cuda())
    res = bp.run()
    its = np.array([r["iters"] for r in res])
    assert np.median(its) < 150
    for r in res:
        if r["iters"] < 150:
            assert r["Q"] == 0
    # truncation keeps the trajectory
    for s in (0, 5, 11):
        k = int(its[s])
        sp = BatchSceneSpec(**{**specs[s].__dict__, "stall_iters": 0, "max_iters": k})
        one = BatchPlanner([sp])
        one.set_inputs([hyper[s]], points[s:s + 1], [circles[s]])
        one.set_starts(prev=torch.from_numpy(prev[s:s + 1]).cuda())
        r1 = one.run()[0]
        assert r1["cost"] == res[s]["cost"] and r1["iters"] == k
        np.testing.assert_array_equal(r1["waypoints"], res[s]["waypoints"])
    ora = []
    for s, sp in enumerate(specs):
        sw = oracle.Swarm(sp.config(), hyper[s])
        sw.load({"has_prev": [1], "prevT": prev[s], "cycle": [1]})
        ora.append(sw.plan(oracle.Scene(points[s, :2], points[s, 2:], circles[s]))["cost"])
    gpu = [r["cost"] for r in res]
    assert abs(np.median(gpu) - np.median(ora)) <= 0.02 * np.median(ora)
