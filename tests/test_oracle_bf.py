"""The oracle's benchmark functions (Table BFs) and DTPSO on them, pinned without a GPU.

BF1-BF4 have no formulas in the paper; their textbook definitions are pinned by hand
values, by the minimum 0 that Table BFs lists, and (Rosenbrock) by the library
routine ``scipy.optimize.rosen``.  The DTPSO iteration is the path planner's (pinned
in test_oracle_mechanisms.py); what is new here -- the box [lo, hi]^D with lo < 0,
an objective without collisions, odd D -- is pinned by the initial ranges, a step
with pure inertia (w = 1, C = 0) that must clip at both ends of the box, and the
invariants of the bests.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300.inputs import (BF_GRIEWANK, BF_NAMES, BF_RASTRIGIN, BF_ROSENBROCK,
                                           BF_SPHERE, TABLE_HYPER8, BFConfig, bf_large,
                                           bf_standard)


def test_hand_values():
    assert oracle.bf_value(BF_SPHERE, [1, 2, 3]) == 14.0
    assert oracle.bf_value(BF_ROSENBROCK, [0, 0]) == 1.0
    assert oracle.bf_value(BF_ROSENBROCK, [1, 2]) == 100.0          # 100 (2 - 1)^2
    assert oracle.bf_value(BF_ROSENBROCK, [-1, 1, 0]) == 104.0      # (4) + (100)
    assert oracle.bf_value(BF_ROSENBROCK, [5.0]) == 0.0             # no pair of coordinates
    assert oracle.bf_value(BF_RASTRIGIN, [0.5] * 7) == pytest.approx(20.25 * 7, rel=1e-14)
    assert oracle.bf_value(BF_RASTRIGIN, [1, -2, 3]) == pytest.approx(14.0, abs=1e-12)
    # Griewank's index starts at 1: cos(x_1 / 1), cos(x_2 / sqrt 2)
    assert oracle.bf_value(BF_GRIEWANK, [math.pi, 0]) == pytest.approx(2 + math.pi ** 2 / 4000, rel=1e-14)
    x2 = 2 * math.pi * math.sqrt(2)
    assert oracle.bf_value(BF_GRIEWANK, [0, x2]) == pytest.approx(x2 ** 2 / 4000, rel=1e-12)


@pytest.mark.parametrize("fn", list(BF_NAMES))
def test_minimum_is_zero(fn):
    # Table BFs: minimum 0, at the origin (Rosenbrock: at x = 1)
    for D in (1, 2, 30, 1000):
        opt = np.ones(D) if fn == BF_ROSENBROCK else np.zeros(D)
        assert oracle.bf_value(fn, opt) == pytest.approx(0.0, abs=1e-12)
        rng = np.random.default_rng(D)
        x = opt + rng.uniform(-1, 1, D)
        if not (fn == BF_ROSENBROCK and D == 1):
            assert oracle.bf_value(fn, x) > 0


def test_rosenbrock_matches_library_routine():
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(5)
    for D in (2, 3, 30, 1000):
        x = rng.uniform(-600, 600, D)
        assert oracle.bf_value(BF_ROSENBROCK, x) == pytest.approx(scipy_opt.rosen(x), rel=1e-13)


def test_sphere_and_rastrigin_closed_forms_on_random_points():
    rng = np.random.default_rng(6)
    x = rng.uniform(-600, 600, 30)
    assert oracle.bf_value(BF_SPHERE, x) == pytest.approx(float(np.sum(x * x)), rel=1e-14)
    k = rng.integers(-600, 601, 30).astype(np.float64)       # cos(2 pi k) = 1
    assert oracle.bf_value(BF_RASTRIGIN, k) == pytest.approx(float(np.sum(k * k)), rel=1e-12)


def _swarm(fn=BF_SPHERE, D=7, G=2, N=5, lo=-600.0, hi=600.0, hyper=None, iters=100):
    cfg = BFConfig(fn=fn, D=D, G=G, N=N, lo=lo, hi=hi, max_iters=iters, seed=3)
    hy = TABLE_HYPER8[:G] if hyper is None else hyper
    return cfg, oracle.BFSwarm(cfg, hy)


def test_initial_swarm_fills_the_box():
    cfg, sw = _swarm(D=31, G=4, N=50, lo=-600.0, hi=200.0)
    sw.init()
    X = sw.s["X"].reshape(-1, cfg.D)
    V = sw.s["V"].reshape(cfg.G, cfg.N, cfg.D)
    assert X.min() >= -600.0 and X.max() <= 200.0
    assert X.min() < -590.0 and X.max() > 190.0
    assert abs(X.mean() - (-200.0)) < 10.0
    for g in range(cfg.G):
        vmax = TABLE_HYPER8[g, 5] * 800.0                    # V_limit x X_range
        assert np.abs(V[g]).max() <= vmax + 1e-9
        assert np.abs(V[g]).max() > 0.9 * vmax
    np.testing.assert_array_equal(sw.s["P"], sw.s["X"])
    assert np.all(np.isinf(sw.s["Pfit"]))


def test_pure_inertia_step_clips_at_both_ends():
    # w = 1, C1 = C2 = C3 = 0: V is kept (clipped to +-Vmax) and X' = clip(X + V, lo, hi)
    hy = np.array([[0, 0, 0, 1, 1, 0.5], [0, 0, 0, 1, 1, 0.3]], np.float32)
    cfg, sw = _swarm(D=5, hyper=hy, lo=-600.0, hi=600.0)
    sw.init()
    X0, V0 = sw.s["X"].copy(), sw.s["V"].copy()
    sw.step(None, 1)
    want = np.clip(X0 + V0, -600.0, 600.0)
    np.testing.assert_array_equal(sw.s["X"], want)
    np.testing.assert_array_equal(sw.s["V"], V0)
    assert np.any(want == -600.0) and np.any(want == 600.0)
    # the fitness of the first iteration is that of the initial positions
    F0 = sw.evaluate(X0)
    assert sw.s["Tfit"][0] == F0.min()
    np.testing.assert_array_equal(sw.s["Pfit"], F0)


@pytest.mark.parametrize("fn", list(BF_NAMES))
def test_run_invariants(fn):
    cfg, sw = _swarm(fn=fn, D=9, G=3, N=6, iters=60)
    hist = sw.run(60)
    assert np.all(np.diff(hist) <= 0)                         # Tbest never gets worse
    s = sw.s
    D = cfg.D
    assert s["k"][0] == 60
    assert s["Tfit"][0] == pytest.approx(oracle.bf_value(fn, s["Tb"]), rel=1e-12)
    for g in range(cfg.G):
        assert s["Gfit"][g] >= s["Tfit"][0]
        assert s["Gfit"][g] == pytest.approx(oracle.bf_value(fn, s["Gb"][g * D:(g + 1) * D]), rel=1e-12)
    P = s["P"].reshape(-1, D)
    np.testing.assert_allclose(s["Pfit"], sw.evaluate(P), rtol=1e-12)
    assert s["Tfit"][0] == s["Gfit"].min() == s["Pfit"].min()
    X = s["X"].reshape(-1, D)
    assert X.min() >= cfg.lo and X.max() <= cfg.hi


def test_standard_runs_improve():
    # 1400 iterations of the standard run reduce every function by orders of magnitude
    for fn in BF_NAMES:
        cfg, hy = bf_standard(fn, trials=1)
        hist = oracle.BFSwarm(cfg, hy).run(200)
        assert hist[-1] < 0.05 * hist[0]


def test_workload_shapes():
    cfg, hy = bf_standard(BF_RASTRIGIN)
    assert (cfg.D, cfg.G, cfg.N, cfg.max_iters, cfg.runs) == (30, 8, 10, 1400, 50)
    assert (cfg.lo, cfg.hi) == (-600.0, 600.0)
    np.testing.assert_array_equal(hy, TABLE_HYPER8)
    cfg, _ = bf_large(BF_GRIEWANK)
    assert cfg.G * cfg.N == 16384 and cfg.D == 1000
