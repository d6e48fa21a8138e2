"""Benchmark-function DTPSO (Table BFs) on the GPU vs the FP64 oracle, through the C ABI.

Tolerances (FP32 kernel vs FP64 oracle):
  * fitness of a row: 2e-6 x the sum of the magnitudes of its terms (the FP32
    rounding of about D additions, and of the cosines' arguments);
  * positions after identical state and one update: 1e-5 relative with a floor of
    1e-5 x the box width; velocities likewise with a floor of 1e-5 x V_range;
  * first iterations of a run: the same, and the same Pbest decisions;
  * whole runs: the trajectories separate after some tens of iterations, so the
    medians of log10(final fitness) over trials agree within 1 (a factor of 10;
    the oracle's own trials spread over two orders of magnitude).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_10169_gb300 import BFPlanner
from paper_2308_10169_gb300.inputs import (BF_GRIEWANK, BF_NAMES, BF_RASTRIGIN, BF_ROSENBROCK,
                                           BF_SPHERE, TABLE_HYPER8, BFConfig, bf_large, bf_standard)
from paper_2308_10169_gb300.planner import bf_evaluate

pytestmark = pytest.mark.gpu


def _scale(fn, X):
    """Sum of the magnitudes of the terms of BF fn, per row (FP64)."""
    X = np.asarray(X, np.float64)
    if fn == BF_SPHERE:
        return np.sum(X * X, axis=1)
    if fn == BF_ROSENBROCK:
        a = X[:, 1:] - X[:, :-1] ** 2
        return np.sum(100 * a * a + 100 * X[:, :-1] ** 4 + (X[:, :-1] - 1) ** 2, axis=1) + 1.0
    if fn == BF_RASTRIGIN:
        return np.sum(X * X + 10, axis=1) + 10 * X.shape[1]
    return 1 + np.sum(X * X, axis=1) / 4000 + 1 + X.shape[1] * 1e-3


def _planner(cfg, hyper):
    pl = BFPlanner(cfg)
    pl.set_hyper(hyper)
    return pl


@pytest.mark.parametrize("fn", list(BF_NAMES))
@pytest.mark.parametrize("D,n", [(1, 7), (2, 33), (3, 5), (30, 1000), (33, 65), (1000, 300)])
def test_evaluate_matches_oracle(native, fn, D, n):
    rng = np.random.default_rng(D * 10 + fn)
    X = rng.uniform(-600, 600, (n, D)).astype(np.float32)
    X[: n // 4] *= np.float32(1e-3)                     # near the optimum too
    ld = D + 3                                          # a row pitch above D
    Xp = np.zeros((n, ld), np.float32)
    Xp[:, :D] = X
    F = bf_evaluate(fn, torch.from_numpy(Xp).cuda()[:, :D]).cpu().numpy()
    ref = np.array([oracle.bf_value(fn, x) for x in X.astype(np.float64)])
    err = np.abs(F - ref)
    assert np.all(err <= 2e-6 * _scale(fn, X) + 1e-30), (np.max(err / _scale(fn, X)))


def _close(a, b, scale, rtol=1e-5):
    np.testing.assert_allclose(np.asarray(a, np.float64), np.asarray(b, np.float64), rtol=rtol,
                               atol=rtol * scale)


@pytest.mark.parametrize("fn", list(BF_NAMES))
@pytest.mark.parametrize("K", [1, 2, 3])
def test_first_iterations_match_oracle(native, fn, K):
    # K = 1: the initial swarm and its bests; K = 2, 3: one and two updates
    cfg = BFConfig(fn=fn, D=37, G=3, N=11, lo=-600.0, hi=400.0, max_iters=K, seed=7)
    hy = np.array(TABLE_HYPER8[:3])
    hy[1, 2] = 0.0                                      # one group without the Tbest term
    pl = _planner(cfg, hy)
    pl.run_async(use_graph=False)
    s = pl.get_state()
    sw = oracle.BFSwarm(cfg, hy)
    hist = sw.run(K)
    o = sw.state()
    width = cfg.hi - cfg.lo
    assert s["k"][0] == K
    _close(s["X"], o["X"], width)
    _close(s["V"], o["V"], float(hy[:, 5].max()) * width)
    _close(s["P"], o["P"], width)
    np.testing.assert_allclose(s["Pfit"], o["Pfit"], rtol=2e-5)
    np.testing.assert_allclose(s["Gfit"], o["Gfit"], rtol=2e-5)
    _close(s["Gb"], o["Gb"], width)
    assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=2e-5)
    _close(s["Tb"], o["Tb"], width)
    np.testing.assert_allclose(pl.history()[:K], hist, rtol=2e-5)


def _consistent_state(cfg, seed):
    """A random mid-run state whose bests are consistent with its Pbests and whose
    next fitness decisions are far from ties (checked with the oracle)."""
    rng = np.random.default_rng(seed)
    G, N, D = cfg.G, cfg.N, cfg.D
    M = G * N
    sw = oracle.BFSwarm(cfg, TABLE_HYPER8[:G])
    for _ in range(200):
        X = rng.uniform(cfg.lo, cfg.hi, (M, D)).astype(np.float32)
        P = rng.uniform(cfg.lo, cfg.hi, (M, D)).astype(np.float32)
        V = rng.uniform(-50, 50, (M, D)).astype(np.float32)
        Pfit = sw.evaluate(P.astype(np.float64)).astype(np.float32)
        never = rng.random(M) < 0.3
        never[::N] = False                              # every group has a finite best
        Pfit[never] = np.inf                            # not improved yet
        P[never] = X[never]
        gi = np.argmin(Pfit.reshape(G, N), axis=1)
        Gfit = Pfit.reshape(G, N)[np.arange(G), gi]
        Gb = P.reshape(G, N, D)[np.arange(G), gi]
        t = int(np.argmin(Gfit))
        st = {"X": X, "V": V, "P": P, "Pfit": Pfit, "Gb": Gb, "Gfit": Gfit, "Tb": Gb[t].copy(),
              "Tfit": np.array([Gfit[t]], np.float32), "k": np.array([7], np.int32)}
        # decisions of the next iteration, from the oracle's own step
        o = oracle.BFSwarm(cfg, TABLE_HYPER8[:G])
        o.load({k: np.asarray(v, np.float64) if k != "k" else v for k, v in st.items()})
        o.step(None, 1)
        F = o.evaluate(o.s["X"].reshape(M, D))
        fin = np.isfinite(Pfit)
        if np.any(np.abs(F[fin] - Pfit[fin]) <= 1e-4 * np.abs(Pfit[fin])):
            continue
        srt = np.sort(np.minimum(Pfit, F).reshape(G, N), axis=1)
        if np.any(srt[:, 1] - srt[:, 0] <= 1e-4 * np.abs(srt[:, 0])):
            continue
        gs = np.sort(srt[:, 0])
        if gs[1] - gs[0] <= 1e-4 * abs(gs[0]):
            continue
        return st, o.state()
    raise AssertionError("no decisive state")


@pytest.mark.parametrize("fn", list(BF_NAMES))
def test_single_step_from_loaded_state(native, fn):
    cfg = BFConfig(fn=fn, D=21, G=4, N=9, max_iters=50, seed=3)
    st, o = _consistent_state(cfg, 50 + fn)
    pl = _planner(cfg, TABLE_HYPER8[:4])
    pl.set_state(st)
    s0 = pl.get_state()
    np.testing.assert_array_equal(s0["Gfit"], st["Gfit"])
    assert s0["Tfit"][0] == st["Tfit"][0]
    pl.step(1)
    s = pl.get_state()
    width = cfg.hi - cfg.lo
    assert s["k"][0] == o["k"][0] == 8
    _close(s["X"], o["X"], width)
    _close(s["V"], o["V"], float(TABLE_HYPER8[:4, 5].max()) * width)
    _close(s["P"], o["P"], width)
    np.testing.assert_allclose(s["Pfit"], o["Pfit"], rtol=2e-5)
    np.testing.assert_allclose(s["Gfit"], o["Gfit"], rtol=2e-5)
    _close(s["Gb"], o["Gb"], width)
    assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=2e-5)
    _close(s["Tb"], o["Tb"], width)


def test_runs_graph_and_steps_are_consistent(native):
    # run r of a multi-run launch = a one-run launch with run_id r; graph replay =
    # plain launches; run(K) = run(K1) then step(K - K1)
    cfg, hy = bf_standard(BF_RASTRIGIN, seed=5, trials=6)
    cfg = cfg.with_(max_iters=120)
    pl = _planner(cfg, hy)
    pl.run_async(use_graph=True)
    multi = [pl.read(r) for r in range(6)]
    pl.run_async(use_graph=True)                        # replay
    again = [pl.read(r) for r in range(6)]
    for a, b in zip(multi, again):
        np.testing.assert_array_equal(a["x"], b["x"])
    for r in (0, 4):
        one = _planner(cfg.with_(runs=1, run_id=r), hy)
        one.run_async(use_graph=False)
        x = one.read(0)
        np.testing.assert_array_equal(x["x"], multi[r]["x"])
        assert x["fit"] == multi[r]["fit"]
    a = _planner(cfg.with_(runs=1, run_id=4), hy)
    a.run_async(use_graph=False)
    a.step(10)
    b = _planner(cfg.with_(runs=1, run_id=4), hy)
    b.run_async(use_graph=True)
    b.step(4)
    b.step(6)
    ra, rb = a.read(0), b.read(0)
    assert ra["iters"] == rb["iters"] == 130
    np.testing.assert_array_equal(ra["x"], rb["x"])
    np.testing.assert_array_equal(a.get_state()["X"], b.get_state()["X"])


@pytest.mark.parametrize("fn", list(BF_NAMES))
def test_standard_runs_match_oracle_statistically(native, fn):
    cfg, hy = bf_standard(fn, seed=1, trials=16)
    pl = _planner(cfg, hy)
    pl.run_async()
    gpu = np.array([pl.read(r)["fit"] for r in range(16)], np.float64)
    ora = np.array([oracle.BFSwarm(cfg.with_(runs=1, run_id=r), hy).run(1400)[-1] for r in range(16)])
    lg = np.log10(np.median(gpu) + 1e-30)
    lo = np.log10(np.median(ora) + 1e-30)
    assert abs(lg - lo) <= 1.0, (np.median(gpu), np.median(ora))
    for r in range(16):
        h = pl.history(r)
        assert np.all(np.diff(h) <= 0)
        res = pl.read(r)
        assert res["iters"] == 1400 and res["fit"] == h[-1]
        ref = oracle.bf_value(fn, res["x"].astype(np.float64))
        assert abs(ref - res["fit"]) <= 2e-6 * _scale(fn, res["x"][None])[0] + 1e-30
        assert h[-1] < 0.05 * h[0]
        assert res["x"].min() >= cfg.lo and res["x"].max() <= cfg.hi


def test_large_scale_first_iterations_on_sampled_particles(native):
    # the full 16K x 1K configuration, two iterations; sampled particles vs the oracle
    cfg, hy = bf_large(BF_SPHERE, seed=2, iters=2)
    pl = _planner(cfg, hy)
    pl.run_async()
    s = pl.get_state()
    sw = oracle.BFSwarm(cfg, hy)
    sw.run(2)
    o = sw.s
    D = cfg.D
    rows = np.arange(0, cfg.G * cfg.N, 97)
    idx = (rows[:, None] * D + np.arange(D)[None, :]).reshape(-1)
    width = cfg.hi - cfg.lo
    _close(s["X"][idx], o["X"][idx], width)
    _close(s["V"][idx], o["V"][idx], float(hy[:, 5].max()) * width)
    np.testing.assert_allclose(s["Pfit"][rows], o["Pfit"][rows], rtol=2e-5)
    np.testing.assert_allclose(s["Gfit"], o["Gfit"], rtol=2e-5)
    assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=2e-5)
