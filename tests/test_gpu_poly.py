"""Path planning among polygon obstacles (Sec. 3.3.1 map model) on the GPU engine vs
the FP64 oracle, through the C ABI.

Tolerances: crossing counts Q bit-exact for paths whose every (segment, edge)
decision is more than 1e-6 (orientation / product of lengths) from flipping;
fitness 1e-5 relative; positions and velocities after identical state as for the
benchmark functions (1e-5 relative, floors of 1e-5 x the map and x V_range); whole
runs: median final cost over 16 runs within 5% of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_10169_gb300 import BFPlanner
from paper_2308_10169_gb300.inputs import (POLYGON_PATH, TABLE_HYPER8_PATH, BFConfig, polygon_edges,
                                           polygon_workload, random_paths)
from paper_2308_10169_gb300.planner import poly_evaluate

pytestmark = pytest.mark.gpu

MARGIN = 1e-6


def _scene(start, target, edges):
    return oracle.Scene(start, target, np.zeros((0, 3)), edges)


def _close(a, b, scale, rtol=1e-5):
    np.testing.assert_allclose(np.asarray(a, np.float64), np.asarray(b, np.float64), rtol=rtol,
                               atol=rtol * scale)


@pytest.mark.parametrize("T,n", [(8, 2000), (1, 300), (33, 257)])
def test_evaluate_matches_oracle(native, T, n):
    cfg, start, target, polys, edges, hy = polygon_workload(1, T=T)
    X = random_paths(7 + T, n, T).astype(np.float32)
    sc = _scene(start, target, edges)
    sw = oracle.BFSwarm(cfg, hy, sc)
    Fo, Qo = sw.evaluate(X.astype(np.float64), with_q=True)
    keep = oracle.poly_margin(cfg, sc, X.astype(np.float64)) > MARGIN
    assert keep.mean() > 0.9
    F, Q = poly_evaluate(torch.from_numpy(X).cuda(), start, target, torch.from_numpy(edges).cuda(),
                         cfg.alpha, cfg.beta)
    F, Q = F.cpu().numpy(), Q.cpu().numpy()
    np.testing.assert_array_equal(Q[keep], Qo[keep])
    np.testing.assert_allclose(F[keep], Fo[keep], rtol=1e-5)
    assert np.unique(Qo[keep]).size >= 3                      # a spread of crossing counts


def _small(seed):
    cfg, start, target, polys, edges, hy = polygon_workload(seed, N=11, iters=3)
    return cfg.with_(G=3), start, target, edges, np.array(hy[:3])


def _margins_ok(cfg, sc, X):
    return np.all(oracle.poly_margin(cfg, sc, np.asarray(X, np.float64).reshape(-1, cfg.D)) > MARGIN)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_first_iterations_match_oracle(native, K):
    # a seed whose evaluated positions all stay clear of flipping decisions
    for seed in range(40):
        cfg, start, target, edges, hy = _small(seed)
        cfg = cfg.with_(max_iters=K)
        sc = _scene(start, target, edges)
        sw = oracle.BFSwarm(cfg, hy, sc)
        sw.init()
        ok = True
        hist = []
        for _ in range(K):
            if not _margins_ok(cfg, sc, sw.s["X"]):
                ok = False
                break
            sw.iteration()
            hist.append(sw.s["Tfit"][0])
        if ok:
            break
    assert ok
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_polygons(start, target, edges)
    pl.run_async(use_graph=False)
    s = pl.get_state()
    o = sw.state()
    vscale = float(hy[:, 5].max()) * 400.0
    _close(s["X"], o["X"], 400.0)
    _close(s["V"], o["V"], vscale)
    _close(s["P"], o["P"], 400.0)
    np.testing.assert_allclose(s["Pfit"], o["Pfit"], rtol=1e-5)
    np.testing.assert_allclose(s["Gfit"], o["Gfit"], rtol=1e-5)
    assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=1e-5)
    _close(s["Tb"], o["Tb"], 400.0)
    np.testing.assert_allclose(pl.history()[:K], hist, rtol=1e-5)


def test_runs_match_oracle_statistically(native):
    cfg, start, target, polys, edges, hy = polygon_workload(2, N=40, iters=100, runs=16)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_polygons(start, target, edges)
    pl.run_async()
    gpu = np.array([pl.read(r)["fit"] for r in range(16)], np.float64)
    sc = _scene(start, target, edges)
    ora = []
    for r in range(16):
        sw = oracle.BFSwarm(cfg.with_(runs=1, run_id=r), hy, sc)
        h = sw.run(100)
        ora.append(h[-1])
        g = pl.history(r)
        assert np.all(np.diff(g) <= 0)
        x = pl.read(r)["x"]
        assert x.min() >= 0.0 and x.max() <= 400.0
    assert abs(np.median(gpu) - np.median(ora)) <= 0.05 * np.median(ora), (np.median(gpu), np.median(ora))


def test_new_polygons_recapture_the_graph(native):
    cfg, start, target, polys, edges, hy = polygon_workload(3, N=20, iters=30, runs=2)
    cfg = cfg.with_(max_edges=200)
    other = polygon_edges(polys[:5])
    a = BFPlanner(cfg)
    a.set_hyper(hy)
    a.set_polygons(start, target, edges)
    a.run_async()
    a.set_polygons(start, target, other)
    a.run_async()
    b = BFPlanner(cfg)
    b.set_hyper(hy)
    b.set_polygons(start, target, other)
    b.run_async(use_graph=False)
    for r in range(2):
        np.testing.assert_array_equal(a.read(r)["x"], b.read(r)["x"])


def test_lane_per_particle_kernel_matches_oracle(native):
    # enough particles (32 plans x 8 x 170) for the lane-per-particle kernel; two
    # iterations of every plan vs the oracle, on the plans whose evaluated positions
    # stay clear of flipping crossing decisions
    cfg, start, target, polys, edges, hy = polygon_workload(4, iters=2, runs=32)
    pl = BFPlanner(cfg)
    assert pl.kernel_name() == "poly_lane_kernel"
    small = BFPlanner(cfg.with_(runs=1))
    assert small.kernel_name() == "bf_iter_kernel<5>"
    pl.set_hyper(hy)
    pl.set_polygons(start, target, edges)
    pl.run_async()
    sc = _scene(start, target, edges)
    checked = 0
    for r in range(0, 32, 4):
        sw = oracle.BFSwarm(cfg.with_(runs=1, run_id=r), hy, sc)
        sw.init()
        ok = True
        for _ in range(2):
            if not _margins_ok(cfg, sc, sw.s["X"]):
                ok = False
                break
            sw.iteration()
        if not ok:
            continue
        checked += 1
        s, o = pl.get_state(r), sw.state()
        _close(s["X"], o["X"], 400.0)
        _close(s["V"], o["V"], float(hy[:, 5].max()) * 400.0)
        np.testing.assert_allclose(s["Pfit"], o["Pfit"], rtol=1e-5)
        np.testing.assert_allclose(s["Gfit"], o["Gfit"], rtol=1e-5)
        assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=1e-5)
        _close(s["Tb"], o["Tb"], 400.0)
    assert checked >= 2


def test_polygon_warm_start_matches_oracle(native):
    # Priori Initialization on objective 5 (Sec. 3.3.3): each run's first
    # ceil(gamma N) particles per group around its previous path, the planning cycle
    # in the counters; two iterations of each run vs the oracle
    cfg, start, target, polys, edges, hy = polygon_workload(5, N=12, iters=2, runs=4)
    cfg = cfg.with_(G=3, pi_gamma=0.25, pi_halfwidth=20.0)
    hy = np.array(hy[:3])
    prev = random_paths(31, 4, cfg.D // 2).astype(np.float32) * np.float32(0.5) + np.float32(100.0)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_polygons(start, target, edges)
    pl.set_warm_start(prev, cycle=5)
    pl.run_async()
    sc = _scene(start, target, edges)
    checked = 0
    for r in range(4):
        c1 = cfg.with_(runs=1, run_id=r)
        sw = oracle.BFSwarm(c1, hy, sc)
        sw.set_previous(prev[r], 5)
        sw.init()
        ok = True
        for _ in range(2):
            if not _margins_ok(c1, sc, sw.s["X"]):
                ok = False
                break
            sw.iteration()
        if not ok:
            continue
        checked += 1
        s, o = pl.get_state(r), sw.state()
        _close(s["X"], o["X"], 400.0)
        _close(s["V"], o["V"], float(hy[:, 5].max()) * 400.0)
        np.testing.assert_allclose(s["Pfit"], o["Pfit"], rtol=1e-5)
        assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=1e-5)
    assert checked >= 2
