"""Path planning in three dimensions among spheres (the Conclusion's extension from
2D to 3D planning; objective 6 of the generic engine) on the GPU vs the FP64 oracle,
through the C ABI.

Tolerances: collision counts Q bit-exact for paths whose every (segment, sphere)
pair is more than 1e-3 from tangency (|dist - r| > 1e-3); fitness 1e-5 relative;
positions and velocities after identical state 1e-5 relative with floors of 1e-5 x
the box and x V_range (as for the other objectives of the engine); whole runs and
planning cycles: median final cost within 5% of the oracle's (FP32 and FP64
trajectories part after a few iterations, so medians are compared).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_10169_gb300 import BFPlanner
from paper_2308_10169_gb300.inputs import advance_spheres, random_paths3, sphere_workload
from paper_2308_10169_gb300.planner import sphere_evaluate

pytestmark = pytest.mark.gpu

MARGIN = 1e-3


def _scene(sc):
    return oracle.Scene3(sc["start"], sc["target"], sc["spheres"])


def _close(a, b, scale, rtol=1e-5):
    np.testing.assert_allclose(np.asarray(a, np.float64), np.asarray(b, np.float64), rtol=rtol,
                               atol=rtol * scale)


@pytest.mark.parametrize("T,n,S", [(16, 2000, 64), (1, 300, 7), (33, 257, 200), (5, 100, 0)])
def test_evaluate_matches_oracle(native, T, n, S):
    cfg, sc, hy = sphere_workload(1, T=T, S=max(S, 1))
    if S == 0:
        sc["spheres"] = np.zeros((0, 4), np.float32)
    X = random_paths3(7 + T, n, T)
    s3 = _scene(sc)
    sw = oracle.BFSwarm(cfg, hy, s3)
    Fo, Qo = sw.evaluate(X.astype(np.float64), with_q=True)
    keep = oracle.sphere_margin(cfg, s3, X.astype(np.float64)) > MARGIN
    assert keep.mean() > 0.9
    sph = torch.from_numpy(sc["spheres"].reshape(-1, 4).copy()).cuda()
    F, Q = sphere_evaluate(torch.from_numpy(X).cuda(), sc["start"], sc["target"], sph, cfg.alpha, cfg.beta)
    F, Q = F.cpu().numpy(), Q.cpu().numpy()
    np.testing.assert_array_equal(Q[keep], Qo[keep])
    np.testing.assert_allclose(F[keep], Fo[keep], rtol=1e-5)
    if S:
        assert np.unique(Qo[keep]).size >= 3                  # a spread of collision counts
    else:
        assert not Qo.any()


def _small(seed, N=11, G=3, T=5):
    cfg, sc, hy = sphere_workload(seed, T=T, N=N, S=24)
    return cfg.with_(G=G), sc, np.array(hy[:G])


def _margins_ok(cfg, s3, X):
    return np.all(oracle.sphere_margin(cfg, s3, np.asarray(X, np.float64).reshape(-1, cfg.D)) > MARGIN)


def _oracle_clear(cfg, s3, hy, K, prev=None, cycle=0):
    """The oracle's swarm after K iterations, or None if an evaluated position came
    within the tangency margin."""
    sw = oracle.BFSwarm(cfg, hy, s3)
    if prev is not None:
        sw.set_previous(prev, cycle)
    elif cycle:
        sw.s["cycle"][0] = cycle
    sw.init()
    hist = []
    for _ in range(K):
        if not _margins_ok(cfg, s3, sw.s["X"]):
            return None, None
        sw.iteration()
        hist.append(sw.s["Tfit"][0])
    return sw, hist


def _compare_state(s, o, hy, box=400.0):
    _close(s["X"], o["X"], box)
    _close(s["V"], o["V"], float(hy[:, 5].max()) * box)
    _close(s["P"], o["P"], box)
    np.testing.assert_allclose(s["Pfit"], o["Pfit"], rtol=1e-5)
    np.testing.assert_allclose(s["Gfit"], o["Gfit"], rtol=1e-5)
    assert s["Tfit"][0] == pytest.approx(o["Tfit"][0], rel=1e-5)
    _close(s["Tb"], o["Tb"], box)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_first_iterations_match_oracle(native, K):
    for seed in range(40):
        cfg, sc, hy = _small(seed)
        cfg = cfg.with_(max_iters=K)
        sw, hist = _oracle_clear(cfg, _scene(sc), hy, K)
        if sw is not None:
            break
    assert sw is not None
    pl = BFPlanner(cfg)
    assert pl.kernel_name() == "bf_iter_kernel<6>"
    pl.set_hyper(hy)
    pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
    pl.run_async(use_graph=False)
    _compare_state(pl.get_state(), sw.state(), hy)
    np.testing.assert_allclose(pl.history()[:K], hist, rtol=1e-5)


def test_warm_start_matches_oracle(native):
    """Priori Initialization around each run's previous path, with the planning cycle
    in the counters: the first two iterations of every run vs the oracle."""
    cfg, sc, hy = _small(3, N=12, G=2)
    cfg = cfg.with_(max_iters=2, runs=4)
    prev = random_paths3(21, 4, 5) * np.float32(0.5) + np.float32(100.0)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
    pl.set_warm_start(prev, cycle=7)
    pl.run_async()
    s3 = _scene(sc)
    checked = 0
    for r in range(4):
        sw, _ = _oracle_clear(cfg.with_(runs=1, run_id=r), s3, hy, 2, prev=prev[r], cycle=7)
        if sw is None:
            continue
        checked += 1
        _compare_state(pl.get_state(r), sw.state(), hy)
    assert checked >= 2
    # the cold start on the same handle is the plain initialisation again
    pl.set_warm_start(None, cycle=0)
    pl.run_async()
    cold = BFPlanner(cfg)
    cold.set_hyper(hy)
    cold.set_spheres(sc["start"], sc["target"], sc["spheres"])
    cold.run_async()
    for r in range(4):
        np.testing.assert_array_equal(pl.read(r)["x"], cold.read(r)["x"])


@pytest.mark.parametrize("S", [4, 5])
def test_lane_per_particle_kernel_matches_oracle(native, S):
    # 32 plans x 8 x 170 particles: the lane-per-particle kernel; two iterations of
    # the plans whose evaluated positions stay clear of tangency, cold and warm.  Four
    # or five spheres (an odd count exercises the pair staging's padding), so that a
    # good share of the 1360-particle plans keeps every one of its evaluations more
    # than 1e-3 from tangency.
    cfg, sc, hy = sphere_workload(4, iters=2, runs=32, S=S)
    pl = BFPlanner(cfg)
    assert pl.kernel_name() == "sphere_lane_kernel"
    assert BFPlanner(cfg.with_(runs=1)).kernel_name() == "bf_iter_kernel<6>"
    pl.set_hyper(hy)
    pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
    s3 = _scene(sc)
    prev = random_paths3(5, 32, 16)
    for warm in (False, True):
        if warm:
            pl.set_warm_start(prev, cycle=3)
        pl.run_async()
        checked = 0
        for r in range(32):
            sw, _ = _oracle_clear(cfg.with_(runs=1, run_id=r), s3, hy, 2,
                                  prev=prev[r] if warm else None, cycle=3 if warm else 0)
            if sw is None:
                continue
            checked += 1
            _compare_state(pl.get_state(r), sw.state(), hy)
        assert checked >= 2


def test_runs_match_oracle_statistically(native):
    cfg, sc, hy = sphere_workload(2, T=8, N=40, iters=100, runs=16)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
    pl.run_async()
    gpu = np.array([pl.read(r)["fit"] for r in range(16)], np.float64)
    s3 = _scene(sc)
    ora = []
    for r in range(16):
        sw = oracle.BFSwarm(cfg.with_(runs=1, run_id=r), hy, s3)
        ora.append(sw.run(100)[-1])
        g = pl.history(r)
        assert np.all(np.diff(g) <= 0)
        x = pl.read(r)["x"]
        assert x.min() >= 0.0 and x.max() <= 400.0
    assert abs(np.median(gpu) - np.median(ora)) <= 0.05 * np.median(ora), (np.median(gpu), np.median(ora))


def test_dynamic_cycles_match_oracle_statistically(native):
    """Three planning cycles among moving spheres, each run warm-started from its own
    previous best path (PI), on the GPU and with the oracle: medians of each cycle's
    costs over 16 runs within 5%."""
    cfg, sc, hy = sphere_workload(5, T=8, N=40, iters=60, runs=16)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    s3 = _scene(sc)
    sph, vel = sc["spheres"], sc["vel"]
    prev_g = prev_o = None
    swarms = [oracle.BFSwarm(cfg.with_(runs=1, run_id=r), hy, s3) for r in range(16)]
    for cycle in range(3):
        if cycle:
            sph, vel = advance_spheres(sph, vel)
        scene = oracle.Scene3(sc["start"], sc["target"], sph)
        pl.set_spheres(sc["start"], sc["target"], sph)
        pl.set_warm_start(prev_g, cycle=cycle)
        pl.run_async()
        prev_g, gfit, _ = pl.read_all()
        ofit, prev_o_new = [], []
        for r, sw in enumerate(swarms):
            sw.set_scene(scene)
            if prev_o is not None:
                sw.set_previous(prev_o[r], cycle)
            sw.init()
            for _ in range(cfg.max_iters):
                sw.iteration()
            ofit.append(sw.s["Tfit"][0])
            prev_o_new.append(sw.s["Tb"].copy())
        prev_o = prev_o_new
        med_g, med_o = float(np.median(gfit)), float(np.median(ofit))
        assert abs(med_g - med_o) <= 0.05 * med_o, (cycle, med_g, med_o)


def test_new_sphere_count_recaptures_the_graph(native):
    cfg, sc, hy = sphere_workload(3, T=6, N=20, iters=30, runs=2)
    cfg = cfg.with_(max_spheres=100)
    other = sc["spheres"][:10]
    a = BFPlanner(cfg)
    a.set_hyper(hy)
    a.set_spheres(sc["start"], sc["target"], sc["spheres"])
    a.run_async()
    a.set_spheres(sc["start"], sc["target"], other)
    a.run_async()
    b = BFPlanner(cfg)
    b.set_hyper(hy)
    b.set_spheres(sc["start"], sc["target"], other)
    b.run_async(use_graph=False)
    for r in range(2):
        np.testing.assert_array_equal(a.read(r)["x"], b.read(r)["x"])


def test_errors(native):
    from paper_2308_10169_gb300 import _native
    from paper_2308_10169_gb300.inputs import polygon_workload
    cfg, sc, hy = sphere_workload(0, T=4, N=8, iters=5)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    with pytest.raises(RuntimeError, match="set_spheres"):
        pl.run_async()
    bad = sc["spheres"].copy()
    bad[0, 3] = -1.0
    with pytest.raises(RuntimeError, match="negative radius"):
        pl.set_spheres(sc["start"], sc["target"], bad)
    with pytest.raises(RuntimeError, match="max_spheres"):
        pl.set_spheres(sc["start"], sc["target"], np.zeros((cfg.max_spheres + 1, 4), np.float32))
    with pytest.raises(RuntimeError, match="pi_gamma"):
        BFPlanner(cfg.with_(pi_gamma=1.5)).set_warm_start(np.zeros((1, cfg.D), np.float32))
    with pytest.raises(RuntimeError, match="D = 3T"):
        BFPlanner(cfg.with_(D=10))
    pcfg = polygon_workload(0)[0]
    with pytest.raises(RuntimeError, match="objective 6"):
        BFPlanner(pcfg).set_spheres(sc["start"], sc["target"], sc["spheres"])
    assert _native.lib() is not None


def _oracle_plan_clear(cfg, s3, hy, margin_fn):
    """The oracle's planning cycle with Auto Truncation, or None when a position it
    evaluated came within the margin of a flipping collision decision."""
    sw = oracle.BFSwarm(cfg, hy, s3)
    sw.s["stall"][0] = 0
    sw.s["prev_lfv"][0] = np.inf
    sw.init()
    for _ in range(cfg.max_iters):
        if not margin_fn(sw.s["X"]):
            return None
        if sw.iteration_stop():
            break
    return sw


@pytest.mark.parametrize("runs,S", [(4, 48), (32, 4)])
def test_auto_truncation_stop_matches_oracle(native, runs, S):
    """Stall limit 1, unreachable tolerance: a run stops at the first iteration after
    the first whose Tbest collides with nothing.  The stopping iteration, the bests
    and the positions it evaluated (nothing moves after it) vs the oracle, on the
    runs whose evaluations stay clear of tangency; warp kernel (4 runs of 3 x 12) and
    lane kernel (32 runs of 8 x 170)."""
    if runs == 4:
        cfg, sc, hy = sphere_workload(6, T=6, N=12, S=S, iters=40, runs=runs)
        cfg, hy = cfg.with_(G=3), np.array(hy[:3])
    else:
        cfg, sc, hy = sphere_workload(7, T=6, S=S, iters=40, runs=runs)
    cfg = cfg.with_(at_stall=1, stall_tol=1e30)
    pl = BFPlanner(cfg)
    assert pl.kernel_name() == ("bf_iter_kernel<6>" if runs == 4 else "sphere_lane_kernel")
    pl.set_hyper(hy)
    pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
    pl.run_async()
    s3 = _scene(sc)
    checked = early = 0
    for r in range(runs):
        sw = _oracle_plan_clear(cfg.with_(runs=1, run_id=r), s3, hy, lambda X: _margins_ok(cfg, s3, X))
        if sw is None:
            continue
        checked += 1
        got = pl.read(r)
        assert got["iters"] == int(sw.s["k"][0]), r
        early += got["iters"] < cfg.max_iters
        st = pl.get_state(r)
        _close(st["X"], sw.s["X"], 400.0)
        _close(st["Tb"], sw.s["Tb"], 400.0)
        assert st["Tfit"][0] == pytest.approx(sw.s["Tfit"][0], rel=1e-5)
    assert checked >= 2 and early >= 1


def test_auto_truncation_matches_oracle_statistically(native):
    """Stall limit 10, tolerance 1 (the dynamic workload's reading): over 16 runs the
    median stopping iteration within 15% + 1 and the median cost within 5% of the
    oracle's."""
    cfg, sc, hy = sphere_workload(8, T=8, N=40, iters=100, runs=16, at_stall=10, stall_tol=1.0)
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
    pl.run_async()
    g_it, g_cost, o_it, o_cost = [], [], [], []
    s3 = _scene(sc)
    for r in range(16):
        got = pl.read(r)
        g_it.append(got["iters"])
        g_cost.append(got["fit"])
        res = oracle.BFSwarm(cfg.with_(runs=1, run_id=r), hy, s3).plan()
        o_it.append(res["iters"])
        o_cost.append(res["cost"])
    assert min(o_it) < cfg.max_iters            # AT acts on this scene
    assert abs(np.median(g_it) - np.median(o_it)) <= 0.15 * np.median(o_it) + 1, (g_it, o_it)
    assert abs(np.median(g_cost) - np.median(o_cost)) <= 0.05 * np.median(o_cost)


def test_polygon_auto_truncation_stop_matches_oracle(native):
    """The same stop rule on objective 5 (paths among polygons)."""
    from paper_2308_10169_gb300.inputs import polygon_workload
    cfg, start, target, polys, edges, hy = polygon_workload(2, N=12, iters=40, runs=4)
    cfg = cfg.with_(G=3, at_stall=1, stall_tol=1e30)
    hy = np.array(hy[:3])
    pl = BFPlanner(cfg)
    pl.set_hyper(hy)
    pl.set_polygons(start, target, edges)
    pl.run_async()
    sc = oracle.Scene(start, target, np.zeros((0, 3)), edges)
    checked = 0
    for r in range(4):
        c1 = cfg.with_(runs=1, run_id=r)
        sw = _oracle_plan_clear(c1, sc, hy, lambda X: np.all(oracle.poly_margin(c1, sc, X.reshape(-1, c1.D)) > 1e-6))
        if sw is None:
            continue
        checked += 1
        got = pl.read(r)
        assert got["iters"] == int(sw.s["k"][0])
        st = pl.get_state(r)
        _close(st["X"], sw.s["X"], 400.0)
        assert st["Tfit"][0] == pytest.approx(sw.s["Tfit"][0], rel=1e-5)
    assert checked >= 2
