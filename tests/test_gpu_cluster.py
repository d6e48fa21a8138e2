"""The two forms of the per-iteration exchange give identical results.

The grid-wide form puts all CTAs of a run behind one barrier per iteration; the
cluster form (every group's C3 = 0, so Eq. TOF_V needs only the group's own
Gbest) runs one thread-block cluster per group with one warp per particle and the
rows in registers, trades the group best inside the cluster and the groups'
(Gfit, Q) through records read two iterations late, with Auto Truncation decided
two iterations late and the state of the stopping iteration restored.  Its
decisions, bests and arithmetic are meant to be those of the grid-wide form, so
results and states are compared bit for bit; the grid-wide form itself is held to
the oracle by test_gpu_parity.py.
"""
import numpy as np
import pytest

from paper_2308_10169_gb300 import Planner, static_workload
from paper_2308_10169_gb300._native import SepsoError
from paper_2308_10169_gb300.inputs import (AT_STD_WINDOW, HSEF_BOX_HI, HSEF_BOX_LO, TABLE_HYPER8,
                                           dynamic_workload, random_state, sample_hyper)

pytestmark = pytest.mark.gpu


def _pair(cfg, scene, hyper, cpg=0):
    out = []
    for ex in (1, 2):
        pl = Planner(cfg.with_(exchange=ex, ctas_per_group=cpg if ex == 2 else 0))
        pl.set_hyper(hyper)
        pl.set_scene(scene)
        out.append(pl)
    assert out[0].exchange_form() == "grid" and out[1].exchange_form() == "cluster"
    return out


def _same_result(a, b):
    assert a["iters"] == b["iters"]
    assert a["Q"] == b["Q"]
    assert a["status"] == b["status"] == 0
    assert np.float32(a["cost"]) == np.float32(b["cost"])
    assert np.float32(a["length"]) == np.float32(b["length"])
    np.testing.assert_array_equal(a["waypoints"], b["waypoints"])


def _same_state(pa, pb, run=0):
    sa, sb = pa.get_state(run), pb.get_state(run)
    for name in sa:
        np.testing.assert_array_equal(sa[name], sb[name], err_msg=name)


@pytest.mark.parametrize("N,cpg", [(170, 0), (170, 12), (96, 8), (48, 4), (48, 16), (30, 2), (1, 0)])
def test_cluster_form_matches_grid_form_dynamic_cycles(native, N, cpg):
    # the dynamic workload: PI, stall-counter AT (cap 300), moving circles; several
    # cycles so that truncation, PI and the carried state all take part; CTAs of
    # 15 down to 3 particle warps, a ragged last CTA (170 = 11 x 15 + 5) and a
    # one-particle group
    cfg, scene, hyper = dynamic_workload(2)
    cfg = cfg.with_(max_iters=120, N=N)
    ga, cl = _pair(cfg, scene, hyper, cpg)
    iters = []
    for cyc in range(4):
        if cyc:
            ga.advance(1)
            cl.advance(1)
        a, b = ga.plan(), cl.plan()
        _same_result(a, b)
        _same_state(ga, cl)
        iters.append(a["iters"])
    ga.sync()
    cl.sync()


def test_cluster_form_truncates_like_grid_form(native):
    # a map with room to reach a collision-free path, stall limit 3: the stall
    # counter stops cycles well before the cap, and the speculative iteration after
    # the stopping one must leave no trace
    cfg, scene, hyper = static_workload(5)
    cfg = cfg.with_(at_mode=2, stall_iters=3, max_iters=200, use_pi=True)
    ga, cl = _pair(cfg, scene, hyper)
    stopped_early = 0
    for cyc in range(6):
        a, b = ga.plan(), cl.plan()
        _same_result(a, b)
        _same_state(ga, cl)
        stopped_early += a["iters"] < cfg.max_iters
    assert stopped_early >= 3


def test_cluster_form_std_window_truncation(native):
    # the paper's std-window criterion (TW = 20, delta = 10) with C3 = 0 rows
    cfg, scene, hyper = static_workload(9)
    cfg = cfg.with_(at_mode=AT_STD_WINDOW, tw=20, delta=10.0, max_iters=150, use_pi=True, alpha=30.0, beta=4)
    ga, cl = _pair(cfg, scene, hyper)
    for cyc in range(5):
        _same_result(ga.plan(), cl.plan())
        _same_state(ga, cl)


@pytest.mark.parametrize("iters", [1, 2, 7])
def test_cluster_form_steps_from_a_loaded_state(native, iters):
    cfg, scene, hyper = dynamic_workload(3)
    st = random_state(41, cfg)
    ga, cl = _pair(cfg, scene, hyper)
    for pl in (ga, cl):
        pl.set_state(st)
        pl.step(iters)
        pl.step(iters)
    _same_state(ga, cl)


def test_cluster_form_several_runs_and_switching_forms(native):
    # four runs (each its own clusters), then the handle alternates between C3 = 0
    # (cluster form) and C3 > 0 (grid-wide form): the barrier counter, group words
    # and records stay consistent across the switches
    cfg, scene, hyper = dynamic_workload(4)
    cfg = cfg.with_(runs=4, N=40, max_iters=60)
    ref = Planner(cfg.with_(exchange=1))
    mix = Planner(cfg.with_(exchange=3))
    hyper_c3 = hyper.copy()
    hyper_c3[:, 2] = 0.5
    for pl in (ref, mix):
        pl.set_scene(scene)
    for cyc, hy in enumerate([hyper, hyper, hyper_c3, hyper, hyper_c3, hyper_c3, hyper]):
        for pl in (ref, mix):
            pl.set_hyper(hy)
        assert mix.exchange_form() == ("grid" if hy[0, 2] else "cluster")
        for pl in (ref, mix):
            pl.plan_async()
        for run in range(cfg.runs):
            _same_result(ref.read_result(run), mix.read_result(run))
            _same_state(ref, mix, run)
        for pl in (ref, mix):
            pl.step(3)
        for run in range(cfg.runs):
            _same_state(ref, mix, run)
    ref.sync()
    mix.sync()


def test_cluster_form_hsef_matches(native):
    # HSEF L-runs (8 runs, no AT, cap 100) in both forms
    cfg, scene, _ = dynamic_workload(0)
    out = []
    for ex in (1, 2):
        hp = Planner(cfg.with_(runs=8, N=24, at_mode=0, use_pi=False, max_iters=100, exchange=ex))
        hp.set_scene(scene, motion=False)
        hist = hp.hsef(HG=2, HN=4, E=3, hhyper=TABLE_HYPER8[:2], lo=HSEF_BOX_LO, hi=HSEF_BOX_HI,
                       l_vlimit=0.05, hseed=77)
        out.append((hist.cpu().numpy(), *hp.hsef_best()))
        assert hp.exchange_form() == ("grid" if ex == 1 else "cluster")
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


def test_cluster_form_refused_when_an_update_needs_tbest(native):
    cfg, scene, hyper = static_workload(1)
    hy = hyper.copy()
    hy[3, 2] = 0.7  # one group with C3 > 0
    pl = Planner(cfg.with_(exchange=2))
    pl.set_scene(scene)
    pl.set_hyper(hy)
    with pytest.raises(SepsoError) as err:
        pl.plan()
    assert err.value.code == -1  # SEPSO_EINVAL
    auto = Planner(cfg.with_(exchange=3))
    auto.set_scene(scene)
    auto.set_hyper(hy)
    assert auto.exchange_form() == "grid"
    auto.set_hyper(sample_hyper(3, cfg.G))
    assert auto.exchange_form() == "cluster"
    auto0 = Planner(cfg)   # the automatic choice: the cluster form whenever it applies
    auto0.set_scene(scene)
    auto0.set_hyper(hy)
    assert auto0.exchange_form() == "grid"
    auto0.set_hyper(sample_hyper(3, cfg.G))
    assert auto0.exchange_form() == "cluster"
    assert Planner(cfg.with_(exchange=1)).exchange_form() == "grid"


def test_cluster_form_refused_when_it_does_not_fit(native):
    cfg, scene, hyper = static_workload(1)
    for bad in (dict(T=32), dict(N=400), dict(runs=64)):
        with pytest.raises(SepsoError) as err:
            Planner(cfg.with_(exchange=2, **bad))
        assert err.value.code == -7  # SEPSO_ERANGE
        pl = Planner(cfg.with_(exchange=3, **bad))   # falls back to the grid-wide form
        pl.set_scene(scene)
        pl.set_hyper(hyper)
        assert pl.exchange_form() == "grid"
