"""The path-planning setting of Sec. 4.3 and its ablation switches (Table ppresult),
checked on the host and through the oracle (no GPU).

SEPSO uses the evolved Table hyper8path rows with Priori Initialization and Auto
Truncation; SEPSO(NoAT) drops AT (every frame runs the cap of 30 iterations);
SEPSO(NoPI) drops PI; DTPSO runs the unevolved Table hyper8 rows with neither.
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300.inputs import (AT_OFF, AT_STD_WINDOW, PAPER_VARIANTS, PARAMS_PATH,
                                           TABLE_HYPER8, TABLE_HYPER8_PATH, paper_workload)


def test_variant_switches():
    for var, sw in PAPER_VARIANTS.items():
        cfg, scene, hyper = paper_workload(0, var)
        assert (cfg.T, cfg.G, cfg.N, cfg.max_iters) == (8, 8, 170, 30)
        assert (cfg.map_w, cfg.map_h) == (366.0, 366.0)
        assert (cfg.alpha, cfg.beta, cfg.pi_gamma, cfg.delta, cfg.tw) == (
            PARAMS_PATH["alpha"], PARAMS_PATH["beta"], PARAMS_PATH["pi_gamma"],
            PARAMS_PATH["delta"], PARAMS_PATH["tw"])
        assert cfg.use_pi == sw["use_pi"]
        assert cfg.at_mode == (AT_STD_WINDOW if sw["at"] else AT_OFF)
        np.testing.assert_array_equal(hyper, TABLE_HYPER8_PATH if var != "DTPSO" else TABLE_HYPER8)
    assert PAPER_VARIANTS["SEPSO"] == dict(hyper="hyper8path", use_pi=True, at=True)
    assert not PAPER_VARIANTS["DTPSO"]["use_pi"] and not PAPER_VARIANTS["DTPSO"]["at"]


def test_scene_shape():
    # the same scene for every variant: 2 static and 6 moving obstacles with speeds in
    # (0, 5], start/target moving 3 and 8 per frame along the vertical axis
    ref = paper_workload(3, "SEPSO")[1]
    for var in PAPER_VARIANTS:
        sc = paper_workload(3, var)[1]
        np.testing.assert_array_equal(sc.circles, ref.circles)
        np.testing.assert_array_equal(sc.circle_vel, ref.circle_vel)
    speed = np.hypot(ref.circle_vel[:, 0], ref.circle_vel[:, 1])
    assert np.all(speed[:2] == 0)
    assert np.all((speed[2:] > 0) & (speed[2:] <= 5.0 + 1e-5))
    assert np.all((ref.circles[:, 2] >= 15) & (ref.circles[:, 2] <= 30))
    np.testing.assert_array_equal(ref.start_vel, [0, 3])
    np.testing.assert_array_equal(ref.target_vel, [0, -8])


def _frames(var, frames, key=100):
    cfg, scene, hyper = paper_workload(0, var)
    sw = oracle.Swarm(cfg.with_(seed=key), hyper)
    c, v, st, sv, tg, tv = (scene.circles, scene.circle_vel, scene.start, scene.start_vel,
                            scene.target, scene.target_vel)
    out = []
    for f in range(frames):
        if f:
            c, v, st, sv, tg, tv = oracle.advance_scene(cfg.map_w, cfg.map_h, c, v, st, sv, tg, tv)
        out.append(sw.plan(oracle.Scene(st, tg, c)))
    return out


@pytest.mark.parametrize("var", ["SEPSO(NoAT)", "DTPSO"])
def test_without_truncation_every_frame_runs_the_cap(var):
    res = _frames(var, 6)
    assert [r["iters"] for r in res] == [30] * 6


def test_truncation_stops_collision_free_frames_early():
    # AT stops only on a collision-free best path (Sec. 3.3.4, second criterion); with
    # the window carried over from the previous frames, later frames stop early
    res = _frames("SEPSO", 8)
    iters = [r["iters"] for r in res]
    assert all(1 <= i <= 30 for i in iters)
    assert min(iters[1:]) < 30
    for r in res:
        if r["iters"] < 30:
            assert r["Q"] == 0
