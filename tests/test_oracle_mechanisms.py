"""Pins of the oracle's PI (Sec. 3.3.3), AT (Sec. 3.3.4), random factors, dynamic
scene step (Fig. PP caption), end-to-end planning and HSEF (Sec. 3.2.1)."""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300.inputs import (AT_STALL, AT_STD_WINDOW, HSEF_BOX_HI, HSEF_BOX_LO,
                                           TABLE_HYPER8, SepsoConfig, static_workload)

# ---------------------------------------------------------------------------
# Random factors
# ---------------------------------------------------------------------------


def test_u01_hand_values():
    # u = (x >> 8) * 2^-24
    assert oracle.u01(0) == 0.0
    assert oracle.u01(0xFF) == 0.0
    assert oracle.u01(0x100) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.u01(0x80000000) == 0.5


def test_philox_known_answers():
    # the generator's published known-answer vectors (tests/golden/philox4x32_10_kat.json)
    import json
    from pathlib import Path
    kat = json.loads((Path(__file__).parent / "golden" / "philox4x32_10_kat.json").read_text())
    for case in kat["cases"]:
        ctr = np.array([[int(w, 16) for w in case["counter"]]], np.uint32)
        k0, k1 = (int(w, 16) for w in case["key"])
        out = oracle.philox(ctr, seed=(k1 << 32) | k0)
        assert [f"{v:08x}" for v in out[0]] == case["output"]


def test_philox_outputs_are_uniform_and_distinct():
    n = 200_000
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n) % 1000
    ctr[:, 1] = np.arange(n) // 1000
    out = oracle.philox(ctr, seed=12345)
    u = (out >> 8).astype(np.float64) * 2.0 ** -24
    flat = u.reshape(-1)
    assert abs(flat.mean() - 0.5) < 4 * np.sqrt(1 / 12 / flat.size)
    assert abs(flat.var() - 1 / 12) < 1e-3
    hist = np.bincount((flat * 64).astype(int), minlength=64)
    e = flat.size / 64
    chi2 = ((hist - e) ** 2 / e).sum()
    assert chi2 < 63 + 6 * np.sqrt(2 * 63)          # 63 dof, ~6 sigma
    # neighbouring counters are uncorrelated, in every output word
    for w in range(4):
        c = np.corrcoef(u[:-1, w], u[1:, w])[0, 1]
        assert abs(c) < 0.01
    # 128-bit outputs of distinct counters do not collide
    assert np.unique(out.view(np.dtype((np.void, 16)))).size == n
    # the key matters
    out2 = oracle.philox(ctr[:1000], seed=12346)
    assert np.mean(out2 == out[:1000]) < 0.01


# ---------------------------------------------------------------------------
# Priori Initialization
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("gamma,N,expect", [(0.25, 170, 43), (0.25, 32, 8), (0.1, 1, 1),
                                            (0.0, 50, 0), (1.0, 7, 7)])
def test_pi_count_is_ceiling(gamma, N, expect):
    # ceil(gamma * N): 42.5 -> 43, 8 -> 8, 0.1 -> 1, 0 -> 0, 7 -> 7
    assert oracle.pi_count(gamma, N) == expect


def _pi_swarm(has_prev, prevT, use_pi=True):
    cfg = SepsoConfig(T=4, G=2, N=16, use_pi=use_pi, pi_gamma=0.25, pi_halfwidth=20.0)
    h = np.tile([1.5, 1.5, 0.0, 0.7, 0.7, 0.05], (2, 1))
    sw = oracle.Swarm(cfg, h)
    sw.load({"has_prev": [has_prev], "prevT": prevT, "cycle": [3]})
    sw.init()
    return cfg, sw.state()


def test_pi_places_first_gamma_fraction_near_previous_best():
    prevT = np.array([10.0, 100.0, 200.0, 395.0, 50.0, 150.0, 250.0, 390.0])
    cfg, s = _pi_swarm(1, prevT)
    X = s["X"].reshape(2, 16, 8)
    n_pi = 4  # ceil(0.25 * 16)
    lo = np.clip(prevT - 20.0, 0, 400)
    hi = np.clip(prevT + 20.0, 0, 400)
    assert np.all(X[:, :n_pi] >= lo - 1e-12) and np.all(X[:, :n_pi] <= hi + 1e-12)
    # the rest are uniform over the map: most lie outside the PI box
    rest = X[:, n_pi:]
    outside = np.any((rest < lo) | (rest > hi), axis=2)
    assert outside.mean() > 0.9
    # waypoints near the border are clipped to the map
    assert np.all(X[:, :n_pi, 3] <= 400.0)
    np.testing.assert_array_equal(s["P"], s["X"])
    assert np.all(np.isinf(s["Pfit"])) and np.isinf(s["Tfit"][0]) and s["k"][0] == 0
    V = s["V"].reshape(2, 16, 8)
    assert np.all(np.abs(V) <= 0.05 * 400 + 1e-12)


def test_no_pi_without_previous_path_or_when_disabled():
    prevT = np.full(8, 200.0)
    for has_prev, use_pi in ((0, True), (1, False)):
        cfg, s = _pi_swarm(has_prev, prevT, use_pi)
        X = s["X"].reshape(2, 16, 8)
        near = np.all(np.abs(X - 200.0) <= 20.0, axis=2)
        assert near.sum() == 0


def test_learned_seed_takes_the_first_particles_then_pi():
    # A second seed of PI's kind (Sec. 3.3.3): n_prior particles per group around
    # priorT (Philox stream 4), then PI's ceil(gamma N) around prevT (stream 3).
    prevT = np.full(8, 100.0)
    priorT = np.full(8, 300.0)
    cfg = SepsoConfig(T=4, G=2, N=16, use_pi=True, pi_gamma=0.25, pi_halfwidth=20.0, seed=9, run_id=2)
    h = np.tile([1.5, 1.5, 0.0, 0.7, 0.7, 0.05], (2, 1))
    sw = oracle.Swarm(cfg, h)
    sw.load({"has_prev": [1], "prevT": prevT, "cycle": [3], "n_prior": [3], "priorT": priorT})
    sw.init()
    X = sw.state()["X"].reshape(2, 16, 8)
    assert np.all(np.abs(X[:, :3] - 300.0) <= 20.0)
    assert np.all(np.abs(X[:, 3:7] - 100.0) <= 20.0)
    far = np.all(np.abs(X[:, 7:] - 100.0) > 20.0, axis=2) | np.any(np.abs(X[:, 7:] - 300.0) > 20.0, axis=2)
    assert far.all()
    # coordinate j of particle p comes from lane j % 4 of Philox block (j // 4, p, 4 << 24 | cycle, run)
    g, n, j = 1, 2, 5
    ctr = np.array([[j // 4, g * 16 + n, (4 << 24) | 3, 2]], np.uint32)
    u = oracle.u01(int(oracle.philox(ctr, 9)[0, j % 4]))
    assert X[g, n, j] == pytest.approx(300.0 + (2 * u - 1) * 20.0, abs=1e-12)
    # without the seed the initialisation is PI's alone
    sw2 = oracle.Swarm(cfg, h)
    sw2.load({"has_prev": [1], "prevT": prevT, "cycle": [3]})
    sw2.init()
    X2 = sw2.state()["X"].reshape(2, 16, 8)
    assert np.all(np.abs(X2[:, :4] - 100.0) <= 20.0)
    np.testing.assert_array_equal(X2[:, 7:], X[:, 7:])


# ---------------------------------------------------------------------------
# Auto Truncation
# ---------------------------------------------------------------------------

def test_window_std_hand_values():
    # population std: [10, 12, 14, 16] -> mean 13, var (9+1+1+9)/4 = 5
    assert oracle.window_std([10, 12, 14, 16]) == pytest.approx(np.sqrt(5.0), rel=1e-15)
    assert oracle.window_std([7, 7]) == 0.0


def _at_swarm(mode, tw=3, delta=1.0, stall_iters=3):
    cfg = SepsoConfig(T=1, G=1, N=1, at_mode=mode, tw=tw, delta=delta, stall_iters=stall_iters)
    return oracle.Swarm(cfg, np.zeros((1, 6)))


def test_std_window_ring_buffer_and_collision_condition():
    sw = _at_swarm(AT_STD_WINDOW, tw=3, delta=1.0)
    seq = [(100.0, 0, False),   # one sample: no decision
           (50.0, 0, False),    # std(100, 50) = 25
           (49.0, 0, False),    # std(100, 50, 49) large
           (49.0, 0, True),     # window (50, 49, 49): std = 0.471 < 1
           (49.0, 2, False),    # std 0 but the best path collides
           (49.0, 0, True)]
    for lfv, q, expect in seq:
        sw.load({"Tfit": [lfv], "TQ": [q]})
        assert sw.at_update() == expect, (lfv, q)
    s = sw.state()
    assert s["win_n"][0] == 3 and s["win_head"][0] == 6 % 3


def test_stall_counter():
    sw = _at_swarm(AT_STALL, stall_iters=3)
    sw.load({"prev_lfv": [np.inf], "stall": [0]})
    seq = [(100.0, 0, 0, False), (90.0, 0, 0, False), (90.0, 0, 1, False), (90.0, 0, 2, False),
           (90.0, 1, 3, False),   # stalled 3 times but colliding
           (90.0, 0, 4, True), (80.0, 0, 0, False)]
    for lfv, q, stall, expect in seq:
        sw.load({"Tfit": [lfv], "TQ": [q]})
        assert sw.at_update() == expect
        assert sw.state()["stall"][0] == stall


# ---------------------------------------------------------------------------
# Dynamic scene
# ---------------------------------------------------------------------------

def test_advance_scene_hand_values():
    circles = [[395.0, 200.0, 3.0], [100.0, 2.0, 5.0], [50.0, 50.0, 10.0]]
    cvel = [[2.0, 0.0], [0.0, -1.5], [0.0, 0.0]]
    c, v, s, sv, t, tv = oracle.advance_scene(400, 400, circles, cvel, (20, 399.5), (0, 1),
                                              (380, 1), (0, -1))
    # 395 + 2 = 397; 397 + 3 = 400 is not beyond the border: velocity kept
    assert c[0, 0] == 397.0 and v[0, 0] == 2.0
    # 2 - 1.5 = 0.5; 0.5 - 5 < 0 while moving down: velocity flips
    assert c[1, 1] == 0.5 and v[1, 1] == 1.5
    np.testing.assert_array_equal(c[2], [50, 50, 10])
    # start 399.5 + 1 = 400.5 > 400 moving up: flips; target 1 - 1 = 0, not below 0: kept
    assert s[1] == 400.5 and sv[1] == -1.0
    assert t[1] == 0.0 and tv[1] == -1.0
    c2, v2, *_ = oracle.advance_scene(400, 400, c, v, s, sv, t, tv)
    assert c2[0, 0] == 399.0 and v2[0, 0] == -2.0


# ---------------------------------------------------------------------------
# End to end
# ---------------------------------------------------------------------------

def test_obstacle_free_plan_reaches_straight_line_optimum():
    cfg, _, hyper = static_workload(0)
    cfg = cfg.with_(max_iters=200)
    sc = oracle.Scene((20, 20), (380, 380), np.zeros((0, 3)))
    res = oracle.Swarm(cfg, hyper).plan(sc)
    opt = 360.0 * np.sqrt(2.0)
    assert res["Q"] == 0
    assert opt - 1e-9 <= res["cost"] <= opt * 1.005


def test_plan_result_is_consistent_and_monotone():
    cfg, scene, hyper = static_workload(1)
    sc = oracle.Scene(scene.start, scene.target, scene.circles)
    sw = oracle.Swarm(cfg, hyper)
    sw.init()
    last = np.inf
    while True:
        stop = sw.iteration(sc, check_stop=True)
        tf = sw.state()["Tfit"][0]
        assert tf <= last
        last = tf
        if stop:
            break
    assert sw.state()["k"][0] == cfg.max_iters
    res = oracle.Swarm(cfg, hyper).plan(sc)
    F, Q, L = oracle.evaluate(cfg, sc, res["waypoints"])
    assert res["cost"] == F[0] and res["Q"] == Q[0] and res["length"] == pytest.approx(L[0])
    assert res["cost"] == last and res["iters"] == cfg.max_iters


def test_plan_warm_state_and_truncation():
    cfg, scene, hyper = static_workload(2)
    cfg = cfg.with_(at_mode=AT_STALL, stall_iters=10, max_iters=300, use_pi=True)
    sc = oracle.Scene(scene.start, scene.target, scene.circles)
    sw = oracle.Swarm(cfg, hyper)
    r1 = sw.plan(sc)
    s = sw.state()
    assert s["cycle"][0] == 1 and s["has_prev"][0] == 1
    np.testing.assert_array_equal(s["prevT"], r1["waypoints"])
    assert r1["iters"] < 300 and r1["Q"] == 0 and s["stall"][0] >= 10
    r2 = sw.plan(sc)
    assert sw.state()["cycle"][0] == 2
    # warm start from the previous best: the second plan starts no worse than the PI box allows
    assert r2["cost"] <= r1["cost"] * 1.05


# ---------------------------------------------------------------------------
# HSEF
# ---------------------------------------------------------------------------

def _small_hsef(E):
    lcfg = SepsoConfig(T=3, G=2, N=6, max_iters=8, alpha=30.0, beta=4)
    rng = np.random.default_rng(9)
    circ = np.column_stack([rng.uniform(60, 340, (6, 2)), rng.uniform(10, 30, 6)])
    sc = oracle.Scene((20, 20), (380, 380), circ)
    return lcfg, sc, oracle.hsef(lcfg, sc, HG=4, HN=2, E=E, hhyper=TABLE_HYPER8[:4],
                                 lo=HSEF_BOX_LO, hi=HSEF_BOX_HI, l_vlimit=0.05, hseed=77)


def test_hsef_best_lfv_non_increasing_and_in_box():
    lcfg, sc, (best, bf, hist) = _small_hsef(6)
    assert np.all(np.diff(hist) <= 0)
    assert bf == hist[-1]
    G = lcfg.G
    for kind in range(3):
        v = best[kind * G:(kind + 1) * G]
        assert np.all(v >= HSEF_BOX_LO[kind] - 1e-12) and np.all(v <= HSEF_BOX_HI[kind] + 1e-12)


def test_hsef_fitness_is_the_lfv_of_an_l_run():
    # Eq. fit_h: the best H-fitness equals the LFV of an L-run with the best
    # H-position's hyper-parameters, on the same random streams (evolution 1).
    lcfg, sc, (best, bf, hist) = _small_hsef(1)
    G = lcfg.G
    h = np.zeros((G, 6))
    h[:, 0], h[:, 1], h[:, 2] = best[G:2 * G], best[2 * G:], 0.0
    # V_limit of the L-runs is passed as FP32 0.05, like every other input
    h[:, 3], h[:, 4], h[:, 5] = best[:G], best[:G], float(np.float32(0.05))
    res = oracle.Swarm(lcfg, h).plan(sc)
    assert res["cost"] == bf


# H-swarm update (Eqs. TOF_omega, TOF_V, TOF_X in the (w, C1, C2) space of Sec. 3.2.1),
# read from the H state after the last update.  After the first evolution every
# H-particle's personal best is its position, so the first update exercises inertia,
# the H-group best and the global best; the C1 term is pinned on the second update.

def _hsef_state(E, c1=0.0, c2=0.0, c3=0.0, w=0.0, vlim=50.0):
    lcfg = SepsoConfig(T=3, G=2, N=6, max_iters=8, alpha=30.0, beta=4)
    rng = np.random.default_rng(9)
    circ = np.column_stack([rng.uniform(60, 340, (6, 2)), rng.uniform(10, 30, 6)])
    sc = oracle.Scene((20, 20), (380, 380), circ)
    hh = np.zeros((4, 6))
    hh[:, 0], hh[:, 1], hh[:, 2], hh[:, 3], hh[:, 4], hh[:, 5] = c1, c2, c3, w, w, vlim
    return oracle.hsef_state(lcfg, sc, HG=4, HN=2, E=E, hhyper=hh, lo=HSEF_BOX_LO, hi=HSEF_BOX_HI,
                             l_vlimit=0.05, hseed=77)


def _box(G):
    lo = np.repeat(np.float32(HSEF_BOX_LO).astype(np.float64), G)
    hi = np.repeat(np.float32(HSEF_BOX_HI).astype(np.float64), G)
    return lo, hi


def _ratio(dv, toward):
    """Per H-particle: dv / toward over the coordinates where toward != 0."""
    out = []
    for h in range(dv.shape[0]):
        m = np.abs(toward[h]) > 1e-9
        out.append(dv[h, m] / toward[h, m] if m.any() else np.zeros(0))
    return out


def test_hsef_inertia_scales_the_velocity():
    v1 = _hsef_state(1, w=1.0)["HV"]
    v6 = _hsef_state(1, w=0.6)["HV"]
    assert np.abs(v1).max() > 0
    np.testing.assert_allclose(v6, 0.6 * v1, rtol=1e-12, atol=1e-12)


def test_hsef_group_and_global_attractors():
    # C2 pulls towards the H-particle's own H-group best, C3 towards the global best,
    # each with one random factor in [0, 1) per H-particle, the two factors distinct
    factors = {}
    for kw, row in (({"c2": 1.0}, "HGb"), ({"c3": 1.0}, "HTb")):
        st = _hsef_state(1, **kw)
        x0 = st["HP"]  # the first fitness improves every personal best from +inf
        target = st["HGb"][np.arange(8) // 2] if row == "HGb" else np.broadcast_to(st["HTb"], x0.shape)
        f = {}
        for h, r in enumerate(_ratio(st["HV"], target - x0)):
            if r.size:
                assert np.ptp(r) < 1e-9 and 0.0 <= r[0] < 1.0
                f[h] = r[0]
        assert f and max(f.values()) > 0.0  # the attractor acts
        factors[row] = f
        # a row that is the particle's own position gives no pull
        same = np.all(np.abs(target - x0) < 1e-12, axis=1)
        assert same.any() and np.all(st["HV"][same] == 0.0)
    both = set(factors["HGb"]) & set(factors["HTb"])
    assert both and all(factors["HGb"][h] != factors["HTb"][h] for h in both)


def test_hsef_velocity_is_the_sum_of_its_terms():
    parts = [_hsef_state(1, w=0.7)["HV"], _hsef_state(1, c2=0.9)["HV"], _hsef_state(1, c3=1.7)["HV"]]
    whole = _hsef_state(1, w=0.7, c2=0.9, c3=1.7)["HV"]
    np.testing.assert_allclose(whole, sum(parts), rtol=1e-12, atol=1e-12)


def test_hsef_personal_best_attractor_on_the_second_update():
    # C1 does not act on the first update (personal best = position), so two runs
    # that differ only in C1 reach the second update in the same state; the
    # velocity difference is C1 r1 (HP - HX) with one factor per H-particle
    # (w is constant, so the state after the first update is that of a one-evolution
    # run; the large V_limit keeps every velocity unclipped)
    base = dict(c2=0.8, c3=0.6, w=0.5)
    a, b = _hsef_state(2, **base), _hsef_state(2, c1=1.3, **base)
    x1 = _hsef_state(1, **base)["HX"]
    np.testing.assert_array_equal(a["HP"], b["HP"])
    dv = b["HV"] - a["HV"]
    ratios = _ratio(dv, a["HP"] - x1)
    seen = []
    for r in ratios:
        if r.size:
            assert np.ptp(r) < 1e-9 and 0.0 <= r[0] < 1.3
            seen.append(r[0])
    assert seen and max(seen) > 0.0


def test_hsef_positions_and_velocities_are_clipped():
    st = _hsef_state(1, w=0.7, c2=0.9, c3=1.7)
    lo, hi = _box(2)
    np.testing.assert_allclose(st["HX"], np.clip(st["HP"] + st["HV"], lo, hi), rtol=0, atol=1e-12)
    small = _hsef_state(1, w=0.7, c2=0.9, c3=1.7, vlim=0.01)
    assert np.all(np.abs(small["HV"]) <= 0.01 * (hi - lo) + 1e-12)
    assert np.any(np.abs(small["HV"]) >= 0.01 * (hi - lo) - 1e-12)

