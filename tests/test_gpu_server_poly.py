"""Polygon requests in the continuous-batching server (sepso_server_submit_polygons:
the request's obstacles are polygon edges, Q counts proper crossings of path
segments and edges, Sec. 3.3.1) beside circle requests, vs the FP64 oracle through
the C ABI.

The oracle reference of an agent's k-th request is its k-th plan with the same seed
and run id (= agent), Priori Initialization around the agent's previous best path
(Sec. 3.3.3).  Tolerances as for the circle requests: cost 1e-4 relative, Q exact,
waypoints 1e-5 relative with a floor of 1e-5 x the map, for the agents whose
evaluated positions stay clear of flipping crossing decisions (more than 1e-6 of
the product of the lengths).
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300 import Server
from paper_2308_10169_gb300.inputs import AT_STALL, SepsoConfig, box, polygon_edges, random_circles, sample_hyper

pytestmark = pytest.mark.gpu

G, N, OMAX = 3, 12, 64


def _agents(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for a in range(n):
        poly = a % 3 != 2
        T = int(rng.choice([1, 4, 8, 20]))
        if poly:
            k = int(rng.choice([0, 2, 6, 10]))
            boxes = [box(*rng.uniform(60, 340, 2), *rng.uniform(10, 30, 2)) for _ in range(k)]
            obst = polygon_edges(boxes) if boxes else np.zeros((0, 4), np.float32)
        else:
            obst = random_circles(rng, int(rng.choice([0, 8, 32])), lo=20, hi=380, r_lo=5, r_hi=25)
        out.append(dict(T=T, poly=poly, obst=obst, hyper=sample_hyper(500 + a, G)))
    return out


def _scenes(ag, n_req, step=7.0):
    """The agent's scene per request: obstacles shifted along x by a fixed step."""
    out = []
    for k in range(n_req):
        o = ag["obst"].copy()
        o[:, 0] = np.clip(o[:, 0] + step * k, 0, 400)
        if ag["poly"]:
            o[:, 2] = np.clip(o[:, 2] + step * k, 0, 400)
        out.append((np.array([20.0, 20.0 + k], np.float32), np.array([380.0, 380.0 - k], np.float32), o))
    return out


def _cfg(ag, agent, max_iters, stall):
    return SepsoConfig(T=ag["T"], G=G, N=N, max_obstacles=max(len(ag["obst"]), 1), alpha=30.0, beta=4,
                       max_iters=max_iters, at_mode=AT_STALL, stall_iters=stall, stall_tol=0.0,
                       use_pi=True, pi_gamma=0.25, pi_halfwidth=20.0, seed=5, run_id=agent,
                       obstacle_kind=1 if ag["poly"] else 0)


def _oscene(ag, s, t, o):
    if ag["poly"]:
        return oracle.Scene(s, t, np.zeros((0, 3)), o)
    return oracle.Scene(s, t, o)


def _serve(agents, ids, n_req, max_iters, stall, max_slots=64):
    sv = Server(n_agents=max(ids) + 1, max_slots=max_slots, G=G, N=N, Tmax=40, Omax=OMAX,
                max_iters=max_iters, stall_iters=stall, seed=5)
    for a in ids:
        sv.set_hyper(agents[a]["hyper"], agent=a)
    for k in range(n_req):
        for a in ids:
            s, t, o = _scenes(agents[a], n_req)[k]
            if agents[a]["poly"]:
                sv.submit_polygons(a, agents[a]["T"], s, t, o, tag=a * 1000 + k)
            else:
                sv.submit(a, agents[a]["T"], s, t, o, tag=a * 1000 + k)
    sv.drain()
    return sv, {d["tag"]: d for d in sv.poll(max_n=100000)}


def _clear(cfg, sc, X, poly):
    X = np.asarray(X, np.float64).reshape(-1, cfg.D)
    if poly:
        return np.all(oracle.poly_margin(cfg, sc, X) > 1e-6)
    return np.all(oracle.tangency_margin(cfg, sc, X) > 1e-3)


def _plan_checked(sw, cfg, sc, poly):
    """One planning cycle of the oracle, step by step as its plan call takes it, or
    None once an evaluated position came within the margin of a flipping decision."""
    st = sw.s
    if st["cycle"][0] == 0:
        st["win_n"][0] = st["win_head"][0] = 0
    st["stall"][0] = 0
    st["prev_lfv"][0] = np.inf
    sw.init()
    while True:
        if not _clear(cfg, sc, st["X"], poly):
            return None
        if sw.iteration(sc, check_stop=True):
            break
    st["prevT"][...] = st["Tb"]
    st["has_prev"][0] = 1
    st["cycle"][0] += 1
    return {"cost": float(st["Tfit"][0]), "Q": int(st["TQ"][0]), "iters": int(st["k"][0]),
            "waypoints": st["Tb"].copy()}


def test_polygon_requests_match_oracle_first_iterations(native):
    agents = _agents(12)
    ids = list(range(12))
    sv, done = _serve(agents, ids, n_req=3, max_iters=2, stall=10)
    assert len(done) == 36
    checked = polys = 0
    for a in ids:
        ag = agents[a]
        cfg = _cfg(ag, a, 2, 10)
        sw = oracle.Swarm(cfg, ag["hyper"])
        plans = [_plan_checked(sw, cfg, _oscene(ag, s, t, o), ag["poly"]) for s, t, o in _scenes(ag, 3)]
        if any(p is None for p in plans):
            continue
        checked += 1
        polys += ag["poly"]
        for k, o in enumerate(plans):
            r = done[a * 1000 + k]
            assert r["agent"] == a and r["iters"] == o["iters"] == 2
            assert r["Q"] == o["Q"], (a, k)
            assert r["cost"] == pytest.approx(o["cost"], rel=1e-4), (a, k)
            np.testing.assert_allclose(r["waypoints"], o["waypoints"], rtol=1e-5, atol=4e-3)
    assert checked >= 6 and polys >= 4


def test_polygon_request_alone_equals_request_in_the_mix(native):
    agents = _agents(30, seed=1)
    _, mix = _serve(agents, list(range(30)), n_req=3, max_iters=60, stall=8, max_slots=12)
    for a in (0, 4, 7):
        assert agents[a]["poly"]
        _, alone = _serve(agents, [a], n_req=3, max_iters=60, stall=8, max_slots=1)
        for k in range(3):
            x, y = alone[a * 1000 + k], mix[a * 1000 + k]
            assert x["cost"] == y["cost"] and x["iters"] == y["iters"] and x["Q"] == y["Q"]
            np.testing.assert_array_equal(x["waypoints"], y["waypoints"])


def test_polygon_request_argument_checks(native):
    sv = Server(n_agents=2, max_slots=4, G=G, N=N, Tmax=40, Omax=OMAX, max_iters=5, stall_iters=3, seed=5)
    s, t = np.array([20.0, 20.0], np.float32), np.array([380.0, 380.0], np.float32)
    e = polygon_edges([box(200, 200, 20, 20)])
    with pytest.raises(RuntimeError, match="edges"):
        sv.submit_polygons(0, 8, s, t, np.zeros((OMAX + 1, 4), np.float32), tag=1)
    bad = e.copy()
    bad[1, 3] = np.inf
    with pytest.raises(RuntimeError, match="edge"):
        sv.submit_polygons(0, 8, s, t, bad, tag=1)
    sv.submit_polygons(0, 8, s, t, e, tag=1)
    sv.drain()
    assert len(sv.poll()) == 1
