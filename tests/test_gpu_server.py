"""Continuous-batching server (sepso_server_*) vs the FP64 oracle, through the C ABI.

A request is one planning cycle of its agent: Priori Initialization around the
agent's previous best path (Sec. 3.3.3), Algorithm 1, Auto Truncation by stall
counter (Sec. 3.3.4) or the cap.  The oracle reference of an agent's k-th request
is its k-th plan with the same seed and run id (= agent).
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300 import Server
from paper_2308_10169_gb300.inputs import AT_STALL, SepsoConfig, random_circles, sample_hyper

pytestmark = pytest.mark.gpu

G, N = 3, 12


def _agent(a, rng, T, O):
    return dict(T=T, O=O, circles=random_circles(rng, O, lo=20, hi=380, r_lo=5, r_hi=25),
                hyper=sample_hyper(300 + a, G))


def _scenes(ag, n_req, step=7.0):
    """The agent's scene per request: circles shifted by a fixed step each time."""
    out = []
    for k in range(n_req):
        c = ag["circles"].copy()
        c[:, 0] = np.clip(c[:, 0] + step * k, 0, 400)
        out.append((np.array([20.0, 20.0 + k], np.float32), np.array([380.0, 380.0 - k], np.float32), c))
    return out


def _cfg(ag, agent, max_iters, stall, tol=0.0):
    return SepsoConfig(T=ag["T"], G=G, N=N, max_obstacles=max(ag["O"], 1), alpha=30.0, beta=4,
                       max_iters=max_iters, at_mode=AT_STALL, stall_iters=stall, stall_tol=tol,
                       use_pi=True, pi_gamma=0.25, pi_halfwidth=20.0, seed=5, run_id=agent)


def _serve(agents, ids, n_req, max_iters, stall, max_slots=64, mem_budget=0, tol=0.0):
    sv = Server(n_agents=max(ids) + 1, max_slots=max_slots, G=G, N=N, Tmax=40, Omax=64,
                max_iters=max_iters, stall_iters=stall, stall_tol=tol, seed=5, mem_budget=mem_budget)
    for a in ids:
        sv.set_hyper(agents[a]["hyper"], agent=a)
    tag = 0
    for k in range(n_req):
        for a in ids:
            s, t, c = _scenes(agents[a], n_req)[k]
            sv.submit(a, agents[a]["T"], s, t, c, tag=a * 1000 + k)
            tag += 1
    sv.drain()
    done = {d["tag"]: d for d in sv.poll(max_n=100000)}
    return sv, done


def _agents(n, seed=0):
    rng = np.random.default_rng(seed)
    return [_agent(a, rng, T=int(rng.choice([1, 4, 8, 20, 40])), O=int(rng.choice([0, 8, 32, 64])))
            for a in range(n)]


def test_server_requests_match_oracle_first_iterations(native):
    agents = _agents(8)
    ids = list(range(8))
    sv, done = _serve(agents, ids, n_req=3, max_iters=2, stall=10)
    assert len(done) == 24
    for a in ids:
        sw = oracle.Swarm(_cfg(agents[a], a, 2, 10), agents[a]["hyper"])
        for k, (s, t, c) in enumerate(_scenes(agents[a], 3)):
            o = sw.plan(oracle.Scene(s, t, c))
            r = done[a * 1000 + k]
            assert r["agent"] == a and r["iters"] == o["iters"] == 2
            assert r["Q"] == o["Q"], (a, k)
            assert r["cost"] == pytest.approx(o["cost"], rel=1e-4), (a, k)
            np.testing.assert_allclose(r["waypoints"], o["waypoints"], rtol=1e-5, atol=4e-3)


def test_request_alone_equals_request_in_the_mix(native):
    agents = _agents(40, seed=1)
    _, mix = _serve(agents, list(range(40)), n_req=3, max_iters=60, stall=8, max_slots=16)
    for a in (0, 7, 23):
        _, alone = _serve(agents, [a], n_req=3, max_iters=60, stall=8, max_slots=1)
        for k in range(3):
            x, y = alone[a * 1000 + k], mix[a * 1000 + k]
            assert x["cost"] == y["cost"] and x["iters"] == y["iters"] and x["Q"] == y["Q"]
            np.testing.assert_array_equal(x["waypoints"], y["waypoints"])


def test_admission_by_memory_budget(native):
    agents = _agents(24, seed=2)
    big = Server(n_agents=24, max_slots=64, G=G, N=N, Tmax=40, Omax=64)
    small_budget = big.workspace.numel() // 6
    sv, done = _serve(agents, list(range(24)), n_req=2, max_iters=20, stall=5, max_slots=64,
                      mem_budget=small_budget)
    st = sv.stats()
    assert st["slots"] < 64 and sv.workspace.numel() <= small_budget
    assert st["completed"] == st["admitted"] == 48 and len(done) == 48


def test_truncation_and_median_cost(native):
    # Stall-counter AT with a tolerance of 1 length unit: easy scenes stop early once
    # collision-free; the median cost of the served plans matches the oracle's within
    # 2% (FP32 and FP64 trajectories separate over many iterations, so medians are
    # compared).
    rng = np.random.default_rng(3)
    agents = [_agent(a, rng, T=8, O=6) for a in range(24)]
    _, done = _serve(agents, list(range(24)), n_req=2, max_iters=150, stall=10, tol=1.0)
    gi = [d["iters"] for d in done.values()]
    assert np.median(gi) < 150
    for d in done.values():
        if d["iters"] < 150:
            assert d["Q"] == 0
    gpu, ora = [], []
    for a in range(24):
        sw = oracle.Swarm(_cfg(agents[a], a, 150, 10, tol=1.0), agents[a]["hyper"])
        for k, (s, t, c) in enumerate(_scenes(agents[a], 2)):
            ora.append(sw.plan(oracle.Scene(s, t, c))["cost"])
            gpu.append(done[a * 1000 + k]["cost"])
    assert abs(np.median(gpu) - np.median(ora)) <= 0.02 * np.median(ora)
