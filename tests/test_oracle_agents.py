"""The oracle's multi-agent extension (the paper's stated future work): agents share
a scene, each leaves its start with the others and reaches one point of its path
per time step, and another agent's path enters an agent's fitness as a moving
obstacle -- Q of Eq. penalty gains one conflict per (other agent, step) in which the
two come closer than the separation.  Pinned by hand cases, a brute-force sampling
of the two motions in time, and a two-agent swap that best-response rounds resolve.
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300.inputs import SepsoConfig, TABLE_HYPER8_PATH


def _q(T, start, target, wp, others, sep, circles=np.zeros((0, 3))):
    cfg = SepsoConfig(T=T, G=1, N=1, alpha=30.0, beta=1, max_obstacles=max(len(circles), 1))
    sc = oracle.Scene(start, target, circles, agents=np.asarray(others, np.float64), sep=sep)
    F, Q, L = oracle.evaluate(cfg, sc, np.asarray(wp, np.float64).reshape(1, -1))
    return int(Q[0]), float(F[0]), float(L[0])


def test_head_on_swap_conflicts_in_both_steps():
    # A: (0,0) -> (5,0) -> (10,0); B: (10,0) -> (5,0) -> (0,0), T = 1: both meet at
    # (5,0) at step 1; the relative motion passes through the origin in both steps
    b = oracle.timed_path((10, 0), (0, 0), [5, 0], 1)
    assert _q(1, (0, 0), (10, 0), [5, 0], [b], sep=1.0)[0] == 2
    # the same points one step apart in time: B waits at its start first
    b_late = oracle.timed_path((10, 0), (5, 0), [10, 0], 1)   # at (5,0) only at step 2
    q, F, L = _q(1, (0, 0), (10, 0), [5, 0], [b_late], sep=1.0)
    # step 0: rel (-10,0)->(-5,0), min 5; step 1: rel (-5,0)->(5,0) passes 0 -> 1 conflict
    assert q == 1
    assert F == pytest.approx(L + 30.0)


def test_parallel_lanes_and_the_strict_separation():
    T = 3
    wp = [10, 20, 30, 0, 0, 0]
    b = oracle.timed_path((0, 5), (40, 5), [10, 20, 30, 5, 5, 5], T)    # 5 apart all the time
    assert _q(T, (0, 0), (40, 0), wp, [b], sep=4.0)[0] == 0
    assert _q(T, (0, 0), (40, 0), wp, [b], sep=6.0)[0] == T + 1
    assert _q(T, (0, 0), (40, 0), wp, [b], sep=5.0)[0] == 0           # exactly sep apart is no conflict
    assert _q(T, (0, 0), (40, 0), wp, [b], sep=0.0)[0] == 0


def test_conflicts_add_to_obstacle_collisions_and_count_each_agent():
    T = 2
    wp = [100, 200, 100, 100]
    start, target = (0, 100), (300, 100)
    circles = np.array([[150.0, 100.0, 10.0]])                        # on segment 1
    b = oracle.timed_path((300, 100), (0, 100), [200, 100, 100, 100], T)
    q_obs = _q(T, start, target, wp, np.zeros((0, 2 * (T + 2))), 5.0, circles)[0]
    q_b = _q(T, start, target, wp, [b], 5.0)[0]
    assert q_obs == 1 and q_b >= 1
    assert _q(T, start, target, wp, [b], 5.0, circles)[0] == q_obs + q_b
    assert _q(T, start, target, wp, [b, b], 5.0, circles)[0] == q_obs + 2 * q_b


def test_conflicts_match_sampling_the_motions_in_time():
    # independent check: sample both agents' positions densely in time (straight
    # moves between consecutive points, one step per time unit) and compare the
    # closest approach per step with sep
    rng = np.random.default_rng(4)
    T = 4
    checked = 0
    for _ in range(300):
        s, t = rng.uniform(0, 100, 2), rng.uniform(0, 100, 2)
        wp = rng.uniform(0, 100, 2 * T)
        b = rng.uniform(0, 100, 2 * (T + 2))
        sep = rng.uniform(5, 40)
        own = oracle.timed_path(s, t, wp, T)
        P = T + 2
        want, near = 0, False
        for st in range(T + 1):
            u = np.linspace(0.0, 1.0, 20001)
            ax = own[st] + u * (own[st + 1] - own[st])
            ay = own[P + st] + u * (own[P + st + 1] - own[P + st])
            bx = b[st] + u * (b[st + 1] - b[st])
            by = b[P + st] + u * (b[P + st + 1] - b[P + st])
            d = np.hypot(ax - bx, ay - by).min()
            near |= abs(d - sep) < 1e-2
            want += d < sep
        if near:
            continue
        checked += 1
        assert _q(T, s, t, wp, [b], sep)[0] == want
    assert checked > 250


def test_best_response_rounds_resolve_a_swap():
    # two agents swapping ends of an empty map: planned alone, both take the straight
    # line and meet in the middle; against each other's paths (sep 30) the rounds
    # reach plans with no conflict that stay close to the straight length
    cfg = SepsoConfig(T=6, G=8, N=40, alpha=30.0, beta=4, max_iters=150, seed=2, max_obstacles=1)
    hy = np.ascontiguousarray(TABLE_HYPER8_PATH, np.float64)
    starts, targets = [(50, 200), (350, 200)], [(350, 200), (50, 200)]
    rounds = oracle.multi_agent_plan(cfg, hy, np.zeros((0, 3)), starts, targets, sep=30.0, rounds=4)
    first, last = rounds[0], rounds[-1]
    assert all(r["Q"] == 0 for r in first)            # alone: nothing to collide with
    paths = [oracle.timed_path(starts[a], targets[a], first[a]["waypoints"], cfg.T) for a in range(2)]
    assert _q(cfg.T, starts[0], targets[0], first[0]["waypoints"], [paths[1]], 30.0)[0] > 0
    assert all(r["Q"] == 0 for r in last)
    fin = [oracle.timed_path(starts[a], targets[a], last[a]["waypoints"], cfg.T) for a in range(2)]
    assert _q(cfg.T, starts[0], targets[0], last[0]["waypoints"], [fin[1]], 30.0)[0] == 0
    assert _q(cfg.T, starts[1], targets[1], last[1]["waypoints"], [fin[0]], 30.0)[0] == 0
    assert all(r["length"] < 1.25 * 300.0 for r in last)
