"""Multi-agent teams on the batch planner (the paper's stated future work) vs the
FP64 oracle: agents of a team share a map, every agent's path enters its mates'
fitness as a moving obstacle (a conflict per mate and step in which the two come
closer than the separation), and the team plans in rounds of simultaneous best
responses, each a planning cycle with PI around the agent's own previous path.
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300 import BatchPlanner
from paper_2308_10169_gb300.inputs import team_workload

pytestmark = pytest.mark.gpu


def _gpu_rounds(specs, hyper, points, circles, first, size, sep, rounds):
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    bp.set_teams(first, size, sep)
    out = []
    for r in range(rounds):
        if r:
            bp.next_round(r)
        bp.run_async(True)
        out.append(bp.read())
    return out


def _oracle_team(specs, hyper, points, circles, m, A, sep, rounds):
    s0 = m * A
    cfg = specs[s0].config()
    return oracle.multi_agent_plan(cfg, hyper[s0], circles[s0], [points[s0 + a, :2] for a in range(A)],
                                   [points[s0 + a, 2:] for a in range(A)], sep, rounds)


@pytest.mark.parametrize("iters", [1, 2])
def test_team_rounds_first_iterations_match_oracle(native, iters):
    # every round stopped after 1-2 iterations: each agent's result after round 0
    # (alone) and after round 1 (against its mates' round-0 paths) vs the oracle's
    A, sep = 4, 25.0
    specs, hyper, points, circles, first, size = team_workload(1, n_teams=3, A=A, N=32, O=8, max_iters=iters,
                                                               stall_iters=0)
    g = _gpu_rounds(specs, hyper, points, circles, first, size, sep, 2)
    for m in range(3):
        o = _oracle_team(specs, hyper, points, circles, m, A, sep, 2)
        for r in range(2):
            for a in range(A):
                rg, ro = g[r][m * A + a], o[r][a]
                assert rg["iters"] == ro["iters"] == iters
                assert rg["Q"] == ro["Q"], (m, r, a)
                assert rg["cost"] == pytest.approx(ro["cost"], rel=1e-4)
                np.testing.assert_allclose(rg["waypoints"], ro["waypoints"], rtol=1e-5, atol=4e-3)


def test_teams_without_rounds_plan_alone(native):
    # before the first next_round the mates' paths do not count: results equal a
    # plain batch of the same scenes, bit for bit
    specs, hyper, points, circles, first, size = team_workload(2, n_teams=4, A=4, N=32, O=8, max_iters=40)
    a = _gpu_rounds(specs, hyper, points, circles, first, size, 25.0, 1)[0]
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    bp.run_async(True)
    b = bp.read()
    for x, y in zip(a, b):
        assert x["cost"] == y["cost"] and x["Q"] == y["Q"] and x["iters"] == y["iters"]
        np.testing.assert_array_equal(x["waypoints"], y["waypoints"])


def test_best_response_rounds_resolve_conflicts_like_the_oracle(native):
    # full rounds (AT stall 10, cap 100): planned alone the agents of a team all cross
    # the centre and conflict; after three rounds against each other most plans are
    # free of conflicts and collisions, on the GPU as with the oracle (4 teams of 4
    # agents; trajectories part, so the fractions and medians are compared)
    A, sep, R, M = 6, 25.0, 4, 6
    specs, hyper, points, circles, first, size = team_workload(3, n_teams=M, A=A, N=32, O=8)
    g = _gpu_rounds(specs, hyper, points, circles, first, size, sep, R)
    ora = [_oracle_team(specs, hyper, points, circles, m, A, sep, R) for m in range(M)]
    # the scenario needs the rounds: the oracle's own round-0 paths (planned alone)
    # conflict with each other
    T = specs[0].T
    n_conf = 0
    for m in range(M):
        paths = [oracle.timed_path(points[m * A + a, :2], points[m * A + a, 2:], ora[m][0][a]["waypoints"], T)
                 for a in range(A)]
        cfg = specs[m * A].config()
        for a in range(A):
            sc = oracle.Scene(points[m * A + a, :2], points[m * A + a, 2:], np.zeros((0, 3)),
                              agents=np.stack([paths[b] for b in range(A) if b != a]), sep=sep)
            n_conf += int(oracle.evaluate(cfg, sc, ora[m][0][a]["waypoints"].reshape(1, -1))[1][0])
    assert n_conf > 0
    for r in range(R):
        gq = np.array([x["Q"] for x in g[r]])
        oq = np.array([ora[m][r][a]["Q"] for m in range(M) for a in range(A)])
        gc = np.median([x["cost"] for x in g[r]])
        oc = np.median([ora[m][r][a]["cost"] for m in range(M) for a in range(A)])
        assert abs(np.mean(gq == 0) - np.mean(oq == 0)) <= 0.25, (r, np.mean(gq == 0), np.mean(oq == 0))
        assert abs(gc - oc) <= 0.05 * oc, (r, gc, oc)
    assert np.mean([x["Q"] == 0 for x in g[-1]]) >= 0.75
