"""The learned prior inside the serving loop (sepso_server_set_prior), through the C ABI.

At admission the server rasterises each request's scene, runs the prior, takes the
proposal at the request's T (itself when T equals the prior's, else resampled at
equal arc length along start -> proposal -> target) and seeds n_prior particles
per group around it when its fitness is below that of the agent's previous path
(the batch planner's gate).  The reference: the proposal from the Python prior API
on the same scene, the resampling restated below in FP64, the gate and the plan by
the FP64 oracle (Priori Initialization, Sec. 3.3.3, plus the second seed).
"""
import numpy as np
import pytest

import oracle
from paper_2308_10169_gb300 import Server
from paper_2308_10169_gb300._native import SepsoError
from paper_2308_10169_gb300.inputs import AT_STALL, SepsoConfig, prior_init_params, random_circles, sample_hyper

pytestmark = pytest.mark.gpu

G, N, TP, N_PRIOR = 3, 12, 20, 4


def _agents(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for a in range(n):
        T, O = int(rng.choice([1, 4, 8, 20, 40])), int(rng.choice([0, 8, 32, 64]))
        out.append(dict(T=T, O=O, circles=random_circles(rng, O, lo=20, hi=380, r_lo=5, r_hi=25),
                        hyper=sample_hyper(300 + a, G)))
    return out


def _scene(ag, k, step=7.0):
    c = ag["circles"].copy()
    c[:, 0] = np.clip(c[:, 0] + step * k, 0, 400)
    return np.array([20.0, 20.0 + k], np.float32), np.array([380.0, 380.0 - k], np.float32), c


def _prior(capacity):
    from paper_2308_10169_gb300.prior import Prior
    pr = Prior(T=TP, hidden1=256, hidden2=128, capacity=capacity, max_batch=64, max_circles=64)
    pr.set_params(prior_init_params(3, pr.K, 256, 128, 2 * TP, out_scale=1.0))
    return pr


def _serve(agents, ids, n_req, max_iters, stall, pr, max_slots=64):
    sv = Server(n_agents=max(ids) + 1, max_slots=max_slots, G=G, N=N, Tmax=40, Omax=64, max_iters=max_iters,
                stall_iters=stall, seed=5)
    sv.set_prior(pr, N_PRIOR, first_row=0)
    for a in ids:
        sv.set_hyper(agents[a]["hyper"], agent=a)
    for k in range(n_req):
        for a in ids:
            s, t, c = _scene(agents[a], k)
            sv.submit(a, agents[a]["T"], s, t, c, tag=a * 1000 + k)
    sv.drain()
    return sv, {d["tag"]: d for d in sv.poll(max_n=100000)}


def _resample(P, start, target, T):
    """The proposal at T waypoints: itself when T = TP, else the points at arc-length
    fractions i / (T + 1), i = 1..T, of the polyline start -> proposal -> target."""
    if T == TP:
        return np.asarray(P, np.float64)
    xs = np.concatenate([[start[0]], P[:TP], [target[0]]]).astype(np.float64)
    ys = np.concatenate([[start[1]], P[TP:], [target[1]]]).astype(np.float64)
    cum = np.concatenate([[0.0], np.cumsum(np.hypot(np.diff(xs), np.diff(ys)))])
    t = cum[-1] * np.arange(1, T + 1) / (T + 1)
    return np.concatenate([np.interp(t, cum, xs), np.interp(t, cum, ys)])


def test_resample_reference_is_a_polyline_walk():
    # the restatement used as the reference: straight proposals stay on the line at
    # equal spacing, the end points are never moved, T = TP is the identity
    line = np.concatenate([np.linspace(20, 380, TP + 2)[1:-1], np.linspace(20, 380, TP + 2)[1:-1]])
    for T in (1, 4, 8, 40):
        r = _resample(line, (20, 20), (380, 380), T)
        np.testing.assert_allclose(r[:T], np.linspace(20, 380, T + 2)[1:-1], atol=1e-9)
        np.testing.assert_allclose(r[:T], r[T:], atol=1e-9)
    P = np.random.default_rng(0).uniform(0, 400, 2 * TP)
    np.testing.assert_array_equal(_resample(P, (0, 0), (1, 1), TP), P)


def test_server_prior_seeds_match_oracle(native):
    agents = _agents(8, seed=11)
    ids = list(range(8))
    n_req = 3
    pr = _prior(capacity=64 + 8 * n_req)
    sv, done = _serve(agents, ids, n_req, max_iters=2, stall=10, pr=pr)
    assert len(done) == 8 * n_req
    row = 64
    checked, used = 0, 0
    for a in ids:
        ag = agents[a]
        T = ag["T"]
        cfg = SepsoConfig(T=T, G=G, N=N, max_obstacles=max(ag["O"], 1), alpha=30.0, beta=4, max_iters=2,
                          at_mode=AT_STALL, stall_iters=10, stall_tol=0.0, use_pi=True, pi_gamma=0.25,
                          pi_halfwidth=20.0, seed=5, run_id=a)
        sw = oracle.Swarm(cfg, ag["hyper"])
        for k in range(n_req):
            s, t, c = _scene(ag, k)
            pr.add_scenes(row, np.concatenate([s, t])[None], [c])
            P = pr.infer(row, 1).cpu().numpy()[0]
            row += 1
            prop = _resample(P, s, t, T)
            sc = oracle.Scene(s, t, c)
            if k == 0:
                use, amb = True, False
            else:
                f, _, _ = oracle.evaluate(cfg, sc, np.stack([prop, sw.s["prevT"]]))
                use, amb = bool(f[0] < f[1]), abs(f[0] - f[1]) <= 1e-3 * max(abs(f[1]), 1.0)
            if amb:
                break  # the two sides may take different branches from here on
            sw.load({"n_prior": [N_PRIOR if use else 0], "priorT": prop})
            o = sw.plan(sc)
            r = done[a * 1000 + k]
            assert r["iters"] == o["iters"] == 2
            assert r["Q"] == o["Q"], (a, k)
            assert r["cost"] == pytest.approx(o["cost"], rel=1e-4), (a, k)
            np.testing.assert_allclose(r["waypoints"][:2 * T], o["waypoints"], rtol=1e-5, atol=4e-3)
            checked += 1
            used += use
    assert checked >= 16 and 8 <= used < checked  # cold requests use it; some later ones do not


def test_server_prior_request_alone_equals_request_in_the_mix(native):
    agents = _agents(40, seed=12)
    pr = _prior(capacity=64)
    _, mix = _serve(agents, list(range(40)), 3, max_iters=40, stall=8, pr=pr, max_slots=16)
    for a in (0, 9, 31):
        _, alone = _serve(agents, [a], 3, max_iters=40, stall=8, pr=pr, max_slots=1)
        for k in range(3):
            x, y = alone[a * 1000 + k], mix[a * 1000 + k]
            assert x["cost"] == y["cost"] and x["iters"] == y["iters"] and x["Q"] == y["Q"], (a, k)
            np.testing.assert_array_equal(x["waypoints"], y["waypoints"])


def test_server_prior_attach_errors(native):
    sv = Server(n_agents=4, max_slots=8, G=G, N=N, Tmax=40, Omax=64, max_iters=5, seed=5)
    pr = _prior(capacity=8)
    with pytest.raises(SepsoError):
        sv.set_prior(pr, N_PRIOR, first_row=1)  # rows [1, 9) beyond the prior's 8
    with pytest.raises(SepsoError):
        sv.set_prior(pr, N + 1, first_row=0)  # more seeds than particles
    small = Server(n_agents=4, max_slots=8, G=G, N=N, Tmax=40, Omax=128, max_iters=5, seed=5)
    with pytest.raises(SepsoError):
        small.set_prior(pr, N_PRIOR, first_row=0)  # requests with more circles than it rasterises
    sv.set_prior(pr, N_PRIOR, first_row=0)
    sv.set_prior(None, 0)
