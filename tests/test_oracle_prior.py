"""Pins of the learned-prior oracle (prior_oracle.c) against values fixed by
hand, by closed forms and by finite differences -- never against itself."""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle

GOLD = Path(__file__).parent / "golden" / "mlp_hand.json"


def _flat(d, names=("W1", "b1", "W2", "b2", "W3", "b3")):
    return np.concatenate([np.asarray(d[n], np.float64).ravel() for n in names])


def test_hand_worked_forward_and_gradient():
    g = json.loads(GOLD.read_text())
    m = oracle.Mlp(**g["dims"])
    p = _flat(g)
    h1, h2, y = m.forward(p, g["x"])
    np.testing.assert_array_equal(h1, g["h1"])
    np.testing.assert_array_equal(h2, g["h2"])
    np.testing.assert_array_equal(y, g["y"])
    loss, grad = m.loss_grad(p, g["x"], g["target"])
    assert loss == g["loss"]
    np.testing.assert_array_equal(grad, _flat(g, ("gW1", "gb1", "gW2", "gb2", "gW3", "gb3")))


def _random_net(rng, K=9, H1=7, H2=5, O=4, B=3):
    m = oracle.Mlp(K, H1, H2, O)
    p = rng.normal(0, 0.6, m.num_params)
    X = rng.normal(0, 1, (B, K))
    T = rng.normal(0, 1, (B, O))
    return m, p, X, T


def test_forward_matches_numpy_matmul():
    rng = np.random.default_rng(0)
    m, p, X, _ = _random_net(rng, K=33, H1=17, H2=11, O=6, B=5)
    w = m.split(p)
    h1 = np.maximum(X @ w["W1"].T + w["b1"], 0)
    h2 = np.maximum(h1 @ w["W2"].T + w["b2"], 0)
    y = h2 @ w["W3"].T + w["b3"]
    a1, a2, ay = m.forward(p, X)
    np.testing.assert_allclose(a1, h1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a2, h2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(ay, y, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(seed)
    m, p, X, T = _random_net(rng)
    loss, g = m.loss_grad(p, X, T)
    eps = 1e-6
    num = np.zeros_like(p)
    for i in range(p.size):
        q = p.copy()
        q[i] += eps
        lp, _ = m.loss_grad(q, X, T)
        q[i] -= 2 * eps
        lm, _ = m.loss_grad(q, X, T)
        num[i] = (lp - lm) / (2 * eps)
    # a ReLU kink inside +-eps of a pre-activation would break the difference; with
    # these draws every pre-activation is far from 0 relative to eps
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-8)
    _, _, y = m.forward(p, X)
    assert loss == pytest.approx(0.5 * np.sum((y - T) ** 2) / X.shape[0], rel=1e-14)


def test_gradient_vanishes_at_the_targets():
    rng = np.random.default_rng(4)
    m, p, X, _ = _random_net(rng)
    _, _, y = m.forward(p, X)
    loss, g = m.loss_grad(p, X, y)
    assert loss == 0.0 and not np.any(g)


def test_adam_first_steps_closed_form():
    # Kingma and Ba, Algorithm 1: after step 1, m_hat = g and v_hat = g^2, so the
    # step is lr * g / (|g| + eps); a constant gradient keeps m_hat = g, v_hat = g^2.
    rng = np.random.default_rng(5)
    n = 64
    w0, g = rng.normal(size=n), rng.normal(size=n)
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    w, mm, vv = oracle.adam(w0, np.zeros(n), np.zeros(n), g, lr, b1, b2, eps, 1)
    np.testing.assert_allclose(w, w0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    np.testing.assert_allclose(mm, (1 - b1) * g, rtol=1e-15)
    np.testing.assert_allclose(vv, (1 - b2) * g * g, rtol=1e-15)
    w2, m2, v2 = oracle.adam(w, mm, vv, g, lr, b1, b2, eps, 2)
    np.testing.assert_allclose(w2, w0 - 2 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)
    np.testing.assert_allclose(m2, (1 - b1 ** 2) * g, rtol=1e-14)


def _disk_cells(grid, W, cx, cy, r):
    """Cells of a g x g grid over [0, W]^2 whose centre lies in one disk, counted
    row by row from the chord half-width (floor/ceil of the chord ends)."""
    cw = W / grid
    n = 0
    for i in range(grid):
        y = (i + 0.5) * cw
        h2 = r * r - (y - cy) ** 2
        if h2 < 0:
            continue
        h = math.sqrt(h2)
        lo = math.ceil((cx - h) / cw - 0.5)
        hi = math.floor((cx + h) / cw - 0.5)
        n += max(0, min(hi, grid - 1) - max(lo, 0) + 1)
    return n


@pytest.mark.parametrize("cx,cy,r", [(200.3, 190.7, 37.1), (13.0, 388.0, 55.5), (101.1, 250.9, 8.3)])
def test_raster_single_disk_lattice_count(cx, cy, r):
    # centres and radii chosen away from cell centres so the FP32 decision agrees
    # with the exact one
    f = oracle.raster(64, 400.0, 400.0, [[cx, cy, r]], (20, 20), (380, 380), 4104)
    assert int(f[:4096].sum()) == _disk_cells(64, 400.0, cx, cy, r)
    assert set(np.unique(f[:4096])) <= {0.0, 1.0}


def test_raster_features_and_degenerate_scenes():
    f = oracle.raster(64, 400.0, 300.0, np.zeros((0, 3)), (20, 30), (380, 270), 4104)
    assert not f[:4096].any()
    np.testing.assert_array_equal(f[4096:4100], [20 / 400, 30 / 300, 380 / 400, 270 / 300])
    assert not f[4100:].any()
    full = oracle.raster(64, 400.0, 400.0, [[200, 200, 300]], (0, 0), (400, 400), 4104)
    assert full[:4096].all()
    # cell (i, j) is row i (y) and column j (x)
    one = oracle.raster(64, 400.0, 400.0, [[3 * 6.25 + 3.125, 10 * 6.25 + 3.125, 1.0]], (0, 0), (1, 1), 4104)
    assert np.flatnonzero(one[:4096]).tolist() == [10 * 64 + 3]


def test_label_encoding():
    T, W, H = 5, 400.0, 300.0
    s, t = (20.0, 30.0), (380.0, 250.0)
    f = np.arange(1, T + 1) / (T + 1)
    line = np.concatenate([s[0] + f * (t[0] - s[0]), s[1] + f * (t[1] - s[1])])
    np.testing.assert_allclose(oracle.prior_encode(T, W, H, s, t, line), 0, atol=1e-13)
    np.testing.assert_allclose(oracle.prior_decode(T, W, H, s, t, np.zeros(2 * T)), line, rtol=1e-15)
    rng = np.random.default_rng(6)
    wp = np.concatenate([rng.uniform(0, W, T), rng.uniform(0, H, T)])
    np.testing.assert_allclose(oracle.prior_decode(T, W, H, s, t, oracle.prior_encode(T, W, H, s, t, wp)), wp,
                               rtol=1e-12)
    far = oracle.prior_decode(T, W, H, s, t, np.full(2 * T, 5.0))
    np.testing.assert_array_equal(far, np.concatenate([np.full(T, W), np.full(T, H)]))
