"""Learned prior on the GPU vs plain references, through the C ABI.

* the tensor-core GEMM (tcgen05, BF16 in, FP32 accumulate) vs a plain PyTorch
  FP32 matmul of the same BF16 values on the CPU;
* features, labels, forward pass and loss gradient of the MLP vs the FP64 oracle
  (prior_oracle.c), which computes its own features from the same scenes;
* one Adam step vs the closed form of Adam's first step on the oracle gradient;
* training lowers the loss;
* the network trained on the planner's own solutions gains over the PI-only start
  on held-out scenes, its proposals judged by the oracle's fitness.

Tolerances.  The GEMM accumulates in FP32: |error| <= K * 2^-24 * sum |a||b|, far
below the 1e-4 relative bound used.  The MLP rounds its weights and activations
to BF16 (8 significant bits, relative rounding error <= 2^-9 per value) before
each tensor-core product; with the oracle given the same BF16 weights, the
remaining differences are the activation roundings, which average out over the
sums: a relative (Frobenius) error of a few 1e-3 per layer.  The bar is 2e-2 per
tensor with a cosine similarity >= 0.999.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2308_10169_gb300.inputs import prior_init_params, prior_scenes
from paper_2308_10169_gb300.prior import Prior, gemm_bf16

pytestmark = pytest.mark.gpu

T, G64, H1, H2 = 20, 64, 1024, 512


def _bf16_values(a: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (200, 136, 200), (40, 512, 256), (13, 7, 8),
                                   (256, 1024, 4104), (1024, 520, 96)])
def test_gemm_matches_fp32_reference(native, M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = (A.double() @ B.double().T)
    Cf, _ = gemm_bf16(A.cuda(), B.cuda())
    got = Cf.cpu().double()
    tol = 1e-4 * np.sqrt(K)
    assert torch.max(torch.abs(got - ref)).item() <= tol


@pytest.mark.parametrize("tile_n", [64, 128, 256, -64, -128, -256])
def test_gemm_tile_widths_agree(native, tile_n):
    # every tile width of the two kernels (positive: persistent with two
    # accumulators; -64 .. -256: one tile per CTA) gives the same products (ragged
    # M, N and K; K spans several pipeline stages and wraps the stage ring; several
    # tiles per CTA; 19 row tiles)
    g = torch.Generator().manual_seed(tile_n)
    M, N, K = 2333, 1300, 1096
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    Cf, _ = gemm_bf16(A.cuda(), B.cuda(), tile_n=tile_n)
    assert torch.max(torch.abs(Cf.cpu().double() - ref)).item() <= 1e-4 * np.sqrt(K)


def test_gemm_epilogue_bias_relu_mask_bf16(native):
    g = torch.Generator().manual_seed(9)
    M, N, K = 300, 260, 136
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    mask = (torch.rand(M, N, generator=g) > 0.5).to(torch.bfloat16)
    pre = 0.5 * (A.double() @ B.double().T) + bias.double()
    Cf, Cb = gemm_bf16(A.cuda(), B.cuda(), alpha=0.5, bias=bias.cuda(), relu=True, mask=mask.cuda(),
                       out_bf16=True)
    ref = torch.where(mask.double() > 0, torch.clamp(pre, min=0), torch.zeros_like(pre))
    assert torch.max(torch.abs(Cf.cpu().double() - ref)).item() <= 1e-4 * np.sqrt(K)
    # the BF16 output is the FP32 result rounded to nearest
    assert torch.equal(Cb.cpu(), Cf.cpu().to(torch.bfloat16))


@pytest.mark.parametrize("tile_n", [0, 64, 128, 256, -64, -128, -256])
@pytest.mark.parametrize("M,N,K", [(300, 260, 136), (4096, 512, 40), (77, 1000, 512)])
def test_gemm_transposed_output_and_column_sums(native, tile_n, M, N, K):
    # the backward pass's masked products: the BF16 output transposed and the
    # column sums of the output, from both kernels' epilogues (ragged M and N,
    # rows beyond M excluded from the sums, several 32-row slabs per tile)
    g = torch.Generator().manual_seed(M + N + K + tile_n)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    mask = (torch.rand(M, N, generator=g) > 0.5).to(torch.bfloat16)
    pre = 0.5 * (A.double() @ B.double().T) + bias.double()
    ref = torch.where(mask.double() > 0, torch.clamp(pre, min=0), torch.zeros_like(pre))
    Cf, Cb, Ct, cs = gemm_bf16(A.cuda(), B.cuda(), alpha=0.5, bias=bias.cuda(), relu=True, mask=mask.cuda(),
                               out_bf16=True, out_t=True, colsum=True, tile_n=tile_n)
    assert torch.max(torch.abs(Cf.cpu().double() - ref)).item() <= 1e-4 * np.sqrt(K)
    # the transposed copy holds exactly the BF16 output's values
    assert torch.equal(Ct.cpu(), Cb.cpu().T)
    # column sums of the FP32 output (32-row slabs in order, then the slabs): at most
    # 32 + ceil(M / 32) FP32 additions per sum of non-negative terms (ReLU), so the
    # error is below (32 + 128) * 2^-24 * sum < 1e-5 * sum
    want = Cf.cpu().double().sum(0)
    assert torch.allclose(cs.cpu().double(), want, rtol=2e-5, atol=1e-6)


@pytest.mark.parametrize("M,N,K,ksplit,tile_n", [(40, 512, 4096, 16, -64), (512, 1024, 4096, 4, -128),
                                                 (130, 70, 1000, 5, 0), (200, 300, 64, 3, -256)])
def test_gemm_split_k_matches_reference(native, M, N, K, ksplit, tile_n):
    # K in slices (the last one ragged; more slices asked than K has blocks), the
    # FP32 products summed in slice order before the epilogue
    g = torch.Generator().manual_seed(K + ksplit)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    mask = (torch.rand(M, N, generator=g) > 0.3).to(torch.bfloat16)
    pre = 2.0 * (A.double() @ B.double().T) + bias.double()
    ref = torch.where(mask.double() > 0, torch.clamp(pre, min=0), torch.zeros_like(pre))
    Cf, Cb, _, _ = gemm_bf16(A.cuda(), B.cuda(), alpha=2.0, bias=bias.cuda(), relu=True, mask=mask.cuda(),
                             out_bf16=True, ksplit=ksplit, tile_n=tile_n)
    assert torch.max(torch.abs(Cf.cpu().double() - ref)).item() <= 2e-4 * np.sqrt(K)
    assert torch.equal(Cb.cpu(), Cf.cpu().to(torch.bfloat16))
    one, _ = gemm_bf16(A.cuda(), B.cuda(), alpha=2.0, bias=bias.cuda(), relu=True, mask=mask.cuda(),
                       tile_n=tile_n)
    assert torch.max(torch.abs(Cf.cpu() - one.cpu())).item() <= 2e-4 * np.sqrt(K)


def _scenes(seed, n):
    sc = prior_scenes(seed, n)
    return sc, [sc["circles"][i] for i in range(n)]


def _paths(seed, n):
    rng = np.random.default_rng(500 + seed)
    return rng.uniform(0, 400, (n, 2 * T)).astype(np.float32)


def _oracle_params(p32: np.ndarray, m: oracle.Mlp) -> np.ndarray:
    """The network the GPU evaluates: BF16 weight matrices, FP32 biases."""
    p = p32.astype(np.float64).copy()
    parts = m.split(p)
    for w in ("W1", "W2", "W3"):
        parts[w][...] = _bf16_values(parts[w])
    return p


def _oracle_features(sc, i):
    p = sc["points"][i]
    return oracle.raster(G64, 400.0, 400.0, sc["circles"][i], p[:2], p[2:], 4104)


def test_features_and_labels_match_oracle(native):
    n = 40
    sc, circ = _scenes(1, n)
    circ[3] = np.zeros((0, 3), np.float32)  # a scene without obstacles
    wp = _paths(1, n)
    pr = Prior(T=T, capacity=64, max_batch=32)
    pr.add_scenes(8, sc["points"], circ, wp)
    f, y = pr.get_rows(8, n)
    for i in range(n):
        p = sc["points"][i]
        ref = oracle.raster(G64, 400.0, 400.0, circ[i], p[:2], p[2:], 4104)
        np.testing.assert_array_equal(f[i, :4096], ref[:4096])
        np.testing.assert_allclose(f[i, 4096:4100], ref[4096:4100], rtol=2 ** -8)
        assert not f[i, 4100:].any()
        lab = oracle.prior_encode(T, 400.0, 400.0, p[:2], p[2:], wp[i])
        np.testing.assert_allclose(y[i], lab, rtol=1e-5, atol=1e-6)


def _prior_with_data(n, seed, capacity=64, max_batch=64):
    sc, circ = _scenes(seed, n)
    wp = _paths(seed, n)
    pr = Prior(T=T, capacity=capacity, max_batch=max_batch)
    pr.add_scenes(0, sc["points"], circ, wp)
    m = oracle.Mlp(4104, H1, H2, 2 * T)
    params = prior_init_params(seed, 4104, H1, H2, 2 * T, out_scale=1.0)
    pr.set_params(params)
    X = np.stack([_oracle_features(sc, i) for i in range(n)])
    Y = np.stack([oracle.prior_encode(T, 400.0, 400.0, sc["points"][i, :2], sc["points"][i, 2:], wp[i])
                  for i in range(n)])
    return pr, m, params, X, Y


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_matches_oracle(native):
    n = 21  # ragged: not a multiple of 8 or of the 128-row tile
    pr, m, params, X, _ = _prior_with_data(n, 2, max_batch=16)  # two chunks
    y = pr.forward(0, n)
    _, _, yo = m.forward(_oracle_params(params, m), X)
    assert _rel(y, yo) < 2e-2
    for i in range(n):
        cos = np.dot(y[i], yo[i]) / (np.linalg.norm(y[i]) * np.linalg.norm(yo[i]))
        assert cos > 0.999


def test_gradient_matches_oracle(native):
    n = 24
    pr, m, params, X, Y = _prior_with_data(n, 3)
    g, loss = pr.grad(0, n)
    lo, go = m.loss_grad(_oracle_params(params, m), X, Y)
    assert loss == pytest.approx(lo, rel=2e-2)
    gs, gos = m.split(g), m.split(go)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        a, b = gs[name].ravel().astype(np.float64), gos[name].ravel()
        assert _rel(a, b) < 2e-2, name
        assert np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.999, name


def test_first_adam_step_is_signed_learning_rate(native):
    # Adam's first step is lr * g / (|g| + eps): -lr * sign(g) wherever |g| >> eps.
    n = 16
    pr, m, params, X, Y = _prior_with_data(n, 4)
    _, go = m.loss_grad(_oracle_params(params, m), X, Y)
    pr.train(steps=1, batch=n, first=0)
    w1 = pr.get_params().astype(np.float64)
    step = w1 - params.astype(np.float64)
    lr = 1e-3
    # entries whose oracle gradient is clearly away from zero (GPU and oracle agree
    # on the sign there): the step is -lr * sign(g) up to FP32 rounding of w
    big = np.abs(go) > 0.05 * np.abs(go).max()
    assert big.sum() > 1000
    np.testing.assert_allclose(step[big], -lr * np.sign(go[big]), rtol=0,
                               atol=4 * np.finfo(np.float32).eps * (np.abs(params[big]).max() + lr))
    assert np.all(np.abs(step) <= lr * (1 + 1e-3) + 4 * np.finfo(np.float32).eps * np.abs(params).max())


def test_training_lowers_the_loss(native):
    n = 256
    pr, _, _, _, _ = _prior_with_data(n, 5, capacity=n, max_batch=64)
    losses = pr.train(steps=300, batch=64, n_rows=n, seed=11)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.5 * losses[:5].mean()
    pr.sync()


def test_trained_prior_gains_over_pi_only(native):
    # The prior trained on the planner's own solutions (self-training rounds) vs the
    # method without it, on held-out scenes of the dynamic workload's kind:
    # cold start (no previous path), iteration budgets, and a short dynamic run.
    # The oracle's fitness judges the proposals themselves.
    from paper_2308_10169_gb300.prior import evaluate_prior, fit_prior
    ntr, nev = 4096, 256
    tr, ev = prior_scenes(20, ntr), prior_scenes(21, nev)
    pr = Prior(T=T, capacity=ntr + nev, max_batch=512)
    init = prior_init_params(0, pr.K, H1, H2, 2 * T)
    pr.set_params(init)
    # proposals of the untrained network, judged by the oracle
    untrained = _oracle_judge(pr, ev, ntr)
    hist = fit_prior(pr, tr, rounds=3, epochs=30, batch=512, seed=1)
    assert hist["label_cost"][-1] < 0.6 * hist["label_cost"][0]
    trained = _oracle_judge(pr, ev, ntr)
    assert np.median(trained) < np.median(untrained)
    res = evaluate_prior(pr, ev, ntr, budgets=(10, 50, 300), cycles=3)
    cold = res["cold"]
    assert cold["prior_pi"]["cost_median"] < 0.6 * cold["pi_only"]["cost_median"]
    assert cold["prior_pi"]["collision_free"] >= cold["pi_only"]["collision_free"]
    conv = res["iters_to_converge"]
    assert conv["prior_pi"] == 10 and (conv["pi_only"] is None or conv["pi_only"] > 10)
    last = {m: res["dynamic"][m][-1]["cost_median"] for m in ("pi_only", "prior_pi")}
    assert last["prior_pi"] < last["pi_only"]


def _oracle_judge(pr, ev, first):
    """Oracle fitness (Sec. 3.3.2, FP64) of the prior's proposed paths."""
    from paper_2308_10169_gb300.inputs import SepsoConfig
    from paper_2308_10169_gb300.prior import propose
    wp = propose(pr, ev, first).cpu().numpy()
    cfg = SepsoConfig(T=T, G=1, N=1, max_obstacles=64, alpha=30.0, beta=4)
    out = []
    for i in range(wp.shape[0]):
        p = ev["points"][i]
        f, _, _ = oracle.evaluate(cfg, oracle.Scene(p[:2], p[2:], ev["circles"][i]), wp[i])
        out.append(f[0])
    return np.array(out)
