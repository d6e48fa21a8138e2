"""Python binding of the learned prior (``sepso_prior_*``) and of the tensor-core
GEMM (``sepso_gemm_bf16``) -- argument marshalling only; every step runs in the
CUDA library.

The prior is a small MLP that maps a scene (occupancy raster + start/target) to a
proposed path, used beside Priori Initialization (Sec. 3.3.3) to seed a cycle's
particles; the paper itself has no learned component.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import check_prior


def _dev(device=None) -> torch.device:
    if not torch.cuda.is_available():
        raise RuntimeError("the SEPSO prior needs a CUDA device (there is no CPU path)")
    return torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())


def _f32(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    return a.reshape(shape) if shape is not None else a


class Prior:
    """MLP x (g*g raster + start/target) -> hidden1 -> hidden2 -> 2T with BF16
    tensor-core kernels, FP32 masters and Adam; dataset rows held on the device."""

    def __init__(self, T: int = 20, grid: int = 64, hidden1: int = 1024, hidden2: int = 512,
                 max_batch: int = 4096, capacity: int = 4096, max_circles: int = 1024,
                 map_w: float = 400.0, map_h: float = 400.0, lr: float = 1e-3, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8, device=None):
        self.device = _dev(device)
        self.cfg = _native.PriorConfig(T=T, grid=grid, hidden1=hidden1, hidden2=hidden2,
                                       max_batch=max_batch, capacity=capacity, max_circles=max_circles,
                                       map_w=map_w, map_h=map_h, lr=lr, beta1=beta1, beta2=beta2, eps=eps)
        self.T, self.grid, self.H1, self.H2 = T, grid, hidden1, hidden2
        self.K = (grid * grid + 4 + 7) // 8 * 8
        self.O = 2 * T
        self.capacity, self.max_batch = capacity, max_batch
        L = _native.lib()
        size = ctypes.c_size_t()
        check_prior(L.sepso_prior_workspace_size(ctypes.byref(self.cfg), ctypes.byref(size)))
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        check_prior(L.sepso_prior_create(ctypes.byref(self.cfg), ctypes.c_void_p(self.workspace.data_ptr()),
                                         size.value, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _native.lib().sepso_prior_destroy(h)
            self._h = None

    @property
    def num_params(self) -> int:
        return int(_native.lib().sepso_prior_num_params(self._h))

    def set_params(self, params) -> None:
        p = _f32(params, (self.num_params,))
        check_prior(_native.lib().sepso_prior_set_params(self._h, _native.fptr(p)))

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params, np.float32)
        check_prior(_native.lib().sepso_prior_get_params(self._h, _native.fptr(p)))
        return p

    def add_scenes(self, first: int, points, circles, waypoints=None) -> None:
        """Rasterise scenes into rows [first, first + n); circles: list of (O, 3)."""
        pts = _f32(points).reshape(-1, 4)
        n = pts.shape[0]
        counts = np.array([np.asarray(c).reshape(-1, 3).shape[0] for c in circles], np.int32)
        assert counts.size == n
        flat = _f32(np.concatenate([np.asarray(c, np.float32).reshape(-1, 3) for c in circles])
                    if n else np.zeros((0, 3), np.float32))
        wp = None if waypoints is None else _f32(waypoints, (n, self.O))
        check_prior(_native.lib().sepso_prior_add_scenes(
            self._h, first, n, _native.fptr(pts), counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            _native.fptr(flat) if flat.size else None, _native.fptr(wp)))

    def set_labels(self, first: int, waypoints: torch.Tensor) -> None:
        """Relabel rows [first, first + n) with the paths of a device tensor (n, >= 2T)."""
        assert waypoints.is_cuda and waypoints.dtype == torch.float32 and waypoints.stride(1) == 1
        check_prior(_native.lib().sepso_prior_set_labels(self._h, first, waypoints.shape[0],
                                                         ctypes.c_void_p(waypoints.data_ptr()),
                                                         waypoints.stride(0)))

    def get_rows(self, first: int, n: int):
        f = np.empty((n, self.K), np.float32)
        y = np.empty((n, self.O), np.float32)
        check_prior(_native.lib().sepso_prior_get_rows(self._h, first, n, _native.fptr(f), _native.fptr(y)))
        return f, y

    def forward(self, first: int, n: int) -> np.ndarray:
        y = np.empty((n, self.O), np.float32)
        check_prior(_native.lib().sepso_prior_forward(self._h, first, n, _native.fptr(y)))
        return y

    def grad(self, first: int, n: int):
        g = np.empty(self.num_params, np.float32)
        loss = np.zeros(1, np.float32)
        check_prior(_native.lib().sepso_prior_grad(self._h, first, n, _native.fptr(g), _native.fptr(loss)))
        return g, float(loss[0])

    def train(self, steps: int, batch: int, n_rows: int | None = None, first: int = -1, seed: int = 0,
              losses: bool = True):
        """Adam steps on minibatches drawn from rows [0, n_rows) (or the fixed rows
        [first, first + batch)); returns the per-step losses when asked."""
        out = np.empty(steps, np.float32) if losses else None
        nr = self.capacity if n_rows is None else n_rows
        check_prior(_native.lib().sepso_prior_train(self._h, nr, first, steps, batch, seed,
                                                    _native.fptr(out)))
        return out

    def infer(self, first: int, n: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """Proposed waypoints of rows [first, first + n) into a device tensor (n, >= 2T)."""
        if out is None:
            out = torch.empty((n, self.O), dtype=torch.float32, device=self.device)
        assert out.is_cuda and out.dtype == torch.float32 and out.dim() == 2 and out.shape[0] >= n
        assert out.stride(1) == 1
        check_prior(_native.lib().sepso_prior_infer(self._h, first, n, ctypes.c_void_p(out.data_ptr()),
                                                    out.stride(0)))
        return out

    def sync(self) -> None:
        check_prior(_native.lib().sepso_prior_sync(self._h))

    def launch_count(self) -> int:
        return int(_native.lib().sepso_prior_launch_count(self._h))


def gemm_bf16(A: torch.Tensor, B: torch.Tensor, alpha: float = 1.0, bias: torch.Tensor | None = None,
              relu: bool = False, mask: torch.Tensor | None = None, out_f32: bool = True,
              out_bf16: bool = False, sync: bool = True, tile_n: int = 0, out_t: bool = False,
              colsum: bool = False, ksplit: int = 1):
    """C = epilogue(alpha * A @ B^T) on the tensor cores; A (M, K), B (N, K) BF16 CUDA.
    tile_n: 0 automatic; 64 / 128 / 256 the persistent kernel; negative, the
    one-tile-per-CTA kernel with that width.  out_t: also a BF16 (N, M) copy of
    the output transposed; colsum: also the N column sums of the output; ksplit:
    K in that many slices (FP32 products summed in slice order).  Returns
    (Cf, Cb), or (Cf, Cb, Ct, colsum) when out_t, colsum or ksplit is asked for."""
    assert A.is_cuda and B.is_cuda and A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    assert A.stride(1) == 1 and B.stride(1) == 1 and A.shape[1] == B.shape[1]
    M, K = A.shape
    N = B.shape[0]
    dev = A.device
    Cf = torch.empty((M, N), dtype=torch.float32, device=dev) if out_f32 else None
    Cb = torch.empty((M, N), dtype=torch.bfloat16, device=dev) if out_bf16 else None
    vp = ctypes.c_void_p
    stream = torch.cuda.current_stream(dev).cuda_stream
    L = _native.lib()
    args = [vp(A.data_ptr()), vp(B.data_ptr()), M, N, K, A.stride(0), B.stride(0), float(alpha),
            vp(bias.data_ptr()) if bias is not None else None, int(relu),
            vp(mask.data_ptr()) if mask is not None else None, mask.stride(0) if mask is not None else 0,
            vp(Cf.data_ptr()) if Cf is not None else None, N, vp(Cb.data_ptr()) if Cb is not None else None, N]
    extended = out_t or colsum or ksplit != 1
    Ct = cs = None
    if not extended:
        check_prior(L.sepso_gemm_bf16(*args, int(tile_n), vp(stream)))
    else:
        Ct = torch.empty((N, M), dtype=torch.bfloat16, device=dev) if out_t else None
        cs = torch.empty(N, dtype=torch.float32, device=dev) if colsum else None
        size = ctypes.c_size_t()
        check_prior(L.sepso_gemm_bf16_ex_workspace(M, N, int(ksplit), int(colsum), ctypes.byref(size)))
        ws = torch.empty(max(size.value, 16), dtype=torch.uint8, device=dev)
        ex = _native.GemmExtra(Ct=Ct.data_ptr() if Ct is not None else None, ldct=M,
                               colsum=cs.data_ptr() if cs is not None else None, ksplit=int(ksplit),
                               workspace=ws.data_ptr(), workspace_bytes=ws.numel())
        check_prior(L.sepso_gemm_bf16_ex(*args, ctypes.byref(ex), int(tile_n), vp(stream)))
    if sync:
        check_prior(L.sepso_gemm_bf16_sync(vp(stream)))
    return (Cf, Cb, Ct, cs) if extended else (Cf, Cb)


# ----------------------------------------------------------------------------
# Pipeline: SEPSO solutions as labels, training, held-out comparison
# ----------------------------------------------------------------------------

def plan_scenes(scenes: dict, T: int = 20, G: int = 8, N: int = 170, hyper=None, max_iters: int = 300,
                stall_iters: int = 10, stall_tol: float = 0.0, seed: int = 0, run0: int = 0, cycle: int = 0,
                prev: torch.Tensor | None = None, prior: torch.Tensor | None = None, n_pi: int = 0,
                n_prior: int = 0, pi_halfwidth: float = 20.0, chunk: int = 8192, shape=None, device=None) -> dict:
    """Plan every scene (points (n,4), circles (n,O,3)) with the batch planner in
    chunks: Algorithm 1 with stall-counter Auto Truncation, PI around prev (rows of
    a device tensor, n_pi particles per group) and the learned seed around prior
    (n_prior particles).  Returns waypoints (device tensor (n, 2T)), cost, iters, Q
    (numpy), the launch shape used and the device seconds of the runs."""
    from .inputs import TABLE_HYPER8_PATH, BatchSceneSpec
    from .planner import BatchPlanner

    hy = np.asarray(TABLE_HYPER8_PATH if hyper is None else hyper, np.float32)[:G]
    pts, circ = scenes["points"], scenes["circles"]
    n, O = pts.shape[0], circ.shape[1]
    dev = _dev(device)
    wp = torch.empty((n, 2 * T), dtype=torch.float32, device=dev)
    cost, iters, Q = np.empty(n, np.float32), np.empty(n, np.int32), np.empty(n, np.int32)
    secs = 0.0
    used = 0
    for c0 in range(0, n, chunk):
        m = min(chunk, n - c0)
        specs = [BatchSceneSpec(T=T, G=G, N=N, O=O, max_iters=max_iters, alpha=30.0, beta=4, seed=seed,
                                run_id=run0 + c0 + i, stall_iters=stall_iters, stall_tol=stall_tol,
                                n_pi=n_pi if prev is not None else 0,
                                n_prior=n_prior if prior is not None else 0, pi_halfwidth=pi_halfwidth,
                                cycle=cycle) for i in range(m)]
        bp = BatchPlanner(specs, device=dev)
        bp.set_inputs([hy] * m, pts[c0:c0 + m], [circ[c0 + i] for i in range(m)])
        if shape is None:
            shape, _ = bp.autotune(trial_launches=3)
        else:
            bp.set_shape(shape["tile"], shape["threads"])
        if prev is not None or prior is not None:
            bp.set_starts(prev=prev[c0:c0 + m] if prev is not None else None,
                          prior=prior[c0:c0 + m] if prior is not None else None)
            if prior is not None:
                used += bp.prior_used()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(bp.stream)
        bp.run_async(use_graph=True)
        ev1.record(bp.stream)
        res = bp.read()
        secs += ev0.elapsed_time(ev1) / 1e3
        wp[c0:c0 + m] = torch.from_numpy(np.stack([r["waypoints"] for r in res])).to(dev)
        cost[c0:c0 + m] = [r["cost"] for r in res]
        iters[c0:c0 + m] = [r["iters"] for r in res]
        Q[c0:c0 + m] = [r["Q"] for r in res]
        bp.close()
    return dict(waypoints=wp, cost=cost, iters=iters, Q=Q, shape=shape, seconds=secs,
                prior_used=used if prior is not None else None)


def fit_prior(prior: Prior, scenes: dict, rounds: int = 3, epochs: int = 30, batch: int = 4096, seed: int = 0,
              n_prior: int = 43, shape=None, **plan_kw) -> dict:
    """Train the prior on SEPSO solutions the planner itself generates, in rounds:
    the first labels are plain SEPSO plans of the scenes; after each training phase
    the scenes are planned again with the prior's proposals as a second seed, and a
    scene's label becomes the new plan when its cost is lower.  Scenes occupy rows
    [0, n).  Returns the label costs per round, the losses and timings."""
    n = scenes["points"].shape[0]
    prior.add_scenes(0, scenes["points"], [scenes["circles"][i] for i in range(n)])
    lab = plan_scenes(scenes, seed=seed, run0=0, shape=shape, **plan_kw)
    shape = lab["shape"]
    labels, cost = lab["waypoints"], lab["cost"]
    hist = dict(label_cost=[float(np.median(cost))], label_iters=[float(np.mean(lab["iters"]))],
                losses=[], plan_s=lab["seconds"], train_s=0.0, steps=0)
    steps = max(1, epochs * n // batch)
    for r in range(rounds):
        prior.set_labels(0, labels)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(prior.stream)
        loss = np.concatenate([prior.train(steps=min(65536, steps - s0), batch=batch, n_rows=n,
                                           seed=seed * 1000 + r) for s0 in range(0, steps, 65536)])
        ev1.record(prior.stream)
        ev1.synchronize()
        hist["train_s"] += ev0.elapsed_time(ev1) / 1e3
        hist["steps"] += steps
        hist["losses"].append([float(loss[:10].mean()), float(loss[-10:].mean())])
        if r + 1 < rounds:
            prop = prior.infer(0, n)
            nl = plan_scenes(scenes, seed=seed, run0=0, cycle=r + 1, prior=prop, n_prior=n_prior, shape=shape,
                             **plan_kw)
            hist["plan_s"] += nl["seconds"]
            better = nl["cost"] < cost
            labels = torch.where(torch.from_numpy(better).to(labels.device)[:, None], nl["waypoints"], labels)
            cost = np.where(better, nl["cost"], cost)
            hist["label_cost"].append(float(np.median(cost)))
            hist["label_iters"].append(float(np.mean(nl["iters"])))
    hist["shape"] = shape
    return hist


def fit_prior_sets(prior: Prior, sets: list, rounds: int = 2, epochs: int = 30, batch: int = 4096, seed: int = 0,
                   n_prior: int = 43, **plan_kw) -> dict:
    """fit_prior over several scene sets (each with its own circle count), laid out
    back to back from row 0: every set is labelled by the planner, the prior trains
    on all rows, and after each training phase every set is planned again with the
    proposals as a second seed, a scene's label becoming the new plan when it is
    cheaper.  Returns the per-round median label cost and collision-free share."""
    offs = np.cumsum([0] + [d["points"].shape[0] for d in sets])
    n = int(offs[-1])
    for d, o in zip(sets, offs[:-1]):
        m = d["points"].shape[0]
        prior.add_scenes(int(o), d["points"], [d["circles"][i] for i in range(m)])
    labs = [plan_scenes(d, seed=seed, run0=int(o), **plan_kw) for d, o in zip(sets, offs[:-1])]
    labels = torch.cat([l_["waypoints"] for l_ in labs])
    cost = np.concatenate([l_["cost"] for l_ in labs])
    q = np.concatenate([l_["Q"] for l_ in labs])
    hist = dict(label_cost=[float(np.median(cost))], label_collision_free=[float(np.mean(q == 0))], losses=[],
                plan_s=sum(l_["seconds"] for l_ in labs), train_s=0.0, steps=0)
    steps = max(1, epochs * n // batch)
    for r in range(rounds):
        prior.set_labels(0, labels)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(prior.stream)
        loss = np.concatenate([prior.train(steps=min(65536, steps - s0), batch=batch, n_rows=n,
                                           seed=seed * 1000 + r) for s0 in range(0, steps, 65536)])
        ev1.record(prior.stream)
        ev1.synchronize()
        hist["train_s"] += ev0.elapsed_time(ev1) / 1e3
        hist["steps"] += steps
        hist["losses"].append([float(loss[:10].mean()), float(loss[-10:].mean())])
        if r + 1 < rounds:
            prop = prior.infer(0, n)
            new = [plan_scenes(d, seed=seed, run0=int(o), cycle=r + 1, prior=prop[int(o):int(o) + d["points"].shape[0]],
                               n_prior=n_prior, **plan_kw) for d, o in zip(sets, offs[:-1])]
            hist["plan_s"] += sum(l_["seconds"] for l_ in new)
            ncost = np.concatenate([l_["cost"] for l_ in new])
            better = ncost < cost
            labels = torch.where(torch.from_numpy(better).to(labels.device)[:, None],
                                 torch.cat([l_["waypoints"] for l_ in new]), labels)
            cost = np.where(better, ncost, cost)
            q = np.where(better, np.concatenate([l_["Q"] for l_ in new]), q)
            hist["label_cost"].append(float(np.median(cost)))
            hist["label_collision_free"].append(float(np.mean(q == 0)))
    return hist


def propose(prior: Prior, scenes: dict, first: int) -> torch.Tensor:
    """The prior's proposals (device (n, 2T)) for scenes loaded into rows [first, first + n)."""
    n = scenes["points"].shape[0]
    prior.add_scenes(first, scenes["points"], [scenes["circles"][i] for i in range(n)])
    return prior.infer(first, n)


def _summary(r: dict, n: int) -> dict:
    return dict(cost_median=float(np.median(r["cost"])), iters_mean=float(np.mean(r["iters"])),
                iters_median=float(np.median(r["iters"])), collision_free=float(np.mean(r["Q"] == 0)),
                seconds=float(r["seconds"]), plans_per_s=float(n / r["seconds"]) if r["seconds"] > 0 else None,
                prior_used=None if r.get("prior_used") is None else float(r["prior_used"] / n))


def evaluate_prior(prior: Prior, scenes: dict, first: int, budgets=(10, 25, 50, 100, 200, 300), cycles: int = 5,
                   n_pi: int = 43, n_prior: int = 43, seed: int = 2, run0: int = 10 ** 6, shape=None,
                   **plan_kw) -> dict:
    """Held-out comparison of the PI-only start with prior + PI.

    cold: a new scene (no previous path, so PI-only is the uniform start), planned
      with Auto Truncation; budgets: median cost after exactly k iterations (no AT)
      for each k, and iterations-to-converge = the smallest budget at which a start
      reaches the PI-only start's median cost at the largest budget.
    dynamic: `cycles` planning cycles of each scene moving as in the dynamic workload
      (the last cycle is the given scene), every cycle warm-started by PI from the
      same method's previous plan; per cycle the AT-run summary of each method.
    Scenes are rasterised into prior rows [first, first + n)."""
    n = scenes["points"].shape[0]
    from .inputs import previous_cycle
    out: dict = {"n": n}
    prop = propose(prior, scenes, first)
    base = plan_scenes(scenes, seed=seed, run0=run0, shape=shape, **plan_kw)
    shape = base["shape"]
    withp = plan_scenes(scenes, seed=seed, run0=run0, prior=prop, n_prior=n_prior, shape=shape, **plan_kw)
    out["cold"] = {"pi_only": _summary(base, n), "prior_pi": _summary(withp, n)}
    kw = {k: v for k, v in plan_kw.items() if k not in ("max_iters", "stall_iters")}
    curve = {"pi_only": [], "prior_pi": []}
    for k in budgets:
        a = plan_scenes(scenes, seed=seed, run0=run0, max_iters=k, stall_iters=0, shape=shape, **kw)
        b = plan_scenes(scenes, seed=seed, run0=run0, max_iters=k, stall_iters=0, prior=prop, n_prior=n_prior,
                        shape=shape, **kw)
        curve["pi_only"].append(dict(_summary(a, n), iters=k))
        curve["prior_pi"].append(dict(_summary(b, n), iters=k))
    target = curve["pi_only"][-1]["cost_median"]
    conv = {}
    for m, pts in curve.items():
        hit = [p["iters"] for p in pts if p["cost_median"] <= target * (1.0 + 1e-6)]
        conv[m] = hit[0] if hit else None
    out["budgets"] = curve
    out["iters_to_converge"] = conv
    out["converged_cost"] = target
    dyn = {"pi_only": [], "prior_pi": []}
    prev = {"pi_only": None, "prior_pi": None}
    prev_before_last = {"pi_only": None, "prior_pi": None}
    for c in range(cycles):
        sc = previous_cycle(scenes, cycles - 1 - c) if c < cycles - 1 else scenes
        pc = propose(prior, sc, first)
        if c == cycles - 1:
            prev_before_last = dict(prev)
        for m in ("pi_only", "prior_pi"):
            use_prior = m == "prior_pi"
            r = plan_scenes(sc, seed=seed, run0=run0, cycle=c, prev=prev[m], n_pi=n_pi,
                            prior=pc if use_prior else None, n_prior=n_prior if use_prior else 0, shape=shape,
                            **plan_kw)
            dyn[m].append(_summary(r, n))
            prev[m] = r["waypoints"]
    out["dynamic"] = dyn
    # the last cycle again with fixed iteration budgets (no AT), each method warm-
    # started by PI from its own plans of the cycle before
    last_prev = {m: prev_before_last[m] for m in prev_before_last}
    sc_last = scenes
    dyn_budgets = {"pi_only": [], "prior_pi": []}
    pc = propose(prior, sc_last, first)
    for k in budgets:
        for m in ("pi_only", "prior_pi"):
            use_prior = m == "prior_pi"
            r = plan_scenes(sc_last, seed=seed, run0=run0, cycle=cycles - 1, prev=last_prev[m], n_pi=n_pi,
                            prior=pc if use_prior else None, n_prior=n_prior if use_prior else 0, shape=shape,
                            max_iters=k, stall_iters=0, **kw)
            dyn_budgets[m].append(dict(_summary(r, n), iters=k))
    out["dynamic_budgets"] = dyn_budgets
    out["shape"] = shape
    return out


def single_scene_dynamic(scenes: dict, n: int = 64, cycles: int = 5, T: int = 20, G: int = 8, N: int = 170,
                         hyper=None, seed: int = 2, run0: int = 10 ** 6, device=None) -> dict:
    """The plain single-scene kernel on the first n held-out scenes, each through the
    same `cycles`-cycle dynamic sequence as evaluate_prior (PI from its own previous
    plan, AT stall 10 / cap 300): median path cost of the last cycle and plans/s
    (device time of the planning calls)."""
    from .inputs import TABLE_HYPER8_PATH, AT_STALL, Scene, SepsoConfig, previous_cycle
    from .planner import Planner
    hy = np.asarray(TABLE_HYPER8_PATH if hyper is None else hyper, np.float32)[:G]
    seqs = [previous_cycle(scenes, cycles - 1 - c) if c < cycles - 1 else scenes for c in range(cycles)]
    costs, ms = [], 0.0
    for i in range(n):
        cfg = SepsoConfig(T=T, G=G, N=N, max_obstacles=scenes["circles"].shape[1], alpha=30.0, beta=4,
                          max_iters=300, at_mode=AT_STALL, stall_iters=10, stall_tol=0.0, use_pi=True,
                          pi_gamma=(43 - 0.5) / N, pi_halfwidth=20.0, seed=seed, run_id=run0 + i)
        pl = Planner(cfg, device=device)
        pl.set_hyper(hy)
        for c in range(cycles):
            sc = seqs[c]
            pt = sc["points"][i]
            pl.set_scene(Scene(start=pt[:2], target=pt[2:], circles=sc["circles"][i]), motion=False)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(pl.stream)
            pl.plan_async()
            e1.record(pl.stream)
            res = pl.read_result()
            if c == cycles - 1:
                ms += e0.elapsed_time(e1)
                costs.append(float(res["cost"]))
    return dict(n=n, cost_median=float(np.median(costs)), plans_per_s=n / (ms / 1e3), ms_per_plan=ms / n)
