"""Python face of libsepso: a Planner owns one handle, its workspace and stream.

PyTorch provides the device memory (the workspace is a torch uint8 tensor) and the
stream; every step of the planner runs in the library's CUDA kernels, reached
through the C ABI of include/sepso.h.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import HsefConfig, Result, check, check_bf, fptr
from .inputs import Scene, SepsoConfig


def _f32(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a.reshape(shape) if shape is not None else a


def state_layout(cfg: SepsoConfig) -> dict:
    """(offset, dtype, count) of every field of one run's serialised state."""
    G, N, D, tw = cfg.G, cfg.N, 2 * cfg.T, cfg.tw
    M = G * N
    spec = [("X", np.float32, M * D), ("V", np.float32, M * D), ("P", np.float32, M * D),
            ("Pfit", np.float32, M), ("PQ", np.int32, M), ("Gb", np.float32, G * D),
            ("Gfit", np.float32, G), ("GQ", np.int32, G), ("Tb", np.float32, D),
            ("Tfit", np.float32, 1), ("TQ", np.int32, 1), ("k", np.int32, 1),
            ("cycle", np.int32, 1), ("has_prev", np.int32, 1), ("prevT", np.float32, D),
            ("win", np.float64, tw), ("win_n", np.int32, 1), ("win_head", np.int32, 1),
            ("stall", np.int32, 1), ("prev_lfv", np.float32, 1)]
    out, off = {}, 0
    for name, dt, n in spec:
        if dt == np.float64:
            off = (off + 7) & ~7
        out[name] = (off, dt, n)
        off += np.dtype(dt).itemsize * n
    out["_total"] = off
    return out


def at_window_test(win, ns, heads, delta: float) -> np.ndarray:
    """The Auto Truncation window criterion (Sec. 3.3.4) evaluated on the device by
    the planner's own code: ``win`` (count, tw) float64 rings, ``ns``/``heads`` the
    fill and head of each; returns bool[count], std of the newest entries < delta."""
    w = np.ascontiguousarray(win, np.float64)
    count, tw = w.shape
    n = np.ascontiguousarray(ns, np.int32).reshape(count)
    h = np.ascontiguousarray(heads, np.int32).reshape(count)
    out = np.zeros(count, np.int32)
    stream = torch.cuda.current_stream().cuda_stream
    check(_native.lib().sepso_at_window_test(w.ctypes.data, n.ctypes.data, h.ctypes.data, count, tw,
                                             ctypes.c_float(delta), out.ctypes.data,
                                             ctypes.c_void_p(stream)))
    return out.astype(bool)


def philox_device(ctr: torch.Tensor, seed: int) -> torch.Tensor:
    """Philox4x32-10 of the counters ``ctr`` (device int32/uint32 tensor (n, 4)) under
    the 64-bit ``seed``, computed on the device by the planner's own generator;
    returns the (n, 4) output words (int32 tensor holding the uint32 bits)."""
    c = ctr.contiguous()
    if c.dim() != 2 or c.shape[1] != 4 or c.element_size() != 4 or not c.is_cuda:
        raise ValueError("ctr must be a CUDA tensor of shape (n, 4) with 32-bit elements")
    out = torch.empty_like(c)
    stream = torch.cuda.current_stream(c.device).cuda_stream
    check(_native.lib().sepso_philox(ctypes.c_void_p(c.data_ptr()), c.shape[0], ctypes.c_uint64(seed),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream)))
    return out


class Planner:
    """One SEPSO planner (``cfg.runs`` swarms sharing one scene) on one GPU."""

    def __init__(self, cfg: SepsoConfig, device=None, stream: torch.cuda.Stream | None = None):
        self.lib = _native.lib()
        self.cfg = cfg
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        c = _native.make_config(cfg)
        size = ctypes.c_size_t()
        check(self.lib.sepso_workspace_size(ctypes.byref(c), ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.sepso_create(ctypes.byref(c), ctypes.c_void_p(self.workspace.data_ptr()),
                                        size.value, ctypes.c_void_p(self.stream.cuda_stream),
                                        ctypes.byref(self._h)))
        self.D = 2 * cfg.T
        self.O = 0
        # host buffers of the per-cycle calls (set_scene_arrays, plan_into) and their
        # pointers, made once
        self._st = np.zeros(2, np.float32)
        self._tg = np.zeros(2, np.float32)
        self._ci = np.zeros((max(cfg.max_obstacles, 1), 3), np.float32)
        self._pst, self._ptg, self._pci = fptr(self._st), fptr(self._tg), fptr(self._ci)
        self._res = Result()
        self._pres = ctypes.byref(self._res)
        self._wp_addr, self._pwp = None, None

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if self._h:
            self.lib.sepso_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- inputs -----------------------------------------------------------
    def set_hyper(self, hyper, run: int = -1):
        h = _f32(hyper, (self.cfg.G, 6))
        check(self.lib.sepso_set_hyper(self._h, run, fptr(h)))

    def set_scene(self, scene: Scene, motion: bool = True):
        circ = _f32(scene.circles, (-1, 3))
        check(self.lib.sepso_set_scene(self._h, fptr(_f32(scene.start)), fptr(_f32(scene.target)),
                                       fptr(circ) if circ.size else None, circ.shape[0]))
        self.O = circ.shape[0]
        if motion:
            cv = _f32(scene.circle_vel, (-1, 2))
            check(self.lib.sepso_set_motion(self._h, fptr(cv) if cv.size else None,
                                            fptr(_f32(scene.start_vel)), fptr(_f32(scene.target_vel))))

    def set_scene_arrays(self, start, target, circles):
        """The per-cycle form of set_scene for a caller that holds plain arrays: start
        (2,), target (2,), circles (O, 3) (cx, cy, r) are copied into host buffers the
        planner keeps, then sepso_set_scene uploads them; the velocities stay as they
        are."""
        O = len(circles)
        self._st[:] = start
        self._tg[:] = target
        if O:
            self._ci[:O] = circles
        check(self.lib.sepso_set_scene(self._h, self._pst, self._ptg, self._pci if O else None, O))
        self.O = O

    def set_polygons(self, scene, motion: bool = True):
        """A scene among polygon obstacles (a handle with obstacle_kind = 1):
        ``scene`` carries start, target, polygons (vertex lists) and velocities."""
        e = _f32(scene.edges, (-1, 4))
        off = np.ascontiguousarray(np.asarray(scene.offsets, np.int32))
        check(self.lib.sepso_set_polygons(self._h, fptr(_f32(scene.start)), fptr(_f32(scene.target)),
                                          fptr(e) if e.size else None, e.shape[0],
                                          off.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), off.size - 1))
        self.O = e.shape[0]
        self.P = off.size - 1
        if motion:
            pv = _f32(scene.poly_vel, (-1, 2))
            check(self.lib.sepso_set_motion(self._h, fptr(pv) if pv.size else None,
                                            fptr(_f32(scene.start_vel)), fptr(_f32(scene.target_vel))))

    def get_polygons(self):
        """(start, target, edges (E, 4), polygon velocities (P, 2)) on the device now."""
        s, t = np.zeros(2, np.float32), np.zeros(2, np.float32)
        e = np.zeros((max(self.O, 1), 4), np.float32)
        v = np.zeros((max(self.P, 1), 2), np.float32)
        check(self.lib.sepso_get_polygons(self._h, fptr(s), fptr(t), fptr(e), fptr(v)))
        return s, t, e[:self.O], v[:self.P]

    def advance(self, steps: int = 1):
        check(self.lib.sepso_advance_scene(self._h, steps))

    def get_scene(self) -> Scene:
        s, t = np.zeros(2, np.float32), np.zeros(2, np.float32)
        c = np.zeros((max(self.O, 1), 3), np.float32)
        v = np.zeros((max(self.O, 1), 2), np.float32)
        check(self.lib.sepso_get_scene(self._h, fptr(s), fptr(t), fptr(c), fptr(v)))
        return Scene(start=s, target=t, circles=c[:self.O], circle_vel=v[:self.O])

    # -- hot path ---------------------------------------------------------
    def plan_async(self):
        check(self.lib.sepso_plan_async(self._h))

    def read_result(self, run: int = 0) -> dict:
        wp = np.zeros(self.D, np.float32)
        res = Result()
        check(self.lib.sepso_read_result(self._h, run, fptr(wp), ctypes.byref(res)))
        return {"waypoints": wp, "cost": res.cost, "length": res.length, "Q": res.Q,
                "iters": res.iters, "status": res.status}

    def plan(self) -> dict:
        self.plan_async()
        return self.read_result(0)

    def plan_into(self, waypoints: np.ndarray) -> Result:
        """One synchronous planning cycle writing into a caller-owned host float32
        array of 2T waypoints; returns the planner's result record (overwritten by the
        next call)."""
        addr = waypoints.ctypes.data
        if addr != self._wp_addr:
            assert waypoints.dtype == np.float32 and waypoints.flags.c_contiguous and waypoints.size >= self.D
            self._wp_addr, self._pwp = addr, fptr(waypoints)
        check(self.lib.sepso_plan(self._h, self._pwp, self._pres))
        return self._res

    def result_device(self, run: int = 0):
        wp, rr = ctypes.c_void_p(), ctypes.c_void_p()
        check(self.lib.sepso_result_device(self._h, run, ctypes.byref(wp), ctypes.byref(rr)))
        return wp.value, rr.value

    def step(self, iters: int = 1):
        check(self.lib.sepso_step(self._h, iters))

    def evaluate(self, X: torch.Tensor):
        """F, Q, length of the rows of a CUDA float32 tensor (n, 2T)."""
        assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous() and X.shape[-1] == self.D
        n = X.numel() // self.D
        F = torch.empty(n, dtype=torch.float32, device=X.device)
        Q = torch.empty(n, dtype=torch.int32, device=X.device)
        L = torch.empty(n, dtype=torch.float32, device=X.device)
        check(self.lib.sepso_evaluate(self._h, ctypes.c_void_p(X.data_ptr()), n,
                                      ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(Q.data_ptr()),
                                      ctypes.c_void_p(L.data_ptr())))
        return F, Q, L

    def sync(self):
        check(self.lib.sepso_sync(self._h))

    # -- state ------------------------------------------------------------
    def get_state(self, run: int = 0) -> dict:
        lay = state_layout(self.cfg)
        buf = np.zeros(lay["_total"], np.uint8)
        check(self.lib.sepso_get_state(self._h, run, buf.ctypes.data_as(ctypes.c_void_p), buf.size))
        out = {}
        for name, spec in lay.items():
            if name.startswith("_"):
                continue
            off, dt, n = spec
            out[name] = np.frombuffer(buf, dtype=dt, count=n, offset=off).copy()
        return out

    def set_state(self, state: dict, run: int = 0):
        """Write the given fields (others keep their current values)."""
        lay = state_layout(self.cfg)
        cur = self.get_state(run)
        cur.update({k: v for k, v in state.items() if k in cur})
        buf = np.zeros(lay["_total"], np.uint8)
        for name, spec in lay.items():
            if name.startswith("_"):
                continue
            off, dt, n = spec
            a = np.ascontiguousarray(np.asarray(cur[name]).reshape(-1).astype(dt))
            if a.size != n:
                raise ValueError(f"state field {name}: {a.size} values, expected {n}")
            buf[off:off + a.nbytes] = a.view(np.uint8)
        check(self.lib.sepso_set_state(self._h, run, buf.ctypes.data_as(ctypes.c_void_p), buf.size))

    # -- HSEF -------------------------------------------------------------
    def hsef(self, HG: int, HN: int, E: int, hhyper, lo, hi, l_vlimit: float, hseed: int,
             history: bool = True):
        hc = HsefConfig(HG=HG, HN=HN, E=E, l_vlimit=l_vlimit, hseed=hseed)
        hh = _f32(hhyper, (HG, 6)).reshape(-1)
        for i, v in enumerate(hh):
            hc.hhyper[i] = float(v)
        for i in range(3):
            hc.lo[i] = float(lo[i])
            hc.hi[i] = float(hi[i])
        hist = torch.zeros(E, dtype=torch.float32, device=self.device) if history else None
        check(self.lib.sepso_hsef(self._h, ctypes.byref(hc),
                                  ctypes.c_void_p(hist.data_ptr()) if hist is not None else None))
        return hist

    def hsef_best(self):
        hy = np.zeros((self.cfg.G, 6), np.float32)
        lfv = np.zeros(1, np.float32)
        check(self.lib.sepso_hsef_best(self._h, fptr(hy), fptr(lfv)))
        return hy, float(lfv[0])

    # -- introspection ----------------------------------------------------
    def launch_shape(self) -> dict:
        v = [ctypes.c_int32() for _ in range(4)]
        check(self.lib.sepso_launch_shape(self._h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("ctas_per_group", "threads", "circle_split", "grid"), [x.value for x in v]))

    def exchange_form(self) -> str:
        """"cluster" when the next plan runs one thread-block cluster per group,
        "grid" for the grid-wide barrier."""
        v = int(self.lib.sepso_exchange_form(self._h))
        if v < 0:
            check(v)
        return "cluster" if v == 2 else "grid"

    def counters(self, run: int = 0) -> tuple[int, int]:
        """(planning cycles finished, iterations run) of one run, cumulative."""
        p, i = ctypes.c_int64(), ctypes.c_int64()
        check(self.lib.sepso_counters(self._h, run, ctypes.byref(p), ctypes.byref(i)))
        return p.value, i.value

    def launch_count(self) -> int:
        return int(self.lib.sepso_launch_count(self._h))


class BFPlanner:
    """DTPSO on a benchmark function of Table BFs (``sepso_bf_*``): ``cfg.runs``
    independent swarms of G x N particles over [lo, hi]^D on one GPU."""

    def __init__(self, cfg, device=None, stream: torch.cuda.Stream | None = None):
        self.lib = _native.lib()
        self.cfg = cfg
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        c = _native.bf_config_struct(cfg)
        size = ctypes.c_size_t()
        check_bf(self.lib.sepso_bf_workspace_size(ctypes.byref(c), ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check_bf(self.lib.sepso_bf_create(ctypes.byref(c), ctypes.c_void_p(self.workspace.data_ptr()),
                                              size.value, ctypes.c_void_p(self.stream.cuda_stream),
                                              ctypes.byref(self._h)))

    def close(self):
        if self._h:
            self.lib.sepso_bf_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hyper(self, hyper, run: int = -1):
        h = _f32(hyper, (self.cfg.G, 6))
        check_bf(self.lib.sepso_bf_set_hyper(self._h, h.ctypes.data, run))

    def set_polygons(self, start, target, edges):
        """Objective 5: obstacle edges (E, 4) float32 (x0, y0, x1, y1), start, target."""
        e = _f32(edges, (-1, 4))
        st, tg = _f32(start, (2,)), _f32(target, (2,))
        check_bf(self.lib.sepso_bf_set_polygons(self._h, st.ctypes.data, tg.ctypes.data,
                                                e.ctypes.data if e.size else None, e.shape[0]))

    def set_spheres(self, start, target, spheres):
        """Objective 6: spheres (S, 4) float32 (cx, cy, cz, r), start and target (3,)."""
        sp = _f32(spheres, (-1, 4))
        st, tg = _f32(start, (3,)), _f32(target, (3,))
        check_bf(self.lib.sepso_bf_set_spheres(self._h, st.ctypes.data, tg.ctypes.data,
                                               sp.ctypes.data if sp.size else None, sp.shape[0]))

    def set_warm_start(self, prev_paths=None, cycle: int = 0):
        """Path objectives: the next run's Priori Initialization around each run's
        previous best path (``prev_paths`` (runs, D); None: a cold start) with the
        config's pi_gamma and pi_halfwidth; ``cycle`` enters the Philox counters."""
        if prev_paths is None:
            check_bf(self.lib.sepso_bf_set_warm_start(self._h, None, ctypes.c_float(0.0), ctypes.c_float(0.0),
                                                      int(cycle)))
            return
        pv = _f32(prev_paths, (self.cfg.runs, self.cfg.D))
        check_bf(self.lib.sepso_bf_set_warm_start(self._h, pv.ctypes.data, ctypes.c_float(self.cfg.pi_gamma),
                                                  ctypes.c_float(self.cfg.pi_halfwidth), int(cycle)))

    def read_all(self):
        """Tbest rows of every run (runs, D), their fitness (runs,) and iteration
        counts (runs,; with Auto Truncation, each run's stopping iteration)."""
        R, D = self.cfg.runs, self.cfg.D
        out, fit, its = np.zeros((R, D), np.float32), np.zeros(R, np.float32), np.zeros(R, np.int32)
        for r in range(R):
            res = self.read(r)
            out[r], fit[r], its[r] = res["x"], res["fit"], res["iters"]
        return out, fit, its

    def run_async(self, use_graph: bool = True):
        check_bf(self.lib.sepso_bf_run_async(self._h, int(use_graph)))

    def step(self, iters: int = 1):
        check_bf(self.lib.sepso_bf_step(self._h, iters))

    def sync(self):
        check_bf(self.lib.sepso_bf_sync(self._h))

    def read(self, run: int = 0) -> dict:
        x = np.zeros(self.cfg.D, np.float32)
        f = np.zeros(1, np.float32)
        k = ctypes.c_int32()
        check_bf(self.lib.sepso_bf_read(self._h, run, x.ctypes.data, f.ctypes.data, ctypes.byref(k)))
        return {"x": x, "fit": float(f[0]), "iters": k.value}

    def history(self, run: int = 0) -> np.ndarray:
        h = np.zeros(self.cfg.max_iters, np.float32)
        check_bf(self.lib.sepso_bf_history(self._h, run, h.ctypes.data))
        return h

    def get_state(self, run: int = 0) -> dict:
        G, N, D = self.cfg.G, self.cfg.N, self.cfg.D
        M = G * N
        st = {"X": np.zeros(M * D, np.float32), "V": np.zeros(M * D, np.float32),
              "P": np.zeros(M * D, np.float32), "Pfit": np.zeros(M, np.float32),
              "Gb": np.zeros(G * D, np.float32), "Gfit": np.zeros(G, np.float32),
              "Tb": np.zeros(D, np.float32), "Tfit": np.zeros(1, np.float32)}
        k = ctypes.c_int32()
        check_bf(self.lib.sepso_bf_get_state(self._h, run, *[st[n].ctypes.data for n in
                                                             ("X", "V", "P", "Pfit", "Gb", "Gfit", "Tb", "Tfit")],
                                             ctypes.byref(k)))
        st["k"] = np.array([k.value], np.int32)
        return st

    def set_state(self, state: dict, run: int = 0):
        G, N, D = self.cfg.G, self.cfg.N, self.cfg.D
        M = G * N
        shapes = {"X": M * D, "V": M * D, "P": M * D, "Pfit": M, "Gb": G * D, "Gfit": G, "Tb": D, "Tfit": 1}
        arrs = {n: _f32(state[n], (sz,)) for n, sz in shapes.items()}
        check_bf(self.lib.sepso_bf_set_state(self._h, run, *[arrs[n].ctypes.data for n in shapes],
                                             int(np.asarray(state["k"]).reshape(-1)[0])))

    def launch_count(self) -> int:
        return int(self.lib.sepso_bf_launch_count(self._h))

    def kernel_name(self) -> str:
        return self.lib.sepso_bf_kernel_name(self._h).decode()


def poly_evaluate(X: torch.Tensor, start, target, edges: torch.Tensor, alpha: float, beta: int):
    """Objective 5 of the rows of a CUDA float32 tensor (n, 2T) among CUDA float32
    edges (E, 4): (fitness, Q) tensors."""
    assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    assert edges.is_cuda and edges.dtype == torch.float32 and edges.is_contiguous()
    n, D = X.shape
    F = torch.empty(n, dtype=torch.float32, device=X.device)
    Q = torch.empty(n, dtype=torch.int32, device=X.device)
    st, tg = _f32(start, (2,)), _f32(target, (2,))
    stream = torch.cuda.current_stream(X.device).cuda_stream
    check_bf(_native.lib().sepso_poly_evaluate(D // 2, n, ctypes.c_void_p(X.data_ptr()), X.stride(0),
                                               st.ctypes.data, tg.ctypes.data,
                                               ctypes.c_void_p(edges.data_ptr()), edges.shape[0],
                                               ctypes.c_float(alpha), beta, ctypes.c_void_p(F.data_ptr()),
                                               ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(stream)))
    return F, Q


def sphere_evaluate(X: torch.Tensor, start, target, spheres: torch.Tensor, alpha: float, beta: int):
    """Objective 6 of the rows of a CUDA float32 tensor (n, 3T) among CUDA float32
    spheres (S, 4) (cx, cy, cz, r): (fitness, Q) tensors."""
    assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    assert spheres.is_cuda and spheres.dtype == torch.float32 and spheres.is_contiguous()
    n, D = X.shape
    F = torch.empty(n, dtype=torch.float32, device=X.device)
    Q = torch.empty(n, dtype=torch.int32, device=X.device)
    st, tg = _f32(start, (3,)), _f32(target, (3,))
    stream = torch.cuda.current_stream(X.device).cuda_stream
    check_bf(_native.lib().sepso_sphere_evaluate(D // 3, n, ctypes.c_void_p(X.data_ptr()), X.stride(0),
                                                 st.ctypes.data, tg.ctypes.data,
                                                 ctypes.c_void_p(spheres.data_ptr()), spheres.shape[0],
                                                 ctypes.c_float(alpha), beta, ctypes.c_void_p(F.data_ptr()),
                                                 ctypes.c_void_p(Q.data_ptr()), ctypes.c_void_p(stream)))
    return F, Q


def bf_evaluate(fn: int, X: torch.Tensor) -> torch.Tensor:
    """BF``fn`` of the rows of a CUDA float32 tensor (n, D), on the current stream."""
    assert X.is_cuda and X.dtype == torch.float32 and X.dim() == 2 and X.stride(1) == 1
    F = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    stream = torch.cuda.current_stream(X.device).cuda_stream
    check_bf(_native.lib().sepso_bf_evaluate(fn, X.shape[1], X.shape[0], ctypes.c_void_p(X.data_ptr()),
                                             X.stride(0), ctypes.c_void_p(F.data_ptr()),
                                             ctypes.c_void_p(stream)))
    return F


class BatchPlanner:
    """Many independent scenes of uneven size planned together (sepso_batch_*)."""

    def __init__(self, specs, map_w: float = 400.0, map_h: float = 400.0, device=None,
                 stream: torch.cuda.Stream | None = None):
        from ._native import BatchScene, check_batch
        self.lib = _native.lib()
        self._check = check_batch
        self.specs = list(specs)
        self.n = len(self.specs)
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        arr = (BatchScene * self.n)()
        for i, sp in enumerate(self.specs):
            arr[i] = BatchScene(T=sp.T, G=sp.G, N=sp.N, O=sp.O, max_iters=sp.max_iters,
                                alpha=sp.alpha, beta=sp.beta, seed=sp.seed, run_id=sp.run_id,
                                stall_iters=sp.stall_iters, stall_tol=sp.stall_tol, n_pi=sp.n_pi,
                                n_prior=sp.n_prior, pi_halfwidth=sp.pi_halfwidth, cycle=sp.cycle,
                                obstacle_kind=sp.obstacle_kind)
        self._arr = arr
        size = ctypes.c_size_t()
        check_batch(self.lib.sepso_batch_workspace_size(arr, self.n, ctypes.byref(size)))
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check_batch(self.lib.sepso_batch_create(arr, self.n, map_w, map_h,
                                                    ctypes.c_void_p(self.workspace.data_ptr()),
                                                    size.value, ctypes.c_void_p(self.stream.cuda_stream),
                                                    ctypes.byref(self._h)))
        self.D = [sp.D for sp in self.specs]

    def close(self):
        if self._h:
            self.lib.sepso_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_inputs(self, hyper, points, circles):
        h = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).reshape(-1) for x in hyper]))
        pts = np.ascontiguousarray(np.asarray(points, np.float32).reshape(self.n, 4))
        cl = [np.asarray(c, np.float32).reshape(-1) for c in circles]
        c = np.ascontiguousarray(np.concatenate(cl)) if sum(x.size for x in cl) else np.zeros(3, np.float32)
        self._check(self.lib.sepso_batch_set_inputs(self._h, fptr(h), fptr(pts), fptr(c)))

    def set_shape(self, tile: int, threads: int):
        from ._native import BatchShape
        sh = BatchShape(tile=tile, threads=threads, lanes=32, reserved=0)
        self._check(self.lib.sepso_batch_set_shape(self._h, ctypes.byref(sh)))

    def shape(self) -> dict:
        from ._native import BatchShape
        sh, n = BatchShape(), ctypes.c_int32()
        self._check(self.lib.sepso_batch_get_shape(self._h, ctypes.byref(sh), ctypes.byref(n)))
        return {"tile": sh.tile, "threads": sh.threads, "lanes": sh.lanes, "work_items": n.value}

    def autotune(self, trial_launches: int = 3):
        from ._native import BatchShape
        sh, ms = BatchShape(), ctypes.c_float()
        self._check(self.lib.sepso_batch_autotune(self._h, trial_launches, ctypes.byref(sh),
                                                  ctypes.byref(ms)))
        return {"tile": sh.tile, "threads": sh.threads, "lanes": sh.lanes}, float(ms.value)

    @property
    def Dmax(self) -> int:
        return max(self.D)

    def set_starts(self, prev: torch.Tensor | None = None, prior: torch.Tensor | None = None,
                   has_prev=None):
        """Warm starts of the next run: device tensors (n, >= Dmax) of previous paths
        (PI centres) and/or learned-prior proposals; has_prev: n flags."""
        ld = None
        for t in (prev, prior):
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.stride(1) == 1
                assert t.shape[0] >= self.n and t.shape[1] >= self.Dmax
                assert ld is None or ld == t.stride(0), "prev and prior need the same row stride"
                ld = t.stride(0)
        hp = None
        if has_prev is not None:
            hp = np.ascontiguousarray(np.asarray(has_prev, np.int32).reshape(self.n))
        self._check(self.lib.sepso_batch_set_starts(
            self._h, ctypes.c_void_p(prev.data_ptr()) if prev is not None else None,
            ctypes.c_void_p(prior.data_ptr()) if prior is not None else None, ld or self.Dmax,
            hp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if hp is not None else None))

    def set_teams(self, team_first, team_size, sep: float):
        """Multi-agent teams: scene s's team is scenes [team_first[s], team_first[s] +
        team_size[s]); agents closer than sep during a step conflict."""
        f = np.ascontiguousarray(np.asarray(team_first, np.int32).reshape(self.n))
        z = np.ascontiguousarray(np.asarray(team_size, np.int32).reshape(self.n))
        self._check(self.lib.sepso_batch_set_teams(self._h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                   z.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                                   ctypes.c_float(sep)))

    def next_round(self, cycle: int):
        """Each scene's last result becomes its agent's path for the mates and its
        PI centre; the next run plans round ``cycle``."""
        self._check(self.lib.sepso_batch_next_round(self._h, ctypes.c_uint32(cycle)))

    def prior_used(self) -> int:
        n = ctypes.c_int32()
        self._check(self.lib.sepso_batch_prior_used(self._h, ctypes.byref(n)))
        return n.value

    def run_async(self, use_graph: bool = True):
        self._check(self.lib.sepso_batch_run_async(self._h, int(use_graph)))

    def read(self):
        total = sum(self.D)
        wp = np.zeros(max(total, 1), np.float32)
        res = (Result * self.n)()
        self._check(self.lib.sepso_batch_read(self._h, fptr(wp), res))
        out, off = [], 0
        for i in range(self.n):
            d = self.D[i]
            out.append({"waypoints": wp[off:off + d].copy(), "cost": res[i].cost,
                        "length": res[i].length, "Q": res[i].Q, "iters": res[i].iters,
                        "status": res[i].status})
            off += d
        return out

    def run(self, use_graph: bool = True):
        self.run_async(use_graph)
        return self.read()

    def launch_count(self) -> int:
        return int(self.lib.sepso_batch_launch_count(self._h))


class Server:
    """Continuous-batching request server (sepso_server_*): submit, tick, poll."""

    def __init__(self, n_agents: int, max_slots: int, G: int = 8, N: int = 32, Tmax: int = 40,
                 Omax: int = 256, max_iters: int = 100, stall_iters: int = 10, stall_tol: float = 0.0,
                 alpha: float = 30.0, beta: int = 4, pi_gamma: float = 0.25,
                 pi_halfwidth: float = 20.0, map_w: float = 400.0, map_h: float = 400.0,
                 seed: int = 0, mem_budget: int = 0, tile: int = 0, threads: int = 0, device=None,
                 stream: torch.cuda.Stream | None = None):
        from ._native import ServerConfig, check_server
        self.lib = _native.lib()
        self._check = check_server
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.cfg = ServerConfig(n_agents=n_agents, max_slots=max_slots, mem_budget=mem_budget, G=G, N=N,
                                Tmax=Tmax, Omax=Omax, max_iters=max_iters, stall_iters=stall_iters,
                                stall_tol=stall_tol, alpha=alpha, beta=beta, pi_gamma=pi_gamma,
                                pi_halfwidth=pi_halfwidth, map_w=map_w, map_h=map_h, seed=seed,
                                tile=tile, threads=threads)
        size, slots = ctypes.c_size_t(), ctypes.c_int32()
        check_server(self.lib.sepso_server_workspace_size(ctypes.byref(self.cfg), ctypes.byref(size),
                                                         ctypes.byref(slots)))
        self.slots = slots.value
        self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check_server(self.lib.sepso_server_create(ctypes.byref(self.cfg),
                                                      ctypes.c_void_p(self.workspace.data_ptr()), size.value,
                                                      ctypes.c_void_p(self.stream.cuda_stream),
                                                      ctypes.byref(self._h)))
        self.Dm = 2 * Tmax
        self.G = G

    def close(self):
        if self._h:
            self.lib.sepso_server_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_hyper(self, hyper, agent: int = -1):
        h = _f32(hyper, (self.G, 6))
        self._check(self.lib.sepso_server_set_hyper(self._h, agent, fptr(h)))

    def set_prior(self, prior, n_prior: int, first_row: int = 0):
        """Attach a learned prior (``prior.Prior`` on this server's stream and map) whose
        proposals seed n_prior particles per group of every admitted request, using
        its dataset rows [first_row, first_row + slots); ``None`` detaches it."""
        h = prior._h if prior is not None else None
        self._check(self.lib.sepso_server_set_prior(self._h, h, int(n_prior), int(first_row)))
        self._prior = prior  # the prior must outlive its attachment

    def submit(self, agent: int, T: int, start, target, circles, tag: int):
        c = _f32(circles, (-1, 3))
        self._check(self.lib.sepso_server_submit(self._h, agent, T, fptr(_f32(start)), fptr(_f32(target)),
                                                 fptr(c) if c.size else None, c.shape[0], tag))

    def submit_at(self, agent: int, T: int, start, target, circles, tag: int, arrival_s: float):
        c = _f32(circles, (-1, 3))
        self._check(self.lib.sepso_server_submit_at(self._h, agent, T, fptr(_f32(start)),
                                                    fptr(_f32(target)), fptr(c) if c.size else None,
                                                    c.shape[0], tag, float(arrival_s)))

    def submit_polygons(self, agent: int, T: int, start, target, edges, tag: int, arrival_s: float = -1.0):
        """A request among polygon obstacles: edges (E, 4) as x0, y0, x1, y1."""
        e = _f32(edges, (-1, 4))
        self._check(self.lib.sepso_server_submit_polygons(self._h, agent, T, fptr(_f32(start)),
                                                          fptr(_f32(target)), fptr(e) if e.size else None,
                                                          e.shape[0], tag, float(arrival_s)))

    def clock(self, restart: bool = False) -> float:
        return float(self.lib.sepso_server_clock(self._h, int(restart)))

    def run(self, max_ticks: int = 100_000_000):
        self._check(self.lib.sepso_server_run(self._h, max_ticks))

    def tick(self):
        a, q = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.sepso_server_tick(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def poll(self, max_n: int = 4096):
        from ._native import ServerDone
        out = (ServerDone * max_n)()
        wp = np.zeros(max_n * self.Dm, np.float32)
        n = ctypes.c_int32()
        self._check(self.lib.sepso_server_poll(self._h, out, fptr(wp), max_n, ctypes.byref(n)))
        res = []
        for i in range(n.value):
            d = out[i]
            res.append({"tag": d.tag, "agent": d.agent, "T": d.T, "cost": d.res.cost,
                        "length": d.res.length, "Q": d.res.Q, "iters": d.res.iters,
                        "status": d.res.status, "arrival_s": d.arrival_s, "finish_s": d.finish_s,
                        "waypoints": wp[i * self.Dm:i * self.Dm + 2 * d.T].copy()})
        return res

    def drain(self, max_ticks: int = 1_000_000):
        self._check(self.lib.sepso_server_drain(self._h, max_ticks))

    def stats(self) -> dict:
        s = ctypes.c_int32()
        v = [ctypes.c_int64() for _ in range(4)]
        self._check(self.lib.sepso_server_stats(self._h, ctypes.byref(s), *[ctypes.byref(x) for x in v]))
        return dict(slots=s.value, admitted=v[0].value, completed=v[1].value, ticks=v[2].value,
                    launches=v[3].value)
