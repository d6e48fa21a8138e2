"""FP64 CPU oracle for the SEPSO hot path (ctypes binding of ``sepso_oracle.c``).

TEST INFRASTRUCTURE ONLY: this package is imported by ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``, never by the
product package ``paper_2308_10169_gb300``.  It shares no code with the CUDA path;
both sides consume the same seeded inputs (plain arrays) and nothing else.

What each function follows (paper: arXiv 2308.10169):

* ``philox`` / ``u01``      -- Philox4x32-10 (Salmon et al., SC'11); supplies the
  uniform R1, R2, R3 of Table EXP_TOF (one scalar per particle per iteration).
* ``seg_point_dist``        -- point-to-segment distance, the plain definition.
* ``evaluate``              -- Eqs. path_fit, lenth, penalty (Sec. 3.3.2).
* ``Swarm.init``            -- Algorithm 1 initialisation with Priori
  Initialization (Sec. 3.3.3).
* ``Swarm.iteration``       -- one pass of Algorithm 1: fitness, P/G/T update,
  Eq. TOF_omega, Eq. TOF_V (clip), Eq. TOF_X (clip).
* ``Swarm.plan``            -- one planning cycle with Auto Truncation (Sec. 3.3.4).
* ``advance_scene``         -- the dynamic simulator step (Fig. PP caption).
* ``bf_value`` / ``BFSwarm`` -- the benchmark functions BF1-BF4 (Table BFs, their
  textbook definitions) and DTPSO on them: the same Algorithm 1 iteration as
  ``Swarm`` with that objective over the box [lo, hi]^D; with ``fn = 5`` the
  objective is a path among polygon obstacles (Sec. 3.3.1, Eq. penalty with Q the
  number of path-segment / obstacle-edge crossings, ``seg_cross``); with ``fn = 6``
  it is a path in three dimensions among spheres (the Conclusion's extension from
  2D to 3D planning: Eqs. path_fit / lenth / penalty with a third coordinate and Q
  the number of (segment, sphere) pairs closer than the radius,
  ``seg_point_dist3``, ``Scene3``).
* ``hsef``                  -- the hierarchical self-evolving framework
  (Sec. 3.2.1, Eq. fit_h).
* ``raster`` / ``prior_encode`` / ``prior_decode`` / ``Mlp`` / ``adam`` -- the
  learned prior (``prior_oracle.c``): occupancy raster features, label encoding,
  MLP forward, loss gradient and the Adam step (Kingma and Ba, 2015).

Parity status of each function is recorded in the tests that pin it
(``tests/test_oracle_*.py``).  HSEF is pinned by its invariants, by Eq. fit_h (the
best H-fitness is the LFV of an L-run with the best hyper-parameters) and by its
H-swarm update (inertia, the three attractors with their own rows and distinct
factors, velocity and box clipping, through ``hsef_state``); the paper prints no
HSEF values to compare with (only a figure).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRCS = [_HERE / "sepso_oracle.c", _HERE / "prior_oracle.c"]
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libsepso_oracle.so"

_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u32p = ctypes.POINTER(ctypes.c_uint32)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (plain -O2, no FMA contraction)."""
    _BUILD.mkdir(exist_ok=True)
    stale = not _LIB_PATH.exists() or any(_LIB_PATH.stat().st_mtime < f.stat().st_mtime for f in _SRCS)
    if force or stale:
        tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(
            ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
             *[str(f) for f in _SRCS], "-o", str(tmp), "-lm"],
            check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Config(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_int32), ("G", ctypes.c_int32), ("N", ctypes.c_int32),
        ("W", ctypes.c_double), ("H", ctypes.c_double),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_int32),
        ("max_iters", ctypes.c_int32),
        ("at_mode", ctypes.c_int32), ("tw", ctypes.c_int32), ("delta", ctypes.c_double),
        ("stall_iters", ctypes.c_int32), ("stall_tol", ctypes.c_double),
        ("use_pi", ctypes.c_int32), ("pi_gamma", ctypes.c_double), ("pi_h", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("run_id", ctypes.c_uint32),
        ("problem", ctypes.c_int32), ("Dbf", ctypes.c_int32),
        ("lo", ctypes.c_double), ("hi", ctypes.c_double),
        ("Z", ctypes.c_double),
    ]


class _Scene(ctypes.Structure):
    _fields_ = [("sx", ctypes.c_double), ("sy", ctypes.c_double),
                ("tx", ctypes.c_double), ("ty", ctypes.c_double),
                ("O", ctypes.c_int32), ("circ", _f64p),
                ("E", ctypes.c_int32), ("edges", _f64p),
                ("A", ctypes.c_int32), ("agents", _f64p), ("sep", ctypes.c_double),
                ("sz", ctypes.c_double), ("tz", ctypes.c_double),
                ("S", ctypes.c_int32), ("spheres", _f64p)]


class _State(ctypes.Structure):
    _fields_ = [(n, _f64p) for n in ("X", "V", "P", "Pfit")] + [("PQ", _i32p)] + \
        [(n, _f64p) for n in ("Gb", "Gfit")] + [("GQ", _i32p)] + \
        [(n, _f64p) for n in ("Tb", "Tfit")] + [("TQ", _i32p), ("k", _i32p)] + \
        [("cycle", _i32p), ("has_prev", _i32p), ("prevT", _f64p), ("win", _f64p),
         ("win_n", _i32p), ("win_head", _i32p), ("stall", _i32p), ("prev_lfv", _f64p),
         ("n_prior", _i32p), ("priorT", _f64p)]


class _HsefCfg(ctypes.Structure):
    _fields_ = [("HG", ctypes.c_int32), ("HN", ctypes.c_int32), ("E", ctypes.c_int32),
                ("hhyper", _f64p), ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("l_vlimit", ctypes.c_double), ("hseed", ctypes.c_uint64)]


class _MlpDims(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("H1", ctypes.c_int32), ("H2", ctypes.c_int32),
                ("O", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(str(build()))
        L.so_philox_batch.argtypes = [ctypes.c_int32, _u32p, ctypes.c_uint64, _u32p]
        L.so_u01.argtypes = [ctypes.c_uint32]
        L.so_u01.restype = ctypes.c_double
        L.so_seg_point_dist.argtypes = [ctypes.c_double] * 6
        L.so_seg_point_dist.restype = ctypes.c_double
        L.so_seg_point_dist3.argtypes = [_f64p, _f64p, _f64p]
        L.so_seg_point_dist3.restype = ctypes.c_double
        L.so_sphere_margin.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene), ctypes.c_int32,
                                       _f64p, _f64p]
        L.so_evaluate.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene), ctypes.c_int32,
                                  _f64p, _f64p, _i32p, _f64p]
        L.so_tangency_margin.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene),
                                         ctypes.c_int32, _f64p, _f64p]
        L.so_pi_count.argtypes = [ctypes.c_double, ctypes.c_int32]
        L.so_pi_count.restype = ctypes.c_int32
        L.so_init_swarm.argtypes = [ctypes.POINTER(_Config), _f64p, ctypes.POINTER(_State)]
        L.so_window_std.argtypes = [_f64p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        L.so_bf_value.argtypes = [ctypes.c_int32, ctypes.c_int32, _f64p]
        L.so_bf_value.restype = ctypes.c_double
        L.so_seg_cross.argtypes = [ctypes.c_double] * 8
        L.so_seg_cross.restype = ctypes.c_int32
        L.so_poly_margin.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene), ctypes.c_int32,
                                     _f64p, _f64p]
        L.so_window_std.restype = ctypes.c_double
        L.so_at_update.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_State)]
        L.so_at_update.restype = ctypes.c_int32
        L.so_iteration.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene), _f64p,
                                   ctypes.POINTER(_State), ctypes.c_int32]
        L.so_iteration.restype = ctypes.c_int32
        L.so_plan.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene), _f64p,
                              ctypes.POINTER(_State), _f64p]
        L.so_step.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene), _f64p,
                              ctypes.POINTER(_State), ctypes.c_int32]
        L.so_advance_scene.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.so_advance_polygons.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int32, _i32p,
                                          _f64p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.so_hsef.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene),
                              ctypes.POINTER(_HsefCfg), _f64p, _f64p, _f64p]
        L.so_hsef_state.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(_Scene),
                                    ctypes.POINTER(_HsefCfg), _f64p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                    _f64p, _f64p]
        L.so_mlp_num_params.argtypes = [ctypes.POINTER(_MlpDims)]
        L.so_mlp_num_params.restype = ctypes.c_long
        L.so_raster.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32, _f64p,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int32, _f64p]
        L.so_prior_encode.argtypes = [ctypes.c_int32] + [ctypes.c_double] * 6 + [_f64p, _f64p]
        L.so_prior_decode.argtypes = [ctypes.c_int32] + [ctypes.c_double] * 6 + [_f64p, _f64p]
        L.so_mlp_forward.argtypes = [ctypes.POINTER(_MlpDims), _f64p, ctypes.c_int32, _f64p, _f64p,
                                     _f64p, _f64p]
        L.so_mlp_loss_grad.argtypes = [ctypes.POINTER(_MlpDims), _f64p, ctypes.c_int32, _f64p, _f64p,
                                       _f64p]
        L.so_mlp_loss_grad.restype = ctypes.c_double
        L.so_adam.argtypes = [ctypes.c_long, _f64p, _f64p, _f64p, _f64p, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        _lib = L
    return _lib


def _p64(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_f64p)


def _p32(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(_i32p)


def _cfg(c) -> _Config:
    """Build the C struct from any object carrying the planner's config fields."""
    return _Config(T=c.T, G=c.G, N=c.N, W=float(np.float32(c.map_w)), H=float(np.float32(c.map_h)),
                   alpha=float(np.float32(c.alpha)), beta=c.beta, max_iters=c.max_iters,
                   at_mode=c.at_mode, tw=c.tw, delta=float(np.float32(c.delta)),
                   stall_iters=c.stall_iters, stall_tol=float(np.float32(c.stall_tol)),
                   use_pi=int(c.use_pi), pi_gamma=float(np.float32(c.pi_gamma)),
                   pi_h=float(np.float32(c.pi_halfwidth)), seed=c.seed, run_id=c.run_id,
                   problem=5 if getattr(c, "obstacle_kind", 0) == 1 else 0)


class Scene:
    """A static scene in FP64 (converted exactly from the FP32 inputs)."""

    def __init__(self, start, target, circles, edges=None, agents=None, sep: float = 0.0):
        """agents: the other agents' timed paths, (A, 2 (T + 2)) -- x of start,
        waypoints, target, then the y's; sep: the separation below which two agents
        conflict (multi-agent extension)."""
        self.start = np.asarray(start, dtype=np.float64).reshape(2).copy()
        self.target = np.asarray(target, dtype=np.float64).reshape(2).copy()
        self.circles = np.ascontiguousarray(np.asarray(circles, dtype=np.float64).reshape(-1, 3))
        e = np.zeros((0, 4)) if edges is None else edges
        self.edges = np.ascontiguousarray(np.asarray(e, dtype=np.float64).reshape(-1, 4))
        a = np.zeros((0, 2)) if agents is None else np.asarray(agents, dtype=np.float64)
        self.agents = np.ascontiguousarray(a if a.ndim == 2 else a.reshape(1, -1))
        self.sep = float(np.float32(sep))

    def c(self) -> _Scene:
        return _Scene(sx=self.start[0], sy=self.start[1], tx=self.target[0], ty=self.target[1],
                      O=self.circles.shape[0], circ=_p64(self.circles),
                      E=self.edges.shape[0], edges=_p64(self.edges),
                      A=self.agents.shape[0], agents=_p64(self.agents), sep=self.sep)


class Scene3:
    """A static 3D scene in FP64 (the Conclusion's 3D extension): start and target
    (3,), spheres (S, 4) rows (cx, cy, cz, r)."""

    def __init__(self, start, target, spheres):
        self.start = np.asarray(start, dtype=np.float64).reshape(3).copy()
        self.target = np.asarray(target, dtype=np.float64).reshape(3).copy()
        self.spheres = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
        self._none = np.zeros((1, 4))

    def c(self) -> _Scene:
        return _Scene(sx=self.start[0], sy=self.start[1], tx=self.target[0], ty=self.target[1],
                      O=0, circ=_p64(self._none), E=0, edges=_p64(self._none), A=0,
                      agents=_p64(self._none), sep=0.0, sz=self.start[2], tz=self.target[2],
                      S=self.spheres.shape[0], spheres=_p64(self.spheres))


# ----------------------------------------------------------------------------
# Philox and uniforms
# ----------------------------------------------------------------------------

def philox(ctr: np.ndarray, seed: int) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib().so_philox_batch(ctr.shape[0], ctr.ctypes.data_as(_u32p), ctypes.c_uint64(seed),
                          out.ctypes.data_as(_u32p))
    return out


def u01(x: int) -> float:
    return lib().so_u01(int(x))


# ----------------------------------------------------------------------------
# Fitness
# ----------------------------------------------------------------------------

def seg_point_dist(a, b, c) -> float:
    return lib().so_seg_point_dist(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                   float(c[0]), float(c[1]))


def seg_point_dist3(a, b, c) -> float:
    """Distance from point c to the closed segment [a, b] in three dimensions."""
    v = [np.ascontiguousarray(np.asarray(u, np.float64).reshape(3)) for u in (a, b, c)]
    return lib().so_seg_point_dist3(_p64(v[0]), _p64(v[1]), _p64(v[2]))


def evaluate(cfg, scene: Scene, X: np.ndarray):
    """Fitness F, collision count Q and length of each row of X (n x 2T)."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 2 * cfg.T))
    n = X.shape[0]
    F = np.zeros(n, np.float64)
    Q = np.zeros(n, np.int32)
    L = np.zeros(n, np.float64)
    c = _cfg(cfg)
    s = scene.c()
    lib().so_evaluate(ctypes.byref(c), ctypes.byref(s), n, _p64(X), _p64(F), _p32(Q), _p64(L))
    return F, Q, L


def tangency_margin(cfg, scene: Scene, X: np.ndarray) -> np.ndarray:
    """Per particle, min over its (segment, circle) pairs of |dist - r|."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, 2 * cfg.T))
    m = np.zeros(X.shape[0])
    c = _cfg(cfg)
    s = scene.c()
    lib().so_tangency_margin(ctypes.byref(c), ctypes.byref(s), X.shape[0], _p64(X), _p64(m))
    return m


def pi_count(gamma: float, N: int) -> int:
    return lib().so_pi_count(float(np.float32(gamma)), N)


def window_std(values) -> float:
    v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
    return lib().so_window_std(_p64(v), v.size, v.size, 0)


# ----------------------------------------------------------------------------
# Swarm state
# ----------------------------------------------------------------------------

STATE_FIELDS = ("X", "V", "P", "Pfit", "PQ", "Gb", "Gfit", "GQ", "Tb", "Tfit", "TQ", "k",
                "cycle", "has_prev", "prevT", "win", "win_n", "win_head", "stall", "prev_lfv",
                "n_prior", "priorT")


class Swarm:
    """Owns the FP64 swarm state of one planner (Table EXP_TOF tensors)."""

    def __init__(self, cfg, hyper):
        self.cfg = cfg
        T, G, N = cfg.T, cfg.G, cfg.N
        D, M = 2 * T, G * N
        self.hyper = np.ascontiguousarray(np.asarray(hyper, dtype=np.float64).reshape(G, 6))
        tw = max(cfg.tw, 1)
        f = np.zeros
        self.s = {
            "X": f(M * D), "V": f(M * D), "P": f(M * D), "Pfit": np.full(M, np.inf),
            "PQ": f(M, np.int32), "Gb": f(G * D), "Gfit": np.full(G, np.inf), "GQ": f(G, np.int32),
            "Tb": f(D), "Tfit": np.full(1, np.inf), "TQ": f(1, np.int32), "k": f(1, np.int32),
            "cycle": f(1, np.int32), "has_prev": f(1, np.int32), "prevT": f(D), "win": f(tw),
            "win_n": f(1, np.int32), "win_head": f(1, np.int32), "stall": f(1, np.int32),
            "prev_lfv": np.full(1, np.inf),
            # optional second seed (a learned prior's proposal): n_prior particles per
            # group start around priorT, before PI's
            "n_prior": f(1, np.int32), "priorT": f(D),
        }
        self._c = _cfg(cfg)

    def _st(self) -> _State:
        kw = {}
        for name in STATE_FIELDS:
            a = self.s[name]
            kw[name] = _p32(a) if a.dtype == np.int32 else _p64(a)
        return _State(**kw)

    def set_hyper(self, hyper):
        self.hyper[...] = np.asarray(hyper, dtype=np.float64).reshape(self.hyper.shape)

    def load(self, state: dict):
        """Copy arrays (any float/int dtype) into the state, by field name."""
        for k, v in state.items():
            if k in self.s:
                self.s[k][...] = np.asarray(v).reshape(self.s[k].shape).astype(self.s[k].dtype)

    def state(self) -> dict:
        return {k: v.copy() for k, v in self.s.items()}

    def init(self):
        st = self._st()
        lib().so_init_swarm(ctypes.byref(self._c), _p64(self.hyper), ctypes.byref(st))

    def iteration(self, scene: Scene, check_stop: bool = False) -> bool:
        st = self._st()
        s = scene.c()
        return bool(lib().so_iteration(ctypes.byref(self._c), ctypes.byref(s), _p64(self.hyper),
                                       ctypes.byref(st), int(check_stop)))

    def step(self, scene: Scene, iters: int):
        st = self._st()
        s = scene.c()
        lib().so_step(ctypes.byref(self._c), ctypes.byref(s), _p64(self.hyper), ctypes.byref(st),
                      int(iters))

    def at_update(self) -> bool:
        st = self._st()
        return bool(lib().so_at_update(ctypes.byref(self._c), ctypes.byref(st)))

    def plan(self, scene: Scene) -> dict:
        D = 2 * self.cfg.T
        res = np.zeros(D + 4)
        st = self._st()
        s = scene.c()
        lib().so_plan(ctypes.byref(self._c), ctypes.byref(s), _p64(self.hyper), ctypes.byref(st),
                      _p64(res))
        return {"waypoints": res[:D].copy(), "cost": float(res[D]), "length": float(res[D + 1]),
                "Q": int(res[D + 2]), "iters": int(res[D + 3])}


# ----------------------------------------------------------------------------
# Benchmark functions (Table BFs) and DTPSO on them
# ----------------------------------------------------------------------------

def bf_value(fn: int, x) -> float:
    """BF1..BF4 (Sphere, Rosenbrock, Rastrigin, Griewank) at one point, FP64."""
    v = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1))
    return lib().so_bf_value(int(fn), v.size, _p64(v))


def _bf_cfg(c) -> _Config:
    """The C config of a run of the generic engine (any object with BFConfig's fields):
    a benchmark function (fn 1..4), a path among polygons (fn 5, D = 2T) or a 3D
    path among spheres (fn 6, D = 3T); Priori Initialization when pi_gamma > 0."""
    f32 = lambda v: float(np.float32(v))
    T = c.D // 2 if c.fn == 5 else (c.D // 3 if c.fn == 6 else 0)
    return _Config(T=T, G=c.G, N=c.N, W=f32(c.map_w), H=f32(c.map_h),
                   alpha=f32(c.alpha), beta=c.beta, max_iters=c.max_iters,
                   at_mode=2 if getattr(c, "at_stall", 0) > 0 else 0, tw=1, delta=0.0,
                   stall_iters=getattr(c, "at_stall", 0), stall_tol=f32(getattr(c, "stall_tol", 0.0)), seed=c.seed,
                   run_id=c.run_id, problem=c.fn, Dbf=c.D,
                   lo=f32(c.lo), hi=f32(c.hi), Z=f32(getattr(c, "map_d", 0.0)),
                   use_pi=int(getattr(c, "pi_gamma", 0.0) > 0.0), pi_gamma=f32(getattr(c, "pi_gamma", 0.0)),
                   pi_h=f32(getattr(c, "pi_halfwidth", 0.0)))


def seg_cross(a, b, c, d) -> bool:
    """Proper crossing of segments ab and cd (Sec. 3.3.1's segment intersection)."""
    return bool(lib().so_seg_cross(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                   float(c[0]), float(c[1]), float(d[0]), float(d[1])))


def poly_margin(cfg, scene: "Scene", X) -> np.ndarray:
    """Per path: distance of its crossing decisions from a flip (parity tests)."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, cfg.D))
    m = np.zeros(X.shape[0])
    c = _cfg(cfg) if hasattr(cfg, "obstacle_kind") else _bf_cfg(cfg)
    s = scene.c()
    lib().so_poly_margin(ctypes.byref(c), ctypes.byref(s), X.shape[0], _p64(X), _p64(m))
    return m


def sphere_margin(cfg, scene: "Scene3", X) -> np.ndarray:
    """Per 3D path (rows of X, D = 3T): min over its (segment, sphere) pairs of |dist - r|."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, cfg.D))
    m = np.zeros(X.shape[0])
    c = _bf_cfg(cfg)
    s = scene.c()
    lib().so_sphere_margin(ctypes.byref(c), ctypes.byref(s), X.shape[0], _p64(X), _p64(m))
    return m


class BFSwarm(Swarm):
    """DTPSO (Algorithm 1 with Table hyper8-style rows) on a benchmark function:
    the iteration of ``Swarm`` with objective BF``fn`` over [lo, hi]^D, no PI, no AT,
    a fixed number of iterations (``max_iters`` is also the T of Eq. TOF_omega)."""

    _EMPTY = None

    def __init__(self, cfg, hyper, scene: "Scene" = None):
        self.cfg = cfg
        G, N, D = cfg.G, cfg.N, cfg.D
        M = G * N
        self.hyper = np.ascontiguousarray(np.asarray(hyper, dtype=np.float64).reshape(G, 6))
        f = np.zeros
        self.s = {
            "X": f(M * D), "V": f(M * D), "P": f(M * D), "Pfit": np.full(M, np.inf),
            "PQ": f(M, np.int32), "Gb": f(G * D), "Gfit": np.full(G, np.inf), "GQ": f(G, np.int32),
            "Tb": f(D), "Tfit": np.full(1, np.inf), "TQ": f(1, np.int32), "k": f(1, np.int32),
            "cycle": f(1, np.int32), "has_prev": f(1, np.int32), "prevT": f(D), "win": f(1),
            "win_n": f(1, np.int32), "win_head": f(1, np.int32), "stall": f(1, np.int32),
            "prev_lfv": np.full(1, np.inf), "n_prior": f(1, np.int32), "priorT": f(D),
        }
        self._c = _bf_cfg(cfg)
        self._none = scene if scene is not None else Scene((0.0, 0.0), (0.0, 0.0), np.zeros((0, 3)))

    def set_scene(self, scene):
        """The scene of the next iterations (a dynamic run's new obstacle positions)."""
        self._none = scene

    def set_previous(self, prevT, cycle: int):
        """Priori Initialization for the next ``init`` (Sec. 3.3.3): the first
        ceil(pi_gamma N) particles of each group start within +-pi_halfwidth of the
        previous best path ``prevT``; ``cycle`` enters every Philox counter."""
        self.s["prevT"][...] = np.asarray(prevT, np.float64).reshape(-1)
        self.s["has_prev"][0] = 1
        self.s["cycle"][0] = int(cycle)

    def evaluate(self, X, with_q: bool = False):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, self.cfg.D))
        F = np.zeros(X.shape[0])
        Q = np.zeros(X.shape[0], np.int32)
        s = self._none.c()
        lib().so_evaluate(ctypes.byref(self._c), ctypes.byref(s), X.shape[0], _p64(X), _p64(F),
                          _p32(Q), None)
        return (F, Q) if with_q else F

    def iteration(self, scene=None, check_stop: bool = False) -> bool:
        return super().iteration(self._none, False)

    def iteration_stop(self) -> bool:
        """One iteration in planning mode (Auto Truncation and the cap); True when the
        cycle ends here (the update of this iteration is then not applied)."""
        return super().iteration(self._none, True)

    def step(self, scene=None, iters: int = 1):
        super().step(self._none, iters)

    def plan(self) -> dict:
        """One planning cycle (Algorithm 1 with Auto Truncation when the config sets
        at_stall, else max_iters iterations): initialise (PI when set_previous gave a
        previous path), iterate until AT fires or the cap is reached; the stopping
        iteration's bests are kept and no particle moves after it."""
        self.s["stall"][0] = 0
        self.s["prev_lfv"][0] = np.inf
        self.init()
        st = self._st()
        s = self._none.c()
        while not lib().so_iteration(ctypes.byref(self._c), ctypes.byref(s), _p64(self.hyper), ctypes.byref(st), 1):
            pass
        return {"iters": int(self.s["k"][0]), "cost": float(self.s["Tfit"][0]), "Q": int(self.s["TQ"][0]),
                "waypoints": self.s["Tb"].copy()}

    def run(self, iters: int) -> np.ndarray:
        """Initialise, then ``iters`` iterations; returns Tfit after each one."""
        self.init()
        hist = np.zeros(iters)
        for i in range(iters):
            super().iteration(self._none, False)
            hist[i] = self.s["Tfit"][0]
        return hist


# ----------------------------------------------------------------------------
# Dynamic scene and HSEF
# ----------------------------------------------------------------------------

def advance_scene(W, H, circles, cvel, start, svel, target, tvel):
    """One dynamic step, in place, on FP64 copies; returns the new arrays."""
    c = np.ascontiguousarray(np.asarray(circles, np.float64).reshape(-1, 3)).copy()
    v = np.ascontiguousarray(np.asarray(cvel, np.float64).reshape(-1, 2)).copy()
    s = np.asarray(start, np.float64).reshape(2).copy()
    sv = np.asarray(svel, np.float64).reshape(2).copy()
    t = np.asarray(target, np.float64).reshape(2).copy()
    tv = np.asarray(tvel, np.float64).reshape(2).copy()
    lib().so_advance_scene(float(np.float32(W)), float(np.float32(H)), c.shape[0], _p64(c), _p64(v),
                           _p64(s), _p64(sv), _p64(t), _p64(tv))
    return c, v, s, sv, t, tv


def timed_path(start, target, waypoints, T: int) -> np.ndarray:
    """An agent's timed path for Scene(agents=...): start, T waypoints ([x..., y...]),
    target -> (2 (T + 2),) = x_0..x_{T+1}, y_0..y_{T+1}."""
    w = np.asarray(waypoints, np.float64).reshape(2 * T)
    xs = np.concatenate([[start[0]], w[:T], [target[0]]])
    ys = np.concatenate([[start[1]], w[T:], [target[1]]])
    return np.concatenate([xs, ys])


def multi_agent_plan(cfg, hyper, circles, starts, targets, sep: float, rounds: int, seeds=None) -> list:
    """The multi-agent extension by rounds of simultaneous best responses: in round 0
    every agent plans alone; in round r each plans (a fresh planning cycle of
    Algorithm 1 with PI around its own previous path) against the other agents'
    paths of round r - 1 as moving obstacles.  Agent a uses Philox run id run_id + a
    (its own streams).  Returns per round the list of each agent's result."""
    A = len(starts)
    T = cfg.T
    sws = [Swarm(replace_cfg(cfg, run_id=cfg.run_id + a), hyper) for a in range(A)]
    out, paths = [], None
    for r in range(rounds):
        res = []
        for a in range(A):
            others = None if paths is None else np.stack([paths[b] for b in range(A) if b != a])
            sc = Scene(starts[a], targets[a], circles, agents=others, sep=sep if others is not None else 0.0)
            res.append(sws[a].plan(sc))
        paths = [timed_path(starts[a], targets[a], res[a]["waypoints"], T) for a in range(A)]
        out.append(res)
    return out


def replace_cfg(cfg, **kw):
    import dataclasses
    return dataclasses.replace(cfg, **kw)


def advance_polygons(W, H, edges, offsets, pvel, start, svel, target, tvel):
    """One dynamic step of polygon obstacles (rigid translation, bounding-box bounce)
    and of start/target, on FP64 copies; returns (edges, pvel, start, svel, target, tvel)."""
    e = np.ascontiguousarray(np.asarray(edges, np.float64).reshape(-1, 4)).copy()
    off = np.ascontiguousarray(np.asarray(offsets, np.int32).reshape(-1))
    v = np.ascontiguousarray(np.asarray(pvel, np.float64).reshape(-1, 2)).copy()
    s = np.asarray(start, np.float64).reshape(2).copy()
    sv = np.asarray(svel, np.float64).reshape(2).copy()
    t = np.asarray(target, np.float64).reshape(2).copy()
    tv = np.asarray(tvel, np.float64).reshape(2).copy()
    if off.size != v.shape[0] + 1 or off[0] != 0 or off[-1] != e.shape[0] or np.any(np.diff(off) < 0):
        raise ValueError("offsets must run from 0 to the edge count, one more entry than polygons")
    lib().so_advance_polygons(float(np.float32(W)), float(np.float32(H)), v.shape[0],
                              off.ctypes.data_as(_i32p), _p64(e), _p64(v), _p64(s), _p64(sv), _p64(t), _p64(tv))
    return e, v, s, sv, t, tv


def hsef(lcfg, scene: Scene, HG: int, HN: int, E: int, hhyper, lo, hi, l_vlimit: float,
         hseed: int):
    """Evolution phase of SEPSO; returns (best H-position, best LFV, per-evolution best)."""
    G = lcfg.G
    if G > 64:
        raise ValueError("oracle HSEF supports G <= 64")
    hh = np.ascontiguousarray(np.asarray(hhyper, np.float64).reshape(HG, 6))
    hc = _HsefCfg(HG=HG, HN=HN, E=E, hhyper=_p64(hh),
                  lo=(ctypes.c_double * 3)(*[float(np.float32(x)) for x in lo]),
                  hi=(ctypes.c_double * 3)(*[float(np.float32(x)) for x in hi]),
                  l_vlimit=float(np.float32(l_vlimit)), hseed=hseed)
    best = np.zeros(3 * G)
    bf = np.zeros(1)
    hist = np.zeros(E)
    c = _cfg(lcfg)
    s = scene.c()
    lib().so_hsef(ctypes.byref(c), ctypes.byref(s), ctypes.byref(hc), _p64(best), _p64(bf),
                  _p64(hist))
    return best, float(bf[0]), hist


def hsef_state(lcfg, scene: Scene, HG: int, HN: int, E: int, hhyper, lo, hi, l_vlimit: float,
               hseed: int) -> dict:
    """hsef() and the H-swarm state after its last update: HX, HV, HP (HG*HN x 3G),
    HGb (HG x 3G), HTb (3G), with best, bf and hist as hsef() returns them."""
    G = lcfg.G
    if G > 64:
        raise ValueError("oracle HSEF supports G <= 64")
    HM, DH = HG * HN, 3 * G
    hh = np.ascontiguousarray(np.asarray(hhyper, np.float64).reshape(HG, 6))
    hc = _HsefCfg(HG=HG, HN=HN, E=E, hhyper=_p64(hh),
                  lo=(ctypes.c_double * 3)(*[float(np.float32(x)) for x in lo]),
                  hi=(ctypes.c_double * 3)(*[float(np.float32(x)) for x in hi]),
                  l_vlimit=float(np.float32(l_vlimit)), hseed=hseed)
    out = {"best": np.zeros(DH), "bf": np.zeros(1), "hist": np.zeros(E), "HX": np.zeros((HM, DH)),
           "HV": np.zeros((HM, DH)), "HP": np.zeros((HM, DH)), "HGb": np.zeros((HG, DH)),
           "HTb": np.zeros(DH)}
    c = _cfg(lcfg)
    s = scene.c()
    lib().so_hsef_state(ctypes.byref(c), ctypes.byref(s), ctypes.byref(hc), _p64(out["best"]),
                        _p64(out["bf"]), _p64(out["hist"]), _p64(out["HX"]), _p64(out["HV"]),
                        _p64(out["HP"]), _p64(out["HGb"]), _p64(out["HTb"]))
    out["bf"] = float(out["bf"][0])
    return out



# ----------------------------------------------------------------------------
# Learned prior (prior_oracle.c)
# ----------------------------------------------------------------------------

def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, np.float64))
    return a.reshape(shape) if shape is not None else a


def raster(grid: int, W: float, H: float, circles, start, target, K: int) -> np.ndarray:
    """Features of one scene: g*g occupancy cells (decided in FP32), then start and
    target over the map extent, then zeros up to K."""
    c = _f64(circles).reshape(-1, 3).copy()
    out = np.zeros(K)
    lib().so_raster(grid, float(W), float(H), c.shape[0], _p64(c), float(start[0]), float(start[1]),
                    float(target[0]), float(target[1]), K, _p64(out))
    return out


def prior_encode(T: int, W: float, H: float, start, target, waypoints) -> np.ndarray:
    """A path's label: offset from the straight start-target line over the extent."""
    wp = _f64(waypoints, (2 * T,))
    y = np.zeros(2 * T)
    lib().so_prior_encode(T, float(W), float(H), float(start[0]), float(start[1]), float(target[0]),
                          float(target[1]), _p64(wp), _p64(y))
    return y


def prior_decode(T: int, W: float, H: float, start, target, y) -> np.ndarray:
    """Waypoints of a network output (inverse of prior_encode, clipped to the map)."""
    yy = _f64(y, (2 * T,))
    wp = np.zeros(2 * T)
    lib().so_prior_decode(T, float(W), float(H), float(start[0]), float(start[1]), float(target[0]),
                          float(target[1]), _p64(yy), _p64(wp))
    return wp


class Mlp:
    """h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3 in FP64, with the
    parameters as one flat vector W1, b1, W2, b2, W3, b3 (row-major)."""

    def __init__(self, K: int, H1: int, H2: int, O: int):
        self.dims = _MlpDims(K=K, H1=H1, H2=H2, O=O)
        self.K, self.H1, self.H2, self.O = K, H1, H2, O

    @property
    def num_params(self) -> int:
        return int(lib().so_mlp_num_params(ctypes.byref(self.dims)))

    def split(self, flat) -> dict:
        """Views of the six tensors of a flat parameter vector."""
        f = np.asarray(flat)
        K, H1, H2, O = self.K, self.H1, self.H2, self.O
        out, o = {}, 0
        for name, shape in (("W1", (H1, K)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)),
                            ("W3", (O, H2)), ("b3", (O,))):
            n = int(np.prod(shape))
            out[name] = f[o:o + n].reshape(shape)
            o += n
        return out

    def forward(self, params, X):
        p = _f64(params, (self.num_params,))
        x = _f64(X).reshape(-1, self.K)
        B = x.shape[0]
        h1, h2, y = np.zeros((B, self.H1)), np.zeros((B, self.H2)), np.zeros((B, self.O))
        lib().so_mlp_forward(ctypes.byref(self.dims), _p64(p), B, _p64(x), _p64(h1), _p64(h2), _p64(y))
        return h1, h2, y

    def loss_grad(self, params, X, targets):
        """(loss, flat gradient) of (1/2B) sum (y - t)^2."""
        p = _f64(params, (self.num_params,))
        x = _f64(X).reshape(-1, self.K)
        t = _f64(targets).reshape(x.shape[0], self.O)
        g = np.zeros(self.num_params)
        loss = lib().so_mlp_loss_grad(ctypes.byref(self.dims), _p64(p), x.shape[0], _p64(x), _p64(t),
                                      _p64(g))
        return float(loss), g


def adam(w, m, v, g, lr: float, b1: float, b2: float, eps: float, t: int):
    """One Adam step t (1-based), in place on FP64 copies; returns (w, m, v)."""
    w, m, v = _f64(w).copy(), _f64(m).copy(), _f64(v).copy()
    gg = _f64(g)
    lib().so_adam(w.size, _p64(w), _p64(m), _p64(v), _p64(gg), float(lr), float(b1), float(b2), float(eps),
                  int(t))
    return w, m, v
