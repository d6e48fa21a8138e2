"""Seeded synthetic inputs for the SEPSO planner: configs, scenes, hyper-parameters.

This module holds no arithmetic of the method.  It only draws inputs with numpy
(`default_rng(seed)`) and writes down the paper's parameter tables, so that the CUDA
library and the CPU oracle can be fed identical FP32 arrays.

Workload shapes (all synthetic; the paper's own simulator scenes are not published):

* ``static_workload``  -- one static scene: 400x400 map, start (20,20), target
  (380,380), T=8 waypoints, G=8 groups x N=32, O=16 circles with centres
  U[60,340]^2 and radii U[10,30], penalty 1000 per intersection (alpha=1000,
  beta=1), 100 iterations, per-group w~U[0.4,0.9], C1,C2~U[1,2.5], Vmax=20.
* ``dynamic_workload`` -- the dynamic planning run: T=20, G=8 x N=170, 64 circles
  (32 static, 32 moving at speed U[0.5,2] per cycle in a random direction,
  bouncing off the walls), start/target drifting 1 unit per cycle vertically,
  Priori Initialization (gamma=0.25) and Auto Truncation by stall counter (10
  stalled iterations, cap 300), alpha=30, beta=4 (Table params_path).
* ``paper_workload``   -- the path-planning setting of Sec. 4.3 with the ablation
  switches of Table ppresult (366x366 map, 8 obstacles of which 6 move, T=8,
  G=8 x N=170, std-window AT, 30 iterations per frame at most).
* ``polygon_workload`` -- path planning among polygon obstacles (12 boxes and 4
  U-shaped non-convex polygons, 80 edges) on the same engine, 100 iterations.
* ``bf_standard`` / ``bf_large`` -- the benchmark functions of Table BFs: D=30 with
  8 x 10 particles (Sec. 4.1.1) and D=1000 with 8 x 2048 particles (Sec. 4.1.2),
  over [-600, 600]^D, Table hyper8 rows, 1400 iterations.

Paper tables reproduced as data (they are inputs of the method):
Table hyper8 (DTPSO / H-SEPSO / DPPSO hyper-parameters) and Table hyper8path
(evolved L-SEPSO hyper-parameters for path planning), rows
(C1, C2, C3, w_init, w_end, V_limit).
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

AT_OFF, AT_STD_WINDOW, AT_STALL = 0, 1, 2


@dataclass
class SepsoConfig:
    """Planner configuration (mirrors ``sepso_config`` in include/sepso.h)."""
    T: int = 8                 # waypoints; a particle has D = 2T coordinates (Eq. coordinate)
    G: int = 8                 # groups
    N: int = 32                # particles per group
    max_obstacles: int = 16
    map_w: float = 400.0
    map_h: float = 400.0
    alpha: float = 1000.0      # Eq. penalty: alpha * Q^beta
    beta: int = 1
    max_iters: int = 100       # iteration cap = T of Eq. TOF_omega
    at_mode: int = AT_OFF
    tw: int = 20               # truncation window (Table params_path)
    delta: float = 10.0
    stall_iters: int = 10
    stall_tol: float = 0.0
    use_pi: bool = False
    pi_gamma: float = 0.25
    pi_halfwidth: float = 20.0
    seed: int = 0              # Philox key
    run_id: int = 0            # Philox counter word 3
    runs: int = 1              # independent swarms on the same scene
    ctas_per_group: int = 0    # 0 = automatic
    threads: int = 0           # 0 = automatic
    circle_split: int = 0      # 0 = automatic
    fitness_mode: int = 0      # 0 = automatic; 1 lane group per particle; 2 items over the CTA
    exchange: int = 0          # 0 automatic and 3: one cluster per group when C3 = 0 and it fits; 1 grid-wide; 2 cluster (required)
    obstacle_kind: int = 0     # 0 circles; 1 polygon edges (max_obstacles = edge capacity)

    @property
    def D(self) -> int:
        return 2 * self.T

    def with_(self, **kw) -> "SepsoConfig":
        return replace(self, **kw)


@dataclass
class Scene:
    """Start, target and circles (cx, cy, r), plus their per-cycle velocities."""
    start: np.ndarray                      # (2,) float32
    target: np.ndarray                     # (2,) float32
    circles: np.ndarray                    # (O, 3) float32
    circle_vel: np.ndarray = field(default=None)   # (O, 2) float32
    start_vel: np.ndarray = field(default=None)    # (2,) float32
    target_vel: np.ndarray = field(default=None)   # (2,) float32

    def __post_init__(self):
        self.start = np.asarray(self.start, np.float32).reshape(2)
        self.target = np.asarray(self.target, np.float32).reshape(2)
        self.circles = np.ascontiguousarray(np.asarray(self.circles, np.float32).reshape(-1, 3))
        O = self.circles.shape[0]
        if self.circle_vel is None:
            self.circle_vel = np.zeros((O, 2), np.float32)
        if self.start_vel is None:
            self.start_vel = np.zeros(2, np.float32)
        if self.target_vel is None:
            self.target_vel = np.zeros(2, np.float32)
        self.circle_vel = np.ascontiguousarray(np.asarray(self.circle_vel, np.float32).reshape(O, 2))
        self.start_vel = np.asarray(self.start_vel, np.float32).reshape(2)
        self.target_vel = np.asarray(self.target_vel, np.float32).reshape(2)

    @property
    def O(self) -> int:
        return self.circles.shape[0]


# Table hyper8: hyper-parameters for DTPSO, H-SEPSO and DPPSO (C1, C2, C3, w_init, w_end, V_limit).
TABLE_HYPER8 = np.array([
    [2, 1, 1, 0.4, 0.2, 0.2],
    [1, 1, 2, 0.7, 0.3, 0.1],
    [2, 2, 1, 0.8, 0.1, 0.6],
    [2, 2, 1, 0.8, 0.6, 0.4],
    [2, 1, 2, 0.2, 0.1, 0.3],
    [2, 1, 2, 0.9, 0.5, 0.5],
    [1, 2, 2, 0.4, 0.1, 0.8],
    [1, 2, 2, 0.9, 0.3, 0.3],
], dtype=np.float32)

# Table hyper8path: evolved L-SEPSO hyper-parameters for path planning.
TABLE_HYPER8_PATH = np.array([
    [1.53, 1.29, 1.34, 0.48, 0.19, 0.35],
    [1.72, 1.53, 1.34, 0.73, 0.28, 0.32],
    [1.34, 1.42, 1.33, 0.48, 0.21, 0.62],
    [1.76, 1.60, 1.21, 0.47, 0.30, 0.63],
    [1.68, 1.27, 1.25, 0.73, 0.36, 0.41],
    [1.66, 1.54, 1.54, 0.39, 0.16, 0.45],
    [1.57, 1.48, 1.75, 0.56, 0.34, 0.38],
    [1.31, 1.71, 1.23, 0.36, 0.25, 0.50],
], dtype=np.float32)

# Table params_path: alpha, beta, gamma, delta, TW.
PARAMS_PATH = dict(alpha=30.0, beta=4, pi_gamma=0.25, delta=10.0, tw=20)

# Search box of the outer (H) swarm over per-group (w, C1, C2).
HSEF_BOX_LO = (0.4, 1.0, 1.0)
HSEF_BOX_HI = (0.9, 2.5, 2.5)


def sample_hyper(seed: int, G: int, w_range=(0.4, 0.9), c_range=(1.0, 2.5),
                 v_limit: float = 0.05) -> np.ndarray:
    """Per-group constant w ~ U[w_range], C1, C2 ~ U[c_range], C3 = 0 -> (G, 6) float32."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(*w_range, G)
    c1 = rng.uniform(*c_range, G)
    c2 = rng.uniform(*c_range, G)
    h = np.zeros((G, 6), np.float32)
    h[:, 0], h[:, 1], h[:, 2] = c1, c2, 0.0
    h[:, 3], h[:, 4], h[:, 5] = w, w, v_limit
    return h


def random_circles(rng, O: int, lo=60.0, hi=340.0, r_lo=10.0, r_hi=30.0) -> np.ndarray:
    c = np.zeros((O, 3), np.float32)
    c[:, 0] = rng.uniform(lo, hi, O)
    c[:, 1] = rng.uniform(lo, hi, O)
    c[:, 2] = rng.uniform(r_lo, r_hi, O)
    return c


def static_workload(seed: int = 0, O: int = 16):
    """The static single-scene workload: (config, scene, hyper)."""
    cfg = SepsoConfig(T=8, G=8, N=32, max_obstacles=max(O, 1), alpha=1000.0, beta=1,
                      max_iters=100, at_mode=AT_OFF, use_pi=False, seed=0)
    rng = np.random.default_rng(1000 + seed)
    scene = Scene(start=(20, 20), target=(380, 380), circles=random_circles(rng, O))
    hyper = sample_hyper(2000 + seed, cfg.G)
    return cfg, scene, hyper


# Auto Truncation of the dynamic workload: an iteration whose Tbest fitness drops by
# less than this (path-length units) counts as stalled.  The paper's own criterion
# (population std of the last TW = 20 LFVs below delta = 10) already stops an LFV that
# falls steadily by 1.7 per iteration, so improvements below 1 are below its scale.
DYNAMIC_STALL_TOL = 1.0


def dynamic_workload(seed: int = 0, n_static: int = 32, n_moving: int = 32, T: int = 20,
                     N: int = 170, r_range=(5.0, 15.0), stall_tol: float = DYNAMIC_STALL_TOL):
    """The dynamic planning workload: (config, scene with velocities, hyper).  The 64
    circles have radii U[5, 15] = U[10, 30] x sqrt(16 / 64): together they cover the
    same share of the map as the static workload's 16 circles of radii U[10, 30]."""
    O = n_static + n_moving
    cfg = SepsoConfig(T=T, G=8, N=N, max_obstacles=O, alpha=PARAMS_PATH["alpha"],
                      beta=PARAMS_PATH["beta"], max_iters=300, at_mode=AT_STALL,
                      stall_iters=10, stall_tol=stall_tol, tw=PARAMS_PATH["tw"],
                      delta=PARAMS_PATH["delta"], use_pi=True, pi_gamma=PARAMS_PATH["pi_gamma"],
                      pi_halfwidth=20.0, seed=seed)
    rng = np.random.default_rng(3000 + seed)
    circles = random_circles(rng, O, r_lo=r_range[0], r_hi=r_range[1])
    vel = np.zeros((O, 2), np.float32)
    speed = rng.uniform(0.5, 2.0, n_moving)
    ang = rng.uniform(0.0, 2.0 * np.pi, n_moving)
    vel[n_static:, 0] = speed * np.cos(ang)
    vel[n_static:, 1] = speed * np.sin(ang)
    scene = Scene(start=(20, 20), target=(380, 380), circles=circles, circle_vel=vel,
                  start_vel=(0.0, 1.0), target_vel=(0.0, -1.0))
    hyper = sample_hyper(4000 + seed, cfg.G)
    return cfg, scene, hyper


# Ablation variants of the path-planning comparison (Table ppresult): hyper-parameter
# table, Priori Initialization, Auto Truncation.  Without AT a frame runs the cap of
# 30 iterations; with AT the cap stays 30 and the std-window rule may stop earlier.
PAPER_VARIANTS = {
    "SEPSO": dict(hyper="hyper8path", use_pi=True, at=True),
    "SEPSO(NoAT)": dict(hyper="hyper8path", use_pi=True, at=False),
    "SEPSO(NoPI)": dict(hyper="hyper8path", use_pi=False, at=True),
    "DTPSO": dict(hyper="hyper8", use_pi=False, at=False),
}


def paper_workload(seed: int = 0, variant: str = "SEPSO", frame_cap: int = 30):
    """The path-planning setting of Sec. 4.3: (config, scene with velocities, hyper).

    366 x 366 map; 8 obstacles (2 static, 6 moving at speed U(0, 5] per frame in a
    random direction, bouncing off the borders) drawn as circles with centres
    U[60, 306]^2 and radii U[15, 30]; start (20, 40) moving 3 per frame and target
    (346, 326) moving 8 per frame along the vertical axis; T = 8 waypoints (D = 16),
    G = 8 groups x N = 170; alpha = 30, beta = 4, gamma = 0.25, delta = 10, TW = 20
    (Table params_path); a frame is one planning cycle with a cap of ``frame_cap``
    iterations.  ``variant`` is a key of ``PAPER_VARIANTS``: SEPSO uses the evolved
    Table hyper8path rows (linear inertia w_init -> w_end, C3 > 0), DTPSO the
    unevolved Table hyper8 rows.
    """
    v = PAPER_VARIANTS[variant]
    cfg = SepsoConfig(T=8, G=8, N=170, max_obstacles=8, map_w=366.0, map_h=366.0,
                      alpha=PARAMS_PATH["alpha"], beta=PARAMS_PATH["beta"], max_iters=frame_cap,
                      at_mode=AT_STD_WINDOW if v["at"] else AT_OFF, tw=PARAMS_PATH["tw"],
                      delta=PARAMS_PATH["delta"], use_pi=v["use_pi"],
                      pi_gamma=PARAMS_PATH["pi_gamma"], pi_halfwidth=20.0, seed=seed)
    rng = np.random.default_rng(5000 + seed)
    n_static, n_moving = 2, 6
    circles = random_circles(rng, n_static + n_moving, lo=60.0, hi=306.0, r_lo=15.0, r_hi=30.0)
    vel = np.zeros((n_static + n_moving, 2), np.float32)
    speed = 5.0 - rng.uniform(0.0, 5.0, n_moving)      # (0, 5]
    ang = rng.uniform(0.0, 2.0 * np.pi, n_moving)
    vel[n_static:, 0] = speed * np.cos(ang)
    vel[n_static:, 1] = speed * np.sin(ang)
    scene = Scene(start=(20, 40), target=(346, 326), circles=circles, circle_vel=vel,
                  start_vel=(0.0, 3.0), target_vel=(0.0, -8.0))
    table = TABLE_HYPER8_PATH if v["hyper"] == "hyper8path" else TABLE_HYPER8
    return cfg, scene, np.ascontiguousarray(table[:cfg.G], dtype=np.float32)


@dataclass
class PolygonScene:
    """Start, target and polygon obstacles (closed vertex lists, the last vertex
    joined back to the first), with per-cycle velocities: one per polygon (it moves
    as one body) and one each for start and target."""
    start: np.ndarray
    target: np.ndarray
    polygons: list
    poly_vel: np.ndarray = field(default=None)     # (P, 2) float32
    start_vel: np.ndarray = field(default=None)
    target_vel: np.ndarray = field(default=None)

    def __post_init__(self):
        self.start = np.asarray(self.start, np.float32).reshape(2)
        self.target = np.asarray(self.target, np.float32).reshape(2)
        self.polygons = [np.asarray(p, np.float32).reshape(-1, 2) for p in self.polygons]
        P = len(self.polygons)
        self.poly_vel = np.zeros((P, 2), np.float32) if self.poly_vel is None else \
            np.ascontiguousarray(np.asarray(self.poly_vel, np.float32).reshape(P, 2))
        self.start_vel = np.zeros(2, np.float32) if self.start_vel is None else \
            np.asarray(self.start_vel, np.float32).reshape(2)
        self.target_vel = np.zeros(2, np.float32) if self.target_vel is None else \
            np.asarray(self.target_vel, np.float32).reshape(2)

    @property
    def edges(self) -> np.ndarray:
        return polygon_edges(self.polygons)

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum([len(p) for p in self.polygons])]).astype(np.int32)


def box(cx: float, cy: float, hw: float, hh: float):
    """The axis-aligned box of centre (cx, cy) and half-sizes (hw, hh) as a vertex list."""
    return [(cx - hw, cy - hh), (cx + hw, cy - hh), (cx + hw, cy + hh), (cx - hw, cy + hh)]


def paper_box_workload(seed: int = 0, variant: str = "SEPSO", frame_cap: int = 30):
    """The path-planning setting of Sec. 4.3 with the paper's own map model, bounding
    boxes (Sec. 3.3.1): 366 x 366 map; 8 axis-aligned boxes (2 static, 6 moving at
    speed U(0, 5] per frame in a random direction, bouncing off the borders by their
    bounding box) with centres U[60, 306]^2 and half-sizes U[15, 30] per axis; start
    (20, 40) moving 3 per frame and target (346, 326) moving 8 per frame along the
    vertical axis; T = 8, G = 8 x N = 170; alpha = 30, beta = 4, gamma = 0.25, delta
    = 10, TW = 20 (Table params_path); Q counts path-segment / box-edge crossings; a
    frame is one planning cycle with a cap of ``frame_cap`` iterations; ``variant``
    as in ``paper_workload`` -> (config, polygon scene, hyper)."""
    v = PAPER_VARIANTS[variant]
    cfg = SepsoConfig(T=8, G=8, N=170, max_obstacles=32, map_w=366.0, map_h=366.0,
                      alpha=PARAMS_PATH["alpha"], beta=PARAMS_PATH["beta"], max_iters=frame_cap,
                      at_mode=AT_STD_WINDOW if v["at"] else AT_OFF, tw=PARAMS_PATH["tw"],
                      delta=PARAMS_PATH["delta"], use_pi=v["use_pi"],
                      pi_gamma=PARAMS_PATH["pi_gamma"], pi_halfwidth=20.0, seed=seed, obstacle_kind=1)
    rng = np.random.default_rng(7000 + seed)
    n_static, n_moving = 2, 6
    n = n_static + n_moving
    cx, cy = rng.uniform(60.0, 306.0, n), rng.uniform(60.0, 306.0, n)
    hw, hh = rng.uniform(15.0, 30.0, n), rng.uniform(15.0, 30.0, n)
    polys = [box(cx[i], cy[i], hw[i], hh[i]) for i in range(n)]
    vel = np.zeros((n, 2), np.float32)
    speed = 5.0 - rng.uniform(0.0, 5.0, n_moving)      # (0, 5]
    ang = rng.uniform(0.0, 2.0 * np.pi, n_moving)
    vel[n_static:, 0] = speed * np.cos(ang)
    vel[n_static:, 1] = speed * np.sin(ang)
    scene = PolygonScene(start=(20, 40), target=(346, 326), polygons=polys, poly_vel=vel,
                         start_vel=(0.0, 3.0), target_vel=(0.0, -8.0))
    table = TABLE_HYPER8_PATH if v["hyper"] == "hyper8path" else TABLE_HYPER8
    return cfg, scene, np.ascontiguousarray(table[:cfg.G], dtype=np.float32)


# Benchmark functions of Table BFs.
BF_SPHERE, BF_ROSENBROCK, BF_RASTRIGIN, BF_GRIEWANK = 1, 2, 3, 4
POLYGON_PATH = 5   # the same engine with a path among polygon obstacles as objective
SPHERE_PATH = 6    # ... and with a path in three dimensions among spheres
BF_NAMES = {BF_SPHERE: "Sphere", BF_ROSENBROCK: "Rosenbrock", BF_RASTRIGIN: "Rastrigin",
            BF_GRIEWANK: "Griewank"}


@dataclass
class BFConfig:
    """DTPSO on a benchmark function (mirrors ``sepso_bf_config`` in include/sepso.h):
    ``runs`` independent swarms of G groups x N particles over [lo, hi]^D, a fixed
    number of iterations (also the T of Eq. TOF_omega), no PI and no AT."""
    fn: int = BF_SPHERE
    D: int = 30
    G: int = 8
    N: int = 10
    lo: float = -600.0
    hi: float = 600.0
    max_iters: int = 1400
    seed: int = 0
    run_id: int = 0            # Philox counter word 3 of run 0; run r uses run_id + r
    runs: int = 1
    # objective POLYGON_PATH only: D = 2T waypoint coordinates in [0, map_w] x [0, map_h],
    # fitness = length + alpha * Q^beta (Eqs. path_fit, lenth, penalty)
    map_w: float = 400.0
    map_h: float = 400.0
    alpha: float = 30.0
    beta: int = 4
    max_edges: int = 0
    # objective SPHERE_PATH only: D = 3T coordinates, z in [0, map_d]
    map_d: float = 400.0
    max_spheres: int = 0
    # path objectives: Priori Initialization of a run that has a previous path (Sec.
    # 3.3.3), ceil(pi_gamma N) particles per group within +-pi_halfwidth of it
    pi_gamma: float = 0.0
    pi_halfwidth: float = 20.0
    # path objectives: Auto Truncation by stall counter (Sec. 3.3.4): stop after
    # at_stall iterations without an improvement of Tbest by more than stall_tol while
    # Tbest collides with nothing (0: off)
    at_stall: int = 0
    stall_tol: float = 0.0

    def with_(self, **kw) -> "BFConfig":
        return replace(self, **kw)


def bf_standard(fn: int, seed: int = 0, trials: int = 50):
    """Standard benchmark run of Sec. 4.1.1: D = 30 over [-600, 600]^30 (Table BFs),
    80 particles as 8 groups x 10 with the Table hyper8 rows, 1400 iterations,
    ``trials`` independent trials as runs of one launch -> (config, hyper)."""
    cfg = BFConfig(fn=fn, D=30, G=8, N=10, max_iters=1400, seed=seed, runs=trials)
    return cfg, np.ascontiguousarray(TABLE_HYPER8, dtype=np.float32)


def bf_large(fn: int, seed: int = 0, iters: int = 1400):
    """Large-scale run of Sec. 4.1.2: N = 16K particles (8 groups x 2048) of D = 1K
    over [-600, 600]^D, Table hyper8 rows, 1400 iterations -> (config, hyper)."""
    cfg = BFConfig(fn=fn, D=1000, G=8, N=2048, max_iters=iters, seed=seed, runs=1)
    return cfg, np.ascontiguousarray(TABLE_HYPER8, dtype=np.float32)


def polygon_edges(polygons) -> np.ndarray:
    """Closed polygons (lists of (x, y) vertices in order) -> (E, 4) float32 edges
    (x0, y0, x1, y1), the last vertex joined back to the first."""
    out = []
    for poly in polygons:
        v = np.asarray(poly, np.float32).reshape(-1, 2)
        for i in range(len(v)):
            a, b = v[i], v[(i + 1) % len(v)]
            out.append((a[0], a[1], b[0], b[1]))
    return np.asarray(out, np.float32).reshape(-1, 4)


def polygon_workload(seed: int = 0, T: int = 8, N: int = 170, n_boxes: int = 12, n_u: int = 4,
                     iters: int = 100, runs: int = 1):
    """Static path planning among polygon obstacles (Sec. 3.3.1's map model: bounding
    boxes and non-convex outlines): 400 x 400 map, start (20, 20), target (380, 380),
    ``n_boxes`` axis-aligned boxes (centres U[60, 340]^2, half-sizes U[10, 30]) and
    ``n_u`` U-shaped non-convex polygons (8 vertices, 60 x 60, opening towards a random
    side); T waypoints, G = 8 x N, Table hyper8path rows, alpha = 30, beta = 4 (Table
    params_path), ``iters`` iterations -> (config, start, target, polygons, edges, hyper)."""
    rng = np.random.default_rng(6000 + seed)
    polys = []
    for _ in range(n_boxes):
        cx, cy = rng.uniform(60, 340, 2)
        hw, hh = rng.uniform(10, 30, 2)
        polys.append([(cx - hw, cy - hh), (cx + hw, cy - hh), (cx + hw, cy + hh), (cx - hw, cy + hh)])
    for _ in range(n_u):
        cx, cy = rng.uniform(80, 320, 2)
        u = np.array([(-30, -30), (30, -30), (30, 30), (15, 30), (15, -15), (-15, -15), (-15, 30), (-30, 30)],
                     np.float64)
        rot = int(rng.integers(0, 4))
        for _ in range(rot):
            u = np.stack([-u[:, 1], u[:, 0]], axis=1)
        polys.append([(cx + a, cy + b) for a, b in u])
    edges = polygon_edges(polys)
    cfg = BFConfig(fn=POLYGON_PATH, D=2 * T, G=8, N=N, lo=0.0, hi=400.0, max_iters=iters, seed=seed,
                   runs=runs, map_w=400.0, map_h=400.0, alpha=PARAMS_PATH["alpha"],
                   beta=PARAMS_PATH["beta"], max_edges=max(len(edges), 1))
    start = np.array([20.0, 20.0], np.float32)
    target = np.array([380.0, 380.0], np.float32)
    hyper = np.ascontiguousarray(TABLE_HYPER8_PATH, dtype=np.float32)
    return cfg, start, target, polys, edges, hyper


def sphere_workload(seed: int = 0, T: int = 16, N: int = 170, S: int = 64, n_moving: int = 32,
                    iters: int = 100, runs: int = 1, pi_gamma: float = 0.25, at_stall: int = 0,
                    stall_tol: float = 1.0):
    """Path planning in three dimensions among spheres (the paper's Conclusion names
    the extension from 2D to 3D planning): a 400^3 box, start (20, 20, 20), target
    (380, 380, 380), ``S`` spheres with centres U[60, 340]^3 and radii U[10, 30] (the
    2D circles' make-up with a third coordinate), of which the last ``n_moving`` move
    at |v| ~ U[0.5, 2] per cycle in a uniformly random direction; T waypoints (D = 3T),
    G = 8 x N with the Table hyper8path rows, alpha = 30, beta = 4 (Table params_path),
    ``iters`` iterations per plan, ``runs`` independent swarms (Philox runs) on the
    same scene, PI with ``pi_gamma`` and a half-width of 20 once a run has a previous
    path, Auto Truncation by a stall counter of ``at_stall`` iterations (tolerance
    ``stall_tol``; 0: ``iters`` iterations) -> (config, scene dict: start, target,
    spheres (S, 4), vel (S, 3); hyper)."""
    rng = np.random.default_rng(8000 + seed)
    sph = np.empty((S, 4), np.float32)
    sph[:, :3] = rng.uniform(60.0, 340.0, (S, 3))
    sph[:, 3] = rng.uniform(10.0, 30.0, S)
    vel = np.zeros((S, 3), np.float32)
    m = min(n_moving, S)
    if m:
        d = rng.normal(size=(m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        vel[S - m:] = d * rng.uniform(0.5, 2.0, (m, 1))
    cfg = BFConfig(fn=SPHERE_PATH, D=3 * T, G=8, N=N, lo=0.0, hi=400.0, max_iters=iters, seed=seed, runs=runs,
                   map_w=400.0, map_h=400.0, map_d=400.0, alpha=PARAMS_PATH["alpha"], beta=PARAMS_PATH["beta"],
                   max_spheres=max(S, 1), pi_gamma=pi_gamma, pi_halfwidth=20.0, at_stall=at_stall,
                   stall_tol=stall_tol)
    scene = {"start": np.array([20.0, 20.0, 20.0], np.float32),
             "target": np.array([380.0, 380.0, 380.0], np.float32), "spheres": sph, "vel": vel}
    return cfg, scene, np.ascontiguousarray(TABLE_HYPER8_PATH, dtype=np.float32)


def advance_spheres(spheres: np.ndarray, vel: np.ndarray, box=(400.0, 400.0, 400.0)):
    """The 3D scene's simulator step (the Fig. PP caption's rule with a third axis):
    each sphere moves by its velocity; a velocity component flips when the sphere
    passes the wall it is moving towards.  FP32, returns new arrays."""
    c = np.array(spheres, np.float32, copy=True)
    v = np.array(vel, np.float32, copy=True)
    for a in range(3):
        c[:, a] += v[:, a]
        lo = (c[:, a] - c[:, 3] < 0.0) & (v[:, a] < 0.0)
        hi = (c[:, a] + c[:, 3] > np.float32(box[a])) & (v[:, a] > 0.0)
        v[lo | hi, a] = -v[lo | hi, a]
    return c, v


def random_paths3(seed: int, n: int, T: int, box=(400.0, 400.0, 400.0)) -> np.ndarray:
    """n random 3D paths (n, 3T) uniform over the box, FP32."""
    rng = np.random.default_rng(seed)
    X = np.empty((n, 3 * T), np.float32)
    for a in range(3):
        X[:, a * T:(a + 1) * T] = rng.uniform(0.0, box[a], (n, T))
    return X


def random_paths(seed: int, n: int, T: int, W: float = 400.0, H: float = 400.0) -> np.ndarray:
    """n random particles (n, 2T) uniform over the map, FP32."""
    rng = np.random.default_rng(seed)
    X = np.empty((n, 2 * T), np.float32)
    X[:, :T] = rng.uniform(0.0, W, (n, T))
    X[:, T:] = rng.uniform(0.0, H, (n, T))
    return X


def random_state(seed: int, cfg: SepsoConfig) -> dict:
    """A random mid-run swarm state (FP32/int32 arrays named as in the state layout).

    Pbest/Gbest/Tbest rows are drawn over the map; their fitness values are drawn
    as plain numbers (the update reads them only through comparisons)."""
    rng = np.random.default_rng(seed)
    T, G, N = cfg.T, cfg.G, cfg.N
    D, M = 2 * T, G * N

    def pos(n):
        a = np.empty((n, D), np.float32)
        a[:, :T] = rng.uniform(0, cfg.map_w, (n, T))
        a[:, T:] = rng.uniform(0, cfg.map_h, (n, T))
        return a.reshape(-1)

    st = {
        "X": pos(M), "P": pos(M),
        "V": rng.uniform(-20, 20, M * D).astype(np.float32),
        "Pfit": rng.uniform(500, 5000, M).astype(np.float32),
        "PQ": rng.integers(0, 5, M).astype(np.int32),
        "Gb": pos(G), "Gfit": rng.uniform(450, 600, G).astype(np.float32),
        "GQ": rng.integers(0, 2, G).astype(np.int32),
        "Tb": pos(1), "TQ": np.zeros(1, np.int32),
        "k": np.array([int(rng.integers(1, 50))], np.int32),
        "cycle": np.array([int(rng.integers(0, 5))], np.int32),
    }
    st["Tfit"] = np.array([st["Gfit"].min() - 1.0], np.float32)
    return st


@dataclass
class BatchSceneSpec:
    """One scene of a batch (mirrors ``sepso_batch_scene`` in include/sepso.h)."""
    T: int
    G: int
    N: int
    O: int
    max_iters: int = 200
    alpha: float = 30.0
    beta: int = 4
    seed: int = 0
    run_id: int = 0
    stall_iters: int = 0      # 0: no Auto Truncation; else stall-counter AT (Sec. 3.3.4)
    stall_tol: float = 0.0
    n_pi: int = 0             # particles per group around the previous path (PI)
    n_prior: int = 0          # particles per group around the learned prior's proposal
    pi_halfwidth: float = 20.0
    cycle: int = 0
    obstacle_kind: int = 0    # 0: O circles; 1: O polygon edges (Sec. 3.3.1)

    @property
    def D(self) -> int:
        return 2 * self.T

    def config(self, map_w: float = 400.0, map_h: float = 400.0, pi_gamma: float | None = None) -> SepsoConfig:
        """The equivalent single-scene configuration.  PI is on when n_pi > 0, with the
        gamma whose ceil(gamma N) is n_pi; AT is the stall counter when stall_iters > 0."""
        use_pi = self.n_pi > 0
        g = pi_gamma if pi_gamma is not None else ((self.n_pi - 0.5) / self.N if use_pi else 0.0)
        return SepsoConfig(T=self.T, G=self.G, N=self.N, max_obstacles=max(self.O, 1),
                           map_w=map_w, map_h=map_h, alpha=self.alpha, beta=self.beta,
                           max_iters=self.max_iters,
                           at_mode=AT_STALL if self.stall_iters > 0 else AT_OFF,
                           stall_iters=max(self.stall_iters, 1), stall_tol=self.stall_tol,
                           use_pi=use_pi, pi_gamma=g, pi_halfwidth=self.pi_halfwidth,
                           seed=self.seed, run_id=self.run_id, obstacle_kind=self.obstacle_kind)


def batch_workload(seed: int = 0, n: int = 4096, T_range=(8, 64), O_range=(16, 1024),
                   N_range=(32, 512), G: int = 8, r_range=(5.0, 30.0), max_iters: int = 200):
    """The batched workload: n independent scenes with T ~ U{T_range}, O ~ U{O_range},
    N per group ~ U{N_range}, G groups, radii U[r_range], centres uniform over the
    400x400 map, start (20,20), target (380,380), per-group w ~ U[0.4,0.9],
    C1, C2 ~ U[1,2.5], C3 = 0, V_limit 0.05, alpha 30, beta 4.  Philox key = seed,
    run id = scene index.  Returns (specs, hyper list, points (n,4), circle list)."""
    rng = np.random.default_rng(5000 + seed)
    specs, hyper, circles = [], [], []
    points = np.zeros((n, 4), np.float32)
    for s in range(n):
        T = int(rng.integers(T_range[0], T_range[1] + 1))
        O = int(rng.integers(O_range[0], O_range[1] + 1))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        specs.append(BatchSceneSpec(T=T, G=G, N=N, O=O, max_iters=max_iters, seed=seed, run_id=s))
        hyper.append(sample_hyper(int(rng.integers(1 << 30)), G))
        circles.append(random_circles(rng, O, lo=0.0, hi=400.0, r_lo=r_range[0], r_hi=r_range[1]))
        points[s] = (20.0, 20.0, 380.0, 380.0)
    return specs, hyper, points, circles


def team_workload(seed: int = 0, n_teams: int = 512, A: int = 8, T: int = 8, G: int = 8, N: int = 32, O: int = 16,
                  max_iters: int = 100, stall_iters: int = 10, ring: float = 170.0):
    """Multi-agent teams (the paper's stated future work): ``n_teams`` maps of 400 x
    400, each shared by A agents that swap sides -- agent a starts at angle 2 pi a /
    A (+ a small jitter) on a circle of radius ``ring`` about the map centre and
    targets the opposite point, so every path crosses the centre -- among O static
    circles (centres U[100,300]^2, radii U[8,15]).  Per agent: T waypoints, G x N
    particles, Table hyper8path rows, AT stall ``stall_iters`` / cap ``max_iters``,
    PI with ceil(0.25 N) particles from the second round on; Philox key = seed, run
    id = team * A + a.  Returns (specs, hyper list, points (n, 4), circle list,
    team_first (n,), team_size (n,))."""
    rng = np.random.default_rng(8000 + seed)
    n = n_teams * A
    specs, hyper, circles = [], [], []
    points = np.zeros((n, 4), np.float32)
    n_pi = int(np.ceil(0.25 * N))
    first = np.repeat(np.arange(n_teams) * A, A).astype(np.int32)
    size = np.full(n, A, np.int32)
    for m in range(n_teams):
        cs = random_circles(rng, O, lo=100.0, hi=300.0, r_lo=8.0, r_hi=15.0)
        ang0 = rng.uniform(0.0, 2.0 * np.pi)
        for a in range(A):
            s = m * A + a
            th = ang0 + 2.0 * np.pi * a / A + rng.uniform(-0.05, 0.05)
            points[s] = (200.0 + ring * np.cos(th), 200.0 + ring * np.sin(th),
                         200.0 - ring * np.cos(th), 200.0 - ring * np.sin(th))
            specs.append(BatchSceneSpec(T=T, G=G, N=N, O=O, max_iters=max_iters, seed=seed, run_id=s,
                                        stall_iters=stall_iters, n_pi=n_pi))
            hyper.append(np.ascontiguousarray(TABLE_HYPER8_PATH[:G], dtype=np.float32))
            circles.append(cs)
    return specs, hyper, points, circles, first, size


def serving_workload(seed: int = 0, n_agents: int = 2048, T_choices=(8, 20, 40), O_choices=(32, 256),
                     r_range=(3.0, 15.0), lo: float = 60.0, hi: float = 340.0):
    """Agents of the serving workload: each has a T in T_choices, a scene of O in
    O_choices circles (centres U[lo,hi]^2 as in the other workloads, so that the
    start and target start clear; radii U[r_range] x sqrt(32 / O), so that both
    obstacle counts cover the same area of the map; velocities U[0.5,2] per request
    in a uniform direction), start (20,20) and target (380,380) drifting 1 unit per
    request vertically, and its own hyper-parameters (w ~ U[0.4,0.9], C1, C2 ~
    U[1,2.5]).  Returns a list of dicts."""
    rng = np.random.default_rng(7000 + seed)
    agents = []
    for a in range(n_agents):
        T = int(rng.choice(T_choices))
        O = int(rng.choice(O_choices))
        sc = float(np.sqrt(32.0 / O))
        c = random_circles(rng, O, lo=lo, hi=hi, r_lo=r_range[0] * sc, r_hi=r_range[1] * sc)
        sp = rng.uniform(0.5, 2.0, O)
        ang = rng.uniform(0, 2 * np.pi, O)
        v = np.stack([sp * np.cos(ang), sp * np.sin(ang)], 1).astype(np.float32)
        agents.append(dict(T=T, O=O, circles=c, circle_vel=v, start=np.array([20.0, 20.0], np.float32),
                           target=np.array([380.0, 380.0], np.float32),
                           start_vel=np.array([0.0, 1.0], np.float32),
                           target_vel=np.array([0.0, -1.0], np.float32),
                           hyper=sample_hyper(int(rng.integers(1 << 30)), 8)))
    return agents


def serving_prior_scenes(seed: int, n: int, O: int, r_range=(3.0, 15.0), drift: int = 100) -> dict:
    """n snapshots shaped like the serving workload's scenes with O circles (centres
    U[60,340]^2, radii U[r_range] x sqrt(32 / O)), start (20, 20 + c) and target
    (380, 380 - c) for a drift c ~ U{0..drift-1}: the training and held-out scenes of
    the prior that seeds served requests.  Returns float32 arrays points (n, 4) and
    circles (n, O, 3)."""
    rng = np.random.default_rng(11000 + seed)
    sc = float(np.sqrt(32.0 / O))
    circ = np.stack([random_circles(rng, O, lo=60.0, hi=340.0, r_lo=r_range[0] * sc, r_hi=r_range[1] * sc)
                     for _ in range(n)]).astype(np.float32)
    c = rng.integers(0, drift, n).astype(np.float32)
    pts = np.stack([np.full(n, 20.0), 20.0 + c, np.full(n, 380.0), 380.0 - c], 1).astype(np.float32)
    return {"points": pts, "circles": circ}


def poisson_arrivals(seed: int, rate: float, duration: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate over [0, duration)."""
    rng = np.random.default_rng(9000 + seed)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    return t[t < duration]


# ----------------------------------------------------------------------------
# Learned prior: scenes shaped like the dynamic workload, initial weights
# ----------------------------------------------------------------------------

def prior_scenes(seed: int, n: int, O: int = 64, n_moving: int = 32, W: float = 400.0,
                 H: float = 400.0) -> dict:
    """n independent snapshots of the dynamic workload: O circles (centres
    U[60,340]^2, radii U[10,30]; the last n_moving with velocities U[0.5,2] per
    cycle in a uniform direction), start (20, 20 + c) and target (380, 380 - c)
    for a cycle c ~ U{0..359} of the 1-unit vertical drift.  Returns float32
    arrays points (n, 4), circles (n, O, 3), vel (n, O, 2)."""
    rng = np.random.default_rng(11000 + seed)
    circles = np.empty((n, O, 3), np.float32)
    vel = np.zeros((n, O, 2), np.float32)
    points = np.empty((n, 4), np.float32)
    for i in range(n):
        circles[i] = random_circles(rng, O)
        sp = rng.uniform(0.5, 2.0, n_moving)
        ang = rng.uniform(0.0, 2.0 * np.pi, n_moving)
        vel[i, O - n_moving:, 0] = sp * np.cos(ang)
        vel[i, O - n_moving:, 1] = sp * np.sin(ang)
        c = float(rng.integers(0, 360))
        points[i] = (20.0, 20.0 + c, W - 20.0, H - 20.0 - c)
    return dict(points=points, circles=circles, vel=vel)


def previous_cycle(scenes: dict, cycles: int = 1) -> dict:
    """The same scenes `cycles` planning cycles earlier (circles moved back along
    their velocities, start/target drifted back), float32."""
    c = scenes["circles"].copy()
    c[..., :2] -= cycles * scenes["vel"]
    p = scenes["points"].copy()
    p[:, 1] -= cycles
    p[:, 3] += cycles
    return dict(points=p, circles=c, vel=scenes["vel"])


def prior_init_params(seed: int, K: int, H1: int, H2: int, O: int, out_scale: float = 0.1) -> np.ndarray:
    """He-normal W1, W2 (std sqrt(2 / fan_in)), W3 scaled by out_scale (the first
    proposals stay near the straight line), zero biases; flat float32 in the order
    W1, b1, W2, b2, W3, b3."""
    rng = np.random.default_rng(13000 + seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / K), H1 * K), np.zeros(H1),
             rng.normal(0.0, np.sqrt(2.0 / H1), H2 * H1), np.zeros(H2),
             rng.normal(0.0, out_scale * np.sqrt(2.0 / H2), O * H2), np.zeros(O)]
    return np.concatenate(parts).astype(np.float32)
