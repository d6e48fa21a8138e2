"""Benchmark of the SEPSO planner on one GB300 (or N independent replicas).

Workload: the dynamic planning run -- 400x400 map, T=20 waypoints, G=8 groups x
N=170 particles, 64 circles (32 static, 32 moving at U[0.5,2] per cycle, bouncing
off the walls), start/target drifting 1 unit per cycle, Priori Initialization
(gamma = 0.25) and Auto Truncation by stall counter (10 stalled iterations, cap
300), alpha = 30, beta = 4.  First the HSEF evolution phase tunes the per-group
(w, C1, C2) (32 H-particles, each an L-run of 300 iterations); then one step =
one planning cycle (scene advance + plan) with the evolved hyper-parameters.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  ``value`` is plans/s with the scene resident on the device;
``e2e`` is the same metric through the C ABI with host buffers (pinned scene in,
waypoints out, every cycle).  ``--impl reference`` times the FP64 CPU oracle on
the host cores instead (bounded sample).

Further sections add objects to the same line (``--sections`` selects them): the
batched scenes, the learned prior, the serving loop, the ablation of the paper's
path-planning comparison (``paper_ablation``), the benchmark functions at the
standard and large scale (``bf``), planning among polygon obstacles (``poly``),
planning in three dimensions among spheres (``plan3d``) and the tensor-core GEMM
alone (``gemm``, not in the default list).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

METRIC = "plans/sec and particle-evals/sec at oracle-matched cost; p50/p99 plan latency"
UNIT = "plans/s"
WORKLOAD = ("dynamic SEPSO run: 400x400 map, T=20 (D=40), G=8 x N=170, 64 circles r~U[5,15] "
            "(32 static, 32 moving |v|~U[0.5,2]/cycle, wall bounce), start/target drift 1/cycle, "
            "PI gamma=0.25 + AT stall 10 (tolerance 1.0) / cap 300, alpha=30 beta=4, HSEF-evolved (w,C1,C2)")

# The kernel that runs a planning cycle, by the form of its per-iteration exchange.
SWARM_KERNEL = {"cluster": "swarm_cluster_kernel", "grid": "swarm_kernel"}
# FP32 lanes per SM of this architecture (the profiling recipe's unit count).
FP32_LANES_PER_SM = 128
_CLOCK = {}  # the SM clock sampled under load in the main section (used by the later sections)


def fp32_peak(sm_mhz=None):
    """(TFLOP/s, source): the FP32 FMA peak of this device from its queried SM count x
    128 FP32 lanes x 2 flop x the SM clock -- the median sampled under load when
    given (or sampled earlier in this run), else the device's maximum clock."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    src = "median sampled under load"
    mhz = sm_mhz or _CLOCK.get("sm_mhz")
    if sm_mhz:
        _CLOCK["sm_mhz"] = sm_mhz
    if not mhz:
        mhz, src = _max_sm_mhz(), "maximum SM clock (nvidia-smi)"
    return (sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12,
            f"derived: {sms} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz ({src})")


def _max_sm_mhz() -> float:
    try:
        out = subprocess.run(["nvidia-smi", "--id=0", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                             capture_output=True, text=True, timeout=20).stdout.strip().splitlines()
        return float(out[0])
    except Exception:
        return 2070.0
# Algorithmic work of one particle evaluation: (T+1) segments x (18 flops per
# segment-circle test x O circles + 8 flops of length), per the scope table.
FLOPS_PER_PAIR, FLOPS_PER_SEGMENT = 18, 8
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of each planning kernel
# on this workload (ncu --set full captures summarised in profiles/); None whenever
# the kernel changed since its capture.
SWARM_TRAFFIC_BYTES = {"swarm_kernel": None, "swarm_cluster_kernel": 85760}
# The same for gemm_tc_kernel on the MLP's grad-W1 product (1024 x 4104 x 4096),
# profiles/gemm_tc_kernel_mlp_gradW1.md.
GEMM_GRADW1_TRAFFIC_BYTES = 42132480


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--hsef-evolutions", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=0, help="0 = same as --steps")
    ap.add_argument("--cost-cycles", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--match-seeds", type=int, default=64,
                    help="Philox keys of the GPU-vs-oracle cost match on the headline workload")
    ap.add_argument("--match-cycles", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-scenes", type=int, default=4096,
                    help="scenes of the batched section (0 = skip it)")
    ap.add_argument("--batch-iters", type=int, default=200)
    ap.add_argument("--serve-rates", type=str, default="20000,5000",
                    help="offered request rates (1/s) of the serving section ('' = skip it)")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-prior-train", type=int, default=8192,
                    help="training snapshots per circle count of the serving prior (0: serve without one)")
    ap.add_argument("--serve-prior-rounds", type=int, default=2)
    ap.add_argument("--serve-radii", type=str, default="3,15",
                    help="circle radii U[a,b] of the serving scenes with 32 circles (scaled by sqrt(32/O))")
    ap.add_argument("--prior-train", type=int, default=16384,
                    help="training scenes of the learned-prior section (0 = skip it; 200000 = full size)")
    ap.add_argument("--prior-eval", type=int, default=2048, help="held-out scenes (10000 = full size)")
    ap.add_argument("--prior-rounds", type=int, default=3)
    ap.add_argument("--prior-epochs", type=int, default=30)
    ap.add_argument("--prior-batch", type=int, default=4096, help="rows per Adam step")
    ap.add_argument("--sections", type=str, default="main,cpu,batch,prior,serve,paper,boxes,agents,bf,poly,plan3d",
                    help="comma list of main, cpu, batch, prior, serve, paper, boxes, agents, bf, poly, gemm "
                         "(paper: the ablation variants of the path-planning comparison; boxes: the same among "
                         "moving bounding boxes; agents: multi-agent teams; bf: the benchmark "
                         "functions; poly: planning among polygon obstacles; gemm: the tensor-core "
                         "GEMM alone)")
    ap.add_argument("--bf-fns", type=str, default="1,2,3,4", help="benchmark functions (1..4) of section bf")
    ap.add_argument("--bf-iters", type=int, default=1400, help="iterations per benchmark-function run")
    ap.add_argument("--bf-trials", type=int, default=50,
                    help="trials of the standard D=30 runs (0 = only the large-scale runs)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled during the timed region.

    NVML is read directly (the driver's libnvidia-ml, through ctypes) every
    ``period`` seconds from a thread, so that even a timed region of a few
    milliseconds gets samples; the first sample is taken as the region starts.
    Where NVML cannot be loaded, ``nvidia-smi -lms 50`` is read instead."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # nvmlClocksEventReasons bits (NVML API): SwPowerCap, HwSlowdown, SwThermal, HwThermal
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40}
    NVML_CLOCK_SM = 1

    def __init__(self, gpu_index: int, period: float = 0.001):
        self.gpu = gpu_index
        self.period = period
        self.proc = None
        self.lines = []
        self.samples = []  # (sm_mhz, sm_max_mhz, reason bits)
        self.source = None
        self._stop = threading.Event()
        self.t = None

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit_v2")
        h = ctypes.c_void_p()
        uuid = None
        try:  # the CUDA device this rank runs on, whatever CUDA_VISIBLE_DEVICES maps
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(self.gpu).uuid)
        except Exception:
            pass
        if not (uuid and lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(h)) == 0):
            if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
                raise RuntimeError("nvmlDeviceGetHandleByIndex_v2")
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(mx))
        return lib, h, reasons, mx.value

    def _poll(self, lib, h, reasons, mx):
        import ctypes
        clk, bits = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        while True:
            ok = lib.nvmlDeviceGetClockInfo(h, self.NVML_CLOCK_SM, ctypes.byref(clk)) == 0
            ok = ok and reasons(h, ctypes.byref(bits)) == 0
            if ok:
                self.samples.append((float(clk.value), float(mx), int(bits.value)))
            if self._stop.wait(self.period):
                break

    def __enter__(self):
        try:
            lib, h, reasons, mx = self._nvml()
            self.source = "NVML, every 1 ms"
            self.t = threading.Thread(target=self._poll, args=(lib, h, reasons, mx), daemon=True)
            self.t.start()
            return self
        except Exception:
            pass
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.source = "nvidia-smi -lms 50"
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        self._stop.set()
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.t is not None:
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for c, m, bits in self.samples:
            sm.append(c)
            mx.append(m)
            reasons.update(n for n, b in self.REASON_BITS.items() if bits & b)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0, "source": self.source}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "source": self.source}


# ----------------------------------------------------------------------------
# Hyper-parameters of the application phase, shared by both arms
# ----------------------------------------------------------------------------

HYPER_FILE = ROOT / "tests" / "golden" / "dynamic_hsef_hyper.json"


def shared_hyper():
    """(G x 6 hyper-parameters, description): the per-group (w, C1, C2) that the
    oracle's HSEF evolution phase found on the dynamic workload's first scene
    (tests/golden/make_dynamic_hsef_hyper.py writes them), so that the GPU planner
    and the FP64 oracle plan the same configuration and their costs compare."""
    d = json.loads(HYPER_FILE.read_text())
    return np.asarray(d["hyper"], np.float32), "HSEF-evolved (w,C1,C2): " + d["source"]


def run_config(K: int, world: int) -> dict:
    """The ``config`` object of both arms' JSON lines (identical by construction)."""
    return {"workload": WORKLOAD, "hyper": shared_hyper()[1], "cycles": K, "replicas": world,
            "l2": "GPU arm: flushed before every step (256 MiB write outside the timed events); "
                  "CPU arm: none"}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------
# Oracle (CPU) arm: independent dynamic runs, one per host core
# ----------------------------------------------------------------------------

def _oracle_run_worker(seed, n_warm, n_timed, seconds, barrier, out):
    """One process of the oracle arm: the dynamic run with Philox key ``seed`` (the
    scene of seed 0, the shared hyper-parameters), n_warm untimed cycles, then --
    after the barrier -- n_timed timed cycles (or cycles until ``seconds`` pass
    when n_timed < 0).  Puts (seed, t_start, t_end, per-cycle seconds, iters,
    costs, Q) on ``out``."""
    import oracle
    from paper_2308_10169_gb300.inputs import dynamic_workload
    cfg, scene, _ = dynamic_workload(0)
    cfg = cfg.with_(seed=seed)
    hyper, _ = shared_hyper()
    sw = oracle.Swarm(cfg, hyper)
    c, v, st, sv, tg, tv = (scene.circles, scene.circle_vel, scene.start, scene.start_vel,
                            scene.target, scene.target_vel)
    cyc = 0

    def one():
        nonlocal c, v, st, sv, tg, tv, cyc
        if cyc:
            c, v, st, sv, tg, tv = oracle.advance_scene(cfg.map_w, cfg.map_h, c, v, st, sv, tg, tv)
        cyc += 1
        return sw.plan(oracle.Scene(st, tg, c))

    for _ in range(n_warm):
        one()
    if barrier is not None:
        barrier.wait()
    times, iters, costs, qs = [], [], [], []
    t0 = time.time()
    while (n_timed >= 0 and len(times) < n_timed) or (n_timed < 0 and time.time() - t0 < seconds):
        t = time.perf_counter()
        r = one()
        times.append(time.perf_counter() - t)
        iters.append(r["iters"])
        costs.append(r["cost"])
        qs.append(r["Q"])
    out.put((seed, t0, time.time(), times, iters, costs, qs))


def oracle_runs(n_workers: int, warm: list, timed: list, seconds: float = 0.0):
    """Runs _oracle_run_worker in n_workers spawned processes (the GPU may already be
    in use by this process, so no fork); returns the merged record."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    barrier = ctx.Barrier(n_workers)
    procs = [ctx.Process(target=_oracle_run_worker, args=(w, warm[w], timed[w], seconds, barrier, out))
             for w in range(n_workers)]
    for p_ in procs:
        p_.start()
    res = [out.get() for _ in procs]
    for p_ in procs:
        p_.join()
    t_start = min(r[1] for r in res)
    t_end = max(r[2] for r in res)
    times = [t for r in res for t in r[3]]
    return {"wall": t_end - t_start, "times": times, "iters": [i for r in res for i in r[4]],
            "costs": [x for r in res for x in r[5]], "Q": [x for r in res for x in r[6]],
            "workers": n_workers}


def plan_stats(iters, costs, qs, cap: int) -> dict:
    """Auto Truncation and quality figures of a set of planning cycles."""
    iters, costs, qs = np.asarray(iters), np.asarray(costs, np.float64), np.asarray(qs)
    return {"cycles": int(iters.size), "iters_per_plan": float(iters.mean()),
            "at_fire_rate": float(np.mean(iters < cap)), "collision_free": float(np.mean(qs == 0)),
            "median_cost": float(np.median(costs))}


def aggregate_timing(total_ms: float, steps: int, world: int):
    """Whole-job timing over the ranks (one replica per GPU, no data exchange): the
    slowest rank's time, and the units all ranks processed over it."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_max = float(t.item())
    return total_max, world * steps / (total_max / 1e3)


def run_reference(args, rank, world):
    """The oracle on the host cores: W warm-up and K timed planning cycles in all,
    spread over one independent dynamic run per core (each run sequential, as PI
    needs its previous cycle); value = K / wall time of the timed phase."""
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    P = max(1, min(host_cores(), K))
    warm = [W // P + (1 if w < W % P else 0) for w in range(P)]
    timed = [K // P + (1 if w < K % P else 0) for w in range(P)]
    r = oracle_runs(P, warm, timed)
    value = K / r["wall"]
    from paper_2308_10169_gb300.inputs import dynamic_workload
    cfg = dynamic_workload(0)[0]
    st = plan_stats(r["iters"], r["costs"], r["Q"], cfg.max_iters)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * r["wall"] / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": run_config(K, world),
        "particle_evals_per_s": sum(r["iters"]) * cfg.G * cfg.N / r["wall"],
        "latency_ms_single_thread": {"mean": 1e3 * float(np.mean(r["times"])),
                                     "p50": 1e3 * float(np.percentile(r["times"], 50))},
        **st,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
                         "sample": f"{K} timed planning cycles after {W} warm-up cycles, spread over {P} "
                                   f"independent dynamic runs (Philox keys 0..{P - 1}, one process per "
                                   f"core, {host_cores()} cores seen), FP64, wall {r['wall']:.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist

    from paper_2308_10169_gb300 import Planner
    from paper_2308_10169_gb300.inputs import (HSEF_BOX_HI, HSEF_BOX_LO, TABLE_HYPER8, Scene,
                                               dynamic_workload)

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    K, W = args.steps, args.warmup
    if W < 3:
        raise SystemExit("--warmup must be >= 3")

    def barrier():
        if world > 1:
            dist.barrier()

    cfg, scene, hyper0 = dynamic_workload(seed=rank)
    app_hyper, _ = shared_hyper()

    # -- evolution phase (HSEF): 8 H-groups x 4 H-particles, Table hyper8 --------
    HG, HN = 8, 4
    hcfg = cfg.with_(runs=HG * HN, at_mode=0, use_pi=False)
    hp = Planner(hcfg, device=dev)
    hp.set_scene(scene, motion=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    hist = hp.hsef(HG=HG, HN=HN, E=args.hsef_evolutions, hhyper=TABLE_HYPER8, lo=HSEF_BOX_LO,
                   hi=HSEF_BOX_HI, l_vlimit=0.05, hseed=1000 + rank)
    e1.record(stream)
    hp.sync()
    hsef_ms = e0.elapsed_time(e1)
    best_hyper, best_lfv = hp.hsef_best()
    hsef_info = {"evolutions": args.hsef_evolutions, "h_particles": HG * HN,
                 "l_run_iters": cfg.max_iters, "ms": hsef_ms,
                 "evolutions_per_s": 1e3 * args.hsef_evolutions / hsef_ms,
                 "lfv_first": float(hist[0].item()), "lfv_best": best_lfv,
                 "exchange": hp.exchange_form(), "launch": hp.launch_shape(),
                 "oracle_hsef_lfv_best": json.loads(HYPER_FILE.read_text())["lfv_best"],
                 "launches": hp.launch_count(),
                 "note": "the application phase plans with the oracle-evolved set (shared with the "
                         "CPU arm); this GPU evolution phase is timed beside it"}
    del hp

    # -- application phase ----------------------------------------------------
    pl = Planner(cfg, device=dev)
    pl.set_hyper(app_hyper)
    pl.set_scene(scene)
    shape = dict(pl.launch_shape(), exchange=pl.exchange_form())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    for i in range(W):
        if i:
            pl.advance(1)
        pl.plan_async()
    pl.sync()
    plans0, iters0 = pl.counters()
    launches0 = pl.launch_count()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    costs = []
    barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        t_wall0 = time.perf_counter()
        for i in range(K):
            flush.zero_()                      # L2 flush, outside the timed events
            a, b, c = ev[i]
            a.record(stream)
            pl.advance(1)
            b.record(stream)
            pl.plan_async()
            c.record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall0
    barrier()
    launches = pl.launch_count() - launches0
    pl.sync()
    plans1, iters1 = pl.counters()
    step_ms = np.array([a.elapsed_time(c) for a, b, c in ev])
    plan_ms = np.array([b.elapsed_time(c) for a, b, c in ev])
    total_ms = float(step_ms.sum())
    last = pl.read_result()
    iters = iters1 - iters0
    assert plans1 - plans0 == K
    # quality of the same run over the next cycles (untimed: each is read back)
    c_iters, c_q = [], []
    for _ in range(args.cost_cycles):
        pl.advance(1)
        pl.plan_async()
        r_ = pl.read_result()
        costs.append(r_["cost"])
        c_iters.append(r_["iters"])
        c_q.append(r_["Q"])

    total_max, value = aggregate_timing(total_ms, K, world)
    pe_local = iters * cfg.G * cfg.N
    flops = iters * cfg.G * cfg.N * (cfg.T + 1) * (FLOPS_PER_PAIR * scene.O + FLOPS_PER_SEGMENT)
    achieved = flops / (plan_ms.sum() / 1e3) / 1e12

    # -- the two forms of the per-iteration exchange on the same cycles -----------
    forms = {}
    for name, ex in (("grid", 1), ("cluster", 2)):
        try:
            fp = Planner(cfg.with_(exchange=ex), device=dev)
        except Exception as e:  # the cluster form may not fit a device
            forms[name] = {"error": str(e)[:120]}
            continue
        fp.set_hyper(app_hyper)
        fp.set_scene(scene)
        for _ in range(3):
            fp.plan_async()
        fp.sync()
        i0 = fp.counters()[1]
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(30):
            fp.advance(1)
            fp.plan_async()
        f1.record(stream)
        fp.sync()
        forms[name] = {"us_per_iteration": 1e3 * f0.elapsed_time(f1) / max(fp.counters()[1] - i0, 1),
                       "launch": fp.launch_shape()}
        del fp

    # -- the planning kernel's per-iteration floor: fixed-length launches (200
    # iterations each) of the same swarm with the scene's circles and with none (no
    # pair test at all), so that the time the exchange takes shows beside the fitness
    floor = {}
    try:
        fl = Planner(cfg.with_(exchange=2 if shape["exchange"] == "cluster" else 1), device=dev)
        fl.set_hyper(app_hyper)
        for label, sc in (("with_circles", scene),
                          ("no_obstacles", Scene(start=scene.start, target=scene.target,
                                                 circles=np.zeros((0, 3), np.float32)))):
            fl.set_scene(sc, motion=False)
            fl.plan()
            for _ in range(3):
                fl.step(200)
            fl.sync()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(10):
                fl.step(200)
            f1.record(stream)
            fl.sync()
            floor[label] = 1e3 * f0.elapsed_time(f1) / 2000
        floor["note"] = ("us per iteration in fixed-length launches of 200 iterations; the difference is what "
                         "the pair tests cost, the rest is the per-iteration exchange")
        del fl
    except Exception as e:
        floor = {"error": str(e)[:120]}

    # -- end to end through the C ABI with host buffers ----------------------------
    Ke = args.e2e_steps or K
    e2e = run_e2e(torch, pl, cfg, scene, app_hyper, dev, Ke, W)
    clocks = clk.summary()
    peak, peak_src = fp32_peak(clocks.get("sm_mhz"))

    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": total_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded scenes shaped like the paper's dynamic environment)",
            "config": run_config(K, world),
            "launch": shape,
            "particle_evals_per_s": world * pe_local / (total_max / 1e3),
            "iters_per_plan": iters / K,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99)),
                           "max": float(step_ms.max())},
            "cost_last": float(last["cost"]),
            "median_cost": float(np.median(costs)) if costs else None,
            "quality": dict(plan_stats(c_iters, costs, c_q, cfg.max_iters),
                            sample=f"the {len(costs)} cycles after the timed ones, read back one by one")
            if costs else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": SWARM_TRAFFIC_BYTES.get(SWARM_KERNEL[shape["exchange"]]),
                         "kernel": SWARM_KERNEL[shape["exchange"]],
                         "peak_source": peak_src},
            "e2e": e2e,
            "exchange_forms": dict(forms, note="30 cycles each, device time per iteration (scene advance "
                                               "included), same hyper-parameters and scene"),
            "iteration_floor": floor,
            "gpu_launches": int(launches),
            "clocks": clocks,
            "hsef": hsef_info,
            "wall_s_timed_loop": t_wall,
            "paper_context": {"plans_per_s": 67, "s_per_plan": 0.015,
                              "note": "the paper's SEPSO on an i9-10850K + RTX 2070 SUPER, 8 box obstacles, "
                                      "8 waypoints, its own (unpublished) scene: another workload and machine, "
                                      "context only (vs_baseline stays null)"},
        }
    return line


def run_e2e(torch, pl_dev, cfg, scene, hyper, dev, K, W):
    """plans/s through set_scene (pinned host scene) + sepso_plan (host waypoints)."""
    from paper_2308_10169_gb300 import Planner
    from paper_2308_10169_gb300.inputs import Scene
    # the scene sequence the host simulator feeds in (produced before timing)
    sim = Planner(cfg, device=dev)
    sim.set_hyper(hyper)
    sim.set_scene(scene)
    O = scene.O
    pin_c = torch.empty((W + K, O, 3), dtype=torch.float32).pin_memory()
    pin_p = torch.empty((W + K, 4), dtype=torch.float32).pin_memory()
    for i in range(W + K):
        if i:
            sim.advance(1)
        sc = sim.get_scene()
        pin_c[i] = torch.from_numpy(sc.circles)
        pin_p[i, :2] = torch.from_numpy(sc.start)
        pin_p[i, 2:] = torch.from_numpy(sc.target)
    del sim
    pl = Planner(cfg, device=dev)
    pl.set_hyper(hyper)
    cn, pn = pin_c.numpy(), pin_p.numpy()
    wp = torch.empty(cfg.D, dtype=torch.float32).pin_memory().numpy()
    lat = []

    def one(i):
        pl.set_scene_arrays(pn[i, :2], pn[i, 2:], cn[i])
        pl.plan_into(wp)

    for i in range(W):
        one(i)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for i in range(W, W + K):
        t = time.perf_counter()
        one(i)
        lat.append(time.perf_counter() - t)
    total = time.perf_counter() - t0
    lat = np.array(lat) * 1e3
    return {"value": K / total, "unit": UNIT, "h2d_bytes_per_step": O * 16 + 8 * 4,
            "d2h_bytes_per_step": cfg.D * 4 + 20,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "path": "sepso_set_scene (pinned staging, async DMA) + sepso_plan (D2H waypoints, sync)"}


def run_batch(n: int, iters: int):
    """The batched workload: n uneven scenes x iters iterations in one CUDA graph."""
    import torch

    from paper_2308_10169_gb300 import BatchPlanner
    from paper_2308_10169_gb300.inputs import batch_workload
    specs, hyper, points, circles = batch_workload(seed=0, n=n, max_iters=iters)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    shape, tune_ms = bp.autotune(trial_launches=3)
    bp.run_async(True)              # warm-up run (captures the graph)
    torch.cuda.synchronize()
    l0 = bp.launch_count()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record()
    bp.run_async(True)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e)
    res = bp.read()
    pairs = sum(sp.G * sp.N * (sp.T + 1) * sp.O for sp in specs) * iters
    segs = sum(sp.G * sp.N * (sp.T + 1) for sp in specs) * iters
    flops = pairs * FLOPS_PER_PAIR + segs * FLOPS_PER_SEGMENT
    achieved = flops / (ms / 1e3) / 1e12
    return {"workload": f"{n} scenes, T~U{{8..64}}, O~U{{16..1024}} r~U[5,30], N/group~U{{32..512}}, "
                        f"G=8, 400x400, {iters} iterations each, one CUDA graph",
            "plans_per_s": n / (ms / 1e3), "ms": ms,
            "particle_evals_per_s": sum(sp.G * sp.N for sp in specs) * iters / (ms / 1e3),
            "pair_tests_per_s": pairs / (ms / 1e3),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak()[0],
                         "unit": "TFLOP/s", "frac": achieved / fp32_peak()[0], "peak_source": fp32_peak()[1],
                         "kernel": "batch_kernel"},
            "shape": bp.shape(), "autotune_ms_per_launch": tune_ms,
            "gpu_launches": bp.launch_count() - l0,
            "median_cost": float(np.median([r["cost"] for r in res])),
            "collision_free": float(np.mean([r["Q"] == 0 for r in res])),
            "collision_free_by_circles": {f"O<={hi}": float(np.mean([r["Q"] == 0 for r, sp in zip(res, specs)
                                                                     if lo < sp.O <= hi]))
                                          for lo, hi in ((0, 64), (64, 256), (256, 1024))},
            "quality_note": "radii U[5,30] (the configuration's) with up to 1024 circles on 400x400: "
                            "the dense scenes admit no collision-free path",
            "l2": f"inputs larger than L2 ({bp.workspace.numel() / 1e9:.1f} GB of batch state)",
            "cpu_baseline": batch_oracle_baseline(specs, hyper, points, circles, n / (ms / 1e3),
                                                  pairs / n)}


def _batch_oracle_worker(args):
    """One sampled scene of the batch on the oracle: initialisation and one
    iteration (Algorithm 1), timed; returns (seconds, pair tests of the iteration)."""
    import oracle
    spec, hyper, pts, circ = args
    sw = oracle.Swarm(spec.config(), hyper)
    scene = oracle.Scene(pts[:2], pts[2:], circ)
    sw.init()
    t0 = time.perf_counter()
    sw.iteration(scene)
    return time.perf_counter() - t0, spec.G * spec.N * (spec.T + 1) * spec.O


def batch_oracle_baseline(specs, hyper, points, circles, gpu_plans_per_s: float, pairs_per_plan: float,
                          sample: int = 64):
    """The FP64 oracle on the batched workload, on every host core: one iteration of
    each of ``sample`` scenes spread over the batch (every n/sample-th), timed in a
    spawned process pool; the batch's plans/s is extrapolated from the pair tests per
    second the oracle sustained and the batch's pair tests per plan."""
    import multiprocessing as mp
    n = len(specs)
    idx = [int(i * n / sample) for i in range(sample)]
    P = min(host_cores(), sample)
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(P) as pool:
        res = pool.map(_batch_oracle_worker, [(specs[i], hyper[i], points[i], circles[i]) for i in idx], chunksize=1)
    wall = time.perf_counter() - t0
    pairs = sum(r[1] for r in res)
    busy = sum(r[0] for r in res)
    rate = pairs / busy * P   # pair tests per second on P cores, each process busy
    value = rate / pairs_per_plan
    return {"value": value, "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": f"one iteration of each of {sample} scenes spread over the batch, FP64, one process per core; "
                      f"extrapolated to whole plans by pair-test count ({pairs_per_plan:.3g} per plan)",
            "pair_tests_per_s": rate, "sample_wall_s": wall, "gpu_vs_oracle": gpu_plans_per_s / value}


def run_paper(frames: int = 100, seed: int = 0):
    """The path-planning comparison of Sec. 4.3 (Table ppresult) with the ablation
    switches: SEPSO, SEPSO(NoAT), SEPSO(NoPI), DTPSO, each over the same seeded
    sequence of ``frames`` frames (one planning cycle each, cap 30 iterations).
    Time per frame = CUDA-event time of scene advance + plan on the device; the
    result is read back after every frame (outside the events)."""
    import torch

    from paper_2308_10169_gb300 import Planner
    from paper_2308_10169_gb300.inputs import PAPER_VARIANTS, paper_workload
    paper = {"SEPSO": (412.0, 0.015, 12.9), "SEPSO(NoAT)": (408.3, 0.036, 30.0),
             "SEPSO(NoPI)": (415.8, 0.033, 26.8), "DTPSO": (413.9, 0.036, 30.0)}
    out = {}
    for var in PAPER_VARIANTS:
        cfg, scene, hyper = paper_workload(seed, var)
        warm = Planner(cfg)
        warm.set_hyper(hyper)
        warm.set_scene(scene)
        for _ in range(3):
            warm.plan()
        del warm
        pl = Planner(cfg)
        pl.set_hyper(hyper)
        pl.set_scene(scene)
        stream = torch.cuda.current_stream()
        l0 = pl.launch_count()
        ms, wall, L, I, Q = [], [], [], [], []
        torch.cuda.synchronize()
        for f in range(frames):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            a.record(stream)
            if f:
                pl.advance(1)
            pl.plan_async()
            b.record(stream)
            r = pl.read_result()
            wall.append(time.perf_counter() - t0)
            ms.append(a.elapsed_time(b))
            L.append(r["length"]); I.append(r["iters"]); Q.append(r["Q"])
        out[var] = {"path_length": float(np.mean(L)), "ms_per_frame": float(np.mean(ms)),
                    "wall_ms_per_frame_with_readback": 1e3 * float(np.mean(wall)),
                    "iters_per_frame": float(np.mean(I)),
                    "collision_free_frames": float(np.mean(np.array(Q) == 0)),
                    "gpu_launches": pl.launch_count() - l0,
                    "paper_context": {"path_length": paper[var][0], "s_per_frame": paper[var][1],
                                      "iters_per_frame": paper[var][2],
                                      "note": "RTX 2070 SUPER, the paper's own (unpublished) scene"}}
    return {"workload": "366x366 map, 8 circles r~U[15,30] (2 static, 6 moving |v|~U(0,5]/frame, "
                        "wall bounce), start/target moving 3 and 8 per frame vertically, T=8 (D=16), "
                        "G=8 x N=170, alpha=30 beta=4, PI gamma=0.25, std-window AT TW=20 delta=10, "
                        f"cap 30 iterations per frame, {frames} frames, seed {seed}",
            "variants": out}


def run_paper_boxes(frames: int = 100, seed: int = 0, oracle_keys: int = 2, oracle_frames: int = 25):
    """Table ppresult's comparison with the paper's own map model: the same variants
    among 8 moving and static bounding boxes (Q = path-segment / box-edge crossings),
    timed as ``run_paper``; beside each variant the FP64 oracle on the first
    ``oracle_frames`` frames under ``oracle_keys`` Philox keys (means compared)."""
    import torch

    import oracle
    from paper_2308_10169_gb300 import Planner
    from paper_2308_10169_gb300.inputs import PAPER_VARIANTS, paper_box_workload
    paper = {"SEPSO": (412.0, 0.015, 12.9), "SEPSO(NoAT)": (408.3, 0.036, 30.0),
             "SEPSO(NoPI)": (415.8, 0.033, 26.8), "DTPSO": (413.9, 0.036, 30.0)}
    out = {}
    for var in PAPER_VARIANTS:
        cfg, scene, hyper = paper_box_workload(seed, var)
        warm = Planner(cfg)
        warm.set_hyper(hyper)
        warm.set_polygons(scene)
        for _ in range(3):
            warm.plan()
        del warm
        pl = Planner(cfg)
        pl.set_hyper(hyper)
        pl.set_polygons(scene)
        stream = torch.cuda.current_stream()
        l0 = pl.launch_count()
        ms, L, I, Q = [], [], [], []
        torch.cuda.synchronize()
        for f in range(frames):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if f:
                pl.advance(1)
            pl.plan_async()
            b.record(stream)
            r = pl.read_result()
            ms.append(a.elapsed_time(b))
            L.append(r["length"]); I.append(r["iters"]); Q.append(r["Q"])
        oL, oI, oQ, gL, gI, gQ = [], [], [], [], [], []
        for key in range(oracle_keys):
            c2 = cfg.with_(seed=1000 + key)
            g2 = Planner(c2)
            g2.set_hyper(hyper)
            g2.set_polygons(scene)
            sw = oracle.Swarm(c2, hyper)
            e, v, st, sv, tg, tv = (scene.edges, scene.poly_vel, scene.start, scene.start_vel, scene.target,
                                    scene.target_vel)
            for f in range(oracle_frames):
                if f:
                    g2.advance(1)
                    e, v, st, sv, tg, tv = oracle.advance_polygons(cfg.map_w, cfg.map_h, e, scene.offsets, v, st,
                                                                   sv, tg, tv)
                rg = g2.plan()
                ro = sw.plan(oracle.Scene(st, tg, np.zeros((0, 3)), e))
                gL.append(rg["length"]); gI.append(rg["iters"]); gQ.append(rg["Q"])
                oL.append(ro["length"]); oI.append(ro["iters"]); oQ.append(ro["Q"])
        out[var] = {"path_length": float(np.mean(L)), "ms_per_frame": float(np.mean(ms)),
                    "iters_per_frame": float(np.mean(I)),
                    "collision_free_frames": float(np.mean(np.array(Q) == 0)),
                    "gpu_launches": pl.launch_count() - l0, "exchange": pl.exchange_form(),
                    "vs_oracle": {"frames": len(oL), "gpu_path_length": float(np.mean(gL)),
                                  "oracle_path_length": float(np.mean(oL)),
                                  "gpu_iters_per_frame": float(np.mean(gI)),
                                  "oracle_iters_per_frame": float(np.mean(oI)),
                                  "gpu_collision_free": float(np.mean(np.array(gQ) == 0)),
                                  "oracle_collision_free": float(np.mean(np.array(oQ) == 0))},
                    "paper_context": {"path_length": paper[var][0], "s_per_frame": paper[var][1],
                                      "iters_per_frame": paper[var][2],
                                      "note": "RTX 2070 SUPER, the paper's own (unpublished) scene"}}
    return {"workload": "366x366 map, 8 axis-aligned boxes with half-sizes U[15,30] (2 static, 6 moving "
                        "|v|~U(0,5]/frame, bounding-box bounce), Q = path-segment / box-edge crossings, "
                        "start/target moving 3 and 8 per frame vertically, T=8 (D=16), G=8 x N=170, alpha=30 "
                        "beta=4, PI gamma=0.25, std-window AT TW=20 delta=10, cap 30 iterations per frame, "
                        f"{frames} frames, seed {seed}",
            "variants": out}


def run_agents(n_teams: int = 512, A: int = 8, rounds: int = 4, sep: float = 25.0, oracle_teams: int = 2):
    """Multi-agent teams (the paper's stated future work) on the batch planner:
    ``n_teams`` maps of A agents swapping sides across the centre, planned in
    ``rounds`` rounds of simultaneous best responses (each a planning cycle with PI
    around the agent's own previous path, its mates' previous paths counting as
    moving obstacles).  Per round: device time (CUDA events) of the batch run,
    agent-plans/s, the share of plans free of collisions and conflicts, median cost;
    beside it the FP64 oracle on the first ``oracle_teams`` teams."""
    import torch

    import oracle
    from paper_2308_10169_gb300 import BatchPlanner
    from paper_2308_10169_gb300.inputs import team_workload
    specs, hyper, points, circles, first, size = team_workload(0, n_teams=n_teams, A=A)
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, circles)
    shape, _ = bp.autotune(trial_launches=3)
    bp.set_teams(first, size, sep)
    bp.run_async(True)        # warm-up: captures the graph; round 0 below repeats it exactly
    bp.read()
    per = []
    n = len(specs)
    for r in range(rounds):
        if r:
            bp.next_round(r)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bp.stream)
        bp.run_async(True)
        e1.record(bp.stream)
        res = bp.read()
        ms = e0.elapsed_time(e1)
        per.append({"round": r, "ms": ms, "agent_plans_per_s": n / (ms / 1e3),
                    "free_of_collisions_and_conflicts": float(np.mean([x["Q"] == 0 for x in res])),
                    "median_cost": float(np.median([x["cost"] for x in res])),
                    "iters_per_plan": float(np.mean([x["iters"] for x in res]))})
    ora = []
    for m in range(oracle_teams):
        s0 = m * A
        out = oracle.multi_agent_plan(specs[s0].config(), hyper[s0], circles[s0],
                                      [points[s0 + a, :2] for a in range(A)],
                                      [points[s0 + a, 2:] for a in range(A)], sep, rounds)
        ora.append(out)
    for r in range(rounds):
        rr = [ora[m][r][a] for m in range(oracle_teams) for a in range(A)]
        per[r]["oracle_sample"] = {"agents": len(rr),
                                   "free_of_collisions_and_conflicts": float(np.mean([x["Q"] == 0 for x in rr])),
                                   "median_cost": float(np.median([x["cost"] for x in rr]))}
    return {"workload": f"{n_teams} teams x {A} agents on 400x400 maps (16 circles r~U[8,15] in the middle), "
                        f"agents swapping sides across the centre, separation {sep}, T=8, G=8 x N=32 per agent, "
                        f"AT stall 10 / cap 100, {rounds} rounds of best responses",
            "scenes": n, "shape": shape, "rounds": per}


def run_bf(fns, iters: int, trials: int, peak_gbs: float):
    """Benchmark functions (Table BFs): the large-scale runs of Sec. 4.1.2 (16K
    particles x 1K coordinates) and the standard runs of Sec. 4.1.1 (80 particles x
    30 coordinates, ``trials`` trials as the runs of one launch), Table hyper8 rows.
    Each run is one CUDA graph (init, iterations, bests), timed with CUDA events after
    one untimed run; the swarm tensors (262 MB at the large size) exceed L2."""
    import torch

    from paper_2308_10169_gb300 import BFPlanner
    from paper_2308_10169_gb300.inputs import BF_NAMES, bf_large, bf_standard
    paper_large = {1: 23.8, 2: 30.3, 3: 29.6, 4: 30.2}
    paper_standard = {1: 0.37, 2: 0.44, 3: 0.42, 4: 0.46}
    out = {"large": {}, "standard": {}}
    for fn in fns:
        cfg, hy = bf_large(fn, iters=iters)
        pl = BFPlanner(cfg)
        pl.set_hyper(hy)
        pl.run_async()
        pl.sync()
        l0 = pl.launch_count()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(pl.stream)
        pl.run_async()
        b.record(pl.stream)
        pl.sync()
        ms = a.elapsed_time(b)
        coords = cfg.G * cfg.N * cfg.D
        algo = 20 * coords                      # X, V, Pbest read + X, V written, per iteration
        # launch 1 reads X and writes every Pbest row (8 B); launches 2..K+1 are updates
        gbs = coords * (20 * iters + 8) / (ms / 1e3) / 1e9
        r = pl.read(0)
        out["large"][BF_NAMES[fn]] = {
            "s_per_run": ms / 1e3, "us_per_iteration": 1e3 * ms / iters, "best": r["fit"],
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s",
                         "frac": gbs / peak_gbs, "kernel": "bf_iter_kernel",
                         "bytes_per_iteration": algo,
                         "traffic": BF_SPHERE_TRAFFIC_BYTES if fn == 1 else None,
                         "note": "20 B per coordinate; Pbest rows written on improvement not counted"},
            "gpu_launches": pl.launch_count() - l0,
            "paper_dtpso_gpu_s": paper_large[fn]}
        del pl
    if trials > 0:
        for fn in fns:
            cfg, hy = bf_standard(fn, trials=trials)
            cfg = cfg.with_(max_iters=iters)
            pl = BFPlanner(cfg)
            pl.set_hyper(hy)
            pl.run_async()
            pl.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(pl.stream)
            pl.run_async()
            b.record(pl.stream)
            pl.sync()
            ms = a.elapsed_time(b)
            fits = [pl.read(r)["fit"] for r in range(trials)]
            out["standard"][BF_NAMES[fn]] = {
                "s_all_trials": ms / 1e3, "s_per_trial_equivalent": ms / 1e3 / trials,
                "us_per_iteration": 1e3 * ms / iters, "median_best": float(np.median(fits)),
                "paper_dtpso_s_per_trial": paper_standard[fn]}
    out["workload"] = (f"large: D=1000, 8 x 2048 particles, {iters} iterations; standard: D=30, 8 x 10 "
                       f"particles, {trials} trials in one launch; [-600,600]^D, Table hyper8 rows; "
                       "paper numbers are other hardware (context only)")
    return out


def run_poly(runs: int = 64, iters: int = 100):
    """Path planning among polygon obstacles (Sec. 3.3.1's map model): ``runs``
    independent plans of one static scene (12 boxes + 4 non-convex U shapes, 80
    edges), T = 8, G = 8 x 170, Table hyper8path, alpha = 30, beta = 4, ``iters``
    iterations, one CUDA graph per batch of runs; also one plan alone (latency)."""
    import torch

    from paper_2308_10169_gb300 import BFPlanner
    from paper_2308_10169_gb300.inputs import polygon_workload
    from paper_2308_10169_gb300.planner import poly_evaluate
    out = {}
    for R in (runs, 1):
        cfg, start, target, polys, edges, hy = polygon_workload(0, iters=iters, runs=R)
        pl = BFPlanner(cfg)
        pl.set_hyper(hy)
        pl.set_polygons(start, target, edges)
        kname = pl.kernel_name()
        pl.run_async()
        pl.sync()
        l0 = pl.launch_count()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(pl.stream)
        pl.run_async()
        b.record(pl.stream)
        pl.sync()
        ms = a.elapsed_time(b)
        best = np.stack([pl.read(r)["x"] for r in range(R)])
        F, Q = poly_evaluate(torch.from_numpy(best).cuda(), start, target, torch.from_numpy(edges).cuda(),
                             cfg.alpha, cfg.beta)
        Q = Q.cpu().numpy()
        M, T, E = cfg.G * cfg.N, cfg.D // 2, edges.shape[0]
        pairs = R * M * (T + 1) * E * iters
        achieved = pairs * 20 / (ms / 1e3) / 1e12
        out["batch" if R == runs else "single"] = {
            "runs": R, "ms": ms, "plans_per_s": R / (ms / 1e3), "us_per_iteration": 1e3 * ms / iters,
            "median_cost": float(np.median(F.cpu().numpy())), "collision_free": float(np.mean(Q == 0)),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak()[0], "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak()[0], "peak_source": fp32_peak()[1], "kernel": kname,
                         "flops_per_pair": 20},
            "gpu_launches": pl.launch_count() - l0}
        del pl
    out["workload"] = (f"400x400 map, 12 boxes + 4 U-shaped polygons (80 edges), T=8, G=8 x 170, "
                       f"{iters} iterations, Table hyper8path, alpha=30 beta=4, {runs} plans per graph")
    out["batched_scenes"] = run_poly_batch()
    return out


def run_poly_batch(n: int = 1024, iters: int = 100, seed: int = 0):
    """Independent polygon scenes in the batched planner (one CUDA graph): each a
    400 x 400 map with 4..16 axis-aligned boxes (centres U[60,340]^2, half-sizes
    U[10,30]), T ~ U{8..32}, G = 8, N per group ~ U{32..170}, sampled hyper-parameters,
    alpha 30, beta 4, ``iters`` iterations."""
    import torch

    from paper_2308_10169_gb300 import BatchPlanner
    from paper_2308_10169_gb300.inputs import BatchSceneSpec, box, polygon_edges, sample_hyper
    rng = np.random.default_rng(9000 + seed)
    specs, hyper, obst = [], [], []
    for i in range(n):
        k = int(rng.integers(4, 17))
        e = polygon_edges([box(*rng.uniform(60, 340, 2), *rng.uniform(10, 30, 2)) for _ in range(k)])
        specs.append(BatchSceneSpec(T=int(rng.integers(8, 33)), G=8, N=int(rng.integers(32, 171)), O=len(e),
                                    max_iters=iters, alpha=30.0, beta=4, seed=seed, run_id=i, obstacle_kind=1))
        hyper.append(sample_hyper(int(rng.integers(1 << 30)), 8))
        obst.append(e)
    points = np.tile(np.array([[20, 20, 380, 380]], np.float32), (n, 1))
    bp = BatchPlanner(specs)
    bp.set_inputs(hyper, points, obst)
    bp.autotune(trial_launches=3)
    bp.run_async(True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    bp.run_async(True)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    res = bp.read()
    pairs = sum(sp.G * sp.N * (sp.T + 1) * sp.O for sp in specs) * iters
    achieved = pairs * 20 / (ms / 1e3) / 1e12
    return {"workload": f"{n} scenes of 4..16 boxes, T~U{{8..32}}, G=8, N/group~U{{32..170}}, {iters} iterations, "
                        "one CUDA graph (batched planner, obstacle_kind = polygons)",
            "plans_per_s": n / (ms / 1e3), "ms": ms, "pair_tests_per_s": pairs / (ms / 1e3),
            "median_cost": float(np.median([r["cost"] for r in res])),
            "collision_free": float(np.mean([r["Q"] == 0 for r in res])),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak()[0], "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak()[0], "peak_source": fp32_peak()[1], "kernel": "batch_kernel",
                         "flops_per_pair": 20},
            "shape": bp.shape()}


# Algorithmic work of a 3D path evaluation: per (segment, sphere) test 24 flops
# (w = c - m: 3; along = w.u: 5; w - along u: 6; max(|along| - h, 0): 2; squared
# distance: 7; compare: 1), per segment 20 (direction 3, squared length 5, square
# root 1, reciprocal 1, unit vector 3, midpoint 6, half-length 1).
FLOPS_PER_PAIR_3D, FLOPS_PER_SEGMENT_3D = 24, 20
# dram__bytes_read.sum + dram__bytes_write.sum of one sphere_lane_kernel launch of the
# 64-plan batch (profiles/sphere_lane_kernel_3d_batch.md).
SPHERE_LANE_TRAFFIC_BYTES = 54078464
# The same for bf_iter_kernel<1>, large-scale Sphere (profiles/bf_iter_kernel_large_sphere.md).
BF_SPHERE_TRAFFIC_BYTES = 302956544


def run_plan3d(runs: int = 64, iters: int = 100, cycles: int = 20):
    """Path planning in three dimensions among spheres (the paper's Conclusion names
    the 2D-to-3D extension as future work): 400^3 box, 64 spheres r~U[10,30] (32
    moving), T = 16 (D = 48), G = 8 x 170, Table hyper8path, alpha = 30, beta = 4,
    ``iters`` iterations.  ``batch``: ``runs`` independent plans of the static scene
    in one CUDA graph; ``single``: one plan alone; ``dynamic``: ``cycles`` planning
    cycles of all runs among the moving spheres, each run warm-started (PI) from its
    own previous best path, through the host API (scene and warm start in, best
    paths out, every cycle)."""
    import torch

    from paper_2308_10169_gb300 import BFPlanner
    from paper_2308_10169_gb300.inputs import advance_spheres, sphere_workload
    from paper_2308_10169_gb300.planner import sphere_evaluate
    out = {}

    def quality(cfg, sc, sph, best):
        F, Q = sphere_evaluate(torch.from_numpy(best).cuda(), sc["start"], sc["target"],
                               torch.from_numpy(np.ascontiguousarray(sph)).cuda(), cfg.alpha, cfg.beta)
        return float(np.median(F.cpu().numpy())), float(np.mean(Q.cpu().numpy() == 0))

    for R in (runs, 1):
        cfg, sc, hy = sphere_workload(0, iters=iters, runs=R)
        pl = BFPlanner(cfg)
        pl.set_hyper(hy)
        pl.set_spheres(sc["start"], sc["target"], sc["spheres"])
        kname = pl.kernel_name()
        pl.run_async()
        pl.sync()
        l0 = pl.launch_count()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(pl.stream)
        pl.run_async()
        b.record(pl.stream)
        pl.sync()
        ms = a.elapsed_time(b)
        best, _, _ = pl.read_all()
        med, cf = quality(cfg, sc, sc["spheres"], best)
        M, T, S = cfg.G * cfg.N, cfg.D // 3, sc["spheres"].shape[0]
        flops = R * M * (T + 1) * (FLOPS_PER_PAIR_3D * S + FLOPS_PER_SEGMENT_3D) * iters
        achieved = flops / (ms / 1e3) / 1e12
        out["batch" if R == runs else "single"] = {
            "runs": R, "ms": ms, "plans_per_s": R / (ms / 1e3), "us_per_iteration": 1e3 * ms / iters,
            "particle_evals_per_s": R * M * iters / (ms / 1e3),
            "median_cost": med, "collision_free": cf,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak()[0], "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak()[0], "peak_source": fp32_peak()[1], "kernel": kname,
                         "flops_per_pair": FLOPS_PER_PAIR_3D, "flops_per_segment": FLOPS_PER_SEGMENT_3D,
                         "traffic": SPHERE_LANE_TRAFFIC_BYTES if kname == "sphere_lane_kernel" else None},
            "gpu_launches": pl.launch_count() - l0}
        del pl
    # dynamic cycles with PI, through the host API; then the same with Auto Truncation
    def dynamic(at_stall):
        cfg, sc, hy = sphere_workload(0, iters=iters, runs=runs, at_stall=at_stall, stall_tol=1.0)
        pl = BFPlanner(cfg)
        pl.set_hyper(hy)
        sph, vel = sc["spheres"], sc["vel"]
        prev, meds, cfs, its = None, [], [], []
        pl.set_spheres(sc["start"], sc["target"], sph)
        pl.run_async()
        pl.sync()
        cms = []
        for cycle in range(cycles):
            if cycle:
                sph, vel = advance_spheres(sph, vel)
            c0 = time.perf_counter()
            pl.set_spheres(sc["start"], sc["target"], sph)
            pl.set_warm_start(prev, cycle=cycle)
            pl.run_async()
            prev, fit, it = pl.read_all()
            cms.append(1e3 * (time.perf_counter() - c0))
            its.append(float(np.mean(it)))
            med, cf = quality(cfg, sc, sph, prev)
            meds.append(med)
            cfs.append(cf)
        return {"runs": runs, "cycles": cycles, "plans_per_s": runs * cycles / (sum(cms) / 1e3),
                "ms_per_cycle": {"p50": float(np.percentile(cms, 50)), "p99": float(np.percentile(cms, 99))},
                "iters_per_plan": float(np.mean(its)),
                "median_cost_first_last": [meds[0], meds[-1]],
                "collision_free_first_last": [cfs[0], cfs[-1]],
                "collision_free_mean": float(np.mean(cfs)),
                "note": "host API per cycle: set_spheres + set_warm_start (PI from each run's previous best) + "
                        "the run's CUDA graph + best paths read back; the sphere motion on the host"
                        + ("; Auto Truncation by stall counter 10, tolerance 1.0 (a stopped plan's later "
                           "launches skip it)" if at_stall else "")}

    out["dynamic"] = dynamic(0)
    out["dynamic_at"] = dynamic(10)
    out["workload"] = (f"400^3 box, 64 spheres r~U[10,30] (32 moving |v|~U[0.5,2]), T=16 (D=48), G=8 x 170, "
                       f"{iters} iterations, Table hyper8path, alpha=30 beta=4, PI gamma=0.25 h=20, "
                       f"{runs} plans per graph")
    return out


def _world_step(ag):
    """The client's simulated world between two requests of an agent: circles and
    start/target move by their velocity and bounce off the map border."""
    c, v = ag["circles"], ag["circle_vel"]
    for d in (0, 1):
        c[:, d] += v[:, d]
        flip = ((c[:, d] - c[:, 2] < 0) & (v[:, d] < 0)) | ((c[:, d] + c[:, 2] > 400.0) & (v[:, d] > 0))
        v[flip, d] *= -1
    for p, pv in (("start", "start_vel"), ("target", "target_vel")):
        ag[p] += ag[pv]
        for d in (0, 1):
            if (ag[p][d] < 0 and ag[pv][d] < 0) or (ag[p][d] > 400 and ag[pv][d] > 0):
                ag[pv][d] *= -1


SERVE_SLOTS = 1024


def train_serving_prior(radii, n_per_set: int, rounds: int, epochs: int = 30):
    """The learned prior that seeds served requests: T = 20 proposals, trained by
    self-training (fit_prior_sets) on snapshots shaped like the serving scenes, both
    circle counts, labelled by the planner itself (G = 8 x N = 170, cap 300, stall AT
    tolerance 1.0, the shared evolved hyper-parameters).  Its rows after the training
    ones are the server's scratch."""
    import torch

    from paper_2308_10169_gb300.inputs import prior_init_params, serving_prior_scenes
    from paper_2308_10169_gb300.prior import Prior, fit_prior_sets
    sets = [serving_prior_scenes(100 + k, n_per_set, O, r_range=radii) for k, O in enumerate((32, 256))]
    n = 2 * n_per_set
    pr = Prior(T=20, hidden1=1024, hidden2=512, capacity=n + SERVE_SLOTS, max_batch=4096, max_circles=256)
    pr.set_params(prior_init_params(0, pr.K, 1024, 512, 40))
    hy, _ = shared_hyper()
    t0 = time.perf_counter()
    hist = fit_prior_sets(pr, sets, rounds=rounds, epochs=epochs, batch=4096, seed=5, n_prior=43, T=20, G=8, N=170,
                          hyper=hy, max_iters=300, stall_iters=10, stall_tol=1.0)
    torch.cuda.synchronize()
    info = {"workload": f"{n} serving-like snapshots ({n_per_set} with 32 circles, {n_per_set} with 256; radii "
                        f"U[{radii[0]:g},{radii[1]:g}] x sqrt(32/O), start/target drift U{{0..99}}), T=20 labels "
                        "by the planner (G=8 x N=170, cap 300, AT stall 10 tolerance 1.0, shared evolved hyper), "
                        f"{rounds} self-training rounds x {epochs} epochs, MLP 4104 -> 1024 -> 512 -> 40",
            "label_median_cost_per_round": hist["label_cost"],
            "label_collision_free_per_round": hist["label_collision_free"],
            "loss_first_last_per_round": hist["losses"], "train_steps": hist["steps"],
            "train_s": hist["train_s"], "label_plan_s": hist["plan_s"], "wall_s": time.perf_counter() - t0}
    return pr, n, info


def run_serve(rate: float, seconds: float, n_agents: int = 2048, radii=(3.0, 15.0), prior=None, prior_row: int = 0,
              n_prior: int = 8):
    """Open-loop serving: Poisson arrivals at `rate`, 2048 agents with mixed T and O;
    with a learned prior attached when one is given."""
    from paper_2308_10169_gb300 import Server
    from paper_2308_10169_gb300.inputs import poisson_arrivals, serving_workload
    agents = serving_workload(0, n_agents, r_range=radii)
    arr = poisson_arrivals(0, rate, seconds)
    who = np.random.default_rng(11).integers(0, n_agents, len(arr))
    sv = Server(n_agents=n_agents, max_slots=SERVE_SLOTS, G=8, N=32, Tmax=40, Omax=256, max_iters=100,
                stall_iters=10)
    if prior is not None:
        sv.set_prior(prior, n_prior, first_row=prior_row)
    for a, ag in enumerate(agents):
        sv.set_hyper(ag["hyper"], agent=a)
    for i, (t, a) in enumerate(zip(arr, who)):
        ag = agents[a]
        _world_step(ag)
        sv.submit_at(int(a), ag["T"], ag["start"], ag["target"], ag["circles"], tag=i, arrival_s=float(t))
    sv.clock(restart=True)
    sv.run()
    done = sv.poll(max_n=len(arr) + 1)
    lat = np.array([d["finish_s"] - d["arrival_s"] for d in done]) * 1e3
    span = max(d["finish_s"] for d in done) - min(d["arrival_s"] for d in done)
    st = sv.stats()
    return {"offered_per_s": rate, "requests": len(arr), "plans_per_s": len(done) / span,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "iters_per_plan": float(np.mean([d["iters"] for d in done])),
            "median_cost": float(np.median([d["cost"] for d in done])),
            "collision_free": float(np.mean([d["Q"] == 0 for d in done])),
            "collision_free_by_T_O": {f"T{T}_O{O}": float(np.mean([d["Q"] == 0 for d in done
                                                                  if d["T"] == T and agents[d["agent"]]["O"] == O]))
                                      for T in (8, 20, 40) for O in (32, 256)},
            "at_fire_rate": float(np.mean([d["iters"] < 100 for d in done])), "slots": st["slots"],
            "ticks": st["ticks"], "gpu_launches": st["launches"],
            "prior": None if prior is None else {"n_prior": n_prior, "proposal_T": 20}}


def serve_single_scene(n: int = 256, n_agents: int = 2048, radii=(3.0, 15.0), prior=None, prior_row: int = 0,
                       n_prior: int = 8):
    """The plain single-scene kernel on the serving mix: the first request of n agents
    (no previous path), one plan at a time through sepso_plan (host scene in,
    waypoints out), with the server's planner settings; and the same n requests as
    one burst through the server.  Same algorithm and random streams, so the median
    costs agree; throughput and latency are the comparison.  With a prior, the burst
    once more with it attached (its proposals seed the requests)."""
    import torch

    from paper_2308_10169_gb300 import Planner, Server
    from paper_2308_10169_gb300.inputs import AT_STALL, Scene, SepsoConfig, serving_workload
    agents = serving_workload(0, n_agents, r_range=radii)[:n]
    lat, costs, its, qs = [], [], [], []
    for a, ag in enumerate(agents):
        cfg = SepsoConfig(T=ag["T"], G=8, N=32, max_obstacles=256, alpha=30.0, beta=4, max_iters=100,
                          at_mode=AT_STALL, stall_iters=10, stall_tol=0.0, use_pi=True, pi_gamma=0.25,
                          pi_halfwidth=20.0, seed=0, run_id=a)
        pl = Planner(cfg)
        pl.set_hyper(ag["hyper"])
        wp = np.zeros(2 * ag["T"], np.float32)
        if a == 0:  # warm-up
            pl.set_scene(Scene(start=ag["start"], target=ag["target"], circles=ag["circles"]), motion=False)
            pl.plan_into(wp)
            pl = Planner(cfg)
            pl.set_hyper(ag["hyper"])
        torch.cuda.synchronize()
        t = time.perf_counter()
        pl.set_scene(Scene(start=ag["start"], target=ag["target"], circles=ag["circles"]), motion=False)
        r = pl.plan_into(wp)
        lat.append(time.perf_counter() - t)
        costs.append(float(r.cost))
        its.append(int(r.iters))
        qs.append(int(r.Q))
    lat = np.array(lat) * 1e3

    def burst(pr):
        sv = Server(n_agents=n_agents, max_slots=SERVE_SLOTS, G=8, N=32, Tmax=40, Omax=256, max_iters=100,
                    stall_iters=10)
        if pr is not None:
            sv.set_prior(pr, n_prior, first_row=prior_row)
        for a, ag in enumerate(agents):
            sv.set_hyper(ag["hyper"], agent=a)
        for a, ag in enumerate(agents):
            sv.submit_at(a, ag["T"], ag["start"], ag["target"], ag["circles"], tag=a, arrival_s=0.0)
        sv.clock(restart=True)
        sv.run()
        done = sv.poll(max_n=n + 1)
        slat = np.array([d["finish_s"] - d["arrival_s"] for d in done]) * 1e3
        span = max(d["finish_s"] for d in done)
        return {"plans_per_s": len(done) / span,
                "latency_ms": {"p50": float(np.percentile(slat, 50)), "p99": float(np.percentile(slat, 99))},
                "median_cost": float(np.median([d["cost"] for d in done])),
                "iters_per_plan": float(np.mean([d["iters"] for d in done])),
                "collision_free": float(np.mean([d["Q"] == 0 for d in done]))}

    out = {"requests": n,
           "single_scene": {"plans_per_s": n / (lat.sum() / 1e3),
                            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                           "p99": float(np.percentile(lat, 99))},
                            "median_cost": float(np.median(costs)), "iters_per_plan": float(np.mean(its)),
                            "collision_free": float(np.mean(np.array(qs) == 0))},
           "server_burst": burst(None)}
    if prior is not None:
        out["server_burst_prior"] = burst(prior)
    return out


def run_prior(n_train: int, n_eval: int, rounds: int, epochs: int, single: dict, B: int = 4096):
    """Learned prior: self-training on the planner's own solutions, held-out
    comparison with the PI-only start, tensor-core GEMM and training throughput."""
    import torch

    from paper_2308_10169_gb300.inputs import prior_init_params, prior_scenes
    from paper_2308_10169_gb300.prior import Prior, evaluate_prior, fit_prior, gemm_bf16
    H1, H2, T = 1024, 512, 20
    tr, ev = prior_scenes(0, n_train), prior_scenes(1, n_eval)
    pr = Prior(T=T, hidden1=H1, hidden2=H2, capacity=n_train + n_eval, max_batch=B)
    pr.set_params(prior_init_params(0, pr.K, H1, H2, 2 * T))
    l0 = pr.launch_count()
    hist = fit_prior(pr, tr, rounds=rounds, epochs=epochs, batch=B, seed=1)
    res = evaluate_prior(pr, ev, n_train)
    K, O = pr.K, 2 * T
    flops_fwd = 2.0 * B * (K * H1 + H1 * H2 + H2 * O)
    flops_step = 3.0 * flops_fwd          # forward + the two backward products per layer
    train = {"steps": hist["steps"], "batch": B, "seconds": hist["train_s"],
             "steps_per_s": hist["steps"] / hist["train_s"],
             "tflops": hist["steps"] * flops_step / hist["train_s"] / 1e12,
             "loss_first_last_per_round": hist["losses"]}
    gem = run_gemm(B, H1, K)
    dom = gem["grad_W1"]
    peak = _bf16_peak()
    roof = {"bound": "tensor", "achieved": dom["tflops"], "peak": peak, "unit": "TFLOP/s",
            "frac": dom["tflops"] / peak, "traffic": GEMM_GRADW1_TRAFFIC_BYTES,
            "kernel": "gemm_tc_kernel (grad_W1 shape)",
            "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured"}
    # batched + prior against the plain single-scene kernel at equal median path
    # cost, on the same held-out dynamic sequences and settings: the single-scene
    # kernel's last-cycle median cost, and the smallest iteration budget at which the
    # batched planner with the prior (warm-started by PI as well) matches it
    from paper_2308_10169_gb300.prior import single_scene_dynamic
    ss = single_scene_dynamic(ev, n=min(64, n_eval))
    hit = [q for q in res["dynamic_budgets"]["prior_pi"] if q["cost_median"] <= ss["cost_median"]]
    hit_pi = [q for q in res["dynamic_budgets"]["pi_only"] if q["cost_median"] <= ss["cost_median"]]
    eq = {"single_scene": ss,
          "batched_prior_pi": ({"iters": hit[0]["iters"], "median_cost": hit[0]["cost_median"],
                                "plans_per_s": hit[0]["plans_per_s"]} if hit else None),
          "batched_pi_only": ({"iters": hit_pi[0]["iters"], "median_cost": hit_pi[0]["cost_median"],
                               "plans_per_s": hit_pi[0]["plans_per_s"]} if hit_pi else None),
          "note": "last cycle of 5-cycle held-out dynamic sequences; Table hyper8 path rows, AT stall 10 / cap 300 "
                  "for the single-scene kernel; budgets without AT for the batched planner"}
    return {"workload": f"MLP 64x64 raster + start/target ({K} features) -> {H1} -> {H2} -> {O}, BF16 "
                        f"weights/activations, FP32 accumulate and masters, Adam; {n_train} training scenes "
                        f"(64 circles r~U[10,30], 32 moving, start/target drift) labelled by the planner "
                        f"(T=20, G=8 x N=170, Table hyper8 path rows, AT stall 10 / cap 300), {rounds} "
                        f"self-training rounds x {epochs} epochs; {n_eval} held-out scenes",
            "labels": {"median_cost_per_round": hist["label_cost"], "plan_seconds": hist["plan_s"]},
            "train": train, "gemm": gem, "roofline": roof, "eval": res, "at_single_scene_cost": eq,
            "gpu_launches": pr.launch_count() - l0}


def _hbm_peak() -> float:
    path = ROOT / "MEASURED_PEAKS.json"
    return float(json.loads(path.read_text()).get("hbm_gbs", 6800.0)) if path.exists() else 6800.0


def _bf16_peak() -> float:
    path = ROOT / "MEASURED_PEAKS.json"
    return float(json.loads(path.read_text()).get("bf16_tflops", 1900.0)) if path.exists() else 1900.0


def run_gemm(B: int = 4096, H1: int = 1024, K: int = 4104, reps: int = 20):
    """The tensor-core GEMM alone on the two largest products of a training step
    (grad W1 first, then forward layer 1), each launch timed with CUDA events after
    an L2 flush.  Operand rows have the training step's pitch (the feature rows and
    W1 are stored at a multiple of 64 elements, 128-byte rows)."""
    import torch

    from paper_2308_10169_gb300.prior import gemm_bf16
    gem = {}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    for name, (M, N, Kd) in {"grad_W1": (H1, K, B), "forward_layer1": (B, H1, K)}.items():
        pitch = (Kd + 63) // 64 * 64
        A = torch.randn(M, pitch, device="cuda").to(torch.bfloat16)[:, :Kd]
        Bm = torch.randn(N, pitch, device="cuda").to(torch.bfloat16)[:, :Kd]
        # warm-up long enough for the clocks to leave their idle state
        t_end = time.perf_counter() + 0.3
        while time.perf_counter() < t_end:
            for _ in range(20):
                gemm_bf16(A, Bm, sync=False)
            torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gemm_bf16(A, Bm, sync=False)
            e1.record()
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.median(ts))
        gem[name] = {"M": M, "N": N, "K": Kd, "ms": ms, "tflops": 2.0 * M * N * Kd / (ms / 1e3) / 1e12,
                     "frac_of_measured_bf16_peak": 2.0 * M * N * Kd / (ms / 1e3) / 1e12 / _bf16_peak()}
    return gem


def cpu_baseline(seconds: float):
    """The oracle on all host cores for a bounded time: one independent dynamic run
    per core (Philox keys 0..P-1, the shared hyper-parameters), cycles until
    ``seconds`` pass in each run; value = cycles / wall time."""
    from paper_2308_10169_gb300.inputs import dynamic_workload
    P = host_cores()
    r = oracle_runs(P, [0] * P, [-1] * P, seconds)
    cfg = dynamic_workload(0)[0]
    n = len(r["times"])
    return {"value": n / r["wall"], "unit": UNIT, "cores": P, "kind": "oracle",
            "sample": f"the first cycles of {P} independent dynamic runs (Philox keys 0..{P - 1}, "
                      f"shared hyper-parameters), one process per core, about {seconds:.0f} s each: "
                      f"{n} cycles in {r['wall']:.1f} s wall, FP64",
            "particle_evals_per_s": sum(r["iters"]) * cfg.G * cfg.N / r["wall"],
            "latency_ms_single_thread": {"mean": 1e3 * float(np.mean(r["times"])),
                                         "p50": 1e3 * float(np.percentile(r["times"], 50))},
            **plan_stats(r["iters"], r["costs"], r["Q"], cfg.max_iters)}


def _oracle_seed_worker(args):
    """The oracle's first ``cycles`` cycles of the dynamic run under Philox key seed."""
    seed, cycles = args
    import oracle
    from paper_2308_10169_gb300.inputs import dynamic_workload
    cfg, scene, _ = dynamic_workload(0)
    hyper, _ = shared_hyper()
    sw = oracle.Swarm(cfg.with_(seed=seed), hyper)
    c, v, st, sv, tg, tv = (scene.circles, scene.circle_vel, scene.start, scene.start_vel,
                            scene.target, scene.target_vel)
    out = []
    for cyc in range(cycles):
        if cyc:
            c, v, st, sv, tg, tv = oracle.advance_scene(cfg.map_w, cfg.map_h, c, v, st, sv, tg, tv)
        r = sw.plan(oracle.Scene(st, tg, c))
        out.append((r["cost"], r["iters"], r["Q"]))
    return out


def cost_match_dynamic(seeds: int = 64, cycles: int = 2):
    """GPU vs oracle path cost on the headline workload with the shared
    hyper-parameters: under each of ``seeds`` Philox keys both plan the first
    ``cycles`` cycles of the dynamic run (a cold start, then PI; AT by stall
    counter, cap 300).  FP32 and FP64 trajectories separate, so the medians over
    the seeds are compared, cycle by cycle."""
    import multiprocessing as mp

    from paper_2308_10169_gb300 import Planner
    from paper_2308_10169_gb300.inputs import dynamic_workload
    cfg, scene, _ = dynamic_workload(0)
    hyper, _ = shared_hyper()
    t0 = time.perf_counter()
    gpu = []
    for s_ in range(seeds):
        pl = Planner(cfg.with_(seed=s_))
        pl.set_hyper(hyper)
        pl.set_scene(scene)
        row = []
        for cyc in range(cycles):
            if cyc:
                pl.advance(1)
            r = pl.plan()
            row.append((r["cost"], r["iters"], r["Q"]))
        gpu.append(row)
    t_gpu = time.perf_counter() - t0
    t0 = time.perf_counter()
    P = min(host_cores(), seeds)
    with mp.get_context("spawn").Pool(P) as pool:
        ora = pool.map(_oracle_seed_worker, [(s_, cycles) for s_ in range(seeds)], chunksize=1)
    t_ora = time.perf_counter() - t0
    per = []
    rng = np.random.default_rng(0)
    for cyc in range(cycles):
        g = [row[cyc] for row in gpu]
        o = [row[cyc] for row in ora]
        gc, oc = np.array([x[0] for x in g]), np.array([x[0] for x in o])
        gm, om = float(np.median(gc)), float(np.median(oc))
        # the spread of the two medians over the seeds: a bootstrap of both samples
        boot = [(np.median(rng.choice(gc, gc.size)) - np.median(rng.choice(oc, oc.size))) / om for _ in range(2000)]
        # the same Philox key on both sides: the per-key differences pair the samples
        d = (gc - oc) / oc
        gq, oq = np.array([x[2] for x in g]), np.array([x[2] for x in o])
        per.append({"cycle": cyc,
                    "gpu": plan_stats([x[1] for x in g], [x[0] for x in g], [x[2] for x in g], cfg.max_iters),
                    "oracle": plan_stats([x[1] for x in o], [x[0] for x in o], [x[2] for x in o], cfg.max_iters),
                    "rel_diff_median_cost": (gm - om) / om,
                    "rel_diff_bootstrap_95": [float(np.percentile(boot, 2.5)), float(np.percentile(boot, 97.5))],
                    "paired": {"median_rel_diff": float(np.median(d)),
                               "share_within_1pct": float(np.mean(np.abs(d) <= 0.01)),
                               "share_same_collision_outcome": float(np.mean((gq == 0) == (oq == 0)))}})
    return {"workload": "the headline dynamic run's first cycles, shared hyper-parameters",
            "seeds": seeds, "cycles": per, "gpu_seconds": t_gpu,
            "oracle_seconds": t_ora, "oracle_processes": P}


def oracle_match(seeds: int = 64):
    """Path cost of the GPU planner beside the FP64 oracle's on the static workload
    (400 x 400 map, T = 8, G = 8 x N = 32, 16 circles, 100 iterations), one plan per
    seed: FP32 and FP64 trajectories separate, so the medians over the seeds are the
    comparison (the parity tests hold them within 1%)."""
    import oracle
    from paper_2308_10169_gb300 import Planner
    from paper_2308_10169_gb300.inputs import static_workload
    gpu, ora = [], []
    t0 = time.perf_counter()
    for s in range(seeds):
        cfg, scene, hyper = static_workload(s)
        cfg = cfg.with_(seed=s)
        pl = Planner(cfg)
        pl.set_hyper(hyper)
        pl.set_scene(scene)
        gpu.append(float(pl.plan()["cost"]))
        ora.append(float(oracle.Swarm(cfg, hyper).plan(oracle.Scene(scene.start, scene.target,
                                                                       scene.circles))["cost"]))
    g, o = float(np.median(gpu)), float(np.median(ora))
    return {"workload": "static: 400x400, T=8, G=8 x N=32, 16 circles, 100 iterations, alpha 1000, beta 1",
            "seeds": seeds, "gpu_median_cost": g, "oracle_median_cost": o, "rel_diff": (g - o) / o,
            "seconds": time.perf_counter() - t0}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    sections = set(x.strip() for x in args.sections.split(",") if x.strip())
    if "main" in sections:
        line = run_ours(args, rank, world, local)
    else:
        line = {"metric": METRIC, "unit": UNIT, "sections": sorted(sections)} if rank == 0 else None
    if rank == 0:
        if world == 1 and "cpu" in sections and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
            line["oracle_match"] = oracle_match()
            line["cost_match"] = cost_match_dynamic(args.match_seeds, args.match_cycles)
        if world == 1 and "batch" in sections and args.batch_scenes > 0:
            line["batch"] = run_batch(args.batch_scenes, args.batch_iters)
        if world == 1 and "prior" in sections and args.prior_train > 0:
            line["prior"] = run_prior(args.prior_train, args.prior_eval, args.prior_rounds, args.prior_epochs,
                                      line, args.prior_batch)
        if world == 1 and "paper" in sections:
            line["paper_ablation"] = run_paper()
        if world == 1 and "boxes" in sections:
            line["paper_ablation_boxes"] = run_paper_boxes()
        if world == 1 and "agents" in sections:
            line["multi_agent"] = run_agents()
        if world == 1 and "poly" in sections:
            line["poly"] = run_poly()
        if world == 1 and "plan3d" in sections:
            line["plan3d"] = run_plan3d()
        if world == 1 and "bf" in sections:
            line["bf"] = run_bf([int(x) for x in args.bf_fns.split(",") if x.strip()], args.bf_iters,
                                args.bf_trials, _hbm_peak())
        if world == 1 and "gemm" in sections:
            line["gemm"] = run_gemm()
        if world == 1 and "serve" in sections and args.serve_rates:
            radii = tuple(float(x) for x in args.serve_radii.split(","))
            rates = [float(r) for r in args.serve_rates.split(",")]
            pr, prow, pinfo = (train_serving_prior(radii, args.serve_prior_train, args.serve_prior_rounds)
                               if args.serve_prior_train > 0 else (None, 0, None))
            line["serve"] = {
                "workload": "2048 agents, Poisson arrivals, T in {8,20,40}, O in {32,256} circles, centres "
                            f"U[60,340]^2, r~U[{radii[0]:g},{radii[1]:g}] x sqrt(32/O), "
                            "obstacles advanced per request, G=8 x N=32, PI warm start on the device, "
                            "AT stall 10 / cap 100, continuous batching (1024 slots)",
                "runs": [run_serve(r, args.serve_seconds, radii=radii) for r in rates],
                "prior": pinfo,
                "runs_prior": [run_serve(r, args.serve_seconds, radii=radii, prior=pr, prior_row=prow)
                               for r in rates] if pr is not None else None,
                "vs_single_scene": serve_single_scene(radii=radii, prior=pr, prior_row=prow)}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
