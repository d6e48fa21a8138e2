"""ctypes binding of ``libsepso.so`` (declared in include/sepso.h).

Argument marshalling only.  There is no fallback: if the library is missing or
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

from . import build as _build

_lib = None

SEPSO_OK = 0
ERRORS = {-1: "EINVAL", -2: "ESTATE", -3: "ENOSPC", -4: "ECUDA", -5: "ETIMEOUT", -6: "ENOMEM",
          -7: "ERANGE", -8: "EBOUNDS"}


class SepsoError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.c_int32), ("G", ctypes.c_int32), ("N", ctypes.c_int32),
        ("max_obstacles", ctypes.c_int32),
        ("map_w", ctypes.c_float), ("map_h", ctypes.c_float),
        ("alpha", ctypes.c_float), ("beta", ctypes.c_int32),
        ("max_iters", ctypes.c_int32),
        ("at_mode", ctypes.c_int32), ("tw", ctypes.c_int32), ("delta", ctypes.c_float),
        ("stall_iters", ctypes.c_int32), ("stall_tol", ctypes.c_float),
        ("use_pi", ctypes.c_int32), ("pi_gamma", ctypes.c_float), ("pi_halfwidth", ctypes.c_float),
        ("seed", ctypes.c_uint64), ("run_id", ctypes.c_uint32),
        ("runs", ctypes.c_int32), ("ctas_per_group", ctypes.c_int32), ("threads", ctypes.c_int32),
        ("circle_split", ctypes.c_int32), ("fitness_mode", ctypes.c_int32),
        ("exchange", ctypes.c_int32), ("obstacle_kind", ctypes.c_int32),
    ]


class Result(ctypes.Structure):
    _fields_ = [("cost", ctypes.c_float), ("length", ctypes.c_float), ("Q", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("status", ctypes.c_int32)]


class HsefConfig(ctypes.Structure):
    _fields_ = [("HG", ctypes.c_int32), ("HN", ctypes.c_int32), ("E", ctypes.c_int32),
                ("hhyper", ctypes.c_float * (32 * 6)), ("lo", ctypes.c_float * 3),
                ("hi", ctypes.c_float * 3), ("l_vlimit", ctypes.c_float),
                ("hseed", ctypes.c_uint64)]


class BatchScene(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("G", ctypes.c_int32), ("N", ctypes.c_int32),
                ("O", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_int32), ("seed", ctypes.c_uint64), ("run_id", ctypes.c_uint32),
                ("stall_iters", ctypes.c_int32), ("stall_tol", ctypes.c_float), ("n_pi", ctypes.c_int32),
                ("n_prior", ctypes.c_int32), ("pi_halfwidth", ctypes.c_float), ("cycle", ctypes.c_uint32),
                ("obstacle_kind", ctypes.c_int32)]


class BatchShape(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("threads", ctypes.c_int32), ("lanes", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("n_agents", ctypes.c_int32), ("max_slots", ctypes.c_int32),
                ("mem_budget", ctypes.c_size_t), ("G", ctypes.c_int32), ("N", ctypes.c_int32),
                ("Tmax", ctypes.c_int32), ("Omax", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("stall_iters", ctypes.c_int32), ("stall_tol", ctypes.c_float),
                ("alpha", ctypes.c_float), ("beta", ctypes.c_int32), ("pi_gamma", ctypes.c_float),
                ("pi_halfwidth", ctypes.c_float), ("map_w", ctypes.c_float), ("map_h", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("tile", ctypes.c_int32), ("threads", ctypes.c_int32)]


class ServerDone(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_int64), ("agent", ctypes.c_int32), ("T", ctypes.c_int32),
                ("res", Result), ("arrival_s", ctypes.c_double), ("finish_s", ctypes.c_double)]


class PriorConfig(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int32), ("grid", ctypes.c_int32), ("hidden1", ctypes.c_int32),
                ("hidden2", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("capacity", ctypes.c_int32),
                ("max_circles", ctypes.c_int32), ("map_w", ctypes.c_float), ("map_h", ctypes.c_float),
                ("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


class GemmExtra(ctypes.Structure):
    _fields_ = [("Ct", ctypes.c_void_p), ("ldct", ctypes.c_int32), ("colsum", ctypes.c_void_p),
                ("ksplit", ctypes.c_int32), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


def make_config(cfg) -> Config:
    return Config(T=cfg.T, G=cfg.G, N=cfg.N, max_obstacles=cfg.max_obstacles, map_w=cfg.map_w,
                  map_h=cfg.map_h, alpha=cfg.alpha, beta=cfg.beta, max_iters=cfg.max_iters,
                  at_mode=cfg.at_mode, tw=cfg.tw, delta=cfg.delta, stall_iters=cfg.stall_iters,
                  stall_tol=cfg.stall_tol, use_pi=int(cfg.use_pi), pi_gamma=cfg.pi_gamma,
                  pi_halfwidth=cfg.pi_halfwidth, seed=cfg.seed, run_id=cfg.run_id, runs=cfg.runs,
                  ctas_per_group=cfg.ctas_per_group, threads=cfg.threads,
                  circle_split=cfg.circle_split, fitness_mode=cfg.fitness_mode,
                  exchange=cfg.exchange, obstacle_kind=cfg.obstacle_kind)


class BFConfig(ctypes.Structure):
    """``sepso_bf_config`` of include/sepso.h."""
    _fields_ = [("fn", ctypes.c_int32), ("D", ctypes.c_int32), ("G", ctypes.c_int32),
                ("N", ctypes.c_int32), ("lo", ctypes.c_float), ("hi", ctypes.c_float),
                ("max_iters", ctypes.c_int32), ("runs", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("run_id", ctypes.c_uint32),
                ("map_w", ctypes.c_float), ("map_h", ctypes.c_float), ("alpha", ctypes.c_float),
                ("beta", ctypes.c_int32), ("max_edges", ctypes.c_int32),
                ("map_d", ctypes.c_float), ("max_spheres", ctypes.c_int32),
                ("at_stall", ctypes.c_int32), ("stall_tol", ctypes.c_float)]


def bf_config_struct(cfg) -> BFConfig:
    return BFConfig(fn=cfg.fn, D=cfg.D, G=cfg.G, N=cfg.N, lo=cfg.lo, hi=cfg.hi,
                    max_iters=cfg.max_iters, runs=cfg.runs, seed=cfg.seed, run_id=cfg.run_id,
                    map_w=cfg.map_w, map_h=cfg.map_h, alpha=cfg.alpha, beta=cfg.beta,
                    max_edges=cfg.max_edges, map_d=cfg.map_d, max_spheres=cfg.max_spheres,
                    at_stall=cfg.at_stall, stall_tol=cfg.stall_tol)


# Every exported entry point with (restype, argtypes); the tests check the list
# against include/sepso.h.
_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_fp = ctypes.POINTER(ctypes.c_float)
SIGNATURES = {
    "sepso_workspace_size": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(_sz)]),
    "sepso_create": (ctypes.c_int, [ctypes.POINTER(Config), _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "sepso_destroy": (None, [_vp]),
    "sepso_set_hyper": (ctypes.c_int, [_vp, _i32, _fp]),
    "sepso_set_scene": (ctypes.c_int, [_vp, _fp, _fp, _fp, _i32]),
    "sepso_set_motion": (ctypes.c_int, [_vp, _fp, _fp, _fp]),
    "sepso_advance_scene": (ctypes.c_int, [_vp, _i32]),
    "sepso_get_scene": (ctypes.c_int, [_vp, _fp, _fp, _fp, _fp]),
    "sepso_plan_async": (ctypes.c_int, [_vp]),
    "sepso_plan": (ctypes.c_int, [_vp, _fp, ctypes.POINTER(Result)]),
    "sepso_read_result": (ctypes.c_int, [_vp, _i32, _fp, ctypes.POINTER(Result)]),
    "sepso_result_device": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "sepso_step": (ctypes.c_int, [_vp, _i32]),
    "sepso_evaluate": (ctypes.c_int, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "sepso_state_size": (ctypes.c_int, [_vp, ctypes.POINTER(_sz)]),
    "sepso_get_state": (ctypes.c_int, [_vp, _i32, _vp, _sz]),
    "sepso_set_state": (ctypes.c_int, [_vp, _i32, _vp, _sz]),
    "sepso_hsef": (ctypes.c_int, [_vp, ctypes.POINTER(HsefConfig), _vp]),
    "sepso_hsef_best": (ctypes.c_int, [_vp, _fp, _fp]),
    "sepso_plan_static": (ctypes.c_int, [ctypes.POINTER(Config), _fp, _fp, _fp, _fp, _i32, _fp,
                                         ctypes.POINTER(Result), _vp]),
    "sepso_sync": (ctypes.c_int, [_vp]),
    "sepso_launch_shape": (ctypes.c_int, [_vp] + [ctypes.POINTER(_i32)] * 4),
    "sepso_counters": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "sepso_launch_count": (_i64, [_vp]),
    "sepso_batch_workspace_size": (ctypes.c_int, [ctypes.POINTER(BatchScene), _i32,
                                                   ctypes.POINTER(_sz)]),
    "sepso_batch_create": (ctypes.c_int, [ctypes.POINTER(BatchScene), _i32, ctypes.c_float,
                                          ctypes.c_float, _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "sepso_batch_destroy": (None, [_vp]),
    "sepso_batch_set_inputs": (ctypes.c_int, [_vp, _fp, _fp, _fp]),
    "sepso_batch_set_shape": (ctypes.c_int, [_vp, ctypes.POINTER(BatchShape)]),
    "sepso_batch_get_shape": (ctypes.c_int, [_vp, ctypes.POINTER(BatchShape),
                                             ctypes.POINTER(_i32)]),
    "sepso_batch_autotune": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(BatchShape),
                                            ctypes.POINTER(ctypes.c_float)]),
    "sepso_batch_set_starts": (ctypes.c_int, [_vp, _vp, _vp, _i32, ctypes.POINTER(_i32)]),
    "sepso_batch_prior_used": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)]),
    "sepso_batch_run_async": (ctypes.c_int, [_vp, _i32]),
    "sepso_batch_read": (ctypes.c_int, [_vp, _fp, ctypes.POINTER(Result)]),
    "sepso_batch_launch_count": (_i64, [_vp]),
    "sepso_batch_last_error": (ctypes.c_char_p, []),
    "sepso_server_workspace_size": (ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_sz),
                                                    ctypes.POINTER(_i32)]),
    "sepso_server_create": (ctypes.c_int, [ctypes.POINTER(ServerConfig), _vp, _sz, _vp,
                                           ctypes.POINTER(_vp)]),
    "sepso_server_destroy": (None, [_vp]),
    "sepso_server_set_hyper": (ctypes.c_int, [_vp, _i32, _fp]),
    "sepso_server_set_prior": (ctypes.c_int, [_vp, _vp, _i32, _i32]),
    "sepso_server_submit": (ctypes.c_int, [_vp, _i32, _i32, _fp, _fp, _fp, _i32, _i64]),
    "sepso_server_submit_at": (ctypes.c_int, [_vp, _i32, _i32, _fp, _fp, _fp, _i32, _i64,
                                              ctypes.c_double]),
    "sepso_server_submit_polygons": (ctypes.c_int, [_vp, _i32, _i32, _fp, _fp, _fp, _i32, _i64,
                                                    ctypes.c_double]),
    "sepso_server_clock": (ctypes.c_double, [_vp, _i32]),
    "sepso_server_run": (ctypes.c_int, [_vp, _i64]),
    "sepso_server_tick": (ctypes.c_int, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "sepso_server_poll": (ctypes.c_int, [_vp, ctypes.POINTER(ServerDone), _fp, _i32,
                                         ctypes.POINTER(_i32)]),
    "sepso_server_drain": (ctypes.c_int, [_vp, _i64]),
    "sepso_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(_i32)] + [ctypes.POINTER(_i64)] * 4),
    "sepso_server_last_error": (ctypes.c_char_p, []),
    "sepso_prior_workspace_size": (ctypes.c_int, [ctypes.POINTER(PriorConfig), ctypes.POINTER(_sz)]),
    "sepso_prior_create": (ctypes.c_int, [ctypes.POINTER(PriorConfig), _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "sepso_prior_destroy": (None, [_vp]),
    "sepso_prior_num_params": (_i64, [_vp]),
    "sepso_prior_set_params": (ctypes.c_int, [_vp, _fp]),
    "sepso_prior_get_params": (ctypes.c_int, [_vp, _fp]),
    "sepso_prior_add_scenes": (ctypes.c_int, [_vp, _i32, _i32, _fp, ctypes.POINTER(_i32), _fp, _fp]),
    "sepso_prior_set_labels": (ctypes.c_int, [_vp, _i32, _i32, _vp, _i32]),
    "sepso_prior_get_rows": (ctypes.c_int, [_vp, _i32, _i32, _fp, _fp]),
    "sepso_prior_forward": (ctypes.c_int, [_vp, _i32, _i32, _fp]),
    "sepso_prior_grad": (ctypes.c_int, [_vp, _i32, _i32, _fp, _fp]),
    "sepso_prior_train": (ctypes.c_int, [_vp, _i32, _i32, _i32, _i32, ctypes.c_uint64, _fp]),
    "sepso_prior_infer": (ctypes.c_int, [_vp, _i32, _i32, _vp, _i32]),
    "sepso_prior_sync": (ctypes.c_int, [_vp]),
    "sepso_prior_launch_count": (_i64, [_vp]),
    "sepso_prior_last_error": (ctypes.c_char_p, []),
    "sepso_gemm_bf16": (ctypes.c_int, [_vp, _vp, _i32, _i32, _i32, _i32, _i32, ctypes.c_float, _vp, _i32,
                                       _vp, _i32, _vp, _i32, _vp, _i32, _i32, _vp]),
    "sepso_gemm_bf16_sync": (ctypes.c_int, [_vp]),
    "sepso_gemm_bf16_ex_workspace": (ctypes.c_int, [_i32, _i32, _i32, _i32, ctypes.POINTER(_sz)]),
    "sepso_gemm_bf16_ex": (ctypes.c_int, [_vp, _vp, _i32, _i32, _i32, _i32, _i32, ctypes.c_float, _vp, _i32,
                                          _vp, _i32, _vp, _i32, _vp, _i32, ctypes.POINTER(GemmExtra), _i32,
                                          _vp]),
    "sepso_exchange_form": (ctypes.c_int, [_vp]),
    "sepso_batch_set_teams": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                             ctypes.c_float]),
    "sepso_batch_next_round": (ctypes.c_int, [_vp, ctypes.c_uint32]),
    "sepso_set_polygons": (ctypes.c_int, [_vp, _fp, _fp, _fp, _i32, ctypes.POINTER(ctypes.c_int32), _i32]),
    "sepso_get_polygons": (ctypes.c_int, [_vp, _fp, _fp, _fp, _fp]),
    "sepso_philox": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_uint64, _vp, _vp]),
    "sepso_at_window_test": (ctypes.c_int, [_vp, _vp, _vp, _i32, _i32, ctypes.c_float, _vp, _vp]),
    "sepso_bf_workspace_size": (ctypes.c_int, [ctypes.POINTER(BFConfig), ctypes.POINTER(_sz)]),
    "sepso_bf_create": (ctypes.c_int, [ctypes.POINTER(BFConfig), _vp, _sz, _vp, ctypes.POINTER(_vp)]),
    "sepso_bf_destroy": (ctypes.c_int, [_vp]),
    "sepso_bf_set_hyper": (ctypes.c_int, [_vp, _vp, _i32]),
    "sepso_bf_run_async": (ctypes.c_int, [_vp, _i32]),
    "sepso_bf_step": (ctypes.c_int, [_vp, _i32]),
    "sepso_bf_sync": (ctypes.c_int, [_vp]),
    "sepso_bf_read": (ctypes.c_int, [_vp, _i32, _vp, _vp, _vp]),
    "sepso_bf_history": (ctypes.c_int, [_vp, _i32, _vp]),
    "sepso_bf_get_state": (ctypes.c_int, [_vp, _i32] + [_vp] * 9),
    "sepso_bf_set_state": (ctypes.c_int, [_vp, _i32] + [_vp] * 8 + [_i32]),
    "sepso_bf_evaluate": (ctypes.c_int, [_i32, _i32, _i32, _vp, _i32, _vp, _vp]),
    "sepso_bf_set_polygons": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32]),
    "sepso_bf_set_spheres": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32]),
    "sepso_bf_set_warm_start": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_uint32]),
    "sepso_sphere_evaluate": (ctypes.c_int, [_i32, _i32, _vp, _i32, _vp, _vp, _vp, _i32, ctypes.c_float,
                                             _i32, _vp, _vp, _vp]),
    "sepso_poly_evaluate": (ctypes.c_int, [_i32, _i32, _vp, _i32, _vp, _vp, _vp, _i32, ctypes.c_float,
                                           _i32, _vp, _vp, _vp]),
    "sepso_bf_launch_count": (ctypes.c_int64, [_vp]),
    "sepso_bf_kernel_name": (ctypes.c_char_p, [_vp]),
    "sepso_bf_last_error": (ctypes.c_char_p, []),
    "sepso_watchdog_selftest": (ctypes.c_int, [_i32, ctypes.POINTER(_i32), _vp]),
    "sepso_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "sepso_last_error": (ctypes.c_char_p, []),
}


def library_path() -> Path:
    return _build.LIB


def lib(rebuild_if_stale: bool = True):
    """Load libsepso.so (building it first if its sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build() if rebuild_if_stale else _build.LIB
        if not Path(path).exists():
            raise RuntimeError(f"libsepso.so not found at {path}; run __graft_entry__.build()")
        L = ctypes.CDLL(os.fspath(path))
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code: int):
    if code != SEPSO_OK:
        msg = lib().sepso_last_error()
        raise SepsoError(code, msg.decode() if msg else "")
    return code


def check_server(code: int):
    if code != SEPSO_OK:
        msg = lib().sepso_server_last_error()
        raise SepsoError(code, msg.decode() if msg else "")
    return code


def check_prior(code: int):
    if code != SEPSO_OK:
        msg = lib().sepso_prior_last_error()
        raise SepsoError(code, msg.decode() if msg else "")
    return code


def check_bf(code: int):
    if code != SEPSO_OK:
        msg = lib().sepso_bf_last_error()
        raise SepsoError(code, msg.decode() if msg else "")
    return code


def check_batch(code: int):
    if code != SEPSO_OK:
        msg = lib().sepso_batch_last_error()
        raise SepsoError(code, msg.decode() if msg else "")
    return code


def fptr(a):
    """float* from a numpy float32 array (None -> NULL)."""
    if a is None:
        return None
    return a.ctypes.data_as(_fp)
