"""sepso_plan_static: planning for callers that cannot allocate device memory.

Such callers (code inside another framework's memory pool, plugins whose host
forbids allocations after start-up, real-time loops) get one entry point whose
workspace is a static device array inside the library.  These tests call it
through the C ABI and compare it with the regular handle-based sepso_plan on the
same inputs, for two calls in a row (the second must not see the first's state).

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2308_10169_gb300 import Planner, static_workload
from paper_2308_10169_gb300._native import Config, Result, fptr, make_config
from paper_2308_10169_gb300.inputs import dynamic_workload

pytestmark = pytest.mark.gpu


def _plan_static(lib, cfg, scene, hyper, stream=None):
    c = make_config(cfg)
    h = np.ascontiguousarray(hyper, dtype=np.float32)
    circ = np.ascontiguousarray(scene.circles, dtype=np.float32).reshape(-1, 3)
    wp = np.zeros(cfg.D, np.float32)
    res = Result()
    rc = lib.sepso_plan_static(ctypes.byref(c), fptr(h), fptr(scene.start), fptr(scene.target),
                               fptr(circ) if circ.size else None, circ.shape[0], fptr(wp),
                               ctypes.byref(res), stream)
    return rc, wp, res


@pytest.mark.parametrize("which", ["static", "dynamic", "no_obstacles", "side_stream"])
def test_static_scratch_plan_matches_handle_plan_twice(native, which):
    stream = None
    if which in ("static", "side_stream"):
        cfg, scene, hyper = static_workload(7)
    elif which == "no_obstacles":
        cfg, scene, hyper = static_workload(3)
        scene = type(scene)(scene.start, scene.target, np.zeros((0, 3), np.float32))
    else:
        cfg, scene, hyper = dynamic_workload(1)
        cfg = cfg.with_(max_iters=40)
    ref = Planner(cfg)
    ref.set_hyper(hyper)
    ref.set_scene(scene)
    r = ref.plan()
    side = None
    if which == "side_stream":
        side = torch.cuda.Stream()
        stream = ctypes.c_void_p(side.cuda_stream)
    free_before = None
    for call in range(2):
        if call == 1:
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
        rc, wp, res = _plan_static(native, cfg, scene, hyper, stream)
        assert rc == 0, native.sepso_last_error()
        assert res.status == 0
        assert res.iters == r["iters"]
        assert res.Q == r["Q"]
        assert res.cost == pytest.approx(r["cost"], rel=1e-4)
        assert res.length == pytest.approx(r["length"], rel=1e-5)
        np.testing.assert_allclose(wp, r["waypoints"], rtol=1e-5, atol=1e-5 * 400)
    # the second call took no device memory (the first may have loaded the module)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before


def test_static_scratch_rejects_negative_v_limit(native):
    cfg, scene, hyper = static_workload(0)
    bad = np.array(hyper, np.float32).reshape(-1, 6).copy()
    bad[2, 5] = -0.05  # group 2's V_limit, refused by sepso_set_hyper too
    rc, _, _ = _plan_static(native, cfg, scene, bad)
    assert rc == -1  # SEPSO_EINVAL
    assert b"V_limit" in native.sepso_last_error()


def test_static_scratch_rejects_oversized_config(native):
    cfg, scene, hyper = dynamic_workload(0)
    big = cfg.with_(N=4000)  # needs more than the 8 MiB static scratch
    rc, _, _ = _plan_static(native, big, scene, hyper)
    assert rc == -3  # SEPSO_ENOSPC
    assert b"static scratch" in native.sepso_last_error()
