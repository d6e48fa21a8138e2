"""The C-ABI library builds, loads and exports every entry point of include/sepso.h;
host-side argument checks reject bad configurations (no GPU needed)."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

from paper_2308_10169_gb300 import _native
from paper_2308_10169_gb300.inputs import SepsoConfig, dynamic_workload, static_workload
from paper_2308_10169_gb300.planner import state_layout

HEADER = Path(__file__).resolve().parents[1] / "include" / "sepso.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sepso_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _native.lib()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), f"{n} declared in sepso.h but not exported"
    assert set(names) == set(_native.SIGNATURES), "binding and header disagree"


def _ws(cfg):
    size = ctypes.c_size_t()
    c = _native.make_config(cfg)
    return _native.lib().sepso_workspace_size(ctypes.byref(c), ctypes.byref(size)), size.value


@pytest.mark.parametrize("bad", [dict(T=0), dict(T=65), dict(G=0), dict(G=33), dict(N=0),
                                 dict(beta=0), dict(max_iters=0), dict(at_mode=3), dict(tw=0),
                                 dict(runs=0), dict(threads=48), dict(pi_gamma=1.5),
                                 dict(map_w=-1.0), dict(max_obstacles=-1)])
def test_bad_configs_rejected(bad):
    rc, _ = _ws(SepsoConfig(**bad))
    assert rc == -1  # SEPSO_EINVAL
    assert _native.lib().sepso_last_error()


def test_workspace_size_grows_with_runs_and_obstacles():
    cfg, _, _ = dynamic_workload(0)
    rc, base = _ws(cfg)
    assert rc == 0 and base > 0 and base % 256 == 0
    assert _ws(cfg.with_(runs=4))[1] > base
    assert _ws(cfg.with_(max_obstacles=1024))[1] > base


def test_state_layout_matches_header_description():
    cfg, _, _ = static_workload(0)
    lay = state_layout(cfg)
    M, D = cfg.G * cfg.N, cfg.D
    assert lay["X"][0] == 0 and lay["V"][0] == 4 * M * D and lay["P"][0] == 8 * M * D
    assert lay["win"][0] % 8 == 0
    assert lay["_total"] == lay["prev_lfv"][0] + 4


def test_strerror_names_codes():
    lib = _native.lib()
    assert lib.sepso_strerror(0) == b"ok"
    assert lib.sepso_strerror(-5) == b"device-side wait timed out"


# ---------------------------------------------------------------------------
# Host-side argument checks of the batch, server and prior entry points (no GPU:
# the checks run before any CUDA call).
# ---------------------------------------------------------------------------

def _batch_size(**kw):
    base = dict(T=8, G=4, N=32, O=16, max_iters=10, alpha=30.0, beta=4, seed=1, run_id=0)
    base.update(kw)
    arr = (_native.BatchScene * 2)(_native.BatchScene(**base), _native.BatchScene(**base))
    size = ctypes.c_size_t()
    return _native.lib().sepso_batch_workspace_size(arr, 2, ctypes.byref(size)), size.value


def test_batch_workspace_size_and_bad_scenes():
    rc, size = _batch_size()
    assert rc == 0 and size > 0 and size % 256 == 0
    assert _batch_size(O=1000)[1] > size and _batch_size(N=64)[1] > size
    for bad in (dict(T=0), dict(T=65), dict(G=33), dict(N=0), dict(O=-1), dict(max_iters=0), dict(beta=9),
                dict(alpha=-1.0), dict(stall_iters=-1), dict(stall_tol=-0.5), dict(n_pi=33), dict(n_prior=-1),
                dict(pi_halfwidth=-1.0)):
        assert _batch_size(**bad)[0] == -1, bad
    assert _native.lib().sepso_batch_last_error()
    size = ctypes.c_size_t()
    assert _native.lib().sepso_batch_workspace_size(None, 0, ctypes.byref(size)) == -1


def _server_size(**kw):
    base = dict(n_agents=16, max_slots=8, mem_budget=0, G=4, N=32, Tmax=20, Omax=64, max_iters=50, stall_iters=10,
                stall_tol=0.0, alpha=30.0, beta=4, pi_gamma=0.25, pi_halfwidth=20.0, map_w=400.0, map_h=400.0,
                seed=0, tile=0, threads=0)
    base.update(kw)
    c = _native.ServerConfig(**base)
    size, slots = ctypes.c_size_t(), ctypes.c_int32()
    rc = _native.lib().sepso_server_workspace_size(ctypes.byref(c), ctypes.byref(size), ctypes.byref(slots))
    return rc, size.value, slots.value


def test_server_slots_follow_the_memory_budget():
    rc, size, slots = _server_size()
    assert rc == 0 and slots == 8 and size > 0
    rc2, size2, slots2 = _server_size(max_slots=64, mem_budget=size)
    assert rc2 == 0 and 1 <= slots2 <= 8 and size2 <= size
    for bad in (dict(n_agents=0), dict(max_slots=0), dict(G=0), dict(N=0), dict(Tmax=0), dict(Tmax=65),
                dict(Omax=-1), dict(max_iters=0), dict(beta=0), dict(pi_gamma=1.5), dict(map_w=0.0)):
        assert _server_size(**bad)[0] == -1, bad
    assert _native.lib().sepso_server_last_error()


def _prior_size(**kw):
    base = dict(T=20, grid=64, hidden1=1024, hidden2=512, max_batch=256, capacity=1000, max_circles=64,
                map_w=400.0, map_h=400.0, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8)
    base.update(kw)
    c = _native.PriorConfig(**base)
    size = ctypes.c_size_t()
    return _native.lib().sepso_prior_workspace_size(ctypes.byref(c), ctypes.byref(size)), size.value


def test_prior_workspace_size_and_bad_configs():
    rc, size = _prior_size()
    # the dataset alone: 1000 rows x 4104 BF16 features
    assert rc == 0 and size > 1000 * 4104 * 2 and size % 256 == 0
    assert _prior_size(capacity=2000)[1] - size >= 1000 * 4104 * 2
    for bad in (dict(T=0), dict(T=65), dict(grid=4), dict(hidden1=100), dict(hidden2=0), dict(max_batch=12),
                dict(capacity=0), dict(max_circles=-1), dict(lr=0.0), dict(beta1=1.0), dict(eps=0.0)):
        assert _prior_size(**bad)[0] == -1, bad
    assert _native.lib().sepso_prior_last_error()


def test_gemm_rejects_bad_shapes_before_any_launch():
    L = _native.lib()
    # K not a multiple of 8, or NULL operands: rejected on the host
    assert L.sepso_gemm_bf16(None, None, 8, 8, 12, 16, 16, 1.0, None, 0, None, 0, None, 8, None, 8, 0, None) == -1
    assert L.sepso_gemm_bf16(None, None, 8, 8, 16, 16, 16, 1.0, None, 0, None, 0, None, 8, None, 8, 0, None) == -1
    assert L.sepso_prior_last_error()


def test_gemm_extra_workspace_and_argument_checks():
    L = _native.lib()
    size = ctypes.c_size_t()
    assert L.sepso_gemm_bf16_ex_workspace(100, 64, 4, 0, ctypes.byref(size)) == 0 and size.value == 4 * 100 * 64 * 4
    assert L.sepso_gemm_bf16_ex_workspace(100, 64, 1, 1, ctypes.byref(size)) == 0 and size.value == 4 * 64 * 4
    assert L.sepso_gemm_bf16_ex_workspace(100, 64, 0, 0, ctypes.byref(size)) == 0 and size.value == 0
    assert L.sepso_gemm_bf16_ex_workspace(0, 64, 1, 0, ctypes.byref(size)) == -1
    # aligned stand-in device addresses: every check below runs before any CUDA call
    A, B, C = ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20), ctypes.c_void_p(3 << 20)
    ws = ctypes.c_void_p(4 << 20)

    def ex(**kw):
        e = _native.GemmExtra(**kw)
        return L.sepso_gemm_bf16_ex(A, B, 100, 64, 32, 32, 32, 1.0, None, 0, None, 0, C, 64, None, 64,
                                    ctypes.byref(e), 0, None)

    assert ex(Ct=C, ldct=99) == -1                                    # transposed row stride below M
    assert ex(ksplit=2, colsum=C, workspace=ws, workspace_bytes=1 << 20) == -1  # split with colsum
    assert ex(ksplit=2, Ct=C, ldct=100, workspace=ws, workspace_bytes=1 << 20) == -1
    assert ex(ksplit=-1) == -1
    assert ex(ksplit=4, workspace=ws, workspace_bytes=4 * 100 * 64 * 4 - 1) == -3   # workspace too small
    assert ex(colsum=C, workspace=None, workspace_bytes=0) == -3
    assert ex(colsum=C, workspace=ctypes.c_void_p((4 << 20) + 8), workspace_bytes=1 << 20) == -3  # misaligned


def test_at_window_test_rejects_bad_arguments_before_any_launch():
    L = _native.lib()
    win = np.zeros((2, 20), np.float64)
    ns = np.array([5, 20], np.int32)
    heads = np.array([5, 0], np.int32)
    out = np.zeros(2, np.int32)

    def call(w=win, n=ns, h=heads, count=2, tw=20, delta=10.0):
        return L.sepso_at_window_test(w.ctypes.data, n.ctypes.data, h.ctypes.data, count, tw,
                                      ctypes.c_float(delta), out.ctypes.data, None)

    assert call(tw=0) == -1 and call(tw=65) == -1
    assert call(n=np.array([5, 21], np.int32)) == -1          # fill above tw
    assert call(n=np.array([0, 5], np.int32)) == -1           # empty window
    assert call(h=np.array([20, 0], np.int32)) == -1          # head outside the ring
    assert call(h=np.array([-1, 0], np.int32)) == -1
    assert call(count=-1) == -1
    assert L.sepso_at_window_test(None, None, None, 3, 20, ctypes.c_float(1.0), None, None) == -1
    assert call(count=0) == 0                                  # nothing to do, no device call


def test_bf_workspace_size_and_bad_configs():
    L = _native.lib()
    from paper_2308_10169_gb300.inputs import BFConfig

    def size(**kw):
        c = _native.bf_config_struct(BFConfig(**kw))
        out = ctypes.c_size_t()
        rc = L.sepso_bf_workspace_size(ctypes.byref(c), ctypes.byref(out))
        return rc, out.value

    rc, s1 = size(fn=1, D=30, G=8, N=10, runs=1)
    assert rc == 0
    rc, s2 = size(fn=1, D=30, G=8, N=10, runs=50)
    assert rc == 0 and s2 > 40 * s1
    rc, big = size(fn=3, D=1000, G=8, N=2048, runs=1)
    assert rc == 0 and big >= 16384 * 1000 * 16        # X, V and two Pbest buffers
    assert size(fn=5, D=16, G=8, N=170, max_edges=80)[0] == 0     # a path among polygons
    assert size(fn=6, D=48, G=8, N=170, max_spheres=64)[0] == 0   # a 3D path among spheres
    for bad in (dict(fn=5, D=15), dict(fn=5, beta=0), dict(fn=5, beta=9), dict(fn=5, max_edges=4097),
                dict(fn=5, map_w=0.0), dict(fn=5, alpha=-1.0), dict(fn=6, D=31), dict(fn=6, D=2),
                dict(fn=6, map_d=0.0), dict(fn=6, map_d=float("inf")), dict(fn=6, max_spheres=4097),
                dict(fn=6, beta=0), dict(fn=6, at_stall=-1), dict(fn=6, at_stall=5, stall_tol=-1.0),
                dict(fn=6, at_stall=5, stall_tol=float("nan")), dict(fn=1, at_stall=5), dict(fn=7), dict(fn=0), dict(D=0), dict(D=16385), dict(G=0), dict(G=33), dict(N=0),
                dict(runs=0), dict(max_iters=0), dict(lo=1.0, hi=1.0), dict(lo=float("nan")),
                dict(hi=float("inf")), dict(runs=600, G=8)):
        assert size(**bad)[0] == -1, bad
    # workspace checks come before any CUDA call
    c = _native.bf_config_struct(BFConfig(fn=1, D=30, G=8, N=10))
    h = ctypes.c_void_p()
    assert L.sepso_bf_create(ctypes.byref(c), ctypes.c_void_p(1 << 20), s1 - 1, None, ctypes.byref(h)) == -3
    assert L.sepso_bf_create(ctypes.byref(c), ctypes.c_void_p((1 << 20) + 16), s1, None, ctypes.byref(h)) == -3
    assert L.sepso_bf_create(ctypes.byref(c), None, s1, None, ctypes.byref(h)) == -3
    X = ctypes.c_void_p(1 << 20)
    assert L.sepso_bf_evaluate(0, 30, 4, X, 30, X, None) == -1
    assert L.sepso_bf_evaluate(1, 30, 4, X, 29, X, None) == -1     # pitch below D
    assert L.sepso_bf_evaluate(1, 30, 0, None, 30, None, None) == 0  # nothing to do
    assert L.sepso_bf_step(None, 1) == -1 and L.sepso_bf_run_async(None, 1) == -1
    st = np.zeros(2, np.float32)
    assert L.sepso_bf_set_polygons(None, st.ctypes.data, st.ctypes.data, None, 0) == -1
    P = st.ctypes.data
    assert L.sepso_poly_evaluate(0, 4, X, 16, P, P, X, 4, ctypes.c_float(30.0), 4, X, None, None) == -1
    assert L.sepso_poly_evaluate(8, 4, X, 15, P, P, X, 4, ctypes.c_float(30.0), 4, X, None, None) == -1
    assert L.sepso_poly_evaluate(8, 4, X, 16, P, P, X, 4, ctypes.c_float(30.0), 0, X, None, None) == -1
    assert L.sepso_poly_evaluate(8, 4, X, 16, P, P, ctypes.c_void_p((1 << 20) + 4), 4, ctypes.c_float(30.0),
                                 4, X, None, None) == -1                 # edges misaligned
    assert L.sepso_poly_evaluate(8, 0, None, 16, P, P, None, 0, ctypes.c_float(30.0), 4, None, None,
                                 None) == 0
    # the 3D objective's calls: argument checks before any CUDA call
    p3 = np.zeros(3, np.float32)
    P3 = p3.ctypes.data
    assert L.sepso_bf_set_spheres(None, P3, P3, None, 0) == -1
    assert L.sepso_bf_set_warm_start(None, None, ctypes.c_float(0.0), ctypes.c_float(0.0), 0) == -1
    assert L.sepso_sphere_evaluate(0, 4, X, 24, P3, P3, X, 4, ctypes.c_float(30.0), 4, X, None, None) == -1
    assert L.sepso_sphere_evaluate(8, 4, X, 23, P3, P3, X, 4, ctypes.c_float(30.0), 4, X, None, None) == -1
    assert L.sepso_sphere_evaluate(8, 4, X, 24, P3, P3, X, 4, ctypes.c_float(30.0), 9, X, None, None) == -1
    assert L.sepso_sphere_evaluate(8, 4, X, 24, P3, P3, X, -1, ctypes.c_float(30.0), 4, X, None, None) == -1
    assert L.sepso_sphere_evaluate(8, 4, X, 24, P3, P3, ctypes.c_void_p((1 << 20) + 8), 4, ctypes.c_float(30.0),
                                   4, X, None, None) == -1               # spheres misaligned
    assert L.sepso_sphere_evaluate(8, 4, X, 24, None, P3, X, 4, ctypes.c_float(30.0), 4, X, None, None) == -1
    assert L.sepso_sphere_evaluate(8, 0, None, 24, P3, P3, None, 0, ctypes.c_float(30.0), 4, None, None,
                                   None) == 0
