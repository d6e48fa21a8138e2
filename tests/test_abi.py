"""The C-ABI library builds, loads and exports every entry point of include/sepso.h;
host-side argument checks reject bad configurations (no GPU needed)."""
import ctypes
import re
from pathlib import Path

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
