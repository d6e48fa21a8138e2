"""Writes ``dynamic_hsef_hyper.json``: the per-group (w, C1, C2) that the oracle's
HSEF evolution phase (Sec. 3.2.1, Eq. fit_h) finds on the dynamic workload's first
scene (400 x 400, T = 20, G = 8 x N = 170, 64 circles, alpha 30, beta 4).

Settings of the evolution phase: 8 H-groups x 4 H-particles with the Table hyper8
rows, H-positions in [0.4, 0.9] x [1, 2.5]^2 per group, L-runs of the 300-iteration
cap with V_limit 0.05, no PI and no AT, H-seed 1000, 20 evolutions.  Both arms of
the benchmark (the GPU planner and the FP64 oracle timed on the host cores) plan
the application phase with this one set, so that their path costs compare.  The
values come from the oracle alone (FP64, about 2 minutes per evolution on one core).

    python tests/golden/make_dynamic_hsef_hyper.py [evolutions]
"""
import json
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parents[2]
sys.path.insert(0, str(ROOT))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2308_10169_gb300.inputs import HSEF_BOX_HI, HSEF_BOX_LO, TABLE_HYPER8, dynamic_workload  # noqa: E402

OUT = Path(__file__).resolve().parent / "dynamic_hsef_hyper.json"


def main(E: int = 20):
    cfg, scene, _ = dynamic_workload(0)
    lcfg = cfg.with_(at_mode=0, use_pi=False)
    sc = oracle.Scene(scene.start, scene.target, scene.circles)
    t0 = time.time()
    best, lfv, hist = oracle.hsef(lcfg, sc, 8, 4, E, TABLE_HYPER8, HSEF_BOX_LO, HSEF_BOX_HI, 0.05, 1000)
    G = cfg.G
    w, c1, c2 = best[:G], best[G:2 * G], best[2 * G:]
    hyper = np.zeros((G, 6))
    hyper[:, 0], hyper[:, 1], hyper[:, 2] = c1, c2, 0.0
    hyper[:, 3], hyper[:, 4], hyper[:, 5] = w, w, 0.05
    OUT.write_text(json.dumps({
        "source": "oracle.hsef on dynamic_workload(0): 8 H-groups x 4 H-particles, Table hyper8, "
                  "box [0.4,0.9] x [1,2.5]^2, L-runs of 300 iterations (V_limit 0.05, no PI, no AT), "
                  f"H-seed 1000, {E} evolutions",
        "layout": "per group: C1, C2, C3, w_init, w_end, V_limit (w_init = w_end = the evolved w)",
        "hyper": [[float(x) for x in row] for row in hyper],
        "lfv_best": float(lfv),
        "lfv_per_evolution": [float(x) for x in hist],
        "seconds": round(time.time() - t0, 1),
    }, indent=1) + "\n")
    print(OUT, lfv)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 20)
