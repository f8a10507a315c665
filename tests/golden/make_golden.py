"""Writes tests/golden/converged_<scene>.json from the FP64 CPU oracle only.

Each file holds the oracle's converged damped-VarPro solution of one seeded
scene (scene seed 0, camera-initialization seed 1, unit-norm cameras,
tangent-space steps) in PoVar series mode with the scene's series length, and
the converged cost of the exact (dense Cholesky) mode from the same start.
The GPU solves are compared against these values; no value here comes from
the CUDA path.

    python tests/golden/make_golden.py [tiny] [mid]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import povar_oracle as O  # noqa: E402
from paper_2405_05079_gb300 import scenes  # noqa: E402

MAX_ITERS = {"tiny": 3000, "mid": 1500}


def run(name):
    sc = scenes.scene_by_name(name, 0)
    P0 = scenes.init_cameras(sc.n_cams, 1, normalize=True)
    pr = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    out = {"scene": name, "scene_seed": 0, "init_seed": 1, "eta": sc.eta, "m": sc.m,
           "manifold": "sphere", "lambda0": 1e-4, "ftol": 1e-12,
           "source": "tests/golden/make_golden.py (oracle/povar_oracle.py only)"}
    for solver in ("series", "exact"):
        prm = O.Params(eta=sc.eta, m=sc.m, manifold=O.SPHERE, solver=solver, lambda0=1e-4)
        t = time.time()
        st, reps = pr.solve(P0, prm, max_iters=MAX_ITERS[name], ftol=1e-12)
        out[solver] = {"F": st.F, "iterations": len(reps), "F0": reps[0].cost_before,
                       "seconds": time.time() - t}
        if solver == "series":
            out[solver]["P"] = st.P.tolist()
        print(name, solver, len(reps), st.F, f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, f"converged_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["tiny", "mid"]):
        run(n)
