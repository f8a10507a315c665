"""Writes tests/golden/converged_<scene>.json from the FP64 CPU oracle only.

Each file holds the oracle's damped-VarPro trajectory of one seeded scene
(scene seed 0, camera-initialization seed 1, cameras iid N(0,1) scaled to
unit norm, unconstrained first-stage cameras as in Sec. 3.2 / 4.2 of the
paper) with the paper's solver settings of Sec. 5.2 (eta of the scene,
lambda0 = 1e-4, series order 20 -> m = 21 terms, series threshold 0.01),
run until a relative decrease below ftol or the iteration cap: the cost of
every iteration ("trace") and the final cost. The large scene is capped at
the paper's 50 iterations per stage (Sec. 5.2) and uses the matrix-free
oracle step (its dense S does not fit); small scenes also record the exact
(dense Cholesky) mode from the same start. No value here comes from the
CUDA path.

"mid_m<k>" runs the mid scene with the series at m = k terms for the paper's
50 iterations (no decrease rule), for the comparison of series lengths.

Every series run also stores its final cameras "P" and the damping state
("lambda", "nu"), so that a later run can resume the oracle exactly.
"large_more" resumes the large scene from the state stored in
converged_large.json and continues until the paper's stop rule (Sec. 5.2:
an accepted step with relative decrease below 1e-6) or 400 more iterations,
so that the cost after the 50-iteration budget can be compared with the
cost at the stop rule.

"midnear_m<k>" is the end-state reference of the mid scene: from the mid
scene's standard start the exact (dense Cholesky) damped solve converges to
a local minimum (relative decrease below 1e-12); every camera entry of that
minimum is perturbed by 1e-3 times the mean absolute entry (seeded normal
noise), and from there the series solve with m = k terms runs until its
relative decrease is below 1e-12 (at most 400 iterations). The file stores
the perturbed start, the final cost and cameras.

    python tests/golden/make_golden.py [tiny] [mid] [large] [mid_m5] [mid_m10] [mid_m20]
                                       [large_more] [midnear_m5] [midnear_m10] [midnear_m20]
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

SETTINGS = {"m": 21, "series_eps": 0.01, "lambda0": 1e-4, "manifold": "euclid"}
FTOL = {"tiny": 1e-12, "mid": 1e-10, "large": 1e-9}
MAX_ITERS = {"tiny": 300, "mid": 3000, "large": 50}


def run(name):
    scene, m, ftol, max_iters = name, SETTINGS["m"], FTOL.get(name), MAX_ITERS.get(name)
    if name.startswith("mid_m"):
        scene, m, ftol, max_iters = "mid", int(name[len("mid_m"):]), 0.0, 50
    sc = scenes.scene_by_name(scene, 0)
    P0 = scenes.init_cameras(sc.n_cams, 1, normalize=True)
    cls = O.MatrixFreeProblem if scene == "large" else O.Problem
    pr = cls(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    out = {"scene": scene, "scene_seed": 0, "init_seed": 1, "eta": sc.eta,
           "ftol": ftol, **SETTINGS, "m": m,
           "source": "tests/golden/make_golden.py (oracle/povar_oracle.py only)"}
    solvers = ("series",) if scene == "large" or name != scene else ("series", "exact")
    for solver in solvers:
        prm = O.Params(eta=sc.eta, m=m, series_eps=SETTINGS["series_eps"],
                       manifold=O.EUCLID, solver=solver, lambda0=SETTINGS["lambda0"])
        t = time.time()
        trace = []

        def cb(st, rep):
            trace.append([rep.cost_after if rep.accepted else rep.cost_before,
                          round(time.time() - t, 2), int(rep.terms_used)])
            print(name, solver, len(trace), trace[-1], flush=True)
        st, reps = pr.solve(P0, prm, max_iters=max_iters, ftol=ftol, callback=cb)
        out[solver] = {"F": st.F, "iterations": len(reps), "F0": reps[0].cost_before,
                       "seconds": time.time() - t, "trace": trace}
        if solver == "series":
            out[solver]["P"] = st.P.tolist()
            out[solver]["lambda"] = st.lam
            out[solver]["nu"] = st.nu
        print(name, solver, len(reps), st.F, f"{time.time() - t:.1f}s", flush=True)
    with open(os.path.join(HERE, f"converged_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)


def run_more(max_more=400, ftol=1e-6):
    """Resume the large scene from its stored 50-iteration state."""
    with open(os.path.join(HERE, "converged_large.json")) as f:
        base = json.load(f)
    sc = scenes.scene_by_name("large", 0)
    pr = O.MatrixFreeProblem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    prm = O.Params(eta=sc.eta, m=base["m"], series_eps=base["series_eps"], manifold=O.EUCLID,
                   solver="series", lambda0=base["lambda0"])
    b = base["series"]
    P = np.asarray(b["P"], dtype=np.float64)
    X = pr.landmarks(P, sc.eta)
    st = O.State(P=P, X=X, F=pr.cost(P, X, sc.eta), lam=b["lambda"], nu=b["nu"],
                 iteration=b["iterations"])
    t = time.time()
    trace = []
    for _ in range(max_more):
        st, rep = pr.step(st, prm)
        trace.append([rep.cost_after if rep.accepted else rep.cost_before,
                      round(time.time() - t, 2), int(rep.terms_used)])
        print("large_more", st.iteration, trace[-1], flush=True)
        if rep.accepted and (rep.cost_before - rep.cost_after) < ftol * rep.cost_before:
            break
        if st.lam > O.LAMBDA_MAX:
            break
    out = {"scene": "large", "resumed_from": "converged_large.json", "start_iteration":
           b["iterations"], "F_start": b["F"], "ftol": ftol, "F": st.F,
           "iterations": st.iteration, "stopped_by_rule": len(trace) < max_more,
           "seconds": time.time() - t, "trace": trace, "lambda": st.lam, "nu": st.nu,
           "source": "tests/golden/make_golden.py (oracle/povar_oracle.py only)"}
    with open(os.path.join(HERE, "converged_large_more.json"), "w") as f:
        json.dump(out, f, indent=1)


def run_near(m):
    """End-state reference of the mid scene at m series terms (see above)."""
    sc = scenes.scene_by_name("mid", 0)
    P0 = scenes.init_cameras(sc.n_cams, 1, normalize=True)
    pr = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    ex = O.Params(eta=sc.eta, m=m, series_eps=SETTINGS["series_eps"], manifold=O.EUCLID,
                  solver="exact", lambda0=SETTINGS["lambda0"])
    st_ex, reps_ex = pr.solve(P0, ex, max_iters=200, ftol=1e-12)
    rng = np.random.default_rng(7)
    Pstart = st_ex.P + 1e-3 * np.abs(st_ex.P).mean() * rng.normal(size=st_ex.P.shape)
    prm = O.Params(eta=sc.eta, m=m, series_eps=SETTINGS["series_eps"], manifold=O.EUCLID,
                   solver="series", lambda0=SETTINGS["lambda0"])
    t = time.time()
    st, reps = pr.solve(Pstart, prm, max_iters=400, ftol=1e-12)
    out = {"scene": "mid", "scene_seed": 0, "init_seed": 1, "eta": sc.eta, "m": m,
           "series_eps": SETTINGS["series_eps"], "lambda0": SETTINGS["lambda0"],
           "manifold": "euclid", "ftol": 1e-12, "perturbation": 1e-3, "perturbation_seed": 7,
           "exact_minimum": {"F": st_ex.F, "iterations": len(reps_ex)},
           "P_start": Pstart.tolist(), "F_start": reps[0].cost_before,
           "series": {"F": st.F, "iterations": len(reps), "P": st.P.tolist(),
                      "stopped_by_rule": len(reps) < 400, "seconds": time.time() - t,
                      "trace": [r.cost_after if r.accepted else r.cost_before for r in reps]},
           "source": "tests/golden/make_golden.py (oracle/povar_oracle.py only)"}
    print(f"midnear_m{m}", st_ex.F, len(reps_ex), st.F, len(reps), flush=True)
    with open(os.path.join(HERE, f"converged_midnear_m{m}.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    for n in (sys.argv[1:] or ["tiny", "mid"]):
        if n == "large_more":
            run_more()
        elif n.startswith("midnear_m"):
            run_near(int(n[len("midnear_m"):]))
        else:
            run(n)
