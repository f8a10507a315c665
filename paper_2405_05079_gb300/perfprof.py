"""Cost-threshold performance profiles of solver variants (Sec. 5, Eq. pp;
Dolan and More's performance profiles).

For a problem p, every solver starts from the same initial cost f0(p); f*(p)
is the smallest cost any solver of the family reached. For a tolerance tau
the threshold is

    f_tau(p) = f*(p) + tau (f0(p) - f*(p)),

T_tau(p, s) is the first time solver s reaches f_tau(p) (infinite if it never
does), and the profile of s at relative runtime alpha is the percentage of
problems that s solves within alpha times the fastest solver on them:

    rho(s, alpha) = 100 / |P| * |{p : T_tau(p, s) <= alpha * min_s' T_tau(p, s')}|.

`threshold`, `time_to`, `best_costs`, `rho` and `profiles` are these
definitions (host code, no GPU). `time_to_targets` measures T_tau with the
GPU solver over a family of seeded synthetic problems; `main` prints the
profiles of the solver variants for each eta.

    python -m paper_2405_05079_gb300.perfprof --problems 24 --eta 0.1 0.2 0.3 0.4
"""
from __future__ import annotations

import dataclasses
import json
import math

import numpy as np

TAUS = (0.01, 0.003, 0.001)
ALPHAS = (1.0, 1.25, 1.5, 2.0, 3.0, 5.0, 10.0)


@dataclasses.dataclass
class Trace:
    """One solver on one problem: the common initial cost and, after every LM
    step, the cumulative solver time (s) and the cost."""
    f0: float
    times: np.ndarray
    costs: np.ndarray


def threshold(f0: float, fstar: float, tau: float) -> float:
    """Eq. pp: f_tau = f* + tau (f0 - f*)."""
    return fstar + tau * (f0 - fstar)


def time_to(trace: Trace, f: float) -> float:
    """First time at which the trace's cost is <= f (0 if the initial cost
    already is; inf if never)."""
    if trace.f0 <= f:
        return 0.0
    hit = np.nonzero(np.asarray(trace.costs) <= f)[0]
    return float(trace.times[hit[0]]) if hit.size else math.inf


def best_costs(traces: dict) -> dict:
    """f*(p): the smallest cost reached on p by any solver."""
    fstar = {}
    for (_, p), tr in traces.items():
        c = min([tr.f0] + list(tr.costs))
        fstar[p] = min(fstar.get(p, math.inf), c)
    return fstar


def rho(T: dict, alphas=ALPHAS) -> dict:
    """rho(s, alpha) for times T[(solver, problem)] = T_tau(p, s): for each
    solver, the percentage of problems with T_tau(p, s) <= alpha times the
    fastest solver's time on p, at every alpha. A problem that no solver
    reaches counts for none of them."""
    solvers = sorted({s for s, _ in T})
    problems = sorted({p for _, p in T})
    best = {p: min(T[s, p] for s in solvers) for p in problems}
    out = {}
    for s in solvers:
        out[s] = [100.0 * sum(1 for p in problems
                              if math.isfinite(T[s, p]) and T[s, p] <= a * best[p])
                  / len(problems) for a in alphas]
    return out


def profiles(traces: dict, taus=TAUS, alphas=ALPHAS) -> dict:
    """{tau: rho} from cost traces keyed by (solver, problem). All solvers
    must start from the same f0 on a problem (a meaningful comparison needs a
    common initial objective, Sec. 5)."""
    solvers = sorted({s for s, _ in traces})
    problems = sorted({p for _, p in traces})
    for p in problems:
        f0s = [traces[s, p].f0 for s in solvers]
        if max(f0s) - min(f0s) > 1e-12 * max(abs(x) for x in f0s):
            raise ValueError(f"solvers start from different costs on problem {p}")
    fstar = best_costs(traces)
    out = {}
    for tau in taus:
        T = {(s, p): time_to(traces[s, p], threshold(traces[s, p].f0, fstar[p], tau))
             for s in solvers for p in problems}
        out[tau] = rho(T, alphas)
    return out


# ------------------------------------------------------------------ GPU runs

def default_solvers(povar):
    """Solver variants of the family: (name, precision, series terms m (or a
    function of the scene giving m), camera parametrization[, extra
    parameters]). Besides PoVar's variants, the two first-stage competitors
    of Sec. 5.2 on the same kernels: PoBA (joint LM, landmark damping equal
    to the camera damping, the same series settings) and the "iterative"
    VarPro baseline (Schur-Jacobi PCG, at most 500 inner iterations, relative
    residual tolerance 0.01)."""
    return [("mixed m=21", povar.MIXED_FP32, 21, povar.EUCLID),
            ("fp64 m=21", povar.FP64, 21, povar.EUCLID),
            ("mixed m=11", povar.MIXED_FP32, 11, povar.EUCLID),
            ("mixed m=6", povar.MIXED_FP32, 6, povar.EUCLID),
            ("mixed m=21 sphere", povar.MIXED_FP32, 21, povar.SPHERE),
            ("poba mixed m=21", povar.MIXED_FP32, 21, povar.EUCLID, {"lambda_l": 1.0}),
            ("iterative mixed pcg500", povar.MIXED_FP32, 500, povar.EUCLID,
             {"solver": povar.SOLVER_PCG})]


def time_to_targets(problems, solvers, eta: float, taus=TAUS, max_iters: int = 50,
                    seed: int = 0):
    """T_tau(p, s) for every tolerance, solver and problem, measured with the
    GPU solver (povar_solve: one graph launch per LM step for the series
    solvers; the PCG solver issues its kernels eagerly, reading a device
    flag every 8 inner iterations).

    Every solver starts problem k from the same cameras (seeded N(0,1)
    entries scaled to unit norm, Sec. 5.2; landmarks from Eq. 8), with
    lambda0 = 1e-4 and series threshold 0.01. First each solver runs
    max_iters iterations (no stopping rule); f*(p) is the smallest final cost.
    Then, for every tau, each solver runs again from the start and stops at
    the first iteration whose cost is <= f_tau(p); T_tau is the device time of
    that solve (CUDA events), inf if it does not get there within max_iters.
    Before the timed solves, one untimed iteration per solver takes the
    one-off schedule autotuning and step-graph capture out of the times.

    Returns (T, f0, fstar): T[tau][(solver, k)] in seconds, f0[k], fstar[k].
    """
    from . import povar, scenes
    T = {tau: {} for tau in taus}
    f0, fstar = {}, {}
    for k, sc in enumerate(problems):
        P0 = scenes.init_cameras(sc.n_cams, seed + k, normalize=True)
        with povar.Problem.from_scene(sc) as pb:
            # m is a number of terms, or a function of the scene (a tuned policy)
            prms = {name: povar.make_params(**{"eta": eta, "lambda0": 1e-4,
                                               "m": int(m(sc) if callable(m) else m),
                                               "series_eps": 0.01, "manifold": man,
                                               "precision": prec, **(extra[0] if extra else {})})
                    for name, prec, m, man, *extra in solvers}
            final = {}
            for name in prms:
                pb.set_cameras(P0, eta)
                f0.setdefault(k, pb.cost(eta))
                pb.solve(prms[name], max_iters=max_iters, ftol=0.0, allow_stall=True)
                final[name] = pb.cost(eta)
            fstar[k] = min([f0[k]] + list(final.values()))
            for tau in taus:
                target = threshold(f0[k], fstar[k], tau)
                for name in prms:
                    pb.set_cameras(P0, eta)
                    pb.solve(prms[name], max_iters=1, ftol=0.0, allow_stall=True)
                    pb.set_cameras(P0, eta)
                    rep, _ = pb.solve(prms[name], max_iters=max_iters, ftol=0.0,
                                      target_cost=target, allow_stall=True)
                    reached = pb.cost(eta) <= target
                    T[tau][name, k] = rep.ms * 1e-3 if reached else math.inf
    return T, f0, fstar


def main(argv=None):
    import argparse
    from . import povar, scenes
    ap = argparse.ArgumentParser(description="cost-threshold performance profiles (GPU)")
    ap.add_argument("--problems", type=int, default=24)
    ap.add_argument("--family", default="serving", choices=("serving", "batched"))
    ap.add_argument("--eta", type=float, nargs="+", default=[0.1, 0.2, 0.3, 0.4])
    ap.add_argument("--max-iters", type=int, default=50)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args(argv)
    fam = scenes.family_scenes(args.family, args.problems, args.seed)
    solvers = default_solvers(povar)
    for eta in args.eta:
        T, f0, fstar = time_to_targets(fam, solvers, eta, TAUS, args.max_iters, args.seed)
        print(json.dumps({
            "family": args.family, "problems": len(fam), "eta": eta, "alphas": list(ALPHAS),
            "profiles": {str(tau): rho(T[tau]) for tau in TAUS},
            "median_ms": {str(tau): {s: float(np.median([1e3 * T[tau][s, k]
                                                         for k in range(len(fam))]))
                                     for s, *_ in solvers} for tau in TAUS},
            "reached": {str(tau): {s: sum(math.isfinite(T[tau][s, k]) for k in range(len(fam)))
                                   for s, *_ in solvers} for tau in TAUS}}), flush=True)


if __name__ == "__main__":
    main()
