"""Series-length autotuner: the number of series terms m per problem size.

The series (Sec. 4.2) trades the cost of an iteration (m - 1 products)
against its accuracy (the truncation of the Neumann sum), and which side
wins depends on the problem and on the accuracy asked for. The tuner
measures it: on a seeded family of problems of the workload's shape it runs
the GPU solver with every candidate m from the same start and takes the time
to the cost threshold f_tau (Eq. pp) of each; per size class of the
problems (observation count) it keeps the m whose performance profile over
the class is best, i.e. the largest mean of rho(m, alpha) over the profile's
alphas (the area under the profile: fastest to the threshold on most
problems, and reaching it at all on the rest). Ties keep the larger m. The
result is a JSON table; `m_for` looks a problem up in it; the serving loop
applies it per request and a batch per problem (povar_batch_solve_each).

    python -m paper_2405_05079_gb300.autotune --family serving --problems 24 \\
        --eta 0.1 --tau 0.001 --out m_table.json
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import perfprof

CANDIDATES = (6, 11, 16, 21)
# upper edges (observations) of the size classes; the last class is open
BIN_EDGES = (20_000, 100_000, 500_000)


def size_class(n_obs: int, edges=BIN_EDGES) -> int:
    """Index of the size class of a problem with n_obs observations."""
    for k, e in enumerate(edges):
        if n_obs <= e:
            return k
    return len(edges)


def profile_score(T: dict) -> dict:
    """Mean of rho(s, alpha) over the profile's alphas for each solver, from
    T[(solver, problem)] = T_tau(p, s)."""
    return {s: float(np.mean(row)) for s, row in perfprof.rho(T).items()}


def choose_m(T: dict) -> int:
    """The candidate m (solvers keyed by their m) with the best profile score
    over the problems of T; ties keep the larger m."""
    score = profile_score(T)
    return max(score, key=lambda m: (round(score[m], 9), m))


def build_table(T: dict, n_obs: dict, tau: float, eta: float, precision: str,
                candidates=CANDIDATES, edges=BIN_EDGES) -> dict:
    """Table from measured times T[(m, k)] and problem sizes n_obs[k]: one
    row per size class that has problems (classes without any take the
    neighbouring row's m at lookup)."""
    rows = []
    for c in range(len(edges) + 1):
        ks = [k for k in n_obs if size_class(n_obs[k], edges) == c]
        if not ks:
            continue
        Tc = {(m, k): T[m, k] for m in candidates for k in ks}
        rows.append({"class": c, "max_obs": edges[c] if c < len(edges) else None,
                     "problems": len(ks), "m": int(choose_m(Tc)),
                     "score": {str(m): v for m, v in profile_score(Tc).items()},
                     "reached": {str(m): int(sum(math.isfinite(Tc[m, k]) for k in ks))
                                 for m in candidates}})
    return {"tau": tau, "eta": eta, "precision": precision, "candidates": list(candidates),
            "edges": list(edges), "rows": rows}


def m_for(table: dict, n_obs: int) -> int:
    """m of the table row for the size class of n_obs (the nearest class
    with a row when that class had no tuning problems)."""
    c = size_class(n_obs, table["edges"])
    rows = table["rows"]
    if not rows:
        raise ValueError("empty m table")
    best = min(rows, key=lambda r: (abs(r["class"] - c), -r["class"]))
    return int(best["m"])


def params_with_m(table: dict, params, n_obs: int):
    """A copy of params whose series length is the table's m for n_obs."""
    from . import povar
    q = povar.Params.from_buffer_copy(params)
    q.m = m_for(table, n_obs)
    return q


def tune(problems, eta: float, tau: float = 0.001, candidates=CANDIDATES,
         precision: str = "mixed", max_iters: int = 50, seed: int = 0) -> dict:
    """Measure T_tau for every candidate m on every problem (GPU) and build
    the table."""
    from . import povar
    prec = {"mixed": povar.MIXED_FP32, "fp64": povar.FP64}[precision]
    solvers = [(m, prec, m, povar.EUCLID) for m in candidates]
    T, _, _ = perfprof.time_to_targets(problems, solvers, eta, (tau,), max_iters, seed)
    n_obs = {k: sc.n_obs for k, sc in enumerate(problems)}
    return build_table(T[tau], n_obs, tau, eta, precision, candidates)


def evaluate(table: dict, problems, eta: float, tau: float, fixed_m: int = 21,
             max_iters: int = 50, seed: int = 0) -> dict:
    """Performance profiles (Eq. pp) of the tuned policy against a fixed m on
    a family of problems (GPU): rho at every alpha, problems reached, median
    time to the threshold."""
    from . import povar
    prec = {"mixed": povar.MIXED_FP32, "fp64": povar.FP64}[table["precision"]]
    solvers = [(f"m={fixed_m}", prec, fixed_m, povar.EUCLID),
               ("tuned", prec, lambda sc: m_for(table, sc.n_obs), povar.EUCLID)]
    T, _, _ = perfprof.time_to_targets(problems, solvers, eta, (tau,), max_iters, seed)
    Tt = T[tau]
    names = [s[0] for s in solvers]
    n = len(problems)
    return {"tau": tau, "eta": eta, "problems": n, "alphas": list(perfprof.ALPHAS),
            "rho": perfprof.rho(Tt),
            "reached": {s: int(sum(math.isfinite(Tt[s, k]) for k in range(n))) for s in names},
            "median_ms": {s: float(np.median([1e3 * Tt[s, k] for k in range(n)]))
                          for s in names},
            "total_ms_both_reached": {
                s: float(sum(1e3 * Tt[s, k] for k in range(n)
                             if all(math.isfinite(Tt[q, k]) for q in names))) for s in names}}


def main(argv=None):
    import argparse
    from . import scenes
    ap = argparse.ArgumentParser(description="series-length autotuner (GPU)")
    ap.add_argument("--family", default="serving", choices=("serving", "batched"))
    ap.add_argument("--problems", type=int, default=24)
    ap.add_argument("--eta", type=float, default=0.1)
    ap.add_argument("--tau", type=float, default=0.001)
    ap.add_argument("--precision", default="mixed", choices=("mixed", "fp64"))
    ap.add_argument("--max-iters", type=int, default=50)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=None)
    ap.add_argument("--evaluate-seed", type=int, default=None,
                    help="after tuning, profile the table against m = 21 on the family of "
                         "this seed (problems not used for tuning)")
    args = ap.parse_args(argv)
    fam = scenes.family_scenes(args.family, args.problems, args.seed)
    table = tune(fam, args.eta, args.tau, CANDIDATES, args.precision, args.max_iters, args.seed)
    table.update({"family": args.family, "family_seed": args.seed, "problems": len(fam)})
    text = json.dumps(table, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    print(text)
    if args.evaluate_seed is not None:
        held = scenes.family_scenes(args.family, args.problems, args.evaluate_seed)
        ev = evaluate(table, held, args.eta, args.tau, 21, args.max_iters, args.evaluate_seed)
        print(json.dumps({"evaluation_family_seed": args.evaluate_seed, **ev}))


if __name__ == "__main__":
    main()
