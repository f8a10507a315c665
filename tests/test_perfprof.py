"""Performance-profile arithmetic (Sec. 5, Eq. pp and the profile rho) on
hand-built cost traces whose thresholds, times to threshold and profiles are
worked out by hand below, plus invariants of the definitions."""
import math

import numpy as np
import pytest

from paper_2405_05079_gb300 import perfprof as pp


def tr(f0, times, costs):
    return pp.Trace(f0, np.array(times, float), np.array(costs, float))


# Problem 0 (f0 = 100): A reaches 50, 20, 10 at t = 1, 2, 3; B reaches 80, 40,
# 12, 11 at t = 0.5, 1, 1.5, 2. f* = 10 (A's last cost).
# Problem 1 (f0 = 10): A reaches 6, 4 at t = 1, 2; B reaches 5, 2 at t = 1, 4.
# f* = 2 (B's last cost).
TRACES = {
    ("A", 0): tr(100.0, [1, 2, 3], [50, 20, 10]),
    ("B", 0): tr(100.0, [0.5, 1.0, 1.5, 2.0], [80, 40, 12, 11]),
    ("A", 1): tr(10.0, [1, 2], [6, 4]),
    ("B", 1): tr(10.0, [1, 4], [5, 2]),
}


def test_threshold_by_hand():
    assert pp.threshold(100.0, 10.0, 0.01) == pytest.approx(10.9)
    assert pp.threshold(100.0, 10.0, 0.1) == pytest.approx(19.0)
    assert pp.threshold(10.0, 2.0, 0.5) == pytest.approx(6.0)
    assert pp.threshold(7.0, 3.0, 0.0) == 3.0     # tau = 0: the best cost itself
    assert pp.threshold(7.0, 3.0, 1.0) == 7.0     # tau = 1: the initial cost


def test_best_costs_by_hand():
    assert pp.best_costs(TRACES) == {0: 10.0, 1: 2.0}


def test_time_to_by_hand():
    # problem 0, tau = 0.1 -> f = 19: A at t = 3 (20 > 19 at t = 2), B at t = 1.5
    assert pp.time_to(TRACES["A", 0], 19.0) == 3.0
    assert pp.time_to(TRACES["B", 0], 19.0) == 1.5
    # tau = 0.01 -> f = 10.9: B's best is 11, it never gets there
    assert pp.time_to(TRACES["B", 0], 10.9) == math.inf
    # the threshold is inclusive (6 <= 6 at t = 1) and the initial cost counts
    assert pp.time_to(TRACES["A", 1], 6.0) == 1.0
    assert pp.time_to(TRACES["A", 1], 10.0) == 0.0


def test_profiles_by_hand():
    prof = pp.profiles(TRACES, taus=(0.01, 0.1, 0.5), alphas=(1.0, 2.0, 3.0))
    # tau = 0.01: p0 only A (t = 3), p1 only B (t = 4): each solver wins one
    assert prof[0.01] == {"A": [50.0, 50.0, 50.0], "B": [50.0, 50.0, 50.0]}
    # tau = 0.1: p0 A = 3, B = 1.5 (A at ratio 2); p1 A never (4 > 2.8), B = 4
    assert prof[0.1] == {"A": [0.0, 50.0, 50.0], "B": [100.0, 100.0, 100.0]}
    # tau = 0.5: p0 f = 55, A and B both at t = 1; p1 f = 6, both at t = 1
    assert prof[0.5] == {"A": [100.0, 100.0, 100.0], "B": [100.0, 100.0, 100.0]}


def test_rho_unreached_problem_counts_for_nobody():
    T = {("A", 0): 1.0, ("B", 0): 2.0, ("A", 1): math.inf, ("B", 1): math.inf}
    assert pp.rho(T, alphas=(1.0, 2.0)) == {"A": [50.0, 50.0], "B": [0.0, 50.0]}


def test_different_initial_costs_rejected():
    bad = dict(TRACES)
    bad["B", 1] = tr(11.0, [1], [2])
    with pytest.raises(ValueError):
        pp.profiles(bad)


def random_traces(rng, n_solvers=4, n_problems=9):
    out = {}
    for p in range(n_problems):
        f0 = float(rng.uniform(10, 1000))
        for s in range(n_solvers):
            n = int(rng.integers(1, 12))
            times = np.cumsum(rng.uniform(0.01, 1.0, n))
            # costs decrease with occasional rejected steps (cost unchanged)
            costs = f0 * np.cumprod(np.where(rng.random(n) < 0.2, 1.0, rng.uniform(0.2, 0.95, n)))
            out[f"s{s}", p] = pp.Trace(f0, times, costs)
    return out


@pytest.mark.parametrize("seed", range(5))
def test_profile_invariants(seed):
    rng = np.random.default_rng(seed)
    traces = random_traces(rng)
    alphas = (1.0, 1.5, 2.0, 4.0, 1e300)
    prof = pp.profiles(traces, taus=(0.0, 0.003, 0.1), alphas=alphas)
    solvers = sorted({s for s, _ in traces})
    problems = sorted({p for _, p in traces})
    for tau, rows in prof.items():
        for s in solvers:
            # non-decreasing in alpha, within [0, 100]
            assert all(0.0 <= a <= b <= 100.0 for a, b in zip(rows[s], rows[s][1:]))
        # f* is reached by construction: every problem has a winner at alpha = 1
        assert sum(rows[s][0] for s in solvers) >= 100.0 - 1e-9
        # alpha -> inf: the share of problems the solver reaches at all
        for s in solvers:
            fstar = pp.best_costs(traces)
            reached = sum(
                min(traces[s, p].costs.min(), traces[s, p].f0)
                <= pp.threshold(traces[s, p].f0, fstar[p], tau) for p in problems)
            assert rows[s][-1] == pytest.approx(100.0 * reached / len(problems))
    # scaling all times of one problem leaves the profiles unchanged
    scaled = {k: (pp.Trace(v.f0, v.times * 7.5, v.costs) if k[1] == problems[0] else v)
              for k, v in traces.items()}
    assert pp.profiles(scaled, taus=(0.0, 0.003, 0.1), alphas=alphas) == prof
