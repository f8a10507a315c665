"""Times to the cost thresholds of Eq. pp measured with the GPU solver on a
small seeded family: the common initial cost is the oracle's, every threshold
is reached by some solver of the family (f* is attained by one of them, and
the solves are deterministic), and reaching a tight threshold implies
reaching the looser ones."""
import math

import numpy as np
import pytest

from oracle import povar_oracle as O
from paper_2405_05079_gb300 import perfprof as pp
from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu


def test_time_to_targets_on_small_family():
    fam = scenes.family_scenes("batched", 3, seed=3)
    solvers = [s for s in pp.default_solvers(povar) if s[0] in (
        "mixed m=21", "fp64 m=21", "mixed m=6", "poba mixed m=21", "iterative mixed pcg500")]
    assert len(solvers) == 5
    eta = 0.2
    T, f0, fstar = pp.time_to_targets(fam, solvers, eta, pp.TAUS, max_iters=20, seed=3)
    names = [s[0] for s in solvers]
    for k, sc in enumerate(fam):
        P0 = scenes.init_cameras(sc.n_cams, 3 + k, normalize=True)
        X = O.landmarks(P0, sc.cam_idx, sc.pt_idx, sc.meas, eta, sc.n_points)
        F0 = O.cost(P0, X, sc.cam_idx, sc.pt_idx, sc.meas, eta)
        assert abs(f0[k] - F0) <= 1e-10 * F0
        assert 0.0 < fstar[k] < f0[k]
        for tau in pp.TAUS:
            assert min(T[tau][s, k] for s in names) < math.inf, (k, tau)
        for s in names:
            reached = [math.isfinite(T[tau][s, k]) for tau in sorted(pp.TAUS)]
            # sorted taus: tightest first; once reached, every looser one is too
            assert reached == sorted(reached), (k, s)
    prof = {tau: pp.rho(T[tau]) for tau in pp.TAUS}
    for tau, rows in prof.items():
        assert sum(r[0] for r in rows.values()) >= 100.0 - 1e-9
        assert all(np.all(np.diff(r) >= 0) for r in rows.values())


def test_series_length_tuner_on_small_family():
    """The tuner's table holds a candidate m for every size class it saw,
    chosen by the profile of the measured times; the tuned policy then runs
    through the same harness."""
    from paper_2405_05079_gb300 import autotune as at
    fam = scenes.family_scenes("batched", 4, seed=5)
    tab = at.tune(fam, eta=0.1, tau=0.003, candidates=(6, 21), max_iters=20, seed=5)
    assert tab["rows"] and all(r["m"] in (6, 21) for r in tab["rows"])
    assert sum(r["problems"] for r in tab["rows"]) == len(fam)
    for r in tab["rows"]:
        assert max(r["reached"].values()) >= 1
    ev = at.evaluate(tab, fam[:2], eta=0.1, tau=0.003, fixed_m=21, max_iters=20, seed=5)
    assert set(ev["rho"]) == {"m=21", "tuned"}
    assert sum(r[0] for r in ev["rho"].values()) >= 100.0 - 1e-9
