"""Series-length autotuner: size classes, the choice of m from measured times
to threshold (worked out by hand from the profile definition of Sec. 5), the
table and its lookup, and the serving loop's use of it (host logic, no GPU)."""
import math

import pytest

from paper_2405_05079_gb300 import autotune as at
from paper_2405_05079_gb300 import povar

INF = math.inf


def test_size_classes():
    assert at.size_class(1, (10, 100)) == 0
    assert at.size_class(10, (10, 100)) == 0
    assert at.size_class(11, (10, 100)) == 1
    assert at.size_class(100, (10, 100)) == 1
    assert at.size_class(101, (10, 100)) == 2


def test_choose_m_by_hand():
    # m = 6 is fastest on problems 0 and 1 and never reaches problem 2;
    # m = 21 is 2x slower on 0 and 1 and the only one on 2. With the alphas
    # (1, 1.25, 1.5, 2, 3, 5, 10): rho(6) = 66.7 at every alpha (mean 66.7);
    # rho(21) = 33.3 for alpha < 2 and 100 from alpha = 2 (mean 71.4).
    T = {(6, 0): 1.0, (6, 1): 1.0, (6, 2): INF, (21, 0): 2.0, (21, 1): 2.0, (21, 2): 3.0}
    sc = at.profile_score(T)
    assert sc[6] == pytest.approx(200.0 / 3.0)
    assert sc[21] == pytest.approx((3 * 100.0 / 3.0 + 4 * 100.0) / 7.0)
    assert at.choose_m(T) == 21
    # when m = 6 also reaches problem 2 in time, it wins everywhere
    T[6, 2] = 2.5
    assert at.choose_m(T) == 6


def test_choose_m_ties_keep_the_larger_m():
    T = {(6, 0): 1.0, (11, 0): 1.0, (21, 0): 1.0}
    assert at.choose_m(T) == 21


def test_table_and_lookup():
    T = {}
    n_obs = {0: 5_000, 1: 8_000, 2: 300_000, 3: 400_000}
    for k in n_obs:
        small = n_obs[k] < 20_000
        for m in (6, 21):
            T[m, k] = (1.0 if m == 6 else 2.0) if small else (1.0 if m == 21 else INF)
    tab = at.build_table(T, n_obs, tau=0.001, eta=0.1, precision="mixed", candidates=(6, 21),
                         edges=(20_000, 100_000))
    assert [r["class"] for r in tab["rows"]] == [0, 2]
    assert [r["m"] for r in tab["rows"]] == [6, 21]
    assert tab["rows"][1]["reached"] == {"6": 0, "21": 2}
    assert at.m_for(tab, 1_000) == 6
    assert at.m_for(tab, 1_000_000) == 21      # above every edge: class 2
    # class 1 has no row: the nearest row, the larger class on a tie
    assert at.m_for(tab, 50_000) == 21
    with pytest.raises(ValueError):
        at.m_for({"edges": [10], "rows": []}, 5)


def test_serving_params_follow_the_table():
    from paper_2405_05079_gb300 import serving
    srv = serving.Server.__new__(serving.Server)   # host logic only (no streams)
    srv.params = povar.make_params(eta=0.1, m=21, precision=povar.MIXED_FP32)
    srv.m_table = {"edges": [20_000], "rows": [{"class": 0, "m": 6}, {"class": 1, "m": 16}]}

    class S:
        def __init__(self, n):
            self.n_obs = n
    assert srv.params_for(S(1_000)).m == 6
    assert srv.params_for(S(90_000)).m == 16
    assert srv.params.m == 21                       # the server's params are not modified
    q = srv.params_for(S(1_000))
    assert (q.eta, q.precision, q.lambda0) == (0.1, povar.MIXED_FP32, srv.params.lambda0)
    srv.m_table = None
    assert srv.params_for(S(1_000)) is srv.params
