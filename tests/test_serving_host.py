"""Host logic of the serving loop (no GPU): Poisson arrivals, the summary,
and admission by slots and device-memory budget, with the solve replaced by a
stand-in that holds its slot for a while."""
import threading
import time

import numpy as np
import pytest

from paper_2405_05079_gb300 import povar, serving


@pytest.fixture(scope="module", autouse=True)
def library():
    """estimate_bytes is a host function of libpovar (built here; no GPU call)."""
    from paper_2405_05079_gb300 import build
    build.build()


def test_poisson_arrivals_seeded_and_increasing():
    a = serving.poisson_arrivals(2000, rate=50.0, seed=3)
    assert np.array_equal(a, serving.poisson_arrivals(2000, rate=50.0, seed=3))
    assert np.all(np.diff(a) > 0)
    # mean gap 1 / rate; for 2000 exponential gaps the standard error is 2.2%
    assert abs(np.mean(np.diff(np.r_[0.0, a])) * 50.0 - 1.0) < 0.1


def test_summary_by_hand():
    res = [serving.Result(rid=k, arrival=0.1 * k, admitted=0.1 * k + 0.01,
                          finished=0.1 * k + 0.21, iterations=5, cost=1.0,
                          cameras=np.zeros((1, 12)), device_bytes=0) for k in range(5)]
    st = serving.summarize(res, wall=1.0)
    assert st["n"] == 5 and st["solves_per_s"] == 5.0
    assert st["latency_p50_s"] == pytest.approx(0.21)
    assert st["solve_p99_s"] == pytest.approx(0.20)
    assert st["mean_iterations"] == 5.0


class Scene:
    def __init__(self, n_cams, n_points, n_obs):
        self.n_cams, self.n_points, self.n_obs = n_cams, n_points, n_obs


def host_server(budget, slots):
    """A Server without CUDA streams whose solve holds its slot for 20 ms
    and records how many solves and bytes were admitted at the same time."""
    srv = serving.Server.__new__(serving.Server)
    srv.params = povar.make_params(eta=0.1)
    srv.budget, srv.slots, srv.max_iters, srv.ftol, srv.m_table = budget, slots, 50, 1e-6, None
    srv.streams = [None] * slots
    srv._free_streams = list(range(slots))
    srv._lock = threading.Lock()
    srv._used = 0
    seen = {"max_active": 0, "max_used": 0, "active": 0}

    def fake_solve(req, slot, t0, admitted, reserved):
        with srv._lock:
            seen["active"] += 1
            seen["max_active"] = max(seen["max_active"], seen["active"])
            seen["max_used"] = max(seen["max_used"], srv._used)
            assert 0 <= slot < slots
        time.sleep(0.02)
        with srv._lock:
            seen["active"] -= 1
            srv._used -= reserved
            srv._free_streams.append(slot)
        return serving.Result(rid=req.rid, arrival=req.arrival, admitted=admitted,
                              finished=time.perf_counter() - t0, iterations=1, cost=0.0,
                              cameras=np.zeros((1, 12)), device_bytes=reserved)
    srv._solve = fake_solve
    return srv, seen


def test_admission_respects_slots_and_budget():
    scs = [Scene(40 + 10 * (k % 3), 2000, 10000) for k in range(12)]
    need = [povar.estimate_bytes(s.n_cams, s.n_points, s.n_obs) for s in scs]
    budget = 2 * max(need) + 1          # never more than two requests' memory at once
    srv, seen = host_server(budget, slots=4)
    reqs = [serving.Request(rid=k, arrival=0.0, scene=s, P0=None) for k, s in enumerate(scs)]
    res = srv.run(reqs)
    assert [r.rid for r in res] == list(range(12))
    assert seen["max_used"] <= budget
    assert seen["max_active"] <= 2
    assert srv._used == 0 and sorted(srv._free_streams) == [0, 1, 2, 3]
    # with room for all, the slot count binds
    srv, seen = host_server(100 * max(need), slots=3)
    srv.run(reqs)
    assert seen["max_active"] == 3


def test_request_over_budget_is_rejected():
    s = Scene(100, 5000, 25000)
    srv, _ = host_server(povar.estimate_bytes(s.n_cams, s.n_points, s.n_obs) - 1, slots=2)
    with pytest.raises(ValueError):
        srv.run([serving.Request(rid=0, arrival=0.0, scene=s, P0=None)])

