"""Continuous-batching request loop for bundle-adjustment problems.

Requests (a scene and its initial cameras) arrive over time. A request is
admitted as soon as it has arrived, a worker slot is free and the device
memory it needs (``povar.estimate_bytes``, an upper bound checked against the
handle's actual footprint after creation) fits in the admission budget next to
the problems already on the GPU. Every admitted problem gets its own CUDA
stream and its state (cameras, landmarks, damping) stays resident on the
device for its whole solve; problems admitted while others are running are
solved concurrently, so their kernels overlap on the device. When a solve
finishes its memory is released and waiting requests are admitted.

Each problem's result depends only on its own data and parameters (no
cross-problem reduction), so it is the same alone and in the mix.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import threading
import time

import numpy as np

from . import povar


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    scene: object           # scenes.Scene
    P0: np.ndarray          # [n_cams, 12]
    target_cost: float = 0.0


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    iterations: int
    cost: float
    cameras: np.ndarray
    device_bytes: int

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def solve_time(self) -> float:
        return self.finished - self.admitted


def poisson_arrivals(n: int, rate: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process with ``rate`` requests per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


class Server:
    """Admission by device-memory budget, one stream and one worker per slot."""

    def __init__(self, params, budget_bytes: int, slots: int = 8, max_iters: int = 50,
                 ftol: float = 1e-6, m_table: dict | None = None):
        """m_table: a series-length table of the autotuner (autotune.py); when
        given, each request runs with the m of its size class instead of
        params.m."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("the serving loop needs a CUDA device")
        self.params = params
        self.m_table = m_table
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_iters = int(max_iters)
        self.ftol = float(ftol)
        self.streams = [torch.cuda.Stream() for _ in range(self.slots)]
        self._free_streams = list(range(self.slots))
        self._lock = threading.Lock()
        self._used = 0

    def params_for(self, scene):
        """Solver parameters of a request: params, with the tuned m of the
        scene's size class when the server has an m table."""
        if self.m_table is None:
            return self.params
        from .autotune import params_with_m
        return params_with_m(self.m_table, self.params, scene.n_obs)

    def _solve(self, req: Request, slot: int, t0: float, admitted: float, reserved: int):
        stream = self.streams[slot].cuda_stream
        sc = req.scene
        try:
            with povar.Problem.from_scene(sc, stream=stream) as pb:
                actual = pb.device_bytes
                pb.set_cameras(req.P0, self.params.eta)
                _, iters = pb.solve(self.params_for(sc), max_iters=self.max_iters,
                                    ftol=self.ftol, target_cost=req.target_cost,
                                    allow_stall=True)
                cost = pb.cost(self.params.eta)
                cams = pb.cameras()
        finally:
            with self._lock:
                self._used -= reserved
                self._free_streams.append(slot)
        return Result(rid=req.rid, arrival=req.arrival, admitted=admitted,
                      finished=time.perf_counter() - t0, iterations=iters, cost=cost,
                      cameras=cams, device_bytes=actual)

    def run(self, requests: list[Request]) -> list[Result]:
        """Serve ``requests`` (sorted by arrival); returns results by request id."""
        pending = sorted(requests, key=lambda r: r.arrival)
        need = {r.rid: povar.estimate_bytes(r.scene.n_cams, r.scene.n_points, r.scene.n_obs)
                for r in pending}
        for r in pending:
            if need[r.rid] > self.budget:
                raise ValueError(f"request {r.rid} needs {need[r.rid]} bytes, over the budget")
        results = {}
        futures = []
        t0 = time.perf_counter()
        with cf.ThreadPoolExecutor(max_workers=self.slots) as ex:
            while pending or futures:
                now = time.perf_counter() - t0
                admitted_any = False
                while pending and pending[0].arrival <= now:
                    r = pending[0]
                    with self._lock:
                        ok = self._free_streams and self._used + need[r.rid] <= self.budget
                        if ok:
                            slot = self._free_streams.pop()
                            self._used += need[r.rid]
                    if not ok:
                        break
                    pending.pop(0)
                    futures.append(ex.submit(self._solve, r, slot, t0, now, need[r.rid]))
                    admitted_any = True
                done = [f for f in futures if f.done()]
                for f in done:
                    res = f.result()
                    results[res.rid] = res
                    futures.remove(f)
                if not admitted_any and not done:
                    wait = 0.0005
                    if pending and not futures:
                        wait = max(0.0, min(0.01, pending[0].arrival - now))
                    time.sleep(wait)
        return [results[k] for k in sorted(results)]


def summarize(results: list[Result], wall: float | None = None) -> dict:
    lat = np.array([r.latency for r in results])
    sol = np.array([r.solve_time for r in results])
    span = wall if wall is not None else max(r.finished for r in results) - min(
        r.arrival for r in results)
    return {"n": len(results), "solves_per_s": len(results) / span,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "solve_p50_s": float(np.percentile(sol, 50)),
            "solve_p99_s": float(np.percentile(sol, 99)),
            "mean_iterations": float(np.mean([r.iterations for r in results]))}


def sequential(requests: list[Request], params, max_iters: int = 50,
               ftol: float = 1e-6) -> list[Result]:
    """The same requests solved one after another (no overlap), for comparison."""
    results = []
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda q: q.arrival):
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        start = time.perf_counter() - t0
        with povar.Problem.from_scene(r.scene) as pb:
            pb.set_cameras(r.P0, params.eta)
            _, iters = pb.solve(params, max_iters=max_iters, ftol=ftol,
                                target_cost=r.target_cost)
            results.append(Result(rid=r.rid, arrival=r.arrival, admitted=start,
                                  finished=time.perf_counter() - t0, iterations=iters,
                                  cost=pb.cost(params.eta), cameras=pb.cameras(),
                                  device_bytes=pb.device_bytes))
    return results
