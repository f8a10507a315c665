"""Thin ctypes binding of libpovar (C ABI in include/povar.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels. The library is loaded from this package directory (built in-tree by
``paper_2405_05079_gb300.build``); if it is missing the binding raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpovar.so")

EUCLID, SPHERE = 0, 1
FP64, MIXED_FP32, MIXED_BF16 = 0, 1, 2
NSCHEDULES = 6            # POVAR_NSCHEDULES
SOLVER_SERIES, SOLVER_PCG = 0, 1

STATUS = {0: "POVAR_OK", 1: "POVAR_EINVAL", 2: "POVAR_ENOMEM", 3: "POVAR_ECUDA",
          4: "POVAR_ENUMERIC", 5: "POVAR_ETIMEOUT", 6: "POVAR_ENOTCONVERGED"}


class PovarError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("eta", C.c_double), ("lambda0", C.c_double), ("series_eps", C.c_double),
                ("lambda_l", C.c_double), ("m", C.c_int32), ("manifold", C.c_int32),
                ("precision", C.c_int32), ("schedule", C.c_int32), ("solver", C.c_int32),
                ("reserved", C.c_int32)]


class StepReport(C.Structure):
    _fields_ = [("cost_before", C.c_double), ("cost_after", C.c_double), ("pred", C.c_double),
                ("rho", C.c_double), ("lambda_used", C.c_double), ("lambda_next", C.c_double),
                ("accepted", C.c_int32), ("terms_used", C.c_int32), ("iteration", C.c_int32),
                ("converged", C.c_int32), ("ms", C.c_float), ("precision", C.c_int32),
                ("fp64_fallback_at", C.c_int32), ("reserved", C.c_float * 1)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None


def lib() -> C.CDLL:
    """Load libpovar.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} not found: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp, u64 = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_double), C.c_uint64
    L.povar_create.argtypes = [i32, i32, i64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), dp, vp,
                               C.POINTER(vp)]
    L.povar_destroy.argtypes = [vp]
    L.povar_destroy.restype = None
    L.povar_last_error.argtypes = [vp]
    L.povar_last_error.restype = C.c_char_p
    L.povar_set_cameras.argtypes = [vp, dp, C.c_double]
    L.povar_init_random.argtypes = [vp, u64, i32, C.c_double]
    L.povar_get_cameras.argtypes = [vp, dp]
    L.povar_get_points.argtypes = [vp, dp]
    L.povar_cost.argtypes = [vp, C.c_double, dp]
    L.povar_step.argtypes = [vp, C.POINTER(Params), C.POINTER(StepReport)]
    L.povar_solve.argtypes = [vp, C.POINTER(Params), i32, C.c_double, C.c_double,
                              C.POINTER(StepReport), C.POINTER(C.c_int32)]
    L.povar_s2_set.argtypes = [vp, dp, dp]
    L.povar_s2_cost.argtypes = [vp, dp]
    L.povar_s2_step.argtypes = [vp, C.POINTER(Params), C.POINTER(StepReport)]
    L.povar_s2_solve.argtypes = [vp, C.POINTER(Params), i32, C.c_double, C.c_double,
                                 C.POINTER(StepReport), C.POINTER(C.c_int32)]
    L.povar_s2_get_points.argtypes = [vp, dp]
    L.povar_metric_upgrade.argtypes = [vp, dp, i32, C.c_double, dp, dp, dp,
                                       C.POINTER(C.c_int32)]
    u32p = C.POINTER(C.c_uint32)
    L.povar_get_orders.argtypes = [vp, u32p, u32p, u32p, u32p]
    L.povar_get_layout.argtypes = [vp, C.POINTER(C.c_int64), u32p, u32p,
                                   C.POINTER(C.c_int32), u32p, u32p, u32p, u32p]
    L.povar_get_last_step.argtypes = [vp, dp, dp, dp]
    L.povar_set_profiling.argtypes = [vp, i32]
    L.povar_get_profile.argtypes = [vp, dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), i32]
    L.povar_get_tuning.argtypes = [vp, i32, C.POINTER(C.c_int32), C.POINTER(C.c_float)]
    L.povar_device_bytes.argtypes = [vp]
    L.povar_device_bytes.restype = i64
    L.povar_estimate_bytes.argtypes = [i32, i32, i64]
    L.povar_estimate_bytes.restype = i64
    L.povar_launch_count.argtypes = [vp]
    L.povar_launch_count.restype = i64
    L.povar_version.restype = C.c_char_p
    L.povar_batch_create.argtypes = [i32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_int32), dp, vp, C.POINTER(vp)]
    L.povar_batch_destroy.argtypes = [vp]
    L.povar_batch_destroy.restype = None
    L.povar_batch_last_error.argtypes = [vp]
    L.povar_batch_last_error.restype = C.c_char_p
    L.povar_batch_problem.argtypes = [vp, i32]
    L.povar_batch_problem.restype = vp
    L.povar_batch_set_cameras.argtypes = [vp, dp, C.c_double]
    L.povar_batch_get_cameras.argtypes = [vp, dp]
    L.povar_batch_cost.argtypes = [vp, C.c_double, dp]
    L.povar_batch_solve.argtypes = [vp, C.POINTER(Params), i32, C.c_double, dp,
                                    C.POINTER(StepReport), C.POINTER(C.c_int32)]
    L.povar_batch_solve_each.argtypes = [vp, C.POINTER(Params), i32, C.c_double, dp,
                                         C.POINTER(StepReport), C.POINTER(C.c_int32)]
    L.povar_release_cached_memory.argtypes = []
    L.povar_release_cached_memory.restype = None
    L.povar_cost_noalloc.argtypes = [i32, i32, i64, vp, vp, vp, vp, C.c_double, vp, vp, vp]
    L.povar_cost_noalloc.restype = C.c_int
    for name in ("povar_batch_create", "povar_batch_set_cameras", "povar_batch_get_cameras",
                 "povar_batch_cost", "povar_batch_solve", "povar_batch_solve_each"):
        getattr(L, name).restype = C.c_int
    for name in ("povar_create", "povar_set_cameras", "povar_init_random", "povar_get_cameras",
                 "povar_get_points", "povar_cost", "povar_step", "povar_solve",
                 "povar_get_orders", "povar_get_layout", "povar_get_last_step",
                 "povar_set_profiling",
                 "povar_get_profile", "povar_get_tuning"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _obs_arrays(cam_idx, pt_idx, meas, n_obs=None):
    """Contiguous int32 / int32 / float64 (n_obs x 2) copies of one problem's
    observation arrays; ValueError when their lengths disagree (the library
    reads n_obs entries of each)."""
    cam = np.ascontiguousarray(cam_idx, dtype=np.int32).reshape(-1)
    pt = np.ascontiguousarray(pt_idx, dtype=np.int32).reshape(-1)
    m = np.ascontiguousarray(meas, dtype=np.float64)
    n = cam.shape[0] if n_obs is None else int(n_obs)
    if cam.shape[0] != n or pt.shape[0] != n or m.size != 2 * n:
        raise ValueError(f"observation arrays disagree: {n} observations, cam_idx "
                         f"{cam.shape[0]}, pt_idx {pt.shape[0]}, meas {m.size} values "
                         f"(2 per observation)")
    return cam, pt, m.reshape(n, 2)


def make_params(eta=0.1, lambda0=1e-4, m=10, series_eps=0.0, manifold=SPHERE,
                precision=MIXED_FP32, schedule=-1, lambda_l=0.0, solver=0) -> Params:
    """Solver parameters (include/povar.h); lambda_l > 0 selects PoBA (joint
    LM with landmark damping lambda_l * lambda) instead of PoVar; solver
    SOLVER_PCG replaces the series by Schur-Jacobi preconditioned conjugate
    gradients (m = maximum inner iterations, series_eps = relative residual
    tolerance)."""
    return Params(eta=eta, lambda0=lambda0, series_eps=series_eps, lambda_l=lambda_l, m=m,
                  manifold=manifold, precision=precision, schedule=schedule, solver=solver,
                  reserved=0)


def make_s2_params(lambda0=1e-4, m=21, series_eps=0.01, lambda_l=1.0,
                   precision=MIXED_FP32, schedule=-1) -> Params:
    """Parameters of the second stage (povar_s2_*): Riemannian PoBA on the
    unit spheres, landmark damping lambda_l * lambda."""
    return Params(eta=0.0, lambda0=lambda0, series_eps=series_eps, lambda_l=lambda_l, m=m,
                  manifold=SPHERE, precision=precision, schedule=schedule, solver=0, reserved=0)


def current_stream_handle() -> int | None:
    """The current torch CUDA stream as a raw cudaStream_t (None without torch/CUDA)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:  # pragma: no cover - torch is optional for the binding
        pass
    return None


class Problem:
    """Owns a ``povar_problem`` handle. Arrays in and out are host numpy arrays."""

    def __init__(self, n_cams: int, n_points: int, cam_idx, pt_idx, meas, stream=None):
        L = lib()
        self.n_cams, self.n_points = int(n_cams), int(n_points)
        cam, pt, m = _obs_arrays(cam_idx, pt_idx, meas)
        self.n_obs = int(cam.shape[0])
        h = C.c_void_p()
        st = L.povar_create(self.n_cams, self.n_points, self.n_obs, _ptr(cam, C.c_int32),
                            _ptr(pt, C.c_int32), _ptr(m, C.c_double),
                            C.c_void_p(stream) if stream else None, C.byref(h))
        if st != 0:
            raise PovarError(st, "povar_create failed")
        self._h = h

    @classmethod
    def from_scene(cls, scene, stream=None) -> "Problem":
        return cls(scene.n_cams, scene.n_points, scene.cam_idx, scene.pt_idx, scene.meas,
                   stream=stream)

    def _check(self, st: int):
        if st != 0:
            raise PovarError(st, lib().povar_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().povar_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_cameras(self, P, eta: float):
        P = np.ascontiguousarray(P, dtype=np.float64).reshape(self.n_cams, 12)
        self._check(lib().povar_set_cameras(self._h, _ptr(P, C.c_double), eta))

    def set_cameras_device(self, ptr: int, eta: float):
        """Cameras from a device buffer (n_cams x 12 doubles) on the handle's device."""
        self._check(lib().povar_set_cameras(self._h, C.cast(C.c_void_p(ptr),
                                                            C.POINTER(C.c_double)), eta))

    PHASES = ("linearize", "camera_blocks", "series", "pred", "update", "landmarks",
              "controller")

    def set_profiling(self, enable: bool):
        self._check(lib().povar_set_profiling(self._h, 1 if enable else 0))

    def profile(self, reset: bool = False, products: bool = False):
        """Summed phase milliseconds and the number of timed steps; with
        ``products`` also the number of series products those steps computed."""
        ms = np.zeros(len(self.PHASES))
        n = C.c_int64()
        k = C.c_int64()
        self._check(lib().povar_get_profile(self._h, _ptr(ms, C.c_double), C.byref(n),
                                            C.byref(k), 1 if reset else 0))
        out = dict(zip(self.PHASES, ms.tolist()))
        return (out, n.value, k.value) if products else (out, n.value)

    def init_random(self, seed: int, manifold: int, eta: float):
        self._check(lib().povar_init_random(self._h, seed, manifold, eta))

    def cameras(self) -> np.ndarray:
        out = np.empty((self.n_cams, 12))
        self._check(lib().povar_get_cameras(self._h, _ptr(out, C.c_double)))
        return out

    def points(self) -> np.ndarray:
        out = np.empty((self.n_points, 3))
        self._check(lib().povar_get_points(self._h, _ptr(out, C.c_double)))
        return out

    def cost(self, eta: float) -> float:
        v = C.c_double()
        self._check(lib().povar_cost(self._h, eta, C.byref(v)))
        return v.value

    def step(self, params: Params) -> StepReport:
        rep = StepReport()
        self._check(lib().povar_step(self._h, C.byref(params), C.byref(rep)))
        return rep

    def solve(self, params: Params, max_iters=50, ftol=1e-6, target_cost=0.0,
              allow_stall=False):
        """povar_solve. With allow_stall, a solve that ends with
        POVAR_ENOTCONVERGED (the damping diverged: no step could lower the
        cost any more) returns its report instead of raising; the cameras and
        cost stay at the last accepted iterate."""
        rep = StepReport()
        it = C.c_int32()
        st = lib().povar_solve(self._h, C.byref(params), max_iters, ftol, target_cost,
                               C.byref(rep), C.byref(it))
        if not (allow_stall and st == 6):
            self._check(st)
        return rep, it.value

    # ---- second stage: projective refinement by Riemannian PoBA
    def s2_set(self, P=None, X=None):
        """povar_s2_set: homogeneous cameras P [n_cams, 12] and landmarks
        X [n_points, 4] (normalized by the library), or neither (start from
        the first stage's result)."""
        if P is None and X is None:
            self._check(lib().povar_s2_set(self._h, None, None))
            return
        Pa = np.ascontiguousarray(np.asarray(P, dtype=np.float64).reshape(self.n_cams, 12))
        Xa = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(self.n_points, 4))
        self._check(lib().povar_s2_set(self._h, _ptr(Pa, C.c_double), _ptr(Xa, C.c_double)))

    def s2_cost(self) -> float:
        out = C.c_double()
        self._check(lib().povar_s2_cost(self._h, C.byref(out)))
        return out.value

    def s2_step(self, params: Params) -> StepReport:
        rep = StepReport()
        self._check(lib().povar_s2_step(self._h, C.byref(params), C.byref(rep)))
        return rep

    def s2_solve(self, params: Params, max_iters=50, ftol=1e-6, target_cost=0.0,
                 allow_stall=False):
        rep = StepReport()
        it = C.c_int32()
        st = lib().povar_s2_solve(self._h, C.byref(params), max_iters, ftol, target_cost,
                                  C.byref(rep), C.byref(it))
        if not (allow_stall and st == 6):
            self._check(st)
        return rep, it.value

    def s2_points(self):
        out = np.empty((self.n_points, 4))
        self._check(lib().povar_s2_get_points(self._h, _ptr(out, C.c_double)))
        return out

    def metric_upgrade(self, K=None, max_iters=100, ftol=1e-12):
        """povar_metric_upgrade on the current cameras: returns (H [4, 4],
        alpha [n_cams], cost, iterations)."""
        H = np.empty(16)
        al = np.empty(self.n_cams)
        cost = C.c_double()
        it = C.c_int32()
        Kp = None
        if K is not None:
            Ka = np.ascontiguousarray(np.asarray(K, dtype=np.float64).reshape(self.n_cams, 9))
            Kp = _ptr(Ka, C.c_double)
        self._check(lib().povar_metric_upgrade(self._h, Kp, max_iters, ftol,
                                               _ptr(H, C.c_double), _ptr(al, C.c_double),
                                               C.byref(cost), C.byref(it)))
        return H.reshape(4, 4), al, cost.value, it.value

    def orders(self):
        no, np_, nc = self.n_obs, self.n_points, self.n_cams
        pp = np.empty(no, np.uint32)
        op = np.empty(np_ + 1, np.uint32)
        pc = np.empty(no, np.uint32)
        oc = np.empty(nc + 1, np.uint32)
        self._check(lib().povar_get_orders(self._h, _ptr(pp, C.c_uint32), _ptr(op, C.c_uint32),
                                           _ptr(pc, C.c_uint32), _ptr(oc, C.c_uint32)))
        return pp, op, pc, oc

    def layout(self) -> dict:
        """povar_get_layout: the SELL-32 landmark layout and the run tables."""
        L = lib()
        sz = np.zeros(6, np.int64)
        u32 = C.c_uint32
        self._check(L.povar_get_layout(self._h, _ptr(sz, C.c_int64), None, None, None, None,
                                       None, None, None))
        np_pad, nsl, nsell, nrows, npart, nvis = (int(x) for x in sz)
        out = {"slot_pt": np.empty(np_pad, np.uint32), "sell_off": np.empty(nsl + 1, np.uint32),
               "sell_cam": np.empty(nsell, np.int32), "row_mask": np.empty(nrows, np.uint32),
               "row_base": np.empty(nrows, np.uint32),
               "cam_part_off": np.empty(self.n_cams + 1, np.uint32),
               "cam_part_idx": np.empty(npart, np.uint32)}
        self._check(L.povar_get_layout(
            self._h, _ptr(sz, C.c_int64), _ptr(out["slot_pt"], u32), _ptr(out["sell_off"], u32),
            _ptr(out["sell_cam"], C.c_int32), _ptr(out["row_mask"], u32),
            _ptr(out["row_base"], u32), _ptr(out["cam_part_off"], u32),
            _ptr(out["cam_part_idx"], u32)))
        out["n_visits"] = nvis
        return out

    def last_step(self):
        U = np.empty((self.n_cams, 12, 12))
        bp = np.empty((self.n_cams, 12))
        d = np.empty((self.n_cams, 12))
        self._check(lib().povar_get_last_step(self._h, _ptr(U, C.c_double),
                                              _ptr(bp, C.c_double), _ptr(d, C.c_double)))
        return U, bp, d

    def tuning(self, precision: int):
        sched = C.c_int32()
        ms = (C.c_float * NSCHEDULES)()
        self._check(lib().povar_get_tuning(self._h, precision, C.byref(sched), ms))
        return sched.value, list(ms)

    @property
    def device_bytes(self) -> int:
        return int(lib().povar_device_bytes(self._h))

    @property
    def launch_count(self) -> int:
        return int(lib().povar_launch_count(self._h))


class Batch:
    """Independent problems solved together (one CUDA-graph launch per iteration)."""

    def __init__(self, scenes_list, stream=None):
        L = lib()
        self.n = len(scenes_list)
        nc = np.array([s.n_cams for s in scenes_list], np.int32)
        npnt = np.array([s.n_points for s in scenes_list], np.int32)
        nob = np.array([s.n_obs for s in scenes_list], np.int64)
        arrs = [_obs_arrays(s.cam_idx, s.pt_idx, s.meas, s.n_obs) for s in scenes_list]
        cam = np.ascontiguousarray(np.concatenate([a[0] for a in arrs]))
        pt = np.ascontiguousarray(np.concatenate([a[1] for a in arrs]))
        m = np.ascontiguousarray(np.concatenate([a[2] for a in arrs]))
        self.n_cams = nc
        self.n_obs = nob
        self.cam0 = np.concatenate([[0], np.cumsum(nc)])
        h = C.c_void_p()
        st = L.povar_batch_create(self.n, _ptr(nc, C.c_int32), _ptr(npnt, C.c_int32),
                                  _ptr(nob, C.c_int64), _ptr(cam, C.c_int32), _ptr(pt, C.c_int32),
                                  _ptr(m, C.c_double), C.c_void_p(stream) if stream else None,
                                  C.byref(h))
        if st != 0:
            raise PovarError(st, "povar_batch_create failed")
        self._h = h

    def _check(self, st):
        if st != 0:
            raise PovarError(st, lib().povar_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().povar_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_cameras(self, P_list, eta):
        Ps = [np.asarray(p).reshape(-1, 12) for p in P_list]
        if len(Ps) != self.n or any(q.shape[0] != int(c) for q, c in zip(Ps, self.n_cams)):
            raise ValueError(f"expected {self.n} camera arrays of {list(map(int, self.n_cams))} "
                             f"cameras, got {[q.shape[0] for q in Ps]}")
        P = np.ascontiguousarray(np.concatenate(Ps), np.float64)
        self._check(lib().povar_batch_set_cameras(self._h, _ptr(P, C.c_double), eta))

    def cameras(self):
        out = np.empty((int(self.cam0[-1]), 12))
        self._check(lib().povar_batch_get_cameras(self._h, _ptr(out, C.c_double)))
        return [out[self.cam0[k]:self.cam0[k + 1]] for k in range(self.n)]

    def costs(self, eta):
        out = np.empty(self.n)
        self._check(lib().povar_batch_cost(self._h, eta, _ptr(out, C.c_double)))
        return out

    def solve(self, params, max_iters=50, ftol=1e-6, target_costs=None):
        """povar_batch_solve; params is one Params for every problem, or a
        sequence of n Params (povar_batch_solve_each)."""
        reps = (StepReport * self.n)()
        its = np.zeros(self.n, np.int32)
        tc = None if target_costs is None else np.ascontiguousarray(target_costs, np.float64)
        tcp = None if tc is None else _ptr(tc, C.c_double)
        if isinstance(params, Params):
            st = lib().povar_batch_solve(self._h, C.byref(params), max_iters, ftol, tcp, reps,
                                         _ptr(its, C.c_int32))
        else:
            arr = (Params * self.n)(*params)
            st = lib().povar_batch_solve_each(self._h, arr, max_iters, ftol, tcp, reps,
                                              _ptr(its, C.c_int32))
        self._check(st)
        return list(reps), its


@dataclasses.dataclass
class SolveResult:
    report: dict
    iterations: int
    cameras: np.ndarray
    points: np.ndarray


def estimate_bytes(n_cams: int, n_points: int, n_obs: int) -> int:
    """Upper-bound device footprint of a problem of these sizes."""
    return int(lib().povar_estimate_bytes(n_cams, n_points, n_obs))


NOALLOC_MAX_POINTS = 4194304   # POVAR_NOALLOC_MAX_POINTS


def cost_noalloc(n_cams: int, n_points: int, n_obs: int, P: int, off_pt: int, cam: int,
                 meas: int, eta: float, X_out: int | None, cost_out: int,
                 stream: int | None = None) -> None:
    """povar_cost_noalloc on raw device addresses (see include/povar.h):
    P (n_cams x 12 f64), off_pt (n_points + 1 u32), cam (n_obs i32), meas
    (n_obs x 2 f64), X_out (n_points x 3 f64 or None), cost_out (1 f64).
    Enqueued on ``stream``; nothing is allocated or synchronized."""
    st = lib().povar_cost_noalloc(n_cams, n_points, n_obs, P, off_pt, cam, meas, eta,
                                  X_out, cost_out, stream)
    if st == 1 and n_points > NOALLOC_MAX_POINTS:
        raise ValueError(f"n_points = {n_points} exceeds the allocation-free limit "
                         f"of {NOALLOC_MAX_POINTS} landmarks")
    if st != 0:
        raise PovarError(st, "povar_cost_noalloc failed")


def release_cached_memory() -> None:
    """povar_release_cached_memory: give the device memory that destroyed
    problems left in the library's pool back to the device."""
    lib().povar_release_cached_memory()


def version() -> str:
    return lib().povar_version().decode()
