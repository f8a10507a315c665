"""Seeded synthetic bundle-adjustment scenes.

This module only *generates inputs*: camera/point index arrays, normalized
2D measurements and random camera initializations. It contains none of the
solver's arithmetic (no pOSE residual, no normal equations, no Schur
complement) so that the FP64 CPU oracle and the CUDA path can both consume
the same inputs without sharing any method code.

The scenes stand in for the BAL problems the paper evaluates on (its
supplementary size table): BAL itself is not available, so every scene is
drawn from a stated recipe with a seed.

Conventions
-----------
* Measurements are normalized image coordinates ``(pixel - pp) / f`` with
  ``f = 500`` px and ``pp = 0``.
* ``cam_idx[k]``, ``pt_idx[k]`` and ``meas[k]`` describe observation ``k``;
  observations are stored in a random order (the solver builds its own
  camera-major and point-major orders).
* Random camera initialization follows the paper's experimental setup
  (Sec. 5.2 "Dataset"): every entry of every 3x4 camera is iid N(0, 1); the
  landmarks are then obtained in closed form by the solver.
"""
from __future__ import annotations

import dataclasses

import numpy as np

FOCAL_PX = 500.0


@dataclasses.dataclass
class Scene:
    name: str
    seed: int
    n_cams: int
    n_points: int
    cam_idx: np.ndarray      # int32 [n_obs]
    pt_idx: np.ndarray       # int32 [n_obs]
    meas: np.ndarray         # float64 [n_obs, 2], normalized coordinates
    eta: float               # pOSE weight the config uses
    m: int                   # series order (number of terms) the config uses
    gt_cams: np.ndarray      # float64 [n_cams, 3, 4] ground-truth [R | t]
    gt_points: np.ndarray    # float64 [n_points, 3]
    outlier_frac: float = 0.0

    @property
    def n_obs(self) -> int:
        return int(self.cam_idx.shape[0])

    def subset_points(self, keep: np.ndarray) -> "Scene":
        """Scene restricted to the points ``keep`` (renumbered 0..len-1),
        keeping every camera. Used to draw bounded samples of a workload."""
        keep = np.asarray(keep, dtype=np.int64)
        newid = -np.ones(self.n_points, dtype=np.int64)
        newid[keep] = np.arange(keep.size)
        sel = newid[self.pt_idx] >= 0
        return Scene(
            name=f"{self.name}[{keep.size}pts]", seed=self.seed,
            n_cams=self.n_cams, n_points=int(keep.size),
            cam_idx=self.cam_idx[sel].copy(),
            pt_idx=newid[self.pt_idx[sel]].astype(np.int32),
            meas=self.meas[sel].copy(), eta=self.eta, m=self.m,
            gt_cams=self.gt_cams, gt_points=self.gt_points[keep],
            outlier_frac=self.outlier_frac)


def _look_at(center: np.ndarray, target: np.ndarray) -> np.ndarray:
    """World-to-camera [R | t] of a camera at ``center`` looking at ``target``
    (camera z axis forward, y axis roughly world-up)."""
    z = target - center
    z = z / np.linalg.norm(z)
    up = np.array([0.0, 1.0, 0.0])
    x = np.cross(up, z)
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ center
    return np.concatenate([R, t[:, None]], axis=1)


def _project(cams: np.ndarray, pts: np.ndarray, cam_idx, pt_idx) -> np.ndarray:
    """Pinhole projection in normalized coordinates and the depth."""
    Rt = cams[cam_idx]                       # [n, 3, 4]
    Xh = np.concatenate([pts[pt_idx], np.ones((pt_idx.size, 1))], axis=1)
    y = np.einsum("nij,nj->ni", Rt, Xh)
    return y[:, :2] / y[:, 2:3], y[:, 2]


def _distinct_views(rng, n_points: int, n_cams: int, lengths: np.ndarray):
    """For point j, ``lengths[j]`` distinct cameras chosen uniformly."""
    cam_rows = []
    for j in range(n_points):
        cam_rows.append(rng.choice(n_cams, size=int(lengths[j]), replace=False))
    cam_idx = np.concatenate(cam_rows).astype(np.int32)
    pt_idx = np.repeat(np.arange(n_points, dtype=np.int32), lengths)
    return cam_idx, pt_idx


def _finish(name, seed, rng, cams, pts, cam_idx, pt_idx, noise_px, eta, m,
            outlier_frac=0.0) -> Scene:
    uv, depth = _project(cams, pts, cam_idx, pt_idx)
    if np.any(depth <= 0):
        raise RuntimeError("scene generator placed a point behind a camera")
    uv = uv + rng.normal(0.0, noise_px / FOCAL_PX, size=uv.shape)
    if outlier_frac > 0:
        n_out = int(round(outlier_frac * uv.shape[0]))
        idx = rng.choice(uv.shape[0], size=n_out, replace=False)
        # uniform over the image extent (+-500 px around the principal point)
        uv[idx] = rng.uniform(-1.0, 1.0, size=(n_out, 2))
    # observations in random order; the solver builds its own orders
    order = rng.permutation(cam_idx.size)
    return Scene(name=name, seed=seed, n_cams=cams.shape[0],
                 n_points=pts.shape[0], cam_idx=cam_idx[order].copy(),
                 pt_idx=pt_idx[order].copy(), meas=uv[order].copy(), eta=eta,
                 m=m, gt_cams=cams, gt_points=pts, outlier_frac=outlier_frac)


def ring_scene(n_cams: int, n_points: int, seed: int, *, track="uniform3to6",
               noise_px=1.0, eta=0.1, m=10, radius=4.0, max_track=None,
               name=None) -> Scene:
    """Cameras on a ring looking at the origin; points uniform in [-1,1]^3.

    ``track="uniform3to6"``: each point seen by U{3..6} distinct cameras.
    ``track="geom3"``: length 2 + Geom(p=1/3) (mean 4, min 2), capped.
    ``track="geom4"``: length 2 + Geom(p=1/4) (mean 5, min 2), capped.
    """
    rng = np.random.default_rng(seed)
    ang = 2.0 * np.pi * np.arange(n_cams) / n_cams
    heights = 0.3 * np.sin(3.0 * ang)
    centers = np.stack([radius * np.sin(ang), heights, -radius * np.cos(ang)], 1)
    cams = np.stack([_look_at(c, np.zeros(3)) for c in centers])
    pts = rng.uniform(-1.0, 1.0, size=(n_points, 3))
    cap = n_cams if max_track is None else min(n_cams, max_track)
    if track == "uniform3to6":
        lengths = rng.integers(3, 7, size=n_points)
    elif track == "geom3":
        lengths = 1 + rng.geometric(1.0 / 3.0, size=n_points)
    elif track == "geom4":
        lengths = 1 + rng.geometric(1.0 / 4.0, size=n_points)
    else:
        raise ValueError(track)
    lengths = np.minimum(lengths, cap)
    cam_idx, pt_idx = _distinct_views(rng, n_points, n_cams, lengths)
    return _finish(name or f"ring{n_cams}x{n_points}", seed, rng, cams, pts,
                   cam_idx, pt_idx, noise_px, eta, m)


def trajectory_scene(n_cams: int, n_points: int, seed: int, *, noise_px=0.5,
                     eta=0.1, m=20, outlier_frac=0.01, max_track=40,
                     p_geom=0.25, radius=20.0, deg_per_cam=None, name=None) -> Scene:
    """Cameras along a closed circular trajectory looking at its centre.

    Each point is seen by a contiguous window of ``L = 1 + Geom(p_geom)``
    consecutive cameras (mean 5, min 2 for p = 1/4), capped at ``max_track``.
    The point is placed in front of the middle camera of its window, so it
    projects inside the +-45 degree field of view of every camera in it.

    With ``deg_per_cam`` the trajectory is an open helix instead (camera i at
    angle i * deg_per_cam, rising 0.05 per camera, looking at the axis at its
    own height) and windows do not wrap around; this keeps the angle spanned
    by a window small for scenes with few cameras.
    """
    rng = np.random.default_rng(seed)
    if deg_per_cam is None:
        ang = 2.0 * np.pi * np.arange(n_cams) / n_cams
        heights = 0.5 * np.sin(5.0 * ang)
        targets = np.zeros((n_cams, 3))
    else:
        ang = np.deg2rad(deg_per_cam) * np.arange(n_cams)
        heights = 0.05 * np.arange(n_cams)
        targets = np.stack([np.zeros(n_cams), heights, np.zeros(n_cams)], 1)
    centers = np.stack([radius * np.sin(ang), heights, -radius * np.cos(ang)], 1)
    cams = np.stack([_look_at(c, t) for c, t in zip(centers, targets)])
    lengths = np.minimum(1 + rng.geometric(p_geom, size=n_points),
                         min(max_track, n_cams))
    if deg_per_cam is None:
        start = rng.integers(0, n_cams, size=n_points)
    else:
        start = rng.integers(0, n_cams - lengths + 1)
    mid = (start + lengths // 2) % n_cams
    depth = rng.uniform(4.0, 8.0, size=n_points)
    lat = rng.uniform(-0.35, 0.35, size=(n_points, 2)) * depth[:, None]
    Rm = cams[mid, :, :3]                      # rows: camera axes in world
    pts = (centers[mid] + depth[:, None] * Rm[:, 2]
           + lat[:, :1] * Rm[:, 0] + lat[:, 1:] * Rm[:, 1])
    pt_idx = np.repeat(np.arange(n_points, dtype=np.int64), lengths)
    first = np.repeat(start, lengths)
    offs = np.arange(pt_idx.size) - np.repeat(np.cumsum(lengths) - lengths,
                                              lengths)
    cam_idx = ((first + offs) % n_cams).astype(np.int32)
    return _finish(name or f"traj{n_cams}x{n_points}", seed, rng, cams, pts,
                   cam_idx, pt_idx.astype(np.int32), noise_px, eta, m,
                   outlier_frac=outlier_frac)


# --------------------------------------------------------------------------
# The configurations the benchmarks and tests use (sizes from the paper's
# BAL table: "mid" ~ ladybug-49, "large" ~ venice-1672).
# --------------------------------------------------------------------------

def tiny_scene(seed: int = 0) -> Scene:
    """10 cameras on a ring (r=4), 500 points in [-1,1]^3, U{3..6} views per
    point (~2,250 observations), 1 px noise, eta = 0.1, m = 10."""
    return ring_scene(10, 500, seed, track="uniform3to6", noise_px=1.0,
                      eta=0.1, m=10, name="tiny")


def mid_scene(seed: int = 0) -> Scene:
    """50 cameras on a ring, 8,000 points, track 2 + Geom(1/3) (mean 4),
    ~32,000 observations, 0.5 px noise, eta = 0.01, m = 10."""
    return ring_scene(50, 8000, seed, track="geom3", noise_px=0.5, eta=0.01,
                      m=10, max_track=50, name="mid")


def large_scene(seed: int = 0, n_cams: int = 1800,
                n_points: int = 1_000_000) -> Scene:
    """1,800 cameras on a trajectory, 1,000,000 points, contiguous-window
    tracks 2 + Geom(1/4) capped at 40 (mean 5, ~5,000,000 observations),
    0.5 px noise, 1% uniform outliers, eta = 0.1, m = 20."""
    return trajectory_scene(n_cams, n_points, seed, noise_px=0.5, eta=0.1,
                            m=20, outlier_frac=0.01, max_track=40,
                            name="large")


def family_scenes(kind: str, n: int, seed: int = 0) -> list:
    """Seeded families of independent problems of uneven sizes.

    ``batched``: cameras log-uniform in [20, 400], 50 points per camera, mean
    track 4 (1 + Geom(1/3)). ``serving``: cameras log-uniform in [10, 1000],
    100 points per camera, mean track 5 (1 + Geom(1/4)). Both are helix
    trajectories (1 degree per camera, contiguous-window tracks capped at 40),
    0.5 px noise, no outliers, eta = 0.1.
    """
    spec = {"batched": (20, 400, 50, 1.0 / 3.0), "serving": (10, 1000, 100, 0.25)}
    lo, hi, ppc, p = spec[kind]
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xFA11]))
    n_cams = np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))).astype(int)
    seeds = rng.integers(0, 2**31 - 1, size=n)
    return [trajectory_scene(int(c), int(c) * ppc, int(s), noise_px=0.5, eta=0.1, m=20,
                             outlier_frac=0.0, max_track=40, p_geom=p, deg_per_cam=1.0,
                             name=f"{kind}{k}")
            for k, (c, s) in enumerate(zip(n_cams, seeds))]


def init_cameras(n_cams: int, seed: int, normalize: bool) -> np.ndarray:
    """Random camera initialization: 3x4 entries iid N(0,1), stored row-major
    as [n_cams, 12] float64; with ``normalize`` each camera is scaled to unit
    Frobenius norm (a point of the unit-norm camera manifold)."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5EED]))
    P = rng.normal(0.0, 1.0, size=(n_cams, 12))
    if normalize:
        P /= np.linalg.norm(P, axis=1, keepdims=True)
    return P


def stage2_start(scene: Scene, seed: int, noise: float = 0.01):
    """A start for the second (projective) stage near the scene's ground
    truth: the cameras [R | t] and the homogeneous points (X, 1) are moved by
    one random projective transformation H = I + 0.2 N(0, 1) (P H, H^-1 X
    keep every projection), then every entry gets relative iid normal noise
    of size `noise` (of the row's RMS). Returns P [n_cams, 12] (row-major
    3x4) and X [n_points, 4]; rows are not normalized."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x57A6E2]))
    while True:
        H = np.eye(4) + 0.2 * rng.normal(size=(4, 4))
        if np.linalg.cond(H) < 10.0:
            break
    P = np.einsum("nab,bc->nac", scene.gt_cams, H).reshape(scene.n_cams, 12)
    Xh = np.concatenate([scene.gt_points, np.ones((scene.n_points, 1))], axis=1)
    X = np.linalg.solve(H, Xh.T).T
    P = P + noise * np.sqrt(np.mean(P * P, axis=1, keepdims=True)) * rng.normal(size=P.shape)
    X = X + noise * np.sqrt(np.mean(X * X, axis=1, keepdims=True)) * rng.normal(size=X.shape)
    return P, X


def scene_by_name(name: str, seed: int = 0) -> Scene:
    return {"tiny": tiny_scene, "mid": mid_scene, "large": large_scene}[name](seed)


def describe(scene: Scene) -> dict:
    L = np.bincount(scene.pt_idx, minlength=scene.n_points)
    return {"name": scene.name, "seed": scene.seed, "n_cams": scene.n_cams,
            "n_points": scene.n_points, "n_obs": scene.n_obs,
            "track_mean": float(L.mean()), "track_max": int(L.max()),
            "eta": scene.eta, "m": scene.m, "outlier_frac": scene.outlier_frac}


__all__ = ["Scene", "ring_scene", "trajectory_scene", "tiny_scene",
           "mid_scene", "large_scene", "family_scenes", "init_cameras", "scene_by_name",
           "describe", "FOCAL_PX"]
