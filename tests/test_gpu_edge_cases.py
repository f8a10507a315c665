"""GPU edge cases against the oracle: landmarks seen once, the pure-projective
limit eta = 0 (a landmark seen once then has a rank-deficient V_j and takes
the pseudo-inverse), the affine limit eta = 1, and tracks longer than 32 slice
rows (several staging chunks in the row-table schedule)."""
import numpy as np
import pytest

from oracle import povar_oracle as O
from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def single_view_scene(eta):
    """The tiny ring scene with landmarks 0..99 reduced to their first
    observation (track length 1); the others keep 3-6 views."""
    base = scenes.tiny_scene(0)
    keep = np.ones(base.n_obs, bool)
    seen = set()
    for k in range(base.n_obs):
        j = int(base.pt_idx[k])
        if j < 100:
            keep[k] = j not in seen
            seen.add(j)
    return scenes.Scene(name=f"single_eta{eta}", seed=0, n_cams=base.n_cams,
                        n_points=base.n_points, cam_idx=base.cam_idx[keep].copy(),
                        pt_idx=base.pt_idx[keep].copy(), meas=base.meas[keep].copy(),
                        eta=eta, m=8, gt_cams=base.gt_cams, gt_points=base.gt_points)


def long_track_scene():
    """Trajectory scene whose tracks are windows of up to 70 cameras (slice
    widths above 32)."""
    return scenes.trajectory_scene(90, 2000, 8, eta=0.1, m=8, p_geom=0.03, max_track=70,
                                   outlier_frac=0.0, name="long")


CASES = {
    "single_eta0.1": lambda: single_view_scene(0.1),
    "single_eta0": lambda: single_view_scene(0.0),
    "tiny_eta1": lambda: single_view_scene(1.0),
    "long": long_track_scene,
}


@pytest.mark.parametrize("name", list(CASES))
def test_landmarks_and_one_step_match_oracle(name):
    sc = CASES[name]()
    if name == "long":
        assert np.bincount(sc.pt_idx).max() > 32
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    X, _, n_pinv = O.landmarks(P0, sc.cam_idx, sc.pt_idx, sc.meas, sc.eta, sc.n_points,
                               return_V=True)
    if name == "single_eta0":
        assert n_pinv >= 100   # every single-view landmark is rank-deficient at eta = 0
    F = orc.cost(P0, X, sc.eta)
    op = O.Params(eta=sc.eta, m=sc.m, manifold=O.EUCLID, series_eps=0.0, lambda0=1e-4)
    st = orc.init_state(P0, op)
    _, orep = orc.step(st, op)
    for sched in range(povar.NSCHEDULES):
        with povar.Problem.from_scene(sc) as pb:
            pb.set_cameras(P0, sc.eta)
            Xg = pb.points()
            Fg = pb.cost(sc.eta)
            assert rel(Xg, X) <= 1e-9, (name, sched)
            assert abs(Fg - F) <= 1e-10 * max(F, 1e-300) + 1e-14, (name, sched)
            rep = pb.step(povar.make_params(eta=sc.eta, m=sc.m, manifold=povar.EUCLID,
                                            precision=povar.FP64, lambda0=1e-4,
                                            schedule=sched))
            _, _, d = pb.last_step()
        assert rel(d, orep.delta) <= 1e-9, (name, sched)
        assert abs(rep.cost_after - orep.cost_after) <= 1e-9 * orep.cost_after + 1e-14
        assert rep.accepted == int(orep.accepted)


def test_mixed_step_on_long_tracks_close_to_fp64():
    sc = long_track_scene()
    P0 = scenes.init_cameras(sc.n_cams, 5, normalize=True)
    out = {}
    for prec in (povar.FP64, povar.MIXED_FP32):
        for sched in range(povar.NSCHEDULES):
            with povar.Problem.from_scene(sc) as pb:
                pb.set_cameras(P0, sc.eta)
                pb.step(povar.make_params(eta=sc.eta, m=sc.m, manifold=povar.EUCLID,
                                          precision=prec, schedule=sched))
                out[prec, sched] = pb.last_step()[2]
    for sched in range(povar.NSCHEDULES):
        assert rel(out[povar.MIXED_FP32, sched], out[povar.FP64, 0]) <= 1e-3, sched
        assert rel(out[povar.FP64, sched], out[povar.FP64, 0]) <= 1e-12, sched
