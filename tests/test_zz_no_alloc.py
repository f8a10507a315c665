"""GPU tests of the allocation-free cost entry (povar_cost_noalloc).

It is compared with the handle path (povar_create + povar_set_cameras +
povar_cost + povar_get_points) on the same cameras, on two calls in a row.
The file name keeps it last in collection order; it also passes alone.
"""
import numpy as np
import pytest

from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# both paths are FP64; they accumulate V_j, h_j in different orders
COST_RTOL = 1e-10
X_RTOL = 1e-8


def landmark_csr(sc):
    """Observations in landmark-major order (stable), as numpy arrays."""
    order = np.argsort(sc.pt_idx, kind="stable")
    off = np.zeros(sc.n_points + 1, np.uint32)
    np.cumsum(np.bincount(sc.pt_idx, minlength=sc.n_points), out=off[1:])
    cam = np.ascontiguousarray(sc.cam_idx[order], np.int32)
    meas = np.ascontiguousarray(sc.meas[order], np.float64)
    return off, cam, meas


def device(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def handle_result(sc, P, eta):
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P, eta)
        return pb.cost(eta), pb.points()


def noalloc_call(sc, dP, doff, dcam, dmeas, eta, stream):
    X = torch.empty((sc.n_points, 3), dtype=torch.float64, device="cuda")
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    povar.cost_noalloc(sc.n_cams, sc.n_points, sc.n_obs, dP.data_ptr(), doff.data_ptr(),
                       dcam.data_ptr(), dmeas.data_ptr(), eta, X.data_ptr(), F.data_ptr(),
                       stream.cuda_stream)
    stream.synchronize()
    return float(F.item()), X.cpu().numpy()


@pytest.mark.parametrize("name,eta", [("tiny", 0.1), ("traj", 0.1), ("mid", 0.01)])
def test_noalloc_cost_matches_handle_two_calls(name, eta):
    sc = {"tiny": scenes.tiny_scene, "mid": scenes.mid_scene,
          "traj": lambda: scenes.trajectory_scene(120, 6000, 3, eta=0.1)}[name]()
    P = scenes.init_cameras(sc.n_cams, 21, normalize=True)
    F_ref, X_ref = handle_result(sc, P, eta)
    off, cam, meas = landmark_csr(sc)
    dP, doff, dcam, dmeas = device(P), device(off), device(cam), device(meas)
    stream = torch.cuda.Stream()
    first = noalloc_call(sc, dP, doff, dcam, dmeas, eta, stream)
    second = noalloc_call(sc, dP, doff, dcam, dmeas, eta, stream)
    for F, X in (first, second):
        assert abs(F - F_ref) <= COST_RTOL * F_ref, (F, F_ref)
        assert np.all(np.abs(X - X_ref) <= X_RTOL * (1.0 + np.abs(X_ref)))
    # the same inputs give the same bits (fixed-order reductions)
    assert first[0] == second[0]
    assert np.array_equal(first[1], second[1])


def test_noalloc_rejects_too_many_points_and_flags_bad_indices():
    sc = scenes.tiny_scene()
    P = scenes.init_cameras(sc.n_cams, 3, normalize=True)
    off, cam, meas = landmark_csr(sc)
    dP, doff, dmeas = device(P), device(off), device(meas)
    F = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    # over the fixed working array: rejected before anything is launched
    with pytest.raises(ValueError, match="allocation-free limit"):
        povar.cost_noalloc(sc.n_cams, povar.NOALLOC_MAX_POINTS + 1, sc.n_obs, dP.data_ptr(),
                           doff.data_ptr(), device(cam).data_ptr(), dmeas.data_ptr(), 0.1, None,
                           F.data_ptr(), stream.cuda_stream)
    # a camera index out of range is skipped on the device and reported as NaN
    bad = cam.copy()
    bad[7] = sc.n_cams
    povar.cost_noalloc(sc.n_cams, sc.n_points, sc.n_obs, dP.data_ptr(), doff.data_ptr(),
                       device(bad).data_ptr(), dmeas.data_ptr(), 0.1, None, F.data_ptr(),
                       stream.cuda_stream)
    stream.synchronize()
    assert np.isnan(F.item())
