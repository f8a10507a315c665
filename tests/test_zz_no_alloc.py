"""GPU tests of the allocation-free cost entry (povar_cost_noalloc).

Some callers cannot allocate device memory at the point of the call (a
latency-critical loop that cannot afford the device synchronization of
cudaMalloc / cudaFree, or a process whose memory is held by another
allocator); this entry point serves them from a fixed array inside the
library. It is compared with the handle path (povar_create +
povar_set_cameras + povar_cost + povar_get_points) on the same cameras, on
two calls in a row, and with the FP64 CPU oracle directly. The file name
keeps it last in collection order; it also passes alone.
"""
import numpy as np
import pytest

from oracle import povar_oracle as O
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


def test_noalloc_matches_the_oracle_directly():
    """Closed-form landmarks and cost against the FP64 CPU oracle on the tiny
    scene (not only through the handle path)."""
    sc = scenes.tiny_scene()
    P = scenes.init_cameras(sc.n_cams, 5, normalize=True)
    X_o = O.landmarks(P, sc.cam_idx, sc.pt_idx, sc.meas, sc.eta, sc.n_points)
    F_o = O.cost(P, X_o, sc.cam_idx, sc.pt_idx, sc.meas, sc.eta)
    off, cam, meas = landmark_csr(sc)
    stream = torch.cuda.Stream()
    F, X = noalloc_call(sc, device(P), device(off), device(cam), device(meas), sc.eta, stream)
    assert abs(F - F_o) <= COST_RTOL * F_o, (F, F_o)
    assert np.all(np.abs(X - X_o) <= X_RTOL * (1.0 + np.abs(X_o)))


def test_noalloc_flags_malformed_offset_tables_as_nan():
    """A decreasing offset pair and a last offset past n_obs are index errors
    found on the device: the cost is NaN and nothing is read out of bounds."""
    sc = scenes.tiny_scene()
    P = scenes.init_cameras(sc.n_cams, 3, normalize=True)
    off, cam, meas = landmark_csr(sc)
    dP, dcam, dmeas = device(P), device(cam), device(meas)
    stream = torch.cuda.Stream()
    decreasing = off.copy()
    decreasing[5] = decreasing[6] + 1          # off[5] > off[6]
    past_end = off.copy()
    past_end[-1] = sc.n_obs + 3                # last landmark runs past n_obs
    for bad in (decreasing, past_end):
        F = torch.zeros(1, dtype=torch.float64, device="cuda")
        povar.cost_noalloc(sc.n_cams, sc.n_points, sc.n_obs, dP.data_ptr(),
                           device(bad).data_ptr(), dcam.data_ptr(), dmeas.data_ptr(), 0.1, None,
                           F.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        assert np.isnan(F.item())


def test_noalloc_calls_leave_free_device_memory_unchanged():
    """After the first call (which looks up the working array's address),
    further calls take no device memory: the device's free-memory count is
    the same before and after them (any cudaMalloc reserves whole pages)."""
    sc = scenes.trajectory_scene(120, 6000, 3, eta=0.1)
    P = scenes.init_cameras(sc.n_cams, 9, normalize=True)
    off, cam, meas = landmark_csr(sc)
    dP, doff, dcam, dmeas = device(P), device(off), device(cam), device(meas)
    X = torch.empty((sc.n_points, 3), dtype=torch.float64, device="cuda")
    F = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    args = (sc.n_cams, sc.n_points, sc.n_obs, dP.data_ptr(), doff.data_ptr(), dcam.data_ptr(),
            dmeas.data_ptr(), 0.1, X.data_ptr(), F.data_ptr(), stream.cuda_stream)
    povar.cost_noalloc(*args)                  # set-up call
    stream.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        povar.cost_noalloc(*args)
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert np.isfinite(F.item())
