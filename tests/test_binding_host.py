"""Marshalling checks of the Python binding (no GPU): the library reads
n_obs entries of each observation array and n_cams x 12 camera values, so the
binding refuses arrays whose sizes disagree before any library call."""
import numpy as np
import pytest

from paper_2405_05079_gb300 import povar


@pytest.fixture(scope="module", autouse=True)
def library():
    """Problem() loads libpovar before it checks its arguments (built here)."""
    from paper_2405_05079_gb300 import build
    build.build()


class Scene:
    def __init__(self, n_cams, n_points, cam_idx, pt_idx, meas):
        self.n_cams, self.n_points, self.n_obs = n_cams, n_points, len(cam_idx)
        self.cam_idx, self.pt_idx, self.meas = cam_idx, pt_idx, meas


def test_observation_arrays_are_checked_and_converted():
    cam, pt, meas = [0, 1, 1], np.array([0, 0, 1], np.int64), np.zeros(6)
    c, p, m = povar._obs_arrays(cam, pt, meas)
    assert (c.dtype, p.dtype, m.dtype, m.shape) == (np.int32, np.int32, np.float64, (3, 2))
    assert c.flags["C_CONTIGUOUS"] and p.flags["C_CONTIGUOUS"] and m.flags["C_CONTIGUOUS"]
    assert np.array_equal(p, [0, 0, 1])
    for args in ((cam, pt[:2], meas), (cam, pt, meas[:4]), (cam[:2], pt, meas)):
        with pytest.raises(ValueError):
            povar._obs_arrays(*args)
    with pytest.raises(ValueError):
        povar._obs_arrays(cam, pt, meas, n_obs=4)


def test_problem_and_batch_refuse_inconsistent_arrays():
    cam, pt, meas = np.array([0, 1, 1]), np.array([0, 0, 1]), np.zeros((3, 2))
    with pytest.raises(ValueError):
        povar.Problem(2, 2, cam, pt[:2], meas)
    with pytest.raises(ValueError):
        povar.Batch([Scene(2, 2, cam, pt, meas), Scene(2, 2, cam, pt, meas[:2])])


def test_batch_cameras_must_match_each_problem():
    b = povar.Batch.__new__(povar.Batch)      # host state only, no handle
    b.n, b.n_cams = 2, np.array([3, 4], np.int32)
    with pytest.raises(ValueError):
        b.set_cameras([np.zeros((3, 12))], 0.1)                     # one array short
    with pytest.raises(ValueError):
        b.set_cameras([np.zeros((4, 12)), np.zeros((3, 12))], 0.1)  # sizes swapped
