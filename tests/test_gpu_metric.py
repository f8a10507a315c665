"""Parity of the GPU metric upgrade (supplementary section "Metric Upgrade")
with the FP64 CPU oracle (oracle/metric_oracle.py), and the stratified
pipeline's last step on a refined reconstruction.

Tolerances: everything is FP64 on both sides; H, the scales and the cost
agree to 1e-9 relative (the linear start's null vector comes from inverse
iteration on the GPU and from an SVD in the oracle, which differ by
rounding; the Levenberg-Marquardt iterations then converge to the same
point)."""
import numpy as np
import pytest

from oracle import metric_oracle as MU
from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu


def distorted(seed, n_cams=12, spread=0.1, noise=0.0):
    sc = scenes.ring_scene(n_cams, 200, seed, track="uniform3to6", noise_px=1.0, eta=0.1, m=10,
                           name="mu")
    rng = np.random.default_rng(seed)
    H = np.eye(4) + spread * rng.normal(size=(4, 4))
    s = rng.uniform(0.5, 2.0, n_cams) * rng.choice([-1.0, 1.0], n_cams)
    P = s[:, None, None] * np.einsum("nab,bc->nac", sc.gt_cams, H)
    P = P.reshape(n_cams, 12)
    P = P + noise * np.abs(P).mean() * rng.normal(size=P.shape)
    return sc, P


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def h_diff(H, Href):
    """Difference of two upgrades of the same cameras. The first three
    columns of H = H_0 [[I, 0], [c^T, 1]] do not depend on how H_0 completes
    the reference camera (a scale k of the completing row scales H_0's last
    column by 1/k and c by k); the last column is the reconstruction's
    global scale and sign, so it is compared up to a factor."""
    d3 = rel(H[:, :3], Href[:, :3])
    h, hr = H[:, 3], Href[:, 3]
    s = np.dot(h, hr) / np.dot(hr, hr)
    return max(d3, rel(h / s, hr))


@pytest.mark.parametrize("seed,noise", [(1, 0.0), (2, 0.0), (3, 1e-3), (4, 1e-2)])
def test_metric_upgrade_matches_oracle(seed, noise):
    sc, P = distorted(seed, noise=noise)
    ref = MU.upgrade(P, max_iters=100, ftol=1e-12)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P, sc.eta)
        H, al, cost, it = pb.metric_upgrade(max_iters=100, ftol=1e-12)
    assert h_diff(H, ref.H) <= 1e-9
    assert rel(al, ref.alpha) <= 1e-9
    if noise == 0.0:
        assert cost < 1e-18 and ref.cost < 1e-18
    else:
        assert abs(cost - ref.cost) <= 1e-9 * ref.cost
        assert it == ref.iterations


def test_metric_upgrade_with_intrinsics_matches_oracle():
    sc, P = distorted(5)
    rng = np.random.default_rng(5)
    n = P.shape[0]
    K = np.zeros((n, 3, 3))
    for i in range(n):
        f = rng.uniform(0.5, 2.0)
        K[i] = [[f, 0.0, rng.uniform(-0.2, 0.2)], [0.0, 1.1 * f, rng.uniform(-0.2, 0.2)],
                [0.0, 0.0, 1.0]]
    PK = np.einsum("nab,nbc->nac", K, P.reshape(n, 3, 4)).reshape(n, 12)
    ref = MU.upgrade(PK, K=K)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(PK, sc.eta)
        H, al, cost, _ = pb.metric_upgrade(K=K)
    assert cost < 1e-18
    assert h_diff(H, ref.H) <= 1e-9


def test_stratified_pipeline_ends_metric():
    """Second stage from a projective start near the optimum, then the
    upgrade: the upgraded cameras are scaled rotations close to the ground
    truth's rotations relative to camera 0."""
    sc = scenes.ring_scene(20, 1500, 11, track="geom3", noise_px=0.5, eta=0.1, m=10, name="pipe")
    P, X = scenes.stage2_start(sc, 3, 0.01)
    with povar.Problem.from_scene(sc) as pb:
        pb.s2_set(P, X)
        pb.s2_solve(povar.make_s2_params(m=21, series_eps=0.01, precision=povar.FP64),
                    max_iters=50, ftol=1e-10)
        Pr = pb.cameras()
        H, al, cost, _ = pb.metric_upgrade()
    R0 = sc.gt_cams[0][:, :3]
    for i in range(sc.n_cams):
        N = (Pr[i].reshape(3, 4) @ H)[:, :3]
        N = N / np.cbrt(np.linalg.det(N))
        assert np.abs(N.T @ N - np.eye(3)).max() < 1e-2, i
        Rrel = sc.gt_cams[i][:, :3] @ R0.T
        err = min(np.abs(N - Rrel).max(), np.abs(N + Rrel).max())
        assert err < 2e-2, (i, err)


def test_metric_upgrade_invalid_calls():
    sc, P = distorted(6)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P, sc.eta)
        K = np.broadcast_to(np.eye(3), (sc.n_cams, 3, 3)).copy()
        K[3] = 0.0
        with pytest.raises(povar.PovarError) as e:
            pb.metric_upgrade(K=K)
        assert e.value.status == 1
        K[3] = np.eye(3)
        K[4, 0, 0] = np.nan
        with pytest.raises(povar.PovarError):
            pb.metric_upgrade(K=K)
        H, _, _, _ = pb.metric_upgrade()       # still usable afterwards
        assert np.isfinite(H).all()
