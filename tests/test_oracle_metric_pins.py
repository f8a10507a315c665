"""Pins of the metric-upgrade oracle (supplementary "Metric Upgrade") against
what the geometry fixes: a projective distortion of metric cameras is undone
exactly (zero cost, cameras that are scaled rotations with the ground
truth's relative rotations), the Jacobian matches central differences of the
literal residual, the closed-form scale is the 1-D least-squares solution,
and the reduced cost ignores the scale of each camera."""
import numpy as np
import pytest

from oracle import metric_oracle as MU
from paper_2405_05079_gb300 import scenes


def distorted(seed, n_cams=12, spread=0.1):
    """Metric ground-truth cameras [R | t] of a ring scene, moved by a random
    projective transformation and scaled per camera (random sign)."""
    sc = scenes.ring_scene(n_cams, 50, seed, track="uniform3to6", noise_px=0.0, eta=0.1, m=10,
                           name="mu")
    rng = np.random.default_rng(seed)
    H = np.eye(4) + spread * rng.normal(size=(4, 4))
    s = rng.uniform(0.5, 2.0, n_cams) * rng.choice([-1.0, 1.0], n_cams)
    P = s[:, None, None] * np.einsum("nab,bc->nac", sc.gt_cams, H)
    return sc, P.reshape(n_cams, 12)


def literal_residual(P, c):
    """The paper's residual alpha_i (P_i H0) H~ H~^T (P_i H0)^T - I with the
    best alpha_i, written out camera by camera (K = I)."""
    H0 = MU.frame_to_reference(P[0])
    Ht = np.vstack([np.eye(3), np.asarray(c)[None, :]])
    out = []
    for i in range(P.shape[0]):
        B = P[i].reshape(3, 4) @ H0
        M = B @ Ht @ Ht.T @ B.T
        a = np.trace(M) / np.sum(M * M)
        out.append((a * M - np.eye(3)).ravel())
    return np.array(out)


def test_linear_start_is_exact_without_noise():
    """Noise-free cameras: the linear estimate of the dual absolute quadric
    already is the metric solution (c = -T[3, :3] / T[3, 3] for the frame map
    T = H_true H_0, read off the construction)."""
    sc, P = distorted(8)
    rng = np.random.default_rng(8)
    H = np.eye(4) + 0.1 * rng.normal(size=(4, 4))
    H0 = MU.frame_to_reference(P[0])
    T = H @ H0
    c_true = -T[3, :3] / T[3, 3]
    B = MU.upgrade_blocks(P, np.broadcast_to(np.eye(3), (P.shape[0], 3, 3)), H0)
    assert np.allclose(MU.linear_start(B), c_true, atol=1e-9)
    assert MU.cost(B, c_true) < 1e-20


def test_reference_camera_becomes_canonical():
    _, P = distorted(1)
    H0 = MU.frame_to_reference(P[0])
    assert np.allclose(P[0].reshape(3, 4) @ H0, np.hstack([np.eye(3), np.zeros((3, 1))]),
                       atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_projective_distortion_is_undone(seed):
    sc, P = distorted(seed)
    res = MU.upgrade(P)
    assert res.cost < 1e-18
    # the upgraded cameras' left 3x3 blocks are scaled rotations carrying the
    # ground truth's rotations relative to camera 0 (up to one global sign)
    R0 = sc.gt_cams[0][:, :3]
    for i in range(P.shape[0]):
        N = (P[i].reshape(3, 4) @ res.H)[:, :3]
        N = N / np.cbrt(np.linalg.det(N))
        assert np.allclose(N.T @ N, np.eye(3), atol=1e-8)
        Rrel = sc.gt_cams[i][:, :3] @ R0.T
        assert np.allclose(N, Rrel, atol=1e-7) or np.allclose(N, -Rrel, atol=1e-7), i


def test_jacobian_matches_central_differences():
    _, P = distorted(4, spread=0.2)
    H0 = MU.frame_to_reference(P[0])
    B = MU.upgrade_blocks(P, np.broadcast_to(np.eye(3), (P.shape[0], 3, 3)), H0)
    c = np.array([0.3, -0.2, 0.1])
    J = MU.jacobian(B, c)
    h = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (literal_residual(P, c + e) - literal_residual(P, c - e)) / (2 * h)
        assert np.allclose(J[:, :, k], fd, rtol=1e-6, atol=1e-8), k
    assert np.allclose(MU.residuals(B, c), literal_residual(P, c), atol=1e-13)


def test_closed_form_scale_is_the_least_squares_scale():
    _, P = distorted(5, spread=0.2)
    H0 = MU.frame_to_reference(P[0])
    B = MU.upgrade_blocks(P, np.broadcast_to(np.eye(3), (P.shape[0], 3, 3)), H0)
    M = MU.m_blocks(B, np.array([0.1, 0.2, -0.3]))
    a = MU.alphas(M)
    for i in range(M.shape[0]):
        ls, *_ = np.linalg.lstsq(M[i].reshape(9, 1), np.eye(3).ravel(), rcond=None)
        assert abs(a[i] - ls[0]) <= 1e-12 * abs(ls[0])


def test_cost_ignores_the_scale_of_each_camera():
    _, P = distorted(6, spread=0.2)
    rng = np.random.default_rng(0)
    P2 = P * rng.uniform(-3.0, 3.0, (P.shape[0], 1))
    P2[0] = P[0]     # the reference frame is defined by camera 0 as given
    K = np.broadcast_to(np.eye(3), (P.shape[0], 3, 3))
    H0 = MU.frame_to_reference(P[0])
    c = np.array([0.2, 0.1, -0.4])
    assert abs(MU.cost(MU.upgrade_blocks(P, K, H0), c)
               - MU.cost(MU.upgrade_blocks(P2, K, H0), c)) <= 1e-12


def test_accepted_steps_never_raise_the_cost():
    _, P = distorted(7, spread=0.3)
    res = MU.upgrade(P, max_iters=60)
    assert all(b <= a for a, b in zip(res.trace, res.trace[1:]))
    assert res.trace[-1] < res.trace[0]


def test_known_intrinsics_are_removed_first():
    """Cameras K_i [R_i | t_i] H with per-camera intrinsics (focal length and
    principal point): given K_i, the upgrade is exact again; ignoring them
    (K = I) leaves a positive cost."""
    sc, P = distorted(9)
    rng = np.random.default_rng(9)
    n = P.shape[0]
    K = np.zeros((n, 3, 3))
    for i in range(n):
        f = rng.uniform(0.5, 2.0)
        K[i] = [[f, 0.0, rng.uniform(-0.2, 0.2)], [0.0, 1.1 * f, rng.uniform(-0.2, 0.2)],
                [0.0, 0.0, 1.0]]
    PK = np.einsum("nab,nbc->nac", K, P.reshape(n, 3, 4)).reshape(n, 12)
    assert MU.upgrade(PK, K=K).cost < 1e-18
    assert MU.upgrade(PK).cost > 1e-6
