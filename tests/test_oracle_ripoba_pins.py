"""Pins of the second-stage (RiPoBA) oracle against what the paper and the
mathematics fix, independently of the oracle's own formulas: finite
differences of the literal reprojection residual, projective invariances,
the joint projected Gauss-Newton system solved densely, Lemma 2, the
tangency of the updates and their basis invariance, and descent."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import ripoba_oracle as R
from paper_2405_05079_gb300 import scenes


@pytest.fixture(scope="module")
def small():
    """A small scene (6 cameras, 60 points) and a perturbed projective start."""
    sc = scenes.ring_scene(6, 60, 3, track="uniform3to6", noise_px=1.0, eta=0.1, m=10,
                           name="ripoba-small")
    P, X = scenes.stage2_start(sc, 2, 0.02)
    pr = R.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    st = pr.init_state(P, X, R.Params())
    return sc, pr, st


def literal_residual(P, X, cam, pt, meas):
    """Eq. second_stage written out per observation with plain Python."""
    out = []
    for k in range(len(cam)):
        Pi = np.asarray(P[cam[k]]).reshape(3, 4)
        y = Pi @ X[pt[k]]
        out.append([y[0] / y[2] - meas[k][0], y[1] / y[2] - meas[k][1]])
    return np.array(out)


def test_residual_is_the_literal_reprojection_error(small):
    sc, pr, st = small
    r = R.residuals(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas)
    assert np.allclose(r, literal_residual(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas),
                       rtol=1e-13, atol=1e-15)


def test_ground_truth_without_noise_has_zero_residual():
    sc = scenes.ring_scene(5, 40, 4, track="uniform3to6", noise_px=0.0, eta=0.1, m=10,
                           name="ripoba-clean")
    P = sc.gt_cams.reshape(-1, 12)
    X = np.concatenate([sc.gt_points, np.ones((sc.n_points, 1))], axis=1)
    assert R.cost(P, X, sc.cam_idx, sc.pt_idx, sc.meas) < 1e-24


def test_projective_invariance(small):
    """pi(a P H  H^-1 X b) = pi(P X) for scalars a, b and any invertible H."""
    sc, pr, st = small
    rng = np.random.default_rng(0)
    H = np.eye(4) + 0.3 * rng.normal(size=(4, 4))
    a = rng.uniform(0.5, 2.0, size=(sc.n_cams, 1))
    b = rng.uniform(-2.0, -0.5, size=(sc.n_points, 1))
    P2 = a * np.einsum("nab,bc->nac", st.P.reshape(-1, 3, 4), H).reshape(-1, 12)
    X2 = b * np.linalg.solve(H, st.X.T).T
    assert abs(pr.cost(P2, X2) - st.F) <= 1e-10 * st.F


def test_jacobians_match_central_differences(small):
    sc, pr, st = small
    Jp, Jl = R.jacobian_blocks(st.P, st.X, sc.cam_idx, sc.pt_idx)
    h = 1e-6
    r0 = lambda P, X: literal_residual(P, X, sc.cam_idx, sc.pt_idx, sc.meas)
    for k in (0, 7, len(sc.cam_idx) - 1):
        i, j = sc.cam_idx[k], sc.pt_idx[k]
        for a in range(12):
            Pp, Pm = st.P.copy(), st.P.copy()
            Pp[i, a] += h
            Pm[i, a] -= h
            fd = (r0(Pp, st.X)[k] - r0(Pm, st.X)[k]) / (2 * h)
            assert np.allclose(Jp[k, :, a], fd, rtol=1e-6, atol=1e-8), (k, a)
        for a in range(4):
            Xp, Xm = st.X.copy(), st.X.copy()
            Xp[j, a] += h
            Xm[j, a] -= h
            fd = (r0(st.P, Xp)[k] - r0(st.P, Xm)[k]) / (2 * h)
            assert np.allclose(Jl[k, :, a], fd, rtol=1e-6, atol=1e-8), (k, a)


def test_scale_directions_are_in_the_jacobians_null_space(small):
    """J_p vec(P_i) = 0 and J_l X_j = 0 per observation (the local scale
    freedom that makes the unprojected normal equation singular, Sec. 4.3)."""
    sc, pr, st = small
    Jp, Jl = R.jacobian_blocks(st.P, st.X, sc.cam_idx, sc.pt_idx)
    assert np.max(np.abs(np.einsum("kra,ka->kr", Jp, st.P[sc.cam_idx]))) < 1e-10
    assert np.max(np.abs(np.einsum("kra,ka->kr", Jl, st.X[sc.pt_idx]))) < 1e-10
    ne = R.normal_equations(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas, sc.n_cams, sc.n_points)
    for i in range(sc.n_cams):
        assert np.linalg.norm(ne.U[i] @ st.P[i]) < 1e-9 * np.linalg.norm(ne.U[i])


def test_gradient_is_twice_J_transpose_r(small):
    """b = J^T r is half the gradient of the cost (central differences)."""
    sc, pr, st = small
    ne = R.normal_equations(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas, sc.n_cams, sc.n_points)
    h = 1e-6
    for (i, a) in ((0, 3), (4, 10)):
        Pp, Pm = st.P.copy(), st.P.copy()
        Pp[i, a] += h
        Pm[i, a] -= h
        fd = (pr.cost(Pp, st.X) - pr.cost(Pm, st.X)) / (2 * h)
        assert abs(fd - 2 * ne.b_p[12 * i + a]) <= 1e-6 * max(abs(fd), 1e-8)
    for (j, a) in ((0, 0), (33, 3)):
        Xp, Xm = st.X.copy(), st.X.copy()
        Xp[j, a] += h
        Xm[j, a] -= h
        fd = (pr.cost(st.P, Xp) - pr.cost(st.P, Xm)) / (2 * h)
        assert abs(fd - 2 * ne.b_l[4 * j + a]) <= 1e-6 * max(abs(fd), 1e-8)


def joint_tangent_step(sc, st, lam, lambda_l):
    """The damped Gauss-Newton step of the full projected system, built from
    the dense Jacobian times dense tangent bases (no Schur complement)."""
    Jp, Jl = R.jacobian_blocks(st.P, st.X, sc.cam_idx, sc.pt_idx)
    J = R.assemble_jacobian(Jp, Jl, sc.cam_idx, sc.pt_idx, sc.n_cams, sc.n_points).toarray()
    r = R.residuals(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas).ravel()
    Qp = R.sphere_tangent_bases(st.P)
    Ql = R.sphere_tangent_bases(st.X)
    Q = sla.block_diag(*Qp, *Ql)
    Jt = J @ Q
    npv = 11 * sc.n_cams
    D = np.concatenate([np.full(npv, lam), np.full(Jt.shape[1] - npv, lambda_l * lam)])
    d = np.linalg.solve(Jt.T @ Jt + np.diag(D), -Jt.T @ r)
    full = Q @ d
    return full[:12 * sc.n_cams].reshape(-1, 12), full[12 * sc.n_cams:].reshape(-1, 4)


@pytest.mark.parametrize("lambda_l", [1.0, 0.3])
def test_schur_step_is_the_joint_projected_gauss_newton_step(small, lambda_l):
    sc, pr, st = small
    st = R.State(P=st.P, X=st.X, F=st.F, lam=1e-3)
    _, rep = pr.step(st, R.Params(solver="exact", lambda_l=lambda_l))
    dP, dX = joint_tangent_step(sc, st, 1e-3, lambda_l)
    assert np.allclose(rep.dP, dP, rtol=1e-7, atol=1e-10 * np.abs(dP).max())
    assert np.allclose(rep.dX, dX, rtol=1e-7, atol=1e-10 * np.abs(dX).max())


def test_lemma2_eigenvalues_in_unit_interval(small):
    sc, pr, st = small
    for lam in (1e-6, 1e-2, 10.0):
        s2 = R.State(P=st.P, X=st.X, F=st.F, lam=lam)
        _, rsys, rs = pr.system(s2, R.Params())
        Uinv = sla.block_diag(*[np.linalg.inv(b) for b in rsys.Ut])
        M = Uinv @ (rs.Wt @ rs.Vinv @ rs.Wt.T).toarray()
        ev = np.linalg.eigvals(M)
        assert np.max(np.abs(ev.imag)) < 1e-8
        assert ev.real.min() > -1e-10 and ev.real.max() < 1.0


def test_series_converges_to_the_exact_step(small):
    """Proposition 1 applied to S~: the truncation error after m terms is
    M^m applied to the exact step, so it decays at least like rho(M)^m."""
    sc, pr, st = small
    s2 = R.State(P=st.P, X=st.X, F=st.F, lam=0.1)
    _, rsys, rs = pr.system(s2, R.Params())
    Uinv = sla.block_diag(*[np.linalg.inv(b) for b in rsys.Ut])
    M = Uinv @ (rs.Wt @ rs.Vinv @ rs.Wt.T).toarray()
    rho = float(np.max(np.abs(np.linalg.eigvals(M))))
    _, ex = pr.step(s2, R.Params(solver="exact"))
    errs = []
    for m in (1, 10, 100, 1000):
        _, se = pr.step(s2, R.Params(m=m))
        errs.append(np.linalg.norm(se.dP - ex.dP) / np.linalg.norm(ex.dP))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6
    # the error is the remainder sum_{i>=m} M^i x0 = M^m d*: exactly
    ex_t = np.linalg.solve(rs.S, rs.g)
    _, se = pr.step(s2, R.Params(m=10))
    rem = np.linalg.matrix_power(M, 10) @ ex_t
    se_t = np.einsum("nab,na->nb", rsys.Qp, se.dP).ravel()
    assert np.allclose(ex_t - se_t, rem, rtol=1e-6, atol=1e-9 * np.abs(ex_t).max())
    assert rho < 1.0


def test_updates_are_tangent_and_retraction_normalizes(small):
    sc, pr, st = small
    new, rep = pr.step(st, R.Params(m=10))
    assert np.max(np.abs(np.sum(rep.dP * st.P, axis=1))) < 1e-12
    assert np.max(np.abs(np.sum(rep.dX * st.X, axis=1))) < 1e-12
    if rep.accepted:
        assert np.allclose(np.linalg.norm(new.P, axis=1), 1.0, atol=1e-14)
        assert np.allclose(np.linalg.norm(new.X, axis=1), 1.0, atol=1e-14)


def test_step_is_invariant_to_the_tangent_basis(small):
    sc, pr, st = small
    ne = R.normal_equations(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas, sc.n_cams, sc.n_points)
    rng = np.random.default_rng(1)
    out = []
    for rot in (False, True):
        Qp = R.sphere_tangent_bases(st.P)
        Ql = R.sphere_tangent_bases(st.X)
        if rot:
            Qp = np.einsum("nab,nbc->nac", Qp, np.linalg.qr(rng.normal(size=(sc.n_cams, 11, 11)))[0])
            Ql = np.einsum("nab,nbc->nac", Ql, np.linalg.qr(rng.normal(size=(sc.n_points, 3, 3)))[0])
        rsys = R.riemannian_system(ne, Qp, Ql, 1e-3, 1.0)
        rs = R.reduced(rsys)
        dp = np.linalg.solve(rs.S, rs.g)
        dl = R.back_substitute(rsys, rs, dp)
        out.append((np.einsum("nab,nb->na", Qp, dp.reshape(sc.n_cams, -1)),
                    np.einsum("nab,nb->na", Ql, dl.reshape(sc.n_points, -1))))
    assert np.allclose(out[0][0], out[1][0], rtol=1e-8, atol=1e-12)
    assert np.allclose(out[0][1], out[1][1], rtol=1e-8, atol=1e-12)


def test_pred_is_the_gauss_newton_model_decrease(small):
    sc, pr, st = small
    _, rep = pr.step(st, R.Params(m=8))
    Jp, Jl = R.jacobian_blocks(st.P, st.X, sc.cam_idx, sc.pt_idx)
    J = R.assemble_jacobian(Jp, Jl, sc.cam_idx, sc.pt_idx, sc.n_cams, sc.n_points)
    r = literal_residual(st.P, st.X, sc.cam_idx, sc.pt_idx, sc.meas).ravel()
    d = np.concatenate([rep.dP.ravel(), rep.dX.ravel()])
    model = r @ r - np.sum((r + J @ d) ** 2)
    assert abs(rep.pred - model) <= 1e-10 * abs(model)
    assert rep.pred > 0


def test_accepted_steps_descend_to_below_the_ground_truth_cost():
    """From a perturbed projective start, RiPoBA's accepted steps never raise
    the cost and end below the cost of the noisy ground truth (the
    maximum-likelihood fit of the noise)."""
    sc = scenes.ring_scene(8, 150, 5, track="uniform3to6", noise_px=1.0, eta=0.1, m=10,
                           name="ripoba-descent")
    P, X = scenes.stage2_start(sc, 3, 0.02)
    pr = R.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    st = pr.init_state(P, X, R.Params())
    st, trace = pr.solve(st, R.Params(m=21, series_eps=0.01), max_iters=40, ftol=1e-10)
    assert all(b <= a for a, b in zip(trace, trace[1:]))
    Pg = sc.gt_cams.reshape(-1, 12)
    Xg = np.concatenate([sc.gt_points, np.ones((sc.n_points, 1))], axis=1)
    assert trace[-1] < pr.cost(Pg, Xg) < trace[0]
