"""Pins for the FP64 CPU oracle: each test checks the oracle against something
other than itself -- finite differences of the literal pOSE residual, the
library least-squares solver, exact quadratic expansions of the residual, the
joint (non-reduced) normal equations, Lemma 1 / Lemma 2, the Proposition 1
error bound, and the textbook affine-factorization optimum.

A plausible mistake in the oracle (dropped term, wrong sign, transposed
operand, wrong index) fails at least one of these.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import povar_oracle as O
from paper_2405_05079_gb300 import scenes


def _state(sc, seed=1, normalize=True, eta=None):
    eta = sc.eta if eta is None else eta
    P = scenes.init_cameras(sc.n_cams, seed, normalize=normalize)
    pr = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    X = pr.landmarks(P, eta)
    return pr, P, X, eta


# --------------------------------------------------------------- Jacobians

def test_jacobian_blocks_match_central_differences(micro):
    pr, P, X, eta = _state(micro)
    Jp, Jl = O.jacobian_blocks(P, X, pr.cam_idx, pr.pt_idx, pr.meas, eta)
    h = 1e-6
    rng = np.random.default_rng(0)
    for k in rng.choice(len(pr.cam_idx), size=12, replace=False):
        i, j = pr.cam_idx[k], pr.pt_idx[k]
        sel = np.array([k])

        def res(Pi, Xj):
            P2 = P.copy(); P2[i] = Pi
            X2 = X.copy(); X2[j] = Xj
            return O.pose_residuals(P2, X2, pr.cam_idx[sel], pr.pt_idx[sel],
                                    pr.meas[sel], eta)[0]
        fd_p = np.stack([(res(P[i] + h * e, X[j]) - res(P[i] - h * e, X[j])) / (2 * h)
                         for e in np.eye(12)], axis=1)
        fd_l = np.stack([(res(P[i], X[j] + h * e) - res(P[i], X[j] - h * e)) / (2 * h)
                         for e in np.eye(3)], axis=1)
        assert np.allclose(Jp[k], fd_p, rtol=1e-7, atol=1e-8 * np.abs(Jp[k]).max())
        assert np.allclose(Jl[k], fd_l, rtol=1e-7, atol=1e-8 * np.abs(Jl[k]).max())


def test_residual_at_ground_truth_without_noise():
    """Noise-free scene with the true cameras [R|t] (normalized coordinates)
    and true points: the OSE rows of Eq. pose vanish for any eta, and the
    affine rows equal sqrt(eta) (z - 1) m, z the point's depth."""
    sc = scenes.ring_scene(5, 30, 7, noise_px=0.0, eta=0.3)
    P = sc.gt_cams.reshape(sc.n_cams, 12)
    Xw = sc.gt_points[sc.pt_idx]
    R = sc.gt_cams[sc.cam_idx, :, :3]
    t = sc.gt_cams[sc.cam_idx, :, 3]
    z = np.einsum("nj,nj->n", R[:, 2], Xw) + t[:, 2]
    for eta in (0.0, 0.3, 1.0):
        r = O.pose_residuals(P, sc.gt_points, sc.cam_idx, sc.pt_idx, sc.meas, eta)
        assert np.abs(r[:, :2]).max() < 1e-12
        assert np.allclose(r[:, 2:], np.sqrt(eta) * (z - 1.0)[:, None] * sc.meas,
                           rtol=1e-12, atol=1e-14)


def test_residual_weights():
    """eta = 1 keeps only the affine rows, eta = 0 only the OSE rows."""
    sc = scenes.ring_scene(3, 10, 2)
    P = scenes.init_cameras(3, 5, normalize=False)
    X = np.random.default_rng(1).normal(size=(10, 3))
    r1 = O.pose_residuals(P, X, sc.cam_idx, sc.pt_idx, sc.meas, 1.0)
    r0 = O.pose_residuals(P, X, sc.cam_idx, sc.pt_idx, sc.meas, 0.0)
    assert np.all(r1[:, :2] == 0) and np.all(r0[:, 2:] == 0)
    # affine rows at eta=1: P^{1:2} x~ - m
    y = np.einsum("nij,nj->ni", P.reshape(-1, 3, 4)[sc.cam_idx],
                  np.c_[X[sc.pt_idx], np.ones(sc.n_obs)])
    assert np.allclose(r1[:, 2:], y[:, :2] - sc.meas)
    # OSE rows at eta=0 vanish when the measurement equals the projection
    m_exact = y[:, :2] / y[:, 2:3]
    r0e = O.pose_residuals(P, X, sc.cam_idx, sc.pt_idx, m_exact, 0.0)
    assert np.abs(r0e).max() < 1e-10


# --------------------------------------------------------------- landmarks

def test_landmarks_match_bruteforce_lstsq(tiny):
    pr, P, X, eta = _state(tiny)
    Xb = O.landmark_bruteforce(P, pr.cam_idx, pr.pt_idx, pr.meas, eta, pr.n_points)
    scale = np.abs(Xb).max(axis=1, keepdims=True)
    assert np.all(np.abs(X - Xb) <= 1e-8 * np.maximum(scale, 1.0))


def test_pseudo_inverse_branch_gives_minimum_norm_landmarks(tiny):
    """At eta = 0 an observation constrains its landmark only through the two
    rows of the projective error (B_k has rank 2), so a landmark seen once
    has a singular V_j (footnote of Sec. 4.2: pseudo-inverse). The minimum-norm
    least-squares solution of its stacked 4k x 3 system -- what the library
    least-squares solver returns -- is V_j^+ (-h_j), so the pseudo-inverse
    branch must reproduce landmark_bruteforce exactly where V_j is singular,
    and the ordinary inverse must reproduce it where it is not."""
    pr0, P, _, _ = _state(tiny)
    keep = np.ones(len(pr0.pt_idx), bool)
    single = np.arange(0, pr0.n_points, 3)            # every third landmark: one view
    for j in single:
        ks = np.nonzero(pr0.pt_idx == j)[0]
        keep[ks[1:]] = False
    cam, pt, meas = pr0.cam_idx[keep], pr0.pt_idx[keep], pr0.meas[keep]
    assert np.all(np.bincount(pt, minlength=pr0.n_points)[single] == 1)
    X, V, n_pinv = O.landmarks(P, cam, pt, meas, 0.0, pr0.n_points, return_V=True)
    assert n_pinv == len(single)                       # exactly the single-view landmarks
    Xb = O.landmark_bruteforce(P, cam, pt, meas, 0.0, pr0.n_points)
    scale = np.maximum(np.abs(Xb).max(axis=1, keepdims=True), 1.0)
    assert np.all(np.abs(X - Xb) <= 1e-8 * scale)
    # the single-view solutions are minimum-norm: orthogonal to the null space of V_j
    for j in single[:20]:
        w, E = np.linalg.eigh(V[j])
        assert abs(E[:, 0] @ X[j]) <= 1e-8 * max(1.0, np.linalg.norm(X[j]))
    # and solve the consistent 2x3 projective system exactly (zero residual)
    F_single = O.cost(P, X, cam, pt, meas, 0.0)
    sel = np.isin(pt, single)
    r = O.pose_residuals(P, X, cam[sel], pt[sel], meas[sel], 0.0)
    assert np.abs(r).max() <= 1e-9 * max(1.0, F_single)


def test_sym_inverse_batch_picks_the_branch_by_condition():
    """Blocks with a known spectrum: a well-conditioned block gets its
    inverse, a block with a zero eigenvalue and one with cond = 1e14 get the
    pseudo-inverse E diag(1/w or 0) E^T, written out from the construction."""
    rng = np.random.default_rng(4)
    E, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    spectra = [np.array([3.0, 2.0, 0.5]), np.array([3.0, 2.0, 0.0]),
               np.array([3.0, 2.0, 3e-14])]
    V = np.stack([E @ np.diag(w) @ E.T for w in spectra])
    inv, n_pinv = O.sym_inverse_batch(V)
    assert n_pinv == 2
    for k, w in enumerate(spectra):
        keep = w > w.max() / O.PINV_COND
        d = np.where(keep, 1.0 / np.where(keep, w, 1.0), 0.0)
        assert np.allclose(inv[k], E @ np.diag(d) @ E.T, rtol=1e-9, atol=1e-9)


def test_landmark_first_order_optimality(tiny):
    """b_l = J_l^T r = 0 at X*(P) (first-order optimality of Eq. update_landmark)."""
    pr, P, X, eta = _state(tiny)
    ne = pr.normal_equations(P, X, eta)
    Jl_scale = np.sqrt(np.einsum("nii->n", ne.V)).repeat(3)
    assert np.all(np.abs(ne.b_l) <= 1e-9 * np.maximum(Jl_scale, 1.0))


def test_landmark_is_minimizer(micro):
    """Random perturbations of X*(P) never lower the cost."""
    pr, P, X, eta = _state(micro)
    F = pr.cost(P, X, eta)
    rng = np.random.default_rng(3)
    for _ in range(20):
        X2 = X + 1e-3 * rng.normal(size=X.shape)
        assert pr.cost(P, X2, eta) >= F - 1e-12 * F


# --------------------------------------------------------------- normal equation

def test_normal_equation_blocks_from_residual_differences(micro):
    """pOSE is linear in the cameras for fixed landmarks and affine in the
    landmarks for fixed cameras, so the residual differences are exact:
    J_p D = r(P + D, X) - r(P, X), J_l E = r(P, X + E) - r(P, X).
    U, V, W, b_p, b_l are pinned through these differences, independently of
    the Jacobian formulas."""
    pr, P, X, eta = _state(micro)
    ne = pr.normal_equations(P, X, eta)
    rng = np.random.default_rng(4)
    r0 = O.pose_residuals(P, X, pr.cam_idx, pr.pt_idx, pr.meas, eta).ravel()
    for _ in range(5):
        D = rng.normal(size=P.shape)
        E = rng.normal(size=X.shape)
        JpD = O.pose_residuals(P + D, X, pr.cam_idx, pr.pt_idx, pr.meas, eta).ravel() - r0
        JlE = O.pose_residuals(P, X + E, pr.cam_idx, pr.pt_idx, pr.meas, eta).ravel() - r0
        d = D.ravel()
        e = E.ravel()
        UD = np.concatenate([ne.U[i] @ D[i] for i in range(pr.n_cams)])
        VE = np.concatenate([ne.V[j] @ E[j] for j in range(pr.n_points)])
        tol = 1e-10 * (np.linalg.norm(JpD) + np.linalg.norm(JlE)) ** 2
        assert abs(d @ UD - JpD @ JpD) <= tol
        assert abs(e @ VE - JlE @ JlE) <= tol
        assert abs(d @ (ne.W @ e) - JpD @ JlE) <= tol
        assert abs(d @ ne.b_p - r0 @ JpD) <= 1e-10 * np.linalg.norm(r0) * np.linalg.norm(JpD)
        assert abs(e @ ne.b_l - r0 @ JlE) <= 1e-10 * np.linalg.norm(r0) * np.linalg.norm(JlE)


def test_b_p_is_half_gradient_of_reduced_cost(micro):
    """Envelope theorem on the reduced VarPro cost F*(P) = min_X F(P, X)
    (Eq. reduced_varpro): dF*/dP = 2 J_p^T r at X*(P), i.e. b_p = grad/2.
    Checked by central differences of F*, which re-solves the landmarks by
    brute-force least squares at every perturbed camera."""
    pr, P, X, eta = _state(micro)
    ne = pr.normal_equations(P, X, eta)

    def Fstar(Pp):
        Xp = O.landmark_bruteforce(Pp, pr.cam_idx, pr.pt_idx, pr.meas, eta, pr.n_points)
        return pr.cost(Pp, Xp, eta)
    h = 1e-6
    rng = np.random.default_rng(5)
    for _ in range(4):
        i, a = rng.integers(pr.n_cams), rng.integers(12)
        Pp = P.copy(); Pp[i, a] += h
        Pm = P.copy(); Pm[i, a] -= h
        g = (Fstar(Pp) - Fstar(Pm)) / (2 * h)
        assert abs(0.5 * g - ne.b_p[12 * i + a]) <= 1e-6 * max(1.0, abs(g))


# --------------------------------------------------------------- reduced system

def _joint_step(pr, P, X, eta, lam, manifold):
    """Solve the joint damped system [[Q^T U Q + lam I, Q^T W], [W^T Q, V]]
    with the library dense solver (no Schur complement) for the camera part."""
    ne = pr.normal_equations(P, X, eta)
    Q = O.tangent_bases(P, manifold)
    k = Q.shape[2]
    Qbd = O.blockdiag(Q).toarray()
    nc = pr.n_cams
    Upp = sla.block_diag(*ne.U)
    H = np.zeros((k * nc + 3 * pr.n_points,) * 2)
    H[:k * nc, :k * nc] = Qbd.T @ Upp @ Qbd + lam * np.eye(k * nc)
    W = ne.W.toarray()
    H[:k * nc, k * nc:] = Qbd.T @ W
    H[k * nc:, :k * nc] = (Qbd.T @ W).T
    H[k * nc:, k * nc:] = sla.block_diag(*ne.V)
    rhs = -np.concatenate([Qbd.T @ ne.b_p, ne.b_l])
    sol = np.linalg.solve(H, rhs)
    return sol[:k * nc], ne, Q


@pytest.mark.parametrize("manifold", [O.EUCLID, O.SPHERE])
@pytest.mark.parametrize("off_optimum", [False, True])
def test_schur_step_equals_joint_normal_equation_solve(micro, manifold, off_optimum):
    """Eq. pose_update (sign reading: S dx = -(b_p - W V^-1 b_l)) and its
    tangent version give the camera block of the joint Gauss-Newton system.
    Off the landmark optimum b_l != 0, so the b_l term is exercised too."""
    pr, P, X, eta = _state(micro)
    if off_optimum:
        X = X + 0.05 * np.random.default_rng(9).normal(size=X.shape)
    lam = 1e-3
    d_joint, ne, Q = _joint_step(pr, P, X, eta, lam, manifold)
    assert np.abs(ne.b_l).max() > (1e-3 if off_optimum else -1)
    rs = O.reduced_system(ne, Q, lam)
    d = O.exact_step(rs)
    assert np.allclose(d, d_joint, rtol=1e-8, atol=1e-10 * np.abs(d_joint).max())


@pytest.mark.parametrize("manifold", [O.EUCLID, O.SPHERE])
def test_lemma_eigenvalues_in_unit_interval(micro, manifold):
    """Lemma 1 (EUCLID) / Lemma 2 (tangent space): eig(U~^-1 W~ V^-1 W~^T) in [0, 1)."""
    pr, P, X, eta = _state(micro)
    ne = pr.normal_equations(P, X, eta)
    Q = O.tangent_bases(P, manifold)
    for lam in (1e-4, 1e-1, 10.0):
        M = O.series_matrix(O.reduced_system(ne, Q, lam))
        mu = np.linalg.eigvals(M)
        assert np.abs(mu.imag).max() < 1e-8
        assert mu.real.min() > -1e-10 and mu.real.max() < 1.0


@pytest.mark.parametrize("manifold", [O.EUCLID, O.SPHERE])
def test_series_converges_with_proposition1_bound(micro, manifold):
    """delta(m) -> S^-1 g, and in the U~-energy norm (where M is self-adjoint)
    ||S^-1 g - delta(m)|| <= rho^m / (1 - rho) ||U~^-1 g|| (Proposition 1 with
    the m-terms index convention)."""
    pr, P, X, eta = _state(micro)
    ne = pr.normal_equations(P, X, eta)
    Q = O.tangent_bases(P, manifold)
    rs = O.reduced_system(ne, Q, 1e-2)
    exact = O.exact_step(rs)
    M = O.series_matrix(rs)
    rho = np.abs(np.linalg.eigvals(M)).max()
    Ubd = sla.block_diag(*rs.Ut)
    x0 = np.linalg.solve(Ubd, rs.g)

    def enorm(v):
        return np.sqrt(v @ Ubd @ v)
    errs = []
    for m in (1, 2, 5, 10, 40, 200):
        d, terms = O.series_step(rs, m, 0.0)
        assert terms == m
        err = enorm(exact - d)
        assert err <= rho ** m / (1 - rho) * enorm(x0) * (1 + 1e-8) + 1e-14
        errs.append(err)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-3 * enorm(exact) or rho > 0.9


def test_exact_step_falls_back_to_floored_eigen_solve():
    """When rounding leaves S numerically indefinite, exact_step solves with
    every eigenvalue floored at lambda (S >= lambda I holds in exact
    arithmetic). S is built from a known orthonormal E and spectrum w with a
    negative entry, so Cholesky fails; the expected step
    E diag(1 / max(w, lambda)) E^T g is written from the construction."""
    rng = np.random.default_rng(5)
    n = 12
    E, _ = np.linalg.qr(rng.normal(size=(n, n)))
    w = np.geomspace(10.0, 1e-3, n)
    w[-1] = -0.02                     # indefinite: Cholesky must fail
    w[-2] = 0.004                     # below lambda: floored too
    lam = 0.01
    S = E @ np.diag(w) @ E.T
    S = 0.5 * (S + S.T)
    g = rng.normal(size=n)
    with pytest.raises(np.linalg.LinAlgError):
        sla.cho_factor(S, lower=True)
    rs = O.ReducedSystem(Ut=None, Wt=None, Vinv=None, S=S, g=g, Q=None, lam=lam)
    d = O.exact_step(rs)
    expect = E @ ((E.T @ g) / np.maximum(w, lam))
    assert np.allclose(d, expect, rtol=1e-10, atol=1e-12 * np.linalg.norm(expect))
    # an SPD S takes the Cholesky branch: the plain solve
    S_pd = E @ np.diag(np.abs(w) + lam) @ E.T
    rs_pd = O.ReducedSystem(Ut=None, Wt=None, Vinv=None, S=0.5 * (S_pd + S_pd.T), g=g, Q=None,
                            lam=lam)
    expect_pd = E @ ((E.T @ g) / (np.abs(w) + lam))
    assert np.allclose(O.exact_step(rs_pd), expect_pd, rtol=1e-9, atol=1e-12)


def test_series_first_term_and_large_damping(micro):
    """m = 1 gives the block-Jacobi step U~^-1 g; very large lambda gives
    delta -> g / lambda (gradient-descent limit)."""
    pr, P, X, eta = _state(micro)
    ne = pr.normal_equations(P, X, eta)
    Q = O.tangent_bases(P, O.SPHERE)
    rs = O.reduced_system(ne, Q, 1e-2)
    d1, _ = O.series_step(rs, 1)
    x0 = np.concatenate([np.linalg.solve(rs.Ut[i], rs.g[11 * i:11 * i + 11])
                         for i in range(pr.n_cams)])
    assert np.allclose(d1, x0, rtol=1e-10, atol=1e-14 * np.abs(x0).max())
    lam = 1e9
    rs = O.reduced_system(ne, Q, lam)
    d, _ = O.series_step(rs, 10)
    assert np.allclose(d * lam, rs.g, rtol=1e-5, atol=1e-5 * np.abs(rs.g).max())


# --------------------------------------------------------------- tangent space

def test_tangent_step_orthogonal_and_normalized(tiny):
    pr, P, X, eta = _state(tiny)
    st = pr.init_state(P, O.Params(eta=eta, m=5, manifold=O.SPHERE))
    _, rep = pr.step(st, O.Params(eta=eta, m=5, manifold=O.SPHERE))
    Phat = P / np.linalg.norm(P, axis=1, keepdims=True)
    dots = np.einsum("na,na->n", Phat, rep.delta)
    assert np.all(np.abs(dots) <= 1e-14 * np.maximum(np.linalg.norm(rep.delta, axis=1), 1e-300) + 1e-15)
    assert np.allclose(np.linalg.norm(rep.P_trial, axis=1), 1.0, atol=1e-14)


def test_tangent_step_basis_invariant(micro):
    """The step is invariant under Q_i -> Q_i R_i, R_i random orthogonal."""
    pr, P, X, eta = _state(micro)
    ne = pr.normal_equations(P, X, eta)
    Q = O.tangent_bases(P, O.SPHERE)
    rng = np.random.default_rng(8)
    R = np.stack([np.linalg.qr(rng.normal(size=(11, 11)))[0] for _ in range(pr.n_cams)])
    Q2 = np.einsum("nab,nbc->nac", Q, R)
    for solver in ("exact", "series"):
        outs = []
        for QQ in (Q, Q2):
            rs = O.reduced_system(ne, QQ, 1e-3)
            d = O.exact_step(rs) if solver == "exact" else O.series_step(rs, 7)[0]
            outs.append(np.einsum("nab,nb->na", QQ, d.reshape(pr.n_cams, 11)))
        assert np.allclose(outs[0], outs[1], rtol=1e-9, atol=1e-12 * np.abs(outs[0]).max())


# --------------------------------------------------------------- LM controller

@pytest.mark.parametrize("manifold", [O.EUCLID, O.SPHERE])
def test_predicted_decrease_is_gauss_newton_model_decrease(micro, manifold):
    """The step's reported pred equals F - ||r + J_p dP + J_l dX||^2, the
    decrease of the linearized (Gauss-Newton) model at the model-optimal
    landmark increment dX = -V^-1 (b_l + W^T dP), evaluated with the sparse
    Jacobian -- independently of the Schur-complement formula."""
    pr, P, X, eta = _state(micro)
    prm = O.Params(eta=eta, m=6, manifold=manifold, lambda0=1e-2)
    st = pr.init_state(P, prm)
    _, rep = pr.step(st, prm)
    ne = pr.normal_equations(P, st.X, eta)
    dP = rep.delta.ravel()
    Vinv = O.blockdiag(O.sym_inverse_batch(ne.V)[0])
    dX = -(Vinv @ (ne.b_l + ne.W.T @ dP))
    Jp, Jl = O.jacobian_blocks(P, st.X, pr.cam_idx, pr.pt_idx, pr.meas, eta)
    J = O.assemble_jacobian(Jp, Jl, pr.cam_idx, pr.pt_idx, pr.n_cams, pr.n_points)
    model = ne.r.ravel() + J @ np.concatenate([dP, dX])
    F = float(np.sum(ne.r ** 2))
    assert abs(rep.pred - (F - model @ model)) <= 1e-9 * F


@pytest.mark.parametrize("manifold,solver", [(O.SPHERE, "series"), (O.EUCLID, "series"),
                                             (O.SPHERE, "exact")])
def test_accepted_steps_never_increase_cost(tiny, manifold, solver):
    pr, P, X, eta = _state(tiny)
    prm = O.Params(eta=eta, m=10, manifold=manifold, solver=solver)
    st, reps = pr.solve(P, prm, max_iters=25)
    costs = [reps[0].cost_before] + [r.cost_after for r in reps if r.accepted]
    assert all(b < a for a, b in zip(costs, costs[1:]))
    assert costs[-1] < 0.01 * costs[0]
    for r in reps:
        if not r.accepted:
            assert r.cost_after >= r.cost_before
        else:
            assert r.pred > 0


def test_affine_factorization_special_case():
    """eta = 1, EUCLID, full visibility: pOSE reduces to affine factorization
    and the global minimum is the squared tail sigma_4^2 + ... of the
    row-centred 2n x m measurement matrix (Tomasi-Kanade, textbook SVD)."""
    n_cams, n_pts = 6, 60
    sc = scenes.ring_scene(n_cams, n_pts, 11, noise_px=3.0, eta=1.0)
    rng = np.random.default_rng(0)
    cam_idx = np.repeat(np.arange(n_cams), n_pts).astype(np.int32)
    pt_idx = np.tile(np.arange(n_pts), n_cams).astype(np.int32)
    y = np.einsum("nij,nj->ni", sc.gt_cams[cam_idx], np.c_[sc.gt_points[pt_idx], np.ones(cam_idx.size)])
    meas = y[:, :2] / y[:, 2:3] + rng.normal(0, 3.0 / 500, size=(cam_idx.size, 2))
    Mm = np.zeros((2 * n_cams, n_pts))
    Mm[2 * cam_idx, pt_idx] = meas[:, 0]
    Mm[2 * cam_idx + 1, pt_idx] = meas[:, 1]
    Mc = Mm - Mm.mean(axis=1, keepdims=True)
    sv = np.linalg.svd(Mc, compute_uv=False)
    Fstar = float(np.sum(sv[3:] ** 2))
    pr = O.Problem(n_cams, n_pts, cam_idx, pt_idx, meas)
    P0 = scenes.init_cameras(n_cams, 2, normalize=False)
    prm = O.Params(eta=1.0, m=10, manifold=O.EUCLID, solver="exact", lambda0=1e-4)
    st, _ = pr.solve(P0, prm, max_iters=100, ftol=1e-14)
    assert abs(st.F - Fstar) <= 1e-8 * Fstar


# --------------------------------------------------------------- matrix-free variant

@pytest.mark.parametrize("manifold", [O.EUCLID, O.SPHERE])
def test_matrix_free_step_equals_dense_step(tiny, manifold):
    """The matrix-free oracle step (used for scenes whose dense S does not
    fit) reproduces the explicit-S step, including the b_l term off the
    landmark optimum and the early-stop rule."""
    pr, P, X, eta = _state(tiny)
    mf = O.MatrixFreeProblem(pr.n_cams, pr.n_points, pr.cam_idx, pr.pt_idx, pr.meas)
    for eps, m in ((0.0, 7), (0.05, 30)):
        prm = O.Params(eta=eta, m=m, manifold=manifold, series_eps=eps, lambda0=1e-3)
        st = pr.init_state(P, prm)
        st_off = O.State(P=st.P, X=st.X + 0.01, F=st.F, lam=st.lam)
        for s0 in (st, st_off):
            _, a = pr.step(s0, prm)
            _, b = mf.step(s0, prm)
            assert a.terms_used == b.terms_used
            assert np.allclose(b.delta, a.delta, rtol=1e-9, atol=1e-12 * np.abs(a.delta).max())
            assert abs(a.cost_after - b.cost_after) <= 1e-10 * a.cost_after
            assert abs(a.pred - b.pred) <= 1e-8 * abs(a.pred)


# --------------------------------------------------------------- PoBA and PCG (Sec. 2, 5.2)

def _off_optimum(pr, P, X, seed=11, scale=1e-2):
    rng = np.random.default_rng(seed)
    return X + scale * rng.normal(size=X.shape)


@pytest.mark.parametrize("manifold", [O.EUCLID, O.SPHERE])
def test_poba_exact_step_is_joint_damped_gauss_newton(micro, manifold):
    """The PoBA step (Schur reduction with damped V, back-substitution) at a
    point off the landmark optimum equals the joint damped Gauss-Newton
    step solved directly from the full Jacobian: with J~ = [J_p Q | J_l] and
    D = diag(lambda I, lambda_l lambda I), (J~^T J~ + D) (d, dX) = -J~^T r."""
    pr, P, X, eta = _state(micro)
    X = _off_optimum(pr, P, X)
    lam, lam_l = 3e-3, 2.0
    st = O.State(P=P, X=X, F=pr.cost(P, X, eta), lam=lam)
    prm = O.Params(eta=eta, manifold=manifold, method="poba", solver="exact", lambda_l=lam_l)
    _, rep = pr.step(st, prm)
    Jp, Jl = O.jacobian_blocks(P, X, pr.cam_idx, pr.pt_idx, pr.meas, eta)
    J = O.assemble_jacobian(Jp, Jl, pr.cam_idx, pr.pt_idx, pr.n_cams, pr.n_points).toarray()
    Q = O.tangent_bases(P, manifold)
    k = Q.shape[2]
    Qbd = sla.block_diag(*Q)
    nc3 = 12 * pr.n_cams
    Jt = np.hstack([J[:, :nc3] @ Qbd, J[:, nc3:]])
    r = O.pose_residuals(P, X, pr.cam_idx, pr.pt_idx, pr.meas, eta).ravel()
    D = np.diag(np.r_[np.full(k * pr.n_cams, lam), np.full(3 * pr.n_points, lam_l * lam)])
    sol = np.linalg.solve(Jt.T @ Jt + D, -Jt.T @ r)
    dP = (Qbd @ sol[:k * pr.n_cams]).reshape(-1, 12)
    assert np.allclose(rep.delta, dP, rtol=1e-8, atol=1e-10 * np.abs(dP).max())
    X_trial = X + sol[k * pr.n_cams:].reshape(-1, 3)
    P_trial = P + dP
    if manifold == O.SPHERE:
        P_trial = P_trial / np.linalg.norm(P_trial, axis=1, keepdims=True)
    assert abs(rep.cost_after - pr.cost(P_trial, X_trial, eta)) <= 1e-9 * rep.cost_after
    # predicted decrease: ||r||^2 - ||r + J D||^2 = -b^T D + D^T Dmp D at the
    # exact damped solution (normal-equation identity)
    b = Jt.T @ r
    assert abs(rep.pred - (-(b @ sol) + sol @ D @ sol)) <= 1e-8 * abs(rep.pred)


def test_poba_series_converges_to_exact_step(micro):
    """The power series on the damped Schur complement converges to the
    exact PoBA step as the number of terms grows."""
    pr, P, X, eta = _state(micro)
    X = _off_optimum(pr, P, X)
    st = O.State(P=P, X=X, F=pr.cost(P, X, eta), lam=1e-1)
    ex = O.Params(eta=eta, manifold=O.SPHERE, method="poba", solver="exact")
    _, rex = pr.step(st, ex)
    errs = []
    for m in (2, 8, 32, 128, 512):
        prm = O.Params(eta=eta, manifold=O.SPHERE, method="poba", solver="series", m=m)
        _, rs = pr.step(st, prm)
        errs.append(np.linalg.norm(rs.delta - rex.delta) / np.linalg.norm(rex.delta))
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] <= 1e-10


def test_poba_accepted_steps_never_increase_cost(micro):
    pr, P, X, eta = _state(micro)
    prm = O.Params(eta=eta, manifold=O.SPHERE, method="poba", solver="series", m=10)
    st, reps = pr.solve(P, prm, max_iters=25, ftol=0.0)
    for rep in reps:
        if rep.accepted:
            assert rep.cost_after < rep.cost_before


def _reduced(pr, P, X, eta, lam):
    ne = pr.normal_equations(P, X, eta)
    return O.reduced_system(ne, O.tangent_bases(P, O.SPHERE), lam)


def test_pcg_reaches_the_exact_step_within_the_dimension(micro):
    """In exact arithmetic conjugate gradients solve the SPD system in at
    most dim steps; in FP64 (which loses conjugacy on this ill-conditioned
    system) 2 dim steps reach the Cholesky solution to 1e-10, and the
    S-energy error never increases."""
    pr, P, X, eta = _state(micro)
    rs = _reduced(pr, P, X, eta, 1e-2)
    exact = O.exact_step(rs)
    n = len(rs.g)
    d, it = O.pcg_step(rs, 2 * n)
    assert it == 2 * n
    assert np.linalg.norm(d - exact) <= 1e-10 * np.linalg.norm(exact)
    energy = []
    for k in range(1, 12):
        dk, _ = O.pcg_step(rs, k)
        e = dk - exact
        energy.append(float(e @ rs.S @ e))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(energy, energy[1:]))


def test_pcg_first_iteration_is_preconditioned_steepest_descent(micro):
    """One PCG iteration from zero is the exact line minimum along the
    preconditioned gradient z = M^-1 g: delta = (g^T z / z^T S z) z, with M
    the block diagonal of S."""
    pr, P, X, eta = _state(micro)
    rs = _reduced(pr, P, X, eta, 1e-2)
    k = rs.Ut.shape[1]
    M = np.zeros_like(rs.S)
    for i in range(rs.Ut.shape[0]):
        sl = slice(k * i, k * i + k)
        M[sl, sl] = rs.S[sl, sl]
    z = np.linalg.solve(M, rs.g)
    expect = (rs.g @ z) / (z @ rs.S @ z) * z
    d, it = O.pcg_step(rs, 1)
    assert it == 1
    assert np.allclose(d, expect, rtol=1e-10, atol=1e-14 * np.abs(expect).max())
