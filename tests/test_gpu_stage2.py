"""Parity of the GPU second stage (projective refinement of Eq. second_stage
by Riemannian PoBA, Sec. 4.3) with the FP64 CPU oracle
(oracle/ripoba_oracle.py).

Tolerances as for the first stage: FP64 1e-10 relative per step (cost,
camera and landmark updates), 1e-9 on pred; mixed precision (FP32 series
terms and camera vectors, FP64 landmark blocks, linearization,
back-substitution and cost) 1e-4 on the step.
"""
import numpy as np
import pytest

from oracle import povar_oracle as O1
from oracle import ripoba_oracle as R
from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SCENES = {
    "tiny": lambda: scenes.tiny_scene(0),
    "ring60": lambda: scenes.ring_scene(60, 4000, 7, track="geom3", noise_px=1.0, eta=0.1, m=10,
                                        name="ring60"),
}


def traj_scene():
    return scenes.trajectory_scene(120, 6000, 3, eta=0.1, m=8, name="traj")


def start(sc, seed=1, noise=0.01):
    P, X = scenes.stage2_start(sc, seed, noise)
    orc = R.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    return P, X, orc


def gauge_free_rel(P, X, dP, dX, dP_ref, dX_ref):
    """Relative difference of two joint steps after removing the directions
    of the projective gauge: P_i -> P_i (I + A), X_j -> (I - A) X_j for any
    4x4 A leaves every projection unchanged, so the reduced system is
    singular along those 16 directions (up to the damping) and steps may
    differ there without changing the cost to first order. The directions
    are projected onto the tangent spaces, the difference is fitted to them
    by least squares and the remainder is compared with the step."""
    nc, npt = P.shape[0], X.shape[0]
    Pm = P.reshape(nc, 3, 4)
    basis = []
    for a in range(4):
        for b in range(4):
            A = np.zeros((4, 4))
            A[a, b] = 1.0
            gp = (Pm @ A).reshape(nc, 12)
            gp -= np.sum(gp * P, axis=1, keepdims=True) * P
            gx = -(X @ A.T)
            gx -= np.sum(gx * X, axis=1, keepdims=True) * X
            basis.append(np.concatenate([gp.ravel(), gx.ravel()]))
    B = np.stack(basis, axis=1)
    diff = np.concatenate([(dP - dP_ref).ravel(), (dX - dX_ref).ravel()])
    c, *_ = np.linalg.lstsq(B, diff, rcond=None)
    ref = np.concatenate([dP_ref.ravel(), dX_ref.ravel()])
    return float(np.linalg.norm(diff - B @ c) / np.linalg.norm(ref))


def oparams(m, eps=0.0, lambda0=1e-4, lambda_l=1.0):
    return R.Params(lambda0=lambda0, m=m, series_eps=eps, lambda_l=lambda_l)


@pytest.mark.parametrize("schedule", [0, 1])
@pytest.mark.parametrize("lambda0", [1e-4, 1e-1])
@pytest.mark.parametrize("name", list(SCENES))
def test_s2_one_step_fp64_matches_oracle(name, lambda0, schedule):
    sc = SCENES[name]()
    P, X, orc = start(sc)
    op = oparams(10, lambda0=lambda0)
    st0 = orc.init_state(P, X, op)
    st1, orep = orc.step(st0, op)
    with povar.Problem.from_scene(sc) as pb:
        pb.s2_set(P, X)
        assert abs(pb.s2_cost() - st0.F) <= 1e-12 * st0.F
        rep = pb.s2_step(povar.make_s2_params(lambda0=lambda0, m=10, series_eps=0.0,
                                              precision=povar.FP64, schedule=schedule))
        U, bp, d = pb.last_step()
        P1, X1 = pb.cameras(), pb.s2_points()
    assert rep.terms_used == 10
    assert abs(rep.cost_before - orep.cost_before) <= 1e-12 * orep.cost_before
    assert abs(rep.cost_after - orep.cost_after) <= 1e-10 * orep.cost_after
    assert abs(rep.pred - orep.pred) <= 1e-9 * abs(orep.pred)
    assert rep.accepted == int(orep.accepted)
    assert abs(rep.lambda_next - orep.lambda_next) <= 1e-9 * orep.lambda_next
    assert rel(d, orep.dP) <= 1e-10
    # per-camera check next to the global one
    for i in range(sc.n_cams):
        assert rel(d[i], orep.dP[i]) <= 1e-8, i
    assert rel(P1, st1.P) <= 1e-10
    assert rel(X1, st1.X) <= 1e-10


def test_s2_normal_equation_blocks_match_oracle():
    """U_i = sum E (x) XX^T and the reduced right-hand side b_p - W G_l b_l
    against the oracle's explicit sparse products."""
    sc = SCENES["tiny"]()
    P, X, orc = start(sc, seed=2)
    op = oparams(1)
    st0 = orc.init_state(P, X, op)
    ne, rsys, rs = orc.system(st0, op)
    Gl = np.einsum("nab,nbc,ndc->nad", rsys.Ql, np.linalg.inv(rsys.Vt), rsys.Ql)
    s = np.einsum("nab,nb->na", Gl, ne.b_l.reshape(-1, 4))
    b_eff = ne.b_p - ne.W @ s.ravel()
    with povar.Problem.from_scene(sc) as pb:
        pb.s2_set(P, X)
        pb.s2_step(povar.make_s2_params(m=1, series_eps=0.0, precision=povar.FP64))
        U, bp, _ = pb.last_step()
    assert rel(U, ne.U) <= 1e-11
    assert rel(bp.ravel(), b_eff) <= 1e-10


def test_s2_trajectory_fp64_matches_oracle():
    sc = SCENES["tiny"]()
    P, X, orc = start(sc, seed=3, noise=0.03)
    op = oparams(21, eps=0.01)
    st = orc.init_state(P, X, op)
    prm = povar.make_s2_params(m=21, series_eps=0.01, precision=povar.FP64)
    with povar.Problem.from_scene(sc) as pb:
        pb.s2_set(P, X)
        for k in range(8):
            st, orep = orc.step(st, op)
            rep = pb.s2_step(prm)
            if abs(orep.cost_after - orep.cost_before) <= 1e-12 * orep.cost_before:
                break   # converged: accept decisions are rounding-level from here
            assert rep.accepted == int(orep.accepted), k
            assert rep.terms_used == orep.terms_used, k
            assert abs(rep.cost_after - orep.cost_after) <= 1e-9 * orep.cost_after, k
            assert rel(pb.cameras(), st.P) <= 1e-9, k
            assert rel(pb.s2_points(), st.X) <= 1e-9, k


def test_s2_step_on_an_ill_conditioned_scene():
    """The trajectory scene (cameras far from their points: nearly affine
    projections) makes the reduced system ill-conditioned (cond ~3e12 at
    lambda = 1e-4, |y3| down to 2e-5 of |y|). There the trial cost is
    sensitive to rounding: in the oracle alone a 1e-15 relative change of P
    moves it by up to ~4e-6 relative, and different summation orders (the
    GPU's) by ~1e-5. What is well-conditioned is compared tightly: the
    cost at the start, the predicted decrease (a quadratic model value,
    1e-9) and the accept decision; the trial cost within 1e-4."""
    sc = traj_scene()
    P, X, orc = start(sc)
    for lambda0 in (1e-4, 1e-1):
        op = oparams(10, lambda0=lambda0)
        st0 = orc.init_state(P, X, op)
        _, orep = orc.step(st0, op)
        with povar.Problem.from_scene(sc) as pb:
            pb.s2_set(P, X)
            rep = pb.s2_step(povar.make_s2_params(lambda0=lambda0, m=10, series_eps=0.0,
                                                  precision=povar.FP64))
        assert abs(rep.cost_before - orep.cost_before) <= 1e-12 * orep.cost_before
        assert abs(rep.pred - orep.pred) <= 1e-9 * abs(orep.pred)
        assert rep.accepted == int(orep.accepted)
        assert abs(rep.cost_after - orep.cost_after) <= 1e-4 * orep.cost_after


@pytest.mark.parametrize("schedule", [0, 1])
def test_s2_mixed_step_close_to_oracle(schedule):
    sc = SCENES["ring60"]()
    P, X, orc = start(sc)
    op = oparams(10)
    _, orep = orc.step(orc.init_state(P, X, op), op)
    st0 = orc.init_state(P, X, op)
    with povar.Problem.from_scene(sc) as pb:
        pb.s2_set(P, X)
        X0 = pb.s2_points()
        rep = pb.s2_step(povar.make_s2_params(m=10, series_eps=0.0, precision=povar.MIXED_FP32,
                                              schedule=schedule))
        _, _, d = pb.last_step()
        X1 = pb.s2_points()
    # the landmark update of the GPU step, from the retracted landmarks
    dX = X1 * np.linalg.norm(st0.X + orep.dX, axis=1, keepdims=True) - X0
    assert gauge_free_rel(st0.P, st0.X, d, dX, orep.dP, orep.dX) <= 1e-4
    assert abs(rep.pred - orep.pred) <= 1e-5 * abs(orep.pred)
    assert abs(rep.cost_after - orep.cost_after) <= 1e-5 * orep.cost_after


@pytest.mark.parametrize("precision", [povar.FP64, povar.MIXED_FP32])
def test_s2_solve_reaches_the_oracle_minimum(precision):
    """Both precisions converge to the oracle's minimum of Eq. second_stage
    (relative decrease below 1e-12): cost within 1e-6, cameras and landmarks
    within 1e-5 (both are unique on the spheres up to sign, fixed by the
    start)."""
    sc = SCENES["tiny"]()
    P, X, orc = start(sc, seed=4, noise=0.02)
    op = oparams(21, eps=0.01)
    st, trace = orc.solve(orc.init_state(P, X, op), op, max_iters=100, ftol=1e-12)
    with povar.Problem.from_scene(sc) as pb:
        pb.s2_set(P, X)
        rep, iters = pb.s2_solve(povar.make_s2_params(m=21, series_eps=0.01, precision=precision),
                                 max_iters=100, ftol=1e-12)
        F = pb.s2_cost()
        P1, X1 = pb.cameras(), pb.s2_points()
    assert abs(F - st.F) <= 1e-6 * st.F, (F, st.F, iters)
    assert np.max(np.abs(P1 - st.P)) <= 1e-5
    assert np.max(np.abs(X1 - st.X)) <= 1e-5


def test_s2_from_first_stage_result():
    """The stratified pipeline on one handle: a first-stage solve, then the
    second stage from its cameras and (X*, 1); the start cost is the
    oracle's reprojection cost there, and the refinement lowers it."""
    sc = SCENES["tiny"]()
    P0 = scenes.init_cameras(sc.n_cams, 1, normalize=True)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        pb.solve(povar.make_params(eta=sc.eta, m=21, series_eps=0.01, manifold=povar.SPHERE,
                                   precision=povar.MIXED_FP32), max_iters=30)
        Pc = pb.cameras()
        pb.s2_set()
        F0 = pb.s2_cost()
        Xs = O1.landmarks(Pc, sc.cam_idx, sc.pt_idx, sc.meas, sc.eta, sc.n_points)
        Xh = np.concatenate([Xs, np.ones((sc.n_points, 1))], axis=1)
        F_or = R.cost(Pc, Xh, sc.cam_idx, sc.pt_idx, sc.meas)
        assert abs(F0 - F_or) <= 1e-9 * F_or
        rep, _ = pb.s2_solve(povar.make_s2_params(m=21, series_eps=0.01), max_iters=20)
        assert pb.s2_cost() < F0
        # a first-stage step afterwards starts from the closed-form landmarks
        P2 = pb.cameras()
        r1 = pb.step(povar.make_params(eta=sc.eta, m=5, manifold=povar.SPHERE,
                                       precision=povar.FP64))
    X2 = O1.landmarks(P2, sc.cam_idx, sc.pt_idx, sc.meas, sc.eta, sc.n_points)
    F2 = O1.cost(P2, X2, sc.cam_idx, sc.pt_idx, sc.meas, sc.eta)
    assert abs(r1.cost_before - F2) <= 1e-10 * F2


def test_s2_invalid_calls_rejected():
    sc = SCENES["tiny"]()
    P, X, _ = start(sc)
    with povar.Problem.from_scene(sc) as pb:
        with pytest.raises(povar.PovarError) as e:
            pb.s2_step(povar.make_s2_params(precision=povar.FP64))
        assert e.value.status == 1
        with pytest.raises(povar.PovarError):
            pb.s2_set()          # no first-stage state yet
        pb.s2_set(P, X)
        bad = [povar.make_s2_params(lambda_l=0.0), povar.make_s2_params(precision=povar.MIXED_BF16)]
        b = povar.make_s2_params()
        b.manifold = povar.EUCLID
        bad.append(b)
        b = povar.make_s2_params()
        b.solver = povar.SOLVER_PCG
        bad.append(b)
        bad.append(povar.make_s2_params(schedule=3))
        for prm in bad:
            with pytest.raises(povar.PovarError) as e:
                pb.s2_step(prm)
            assert e.value.status == 1
        Xbad = X.copy()
        Xbad[3, 1] = np.nan
        with pytest.raises(povar.PovarError):
            pb.s2_set(P, Xbad)
