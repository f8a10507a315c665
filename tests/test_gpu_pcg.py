"""Parity of the GPU conjugate-gradient solver (the "iterative" VarPro
baseline of Sec. 5.2: Schur-Jacobi preconditioned CG on the reduced camera
system) with the FP64 CPU oracle's pcg_step.

Tolerances: FP64 1e-10 relative on the step up to 10 iterations (the
iterations are the oracle's up to rounding order); later iterates are
compared by what CG minimizes (check_late_iterates). Mixed precision (FP32
vectors and landmark pass, FP64 dot products and preconditioner) 1e-3 after
10 iterations, the FP32 rounding of the iteration vectors.
"""
import numpy as np
import pytest

from oracle import povar_oracle as O
from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SCENES = {
    "tiny": lambda: scenes.tiny_scene(0),
    "traj": lambda: scenes.trajectory_scene(120, 6000, 3, eta=0.1, m=8, name="traj"),
}


def oracle_params(sc, manifold, iters, tol, method="varpro", lambda0=1e-4):
    return O.Params(eta=sc.eta, m=1, manifold=manifold, lambda0=lambda0, solver="pcg",
                    pcg_iters=iters, pcg_tol=tol, method=method, lambda_l=1.0)


def gpu_params(sc, manifold, iters, tol, precision, lambda_l=0.0, lambda0=1e-4):
    return povar.make_params(eta=sc.eta, m=iters, series_eps=tol, manifold=manifold,
                             precision=precision, lambda0=lambda0, lambda_l=lambda_l,
                             solver=povar.SOLVER_PCG)


def one_step(sc, P0, prm):
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        rep = pb.step(prm)
        _, _, d = pb.last_step()
        return rep, d, pb.cameras(), pb.points()


def reduced(orc, st, sc, manifold):
    ne = orc.normal_equations(st.P, st.X, sc.eta)
    Q = O.tangent_bases(st.P, manifold)
    return O.reduced_system(ne, Q, st.lam), Q


@pytest.mark.parametrize("iters", [1, 10])
@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
@pytest.mark.parametrize("name", list(SCENES))
def test_pcg_fixed_iterations_fp64_matches_oracle(name, manifold, iters):
    sc = SCENES[name]()
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, manifold, iters, 0.0)
    st1, orep = orc.step(orc.init_state(P0, op), op)
    rep, d, P1, _ = one_step(sc, P0, gpu_params(sc, manifold, iters, 0.0, povar.FP64))
    assert rep.terms_used == iters == orep.terms_used
    assert rel(d, orep.delta) <= 1e-10
    assert abs(rep.cost_after - orep.cost_after) <= 1e-10 * orep.cost_after
    assert abs(rep.pred - orep.pred) <= 1e-9 * abs(orep.pred)
    assert rep.accepted == int(orep.accepted)
    assert rel(P1, st1.P) <= 1e-10


def check_late_iterates(orc, st0, sc, manifold, orep, rep, d):
    """Past 10 - 20 iterations CG iterates are chaotic in the rounding: in the
    oracle itself a 1e-15 relative change of g moves the step after 40 - 44
    iterations by up to 5e-3 relative (traj scene, sphere). What stays put is
    what CG minimizes: the model value g^T d - d^T S d / 2 (moved by at most
    1.4e-6 there) and the energy error ||d - d*||_S (at most 2e-2). So the
    GPU step must give the oracle's predicted decrease to 1e-5 and an energy
    error within 25 % of the oracle's."""
    rs, Q = reduced(orc, st0, sc, manifold)
    dstar = O.exact_step(rs)
    en = float(dstar @ rs.S @ dstar)

    def energy(dd):
        t = np.einsum("nab,na->nb", Q, np.asarray(dd).reshape(-1, 12)).ravel() - dstar
        return float(t @ rs.S @ t)

    e_gpu, e_orc = energy(d), energy(orep.delta)
    assert abs(rep.pred - orep.pred) <= 1e-5 * abs(orep.pred)
    assert e_gpu <= 1.25 * e_orc + 1e-12 * en, (e_gpu / en, e_orc / en)


@pytest.mark.parametrize("iters", [20, 40, 100])
@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
@pytest.mark.parametrize("name", list(SCENES))
def test_pcg_late_iterations_fp64_match_what_cg_minimizes(name, manifold, iters):
    sc = SCENES[name]()
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, manifold, iters, 0.0)
    st0 = orc.init_state(P0, op)
    _, orep = orc.step(st0, op)
    rep, d, _, _ = one_step(sc, P0, gpu_params(sc, manifold, iters, 0.0, povar.FP64))
    assert rep.terms_used == iters == orep.terms_used
    check_late_iterates(orc, st0, sc, manifold, orep, rep, d)


@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
def test_pcg_tolerance_stop_matches_oracle(manifold):
    """With a relative residual tolerance both sides stop after the same
    iteration (unchanged under 1e-15 perturbations of g in the oracle)."""
    sc = SCENES["traj"]()
    P0 = scenes.init_cameras(sc.n_cams, 5, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, manifold, 500, 1e-3)
    st0 = orc.init_state(P0, op)
    _, orep = orc.step(st0, op)
    assert 1 < orep.terms_used < 500
    rep, d, _, _ = one_step(sc, P0, gpu_params(sc, manifold, 500, 1e-3, povar.FP64))
    assert rep.terms_used == orep.terms_used
    check_late_iterates(orc, st0, sc, manifold, orep, rep, d)


@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
def test_pcg_converged_equals_exact_step(manifold):
    """CG run to a residual of 1e-12 gives the exact (Cholesky) step of the
    damped reduced system: an invariant independent of the CG recurrences."""
    sc = SCENES["tiny"]()
    P0 = scenes.init_cameras(sc.n_cams, 6, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = O.Params(eta=sc.eta, manifold=manifold, lambda0=1e-2, solver="exact")
    _, orep = orc.step(orc.init_state(P0, op), op)
    rep, d, _, _ = one_step(sc, P0, gpu_params(sc, manifold, 2000, 1e-12, povar.FP64,
                                               lambda0=1e-2))
    assert rep.terms_used < 2000
    assert rel(d, orep.delta) <= 1e-8


@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
def test_pcg_mixed_close_to_oracle(manifold):
    sc = SCENES["traj"]()
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, manifold, 10, 0.0)
    _, orep = orc.step(orc.init_state(P0, op), op)
    rep, d, _, _ = one_step(sc, P0, gpu_params(sc, manifold, 10, 0.0, povar.MIXED_FP32))
    assert rep.terms_used == 10
    assert rel(d, orep.delta) <= 1e-3
    assert abs(rep.cost_after - orep.cost_after) <= 1e-4 * orep.cost_after


@pytest.mark.parametrize("precision,tol_d", [(povar.FP64, 1e-10), (povar.MIXED_FP32, 1e-3)])
def test_poba_pcg_step_matches_oracle(precision, tol_d):
    """PoBA's damped Schur complement solved by PCG (both comparison systems
    of Sec. 5.2 on the same kernels)."""
    sc = SCENES["traj"]()
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, O.SPHERE, 10, 0.0, method="poba")
    st1, orep = orc.step(orc.init_state(P0, op), op)
    rep, d, _, X1 = one_step(sc, P0, gpu_params(sc, O.SPHERE, 10, 0.0, precision, lambda_l=1.0))
    assert rel(d, orep.delta) <= tol_d
    assert abs(rep.cost_after - orep.cost_after) <= max(1e-10, tol_d / 10) * orep.cost_after
    if precision == povar.FP64:
        assert rel(X1, st1.X) <= 1e-9


def test_pcg_trajectory_fp64_matches_oracle():
    """Eight LM steps with 10 PCG iterations each (accepts and rejects)."""
    sc = SCENES["tiny"]()
    P0 = scenes.init_cameras(sc.n_cams, 1, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, O.SPHERE, 10, 0.0)
    st = orc.init_state(P0, op)
    prm = gpu_params(sc, O.SPHERE, 10, 0.0, povar.FP64)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        for k in range(8):
            st, orep = orc.step(st, op)
            rep = pb.step(prm)
            assert rep.accepted == int(orep.accepted), k
            assert abs(rep.cost_after - orep.cost_after) <= 1e-9 * orep.cost_after, k
            assert rel(pb.cameras(), st.P) <= 1e-9, k


def test_pcg_solve_reaches_the_series_target_on_tiny():
    """A PCG solve runs to the oracle's converged cost of the tiny scene."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "converged_tiny.json")) as f:
        g = json.load(f)
    sc = scenes.scene_by_name("tiny", g["scene_seed"])
    P0 = scenes.init_cameras(sc.n_cams, g["init_seed"], normalize=True)
    prm = povar.make_params(eta=g["eta"], m=500, series_eps=1e-6, lambda0=g["lambda0"],
                            manifold=povar.EUCLID, precision=povar.FP64,
                            solver=povar.SOLVER_PCG)
    target = g["series"]["F"] * (1.0 + 1e-5)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        rep, iters = pb.solve(prm, max_iters=300, ftol=0.0, target_cost=target)
        assert rep.cost_after <= target or pb.cost(sc.eta) <= target * (1 + 1e-9), iters


def test_pcg_invalid_params_rejected():
    sc = SCENES["tiny"]()
    P0 = scenes.init_cameras(sc.n_cams, 2, normalize=True)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        for kw in ({"solver": 2}, {"solver": povar.SOLVER_PCG, "precision": povar.MIXED_BF16}):
            prm = povar.make_params(eta=sc.eta, m=10, **kw)
            with pytest.raises(povar.PovarError) as e:
                pb.step(prm)
            assert e.value.status == 1
        prm = povar.make_params(eta=sc.eta, m=10)
        prm.reserved = 7
        with pytest.raises(povar.PovarError):
            pb.step(prm)


def test_pcg_not_available_in_a_batch():
    scs = [scenes.tiny_scene(0), scenes.tiny_scene(1)]
    with povar.Batch(scs) as b:
        b.set_cameras([scenes.init_cameras(s.n_cams, 3, normalize=True) for s in scs], 0.1)
        prm = povar.make_params(eta=0.1, m=10, solver=povar.SOLVER_PCG, precision=povar.FP64)
        with pytest.raises(povar.PovarError) as e:
            b.solve(prm, max_iters=2)
        assert e.value.status == 1
