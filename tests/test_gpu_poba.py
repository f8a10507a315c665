"""Parity of the GPU PoBA comparison solver (joint Levenberg-Marquardt with
the power series on the damped Schur complement, Sec. 2 / Sec. 5.2 of the
paper) with the FP64 CPU oracle's PoBA step.

Tolerances as for PoVar: FP64 1e-10 relative per step; mixed precision
(FP32 linearization and series, FP64 landmark blocks and back-substitution)
1e-4 on the step.
"""
import numpy as np
import pytest

from oracle import povar_oracle as O
from paper_2405_05079_gb300 import povar, scenes

pytestmark = pytest.mark.gpu

LAMBDA_L = 1.0   # joint damping: the landmarks get the camera damping


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


SCENES = {
    "tiny": lambda: scenes.tiny_scene(0),
    "traj": lambda: scenes.trajectory_scene(120, 6000, 3, eta=0.1, m=8, name="traj"),
}


def oracle_params(sc, manifold, m):
    return O.Params(eta=sc.eta, m=m, manifold=manifold, series_eps=0.0, lambda0=1e-4,
                    method="poba", solver="series", lambda_l=LAMBDA_L)


def gpu_params(sc, manifold, m, precision, schedule=-1):
    return povar.make_params(eta=sc.eta, m=m, manifold=manifold, precision=precision,
                             lambda0=1e-4, schedule=schedule, lambda_l=LAMBDA_L)


@pytest.mark.parametrize("schedule", [0, 1, 5])
@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
@pytest.mark.parametrize("name", list(SCENES))
def test_poba_one_step_fp64_matches_oracle(name, manifold, schedule):
    sc = SCENES[name]()
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, manifold, sc.m)
    st0 = orc.init_state(P0, op)
    st1, orep = orc.step(st0, op)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        rep = pb.step(gpu_params(sc, manifold, sc.m, povar.FP64, schedule))
        _, _, d = pb.last_step()
        X = pb.points()
    assert rel(d, orep.delta) <= 1e-10
    assert abs(rep.cost_before - orep.cost_before) <= 1e-10 * orep.cost_before
    assert abs(rep.cost_after - orep.cost_after) <= 1e-10 * orep.cost_after
    assert abs(rep.pred - orep.pred) <= 1e-9 * abs(orep.pred)
    assert rep.accepted == int(orep.accepted)
    assert abs(rep.lambda_next - orep.lambda_next) <= 1e-9 * orep.lambda_next
    # the landmarks of the new iterate: back-substituted when accepted
    assert rel(X, st1.X) <= 1e-10


def test_poba_trajectory_fp64_matches_oracle():
    """Ten PoBA steps (accepts and rejects) from the random start stay at
    1e-10 per step: costs, cameras and landmarks."""
    sc = SCENES["tiny"]()
    P0 = scenes.init_cameras(sc.n_cams, 1, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, O.SPHERE, sc.m)
    st = orc.init_state(P0, op)
    prm = gpu_params(sc, povar.SPHERE, sc.m, povar.FP64, 1)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        for k in range(10):
            st, orep = orc.step(st, op)
            rep = pb.step(prm)
            assert rep.accepted == int(orep.accepted), k
            assert abs(rep.cost_after - orep.cost_after) <= 1e-10 * orep.cost_after, k
            assert rel(pb.cameras(), st.P) <= 1e-10, k
            assert rel(pb.points(), st.X) <= 1e-9, k


@pytest.mark.parametrize("manifold", [O.SPHERE, O.EUCLID])
def test_poba_one_step_mixed_close_to_oracle(manifold):
    sc = SCENES["traj"]()
    P0 = scenes.init_cameras(sc.n_cams, 4, normalize=True)
    orc = O.Problem(sc.n_cams, sc.n_points, sc.cam_idx, sc.pt_idx, sc.meas)
    op = oracle_params(sc, manifold, sc.m)
    _, orep = orc.step(orc.init_state(P0, op), op)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        rep = pb.step(gpu_params(sc, manifold, sc.m, povar.MIXED_FP32, 1))
        _, _, d = pb.last_step()
    assert rel(d, orep.delta) <= 1e-4
    assert abs(rep.cost_after - orep.cost_after) <= 1e-5 * orep.cost_after


def test_povar_step_after_poba_steps_starts_from_closed_form_landmarks():
    """After PoBA steps the landmarks are PoBA iterates; a PoVar step then
    re-solves them in closed form first and equals a PoVar step from the
    same cameras on a fresh handle."""
    sc = SCENES["tiny"]()
    P0 = scenes.init_cameras(sc.n_cams, 7, normalize=True)
    poba = gpu_params(sc, povar.SPHERE, 6, povar.FP64, 1)
    povar_prm = povar.make_params(eta=sc.eta, m=6, manifold=povar.SPHERE, precision=povar.FP64,
                                  schedule=1)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        for _ in range(3):
            pb.step(poba)
        P1 = pb.cameras()
        rep = pb.step(povar_prm)
    with povar.Problem.from_scene(sc) as fresh:
        fresh.set_cameras(P1, sc.eta)
        assert abs(fresh.cost(sc.eta) - rep.cost_before) <= 1e-12 * rep.cost_before


def test_poba_solve_reaches_the_povar_target_on_tiny():
    """The PoBA graph solve runs to the oracle's converged PoVar cost of the
    tiny scene (both minimize the same pOSE cost)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "converged_tiny.json")) as f:
        g = json.load(f)
    sc = scenes.scene_by_name("tiny", g["scene_seed"])
    P0 = scenes.init_cameras(sc.n_cams, g["init_seed"], normalize=True)
    prm = povar.make_params(eta=g["eta"], m=g["m"], series_eps=g["series_eps"],
                            lambda0=g["lambda0"], manifold=povar.EUCLID, precision=povar.FP64,
                            lambda_l=LAMBDA_L)
    target = g["series"]["F"] * (1.0 + 1e-5)
    with povar.Problem.from_scene(sc) as pb:
        pb.set_cameras(P0, sc.eta)
        rep, iters = pb.solve(prm, max_iters=300, ftol=0.0, target_cost=target)
        assert rep.cost_after <= target or pb.cost(sc.eta) <= target * (1 + 1e-9), iters
