"""FP64 CPU oracle for the second stage of the stratified problem: projective
refinement by Riemannian PoBA (RiPoBA).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. The
product path (the C-ABI CUDA library and its Python binding) never imports,
links or calls it, and this module imports nothing from the product.

What it computes (paper: Weber, Hong, Cremers, ECCV 2024):

* the projective reprojection cost of Eq. second_stage: for every
  observation (i, j, m_ij) with homogeneous camera P_i (3x4, vec(P_i) on the
  unit sphere of R^12) and homogeneous landmark X_j (on the unit sphere of
  R^4), the residual pi(P_i X_j) - m_ij with pi(y) = (y1 / y3, y2 / y3);
* the residual Jacobians J_p (2x12) and J_l (2x4) by the chain rule;
* the normal equation U, V, W, b_p, b_l and its restriction to the tangent
  spaces of both spheres (Sec. 4.3, Eq. riemannian_normal): tangent bases
  Q_p (12x11) and Q_l (4x3) with Q^T x = 0, projected damping
  Q^T (lambda I) Q = lambda I (D = I), U~ = Q_p^T U Q_p + lambda I,
  V~ = Q_l^T V Q_l + lambda_l lambda I, W~ = Q_p^T W Q_l, b~ = Q^T b;
* the Riemannian Schur complement S~ = U~ - W~ V~^-1 W~^T formed EXPLICITLY
  (dense), solved exactly (Cholesky), by the power series of Lemma 2 /
  Proposition 1, or by Schur-Jacobi preconditioned conjugate gradients;
  landmark updates by back-substitution;
* back-projection of the tangent updates, retraction by normalizing every
  camera and landmark vector, the trial cost, the Gauss-Newton predicted
  decrease, accept/reject and the damping rule of the first stage.

Readings where the paper is silent:

* The cost is the plain sum of squared residuals (no 1/2), as in stage 1.
* Landmark damping: the paper projects one lambda onto both tangent spaces;
  ``lambda_l`` scales the landmark share (1 = the paper's joint damping).
* The right-hand side is -(b~_p - W~ V~^-1 b~_l), the landmark update
  dl = -V~^-1 (b~_l + W~^T dp) (back-substitution); both are the joint
  Gauss-Newton step of the projected system (pinned).
* pred = ||r||^2 - ||r + J_p dP + J_l dX||^2 (the Gauss-Newton model
  decrease of the joint step, with the ambient updates dP = Q_p dp,
  dX = Q_l dl); accept iff the cost decreases; the damping rule, its floor
  and the series threshold rule are the first stage's conventions.

Parity status: every function is pinned by tests/test_oracle_ripoba_pins.py
except the conventions above (damping rule, threshold rule, vec order:
row-major P), which are "parity unpinned -- convention".
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .povar_oracle import (LAMBDA_MAX, LAMBDA_MIN, ReducedSystem, blockdiag, exact_step,
                           pcg_step, series_step)


# ---------------------------------------------------------------------------
# Residual and cost: Eq. second_stage
# ---------------------------------------------------------------------------

def project(P, X, cam_idx, pt_idx):
    """y = P_i X_j per observation (homogeneous image point), [n_obs, 3]."""
    Pm = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)
    return np.einsum("kab,kb->ka", Pm[cam_idx], np.asarray(X, dtype=np.float64)[pt_idx])


def residuals(P, X, cam_idx, pt_idx, meas):
    """pi(P_i X_j) - m_ij, pi(y) = (y1 / y3, y2 / y3); [n_obs, 2]."""
    y = project(P, X, cam_idx, pt_idx)
    return y[:, :2] / y[:, 2:3] - np.asarray(meas, dtype=np.float64)


def cost(P, X, cam_idx, pt_idx, meas):
    """Eq. second_stage: sum of squared reprojection residuals."""
    r = residuals(P, X, cam_idx, pt_idx, meas)
    return float(np.sum(r * r))


def dpi_dy(y):
    """Jacobian of pi at y, [n_obs, 2, 3]:
    [[1/y3, 0, -y1/y3^2], [0, 1/y3, -y2/y3^2]]."""
    n = y.shape[0]
    D = np.zeros((n, 2, 3))
    inv = 1.0 / y[:, 2]
    D[:, 0, 0] = inv
    D[:, 1, 1] = inv
    D[:, 0, 2] = -y[:, 0] * inv * inv
    D[:, 1, 2] = -y[:, 1] * inv * inv
    return D


def jacobian_blocks(P, X, cam_idx, pt_idx):
    """J_p = D (I_3 (x) X^T) (2x12, row-major vec(P)) and J_l = D P_i (2x4)."""
    Pm = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)
    Xk = np.asarray(X, dtype=np.float64)[pt_idx]
    y = np.einsum("kab,kb->ka", Pm[cam_idx], Xk)
    D = dpi_dy(y)
    Jp = np.einsum("kra,kb->krab", D, Xk).reshape(-1, 2, 12)
    Jl = np.einsum("kra,kab->krb", D, Pm[cam_idx])
    return Jp, Jl


def assemble_jacobian(Jp, Jl, cam_idx, pt_idx, n_cams, n_points):
    """Sparse J = [J_p | J_l] of shape (2 n_obs, 12 n_cams + 4 n_points)."""
    n = Jp.shape[0]
    rows = np.repeat(np.arange(2 * n).reshape(n, 2, 1), 12, axis=2)
    cols = (12 * np.asarray(cam_idx)[:, None, None] + np.arange(12)[None, None, :])
    cols = np.broadcast_to(cols, (n, 2, 12))
    rows_l = np.repeat(np.arange(2 * n).reshape(n, 2, 1), 4, axis=2)
    cols_l = (12 * n_cams + 4 * np.asarray(pt_idx)[:, None, None] + np.arange(4)[None, None, :])
    cols_l = np.broadcast_to(cols_l, (n, 2, 4))
    r = np.concatenate([rows.ravel(), rows_l.ravel()])
    c = np.concatenate([cols.ravel(), cols_l.ravel()])
    v = np.concatenate([Jp.ravel(), Jl.ravel()])
    return sp.csr_matrix((v, (r, c)), shape=(2 * n, 12 * n_cams + 4 * n_points))


# ---------------------------------------------------------------------------
# Normal equation and its Riemannian restriction (Sec. 4.3)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class NormalEquations:
    U: np.ndarray          # [n_cams, 12, 12]  J_p^T J_p summed per camera
    V: np.ndarray          # [n_points, 4, 4]  J_l^T J_l summed per landmark
    W: sp.csr_matrix       # [12 n_cams, 4 n_points]  J_p^T J_l
    b_p: np.ndarray        # [12 n_cams]  J_p^T r
    b_l: np.ndarray        # [4 n_points] J_l^T r
    r: np.ndarray          # [n_obs, 2]


def normal_equations(P, X, cam_idx, pt_idx, meas, n_cams, n_points):
    """U, V, W, b_p, b_l from the sparse Jacobian J = [J_p | J_l] by explicit
    sparse products (the block structure is read off J^T J)."""
    r = residuals(P, X, cam_idx, pt_idx, meas)
    Jp, Jl = jacobian_blocks(P, X, cam_idx, pt_idx)
    J = assemble_jacobian(Jp, Jl, cam_idx, pt_idx, n_cams, n_points)
    H = (J.T @ J).tocsr()
    b = J.T @ r.ravel()
    npc = 12 * n_cams
    Hd = H[:npc, :npc].toarray()
    U = np.stack([Hd[12 * i:12 * i + 12, 12 * i:12 * i + 12] for i in range(n_cams)])
    Hl = H[npc:, npc:]
    V = np.stack([Hl[4 * j:4 * j + 4, 4 * j:4 * j + 4].toarray() for j in range(n_points)])
    W = H[:npc, npc:].tocsr()
    return NormalEquations(U=U, V=V, W=W, b_p=b[:npc], b_l=b[npc:], r=r)


def sphere_tangent_bases(Xs):
    """Orthonormal bases of the tangent spaces {v : x^T v = 0} of the unit
    spheres at the rows of Xs: [n, d, d-1] with Q^T x = 0 and Q^T Q = I
    (the last d-1 right singular vectors of the 1 x d matrix x^T)."""
    Xs = np.asarray(Xs, dtype=np.float64)
    n, d = Xs.shape
    Q = np.empty((n, d, d - 1))
    for i in range(n):
        _, _, Vt = np.linalg.svd(Xs[i][None, :])
        Q[i] = Vt[1:].T
    return Q


@dataclasses.dataclass
class RiemannianSystem:
    Ut: np.ndarray          # [n_cams, 11, 11]  Q_p^T U Q_p + lambda I
    Vt: np.ndarray          # [n_points, 3, 3]  Q_l^T V Q_l + lambda_l lambda I
    Wt: sp.csr_matrix       # [11 n_cams, 3 n_points]
    bp: np.ndarray          # [11 n_cams]
    bl: np.ndarray          # [3 n_points]
    Qp: np.ndarray
    Ql: np.ndarray
    lam: float


def riemannian_system(ne: NormalEquations, Qp, Ql, lam, lambda_l=1.0):
    """Eq. riemannian_normal with the projected damping (D_p = D_l = I)."""
    kp, kl = Qp.shape[2], Ql.shape[2]
    Ut = np.einsum("nai,nab,nbj->nij", Qp, ne.U, Qp) + lam * np.eye(kp)[None]
    Vt = np.einsum("nai,nab,nbj->nij", Ql, ne.V, Ql) + lambda_l * lam * np.eye(kl)[None]
    Wt = (blockdiag(Qp).T @ ne.W @ blockdiag(Ql)).tocsr()
    bp = np.einsum("nab,na->nb", Qp, ne.b_p.reshape(-1, 12)).ravel()
    bl = np.einsum("nab,na->nb", Ql, ne.b_l.reshape(-1, 4)).ravel()
    return RiemannianSystem(Ut=Ut, Vt=Vt, Wt=Wt, bp=bp, bl=bl, Qp=Qp, Ql=Ql, lam=lam)


def reduced(rsys: RiemannianSystem) -> ReducedSystem:
    """The Riemannian Schur complement S~ = U~ - W~ V~^-1 W~^T (dense) and
    g = -(b~_p - W~ V~^-1 b~_l), in the first stage's ReducedSystem form so
    that its exact / series / PCG solvers apply unchanged."""
    Vinv = blockdiag(np.linalg.inv(rsys.Vt))
    S = sla.block_diag(*rsys.Ut) - (rsys.Wt @ Vinv @ rsys.Wt.T).toarray()
    g = -(rsys.bp - rsys.Wt @ (Vinv @ rsys.bl))
    return ReducedSystem(Ut=rsys.Ut, Wt=rsys.Wt, Vinv=Vinv, S=S, g=g, Q=rsys.Qp, lam=rsys.lam)


def back_substitute(rsys: RiemannianSystem, rs: ReducedSystem, dp):
    """Tangent landmark update dl = -V~^-1 (b~_l + W~^T dp)."""
    return -(rs.Vinv @ (rsys.bl + rsys.Wt.T @ dp))


def normalize_rows(A):
    A = np.asarray(A, dtype=np.float64)
    return A / np.linalg.norm(A, axis=1, keepdims=True)


# ---------------------------------------------------------------------------
# One RiPoBA iteration and the solve loop
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    lambda0: float = 1e-4
    m: int = 21                 # number of series terms
    series_eps: float = 0.0     # 0: exactly m terms
    lambda_l: float = 1.0       # landmark damping lambda_l * lambda
    solver: str = "series"      # "series" | "exact" | "pcg"
    pcg_iters: int = 500
    pcg_tol: float = 0.0


@dataclasses.dataclass
class State:
    P: np.ndarray               # [n_cams, 12] unit rows
    X: np.ndarray               # [n_points, 4] unit rows
    F: float
    lam: float
    nu: float = 2.0
    iteration: int = 0


@dataclasses.dataclass
class StepReport:
    cost_before: float
    cost_after: float
    pred: float
    rho: float
    lambda_used: float
    lambda_next: float
    accepted: bool
    terms_used: int
    dP: np.ndarray              # [n_cams, 12] ambient camera update
    dX: np.ndarray              # [n_points, 4] ambient landmark update


class Problem:
    def __init__(self, n_cams, n_points, cam_idx, pt_idx, meas):
        self.n_cams, self.n_points = int(n_cams), int(n_points)
        self.cam_idx = np.asarray(cam_idx, dtype=np.int64)
        self.pt_idx = np.asarray(pt_idx, dtype=np.int64)
        self.meas = np.asarray(meas, dtype=np.float64)

    def cost(self, P, X):
        return cost(P, X, self.cam_idx, self.pt_idx, self.meas)

    def init_state(self, P, X, params: Params) -> State:
        P = normalize_rows(np.asarray(P, dtype=np.float64).reshape(self.n_cams, 12))
        X = normalize_rows(np.asarray(X, dtype=np.float64).reshape(self.n_points, 4))
        return State(P=P, X=X, F=self.cost(P, X), lam=params.lambda0)

    def system(self, st: State, params: Params):
        ne = normal_equations(st.P, st.X, self.cam_idx, self.pt_idx, self.meas,
                              self.n_cams, self.n_points)
        Qp = sphere_tangent_bases(st.P)
        Ql = sphere_tangent_bases(st.X)
        rsys = riemannian_system(ne, Qp, Ql, st.lam, params.lambda_l)
        return ne, rsys, reduced(rsys)

    def step(self, st: State, params: Params):
        """One RiPoBA iteration from (P, X) with damping st.lam."""
        ne, rsys, rs = self.system(st, params)
        if params.solver == "exact":
            dp, terms = exact_step(rs), 0
        elif params.solver == "pcg":
            dp, terms = pcg_step(rs, params.pcg_iters, params.pcg_tol)
        else:
            dp, terms = series_step(rs, params.m, params.series_eps)
        dl = back_substitute(rsys, rs, dp)
        dP = np.einsum("nab,nb->na", rsys.Qp, dp.reshape(self.n_cams, -1))
        dX = np.einsum("nab,nb->na", rsys.Ql, dl.reshape(self.n_points, -1))
        P_new = normalize_rows(st.P + dP)
        X_new = normalize_rows(st.X + dX)
        F_new = self.cost(P_new, X_new)
        Jp, Jl = jacobian_blocks(st.P, st.X, self.cam_idx, self.pt_idx)
        lin = (ne.r + np.einsum("kra,ka->kr", Jp, dP[self.cam_idx])
               + np.einsum("kra,ka->kr", Jl, dX[self.pt_idx]))
        pred = float(np.sum(ne.r * ne.r) - np.sum(lin * lin))
        rho = (st.F - F_new) / pred if pred > 0 else 0.0
        accepted = F_new < st.F
        rep = StepReport(cost_before=st.F, cost_after=F_new, pred=pred, rho=rho,
                         lambda_used=st.lam, lambda_next=0.0, accepted=bool(accepted),
                         terms_used=terms, dP=dP, dX=dX)
        if accepted:
            lam = max(st.lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), LAMBDA_MIN)
            new = State(P=P_new, X=X_new, F=F_new, lam=lam, nu=2.0,
                        iteration=st.iteration + 1)
        else:
            new = State(P=st.P, X=st.X, F=st.F, lam=st.lam * st.nu, nu=2.0 * st.nu,
                        iteration=st.iteration + 1)
        rep.lambda_next = new.lam
        return new, rep

    def solve(self, st: State, params: Params, max_iters=50, ftol=1e-6):
        """LM loop of Sec. 5.2: at most max_iters iterations, stopping after
        an accepted step whose relative decrease is below ftol."""
        trace = [st.F]
        for _ in range(max_iters):
            st, rep = self.step(st, params)
            trace.append(st.F)
            if rep.accepted and (rep.cost_before - rep.cost_after) < ftol * rep.cost_before:
                break
            if st.lam > LAMBDA_MAX:
                break
        return st, trace
