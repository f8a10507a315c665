"""FP64 CPU oracle for the Power Variable Projection (PoVar) inner solve.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. The
product path (the C-ABI CUDA library ``libpovar`` and its Python binding) never
imports, links or calls it, and this module imports nothing from the product.

What it computes (paper: Weber, Hong, Cremers, "Power Variable Projection for
Initialization-Free Large-Scale Bundle Adjustment", ECCV 2024):

* the pOSE residual and cost of the first, separable stage
  (Eq. ba_first_stage and Eq. pose, Sec. 3.2);
* the closed-form landmark of Variable Projection (Eq. update_landmark,
  Sec. 4.1), solved from the per-landmark 3x3 normal equations;
* the RW2 normal equation U_lambda, V_0, W, b_p, b_l (Sec. 4.1), built from
  the residual Jacobians J_p, J_l by explicit sparse products;
* the tangent-space restriction of the camera block to the unit-norm camera
  manifold (Sec. 4.3: tangent basis, projected normal equation, damping
  projected as Q^T (lambda I) Q = lambda I, back-projection, retraction by
  normalization) -- used when ``manifold == SPHERE``;
* the Schur complement S formed EXPLICITLY as a dense matrix (Eq. schur_varpro
  and its Riemannian version S~ of Sec. 4.3), solved either exactly by dense
  Cholesky or by the truncated power series of Proposition 1 / the PoVar
  series x(m) (Sec. 4.2);
* one damped VarPro step: pose update, closed-form landmark re-solve at the new
  cameras (Sec. 4.2: the landmarks are eliminated in closed form),
  gain ratio, accept/reject and damping update;
* the comparison solvers of Sec. 5.2 on the same problem: PoBA (joint
  Levenberg-Marquardt whose damped Schur complement is inverted by the
  power series, landmarks updated by back-substitution; Sec. 2) and the
  "iterative" VarPro baseline (conjugate gradients on the reduced camera
  system with the Schur-Jacobi preconditioner).

Readings where the paper is silent or garbled:

* Sign of the right-hand side of Eq. pose_update: the paper's series x(m)
  carries a leading minus, so the step solves S dx = -(b_p - W V^-1 b_l).
* Series length: ``m`` is the NUMBER of terms, sum_{i<m}; the paper's
  "order 20" corresponds to m = 21.
* Series threshold ("threshold 0.01", Sec. 5.2): after term k the series stops
  when ||x_k||_2 <= eps * ||delta_k||_2; eps = 0 runs exactly m terms.
* D_p = I; the damping update is the Madsen-Nielsen rule (on accept:
  lambda *= max(1/3, 1 - (2 rho - 1)^3), nu = 2; on reject: lambda *= nu,
  nu *= 2), with lambda kept >= LAMBDA_MIN = 1e-8; a step is accepted iff
  the cost decreases.
* The predicted decrease is pred = 2 g^T d - d^T (S - lambda I) d.
* vec(P) is row-major (rows p1, p2, p3 of the 3x4 camera).
* Rank-deficient V_j: pseudo-inverse when cond(V_j) > 1e12 (footnote of
  Sec. 4.2); it never triggers on the configured scenes.

Parity status: every function is pinned by tests/test_oracle_pins.py except
the conventions above (damping rule, series threshold rule, vec order), which
are "parity unpinned -- convention": the CUDA path implements the same
convention and nothing in the paper fixes them.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

EUCLID = 0
SPHERE = 1
PINV_COND = 1e12
LAMBDA_MIN = 1e-8    # damping floor (convention; the paper gives no bound)
LAMBDA_MAX = 1e30    # damping ceiling: the solve stops as diverged above it


# ---------------------------------------------------------------------------
# Residual and cost: Eq. pose / Eq. ba_first_stage (Sec. 3.2)
# ---------------------------------------------------------------------------

def pose_residuals(P, X, cam_idx, pt_idx, meas, eta):
    """pOSE residual per observation, literally as Eq. pose writes it.

    For observation (i, j, m_ij) with camera x_p^i (3x4) and landmark
    x~_l^j = (X_j, 1):
        rows 0-1: sqrt(1 - eta) * (x_p^{i,1:2} x~ - (x_p^{i,3} x~) m_ij)
        rows 2-3: sqrt(eta)     * (x_p^{i,1:2} x~ - m_ij)
    Returns an [n_obs, 4] array.
    """
    Pc = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)[cam_idx]
    xt = np.concatenate([X[pt_idx], np.ones((len(pt_idx), 1))], axis=1)
    y = np.einsum("nij,nj->ni", Pc, xt)
    r = np.empty((len(cam_idx), 4))
    r[:, 0:2] = np.sqrt(1.0 - eta) * (y[:, 0:2] - y[:, 2:3] * meas)
    r[:, 2:4] = np.sqrt(eta) * (y[:, 0:2] - meas)
    return r


def cost(P, X, cam_idx, pt_idx, meas, eta):
    """F = ||r||_2^2 (Eq. ba_first_stage with the pOSE residual)."""
    r = pose_residuals(P, X, cam_idx, pt_idx, meas, eta)
    return float(np.sum(r * r))


# ---------------------------------------------------------------------------
# Jacobians of the residual (chain rule through y = x_p^i x~_j)
# ---------------------------------------------------------------------------

def dresidual_dy(meas, eta):
    """B_k = d r_k / d y_k, where y_k = x_p^i x~_j (3-vector); Eq. pose is
    linear in y, so B_k depends only on m_ij and eta. Returns [n, 4, 3]."""
    s1, s2 = np.sqrt(1.0 - eta), np.sqrt(eta)
    n = meas.shape[0]
    B = np.zeros((n, 4, 3))
    B[:, 0, 0] = s1
    B[:, 0, 2] = -s1 * meas[:, 0]
    B[:, 1, 1] = s1
    B[:, 1, 2] = -s1 * meas[:, 1]
    B[:, 2, 0] = s2
    B[:, 3, 1] = s2
    return B


def jacobian_blocks(P, X, cam_idx, pt_idx, meas, eta):
    """Per-observation Jacobian blocks of the pOSE residual.

    J_p (4x12): derivative w.r.t. the row-major vec of camera i; since
    y = x_p x~, dy_a / dP[a, b] = x~_b, so J_p[:, 4a + b] = B[:, a] x~_b.
    J_l (4x3):  derivative w.r.t. the inhomogeneous landmark X_j (the last
    homogeneous coordinate is fixed to 1), J_l = B P[:, 0:3].
    """
    B = dresidual_dy(meas, eta)
    Pc = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)[cam_idx]
    xt = np.concatenate([X[pt_idx], np.ones((len(pt_idx), 1))], axis=1)
    Jp = np.einsum("nra,nb->nrab", B, xt).reshape(-1, 4, 12)
    Jl = np.einsum("nra,nac->nrc", B, Pc[:, :, 0:3])
    return Jp, Jl


def assemble_jacobian(Jp, Jl, cam_idx, pt_idx, n_cams, n_points):
    """Sparse J = [J_p | J_l] with 4 rows per observation, the 12 n_cams
    camera columns first and the 3 n_points landmark columns after them."""
    n = len(cam_idx)
    rows = np.arange(4 * n).reshape(n, 4)
    r_p = np.repeat(rows[:, :, None], 12, axis=2)
    c_p = (12 * cam_idx[:, None, None] + np.arange(12)[None, None, :]) \
        + np.zeros((n, 4, 12), dtype=np.int64)
    r_l = np.repeat(rows[:, :, None], 3, axis=2)
    c_l = (12 * n_cams + 3 * pt_idx[:, None, None] + np.arange(3)[None, None, :]) \
        + np.zeros((n, 4, 3), dtype=np.int64)
    data = np.concatenate([Jp.ravel(), Jl.ravel()])
    ri = np.concatenate([r_p.ravel(), r_l.ravel()])
    ci = np.concatenate([c_p.ravel(), c_l.ravel()])
    return sp.csr_matrix((data, (ri, ci)), shape=(4 * n, 12 * n_cams + 3 * n_points))


# ---------------------------------------------------------------------------
# Closed-form landmarks: Eq. update_landmark (Sec. 4.1)
# ---------------------------------------------------------------------------

def sym_inverse_batch(V):
    """Inverses of a stack of symmetric PSD 3x3 blocks; the Moore-Penrose
    pseudo-inverse for blocks that are numerically rank-deficient
    (cond > PINV_COND; footnote of Sec. 4.2). Returns (inverses, n_pinv)."""
    V = np.asarray(V, dtype=np.float64)
    w = np.linalg.eigvalsh(V)
    bad = (w[:, -1] <= 0) | (w[:, 0] <= w[:, -1] / PINV_COND)
    out = np.empty_like(V)
    if np.any(~bad):
        out[~bad] = np.linalg.inv(V[~bad])
    if np.any(bad):
        out[bad] = np.linalg.pinv(V[bad], rcond=1.0 / PINV_COND, hermitian=True)
    return out, int(bad.sum())


def landmarks(P, cam_idx, pt_idx, meas, eta, n_points, return_V=False):
    """x~_l^*(x_p) = argmin ||G(x_p) x~_l - z(x_p)||^2 with the last
    coordinate of x~_l fixed to 1 (Eq. update_landmark).

    With the camera fixed, the residual is affine in X_j: r = J_l X + r(X=0).
    Each landmark's least-squares problem is solved from its 3x3 normal
    equations V_j X_j = -h_j, V_j = sum J_l^T J_l, h_j = sum J_l^T r(X=0).
    """
    X0 = np.zeros((n_points, 3))
    r0 = pose_residuals(P, X0, cam_idx, pt_idx, meas, eta)
    _, Jl = jacobian_blocks(P, X0, cam_idx, pt_idx, meas, eta)
    V = np.zeros((n_points, 3, 3))
    h = np.zeros((n_points, 3))
    np.add.at(V, pt_idx, np.einsum("nra,nrb->nab", Jl, Jl))
    np.add.at(h, pt_idx, np.einsum("nra,nr->na", Jl, r0))
    Vi, n_pinv = sym_inverse_batch(V)
    X = -np.einsum("nab,nb->na", Vi, h)
    if return_V:
        return X, V, n_pinv
    return X


def landmark_bruteforce(P, cam_idx, pt_idx, meas, eta, n_points):
    """Pin for ``landmarks``: stack every observation of landmark j into a
    4k x 4 homogeneous system and call the library least-squares solver on
    the 4k x 3 part with the fourth column moved to the right-hand side."""
    Pm = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)
    X = np.empty((n_points, 3))
    s1, s2 = np.sqrt(1.0 - eta), np.sqrt(eta)
    for j in range(n_points):
        ks = np.nonzero(pt_idx == j)[0]
        rows, rhs = [], []
        for k in ks:
            Pi = Pm[cam_idx[k]]
            u, v = meas[k]
            # the four residual rows of Eq. pose as functions of (X, 1)
            rows.append(s1 * (Pi[0] - u * Pi[2]))
            rows.append(s1 * (Pi[1] - v * Pi[2]))
            rows.append(s2 * Pi[0])
            rows.append(s2 * Pi[1])
            rhs.extend([0.0, 0.0, s2 * u, s2 * v])
        A = np.array(rows)
        b = np.array(rhs)
        X[j] = np.linalg.lstsq(A[:, :3], b - A[:, 3], rcond=None)[0]
    return X


# ---------------------------------------------------------------------------
# RW2 normal equation (Sec. 4.1)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class NormalEquations:
    U: np.ndarray        # [n_cams, 12, 12]  J_p^T J_p (undamped)
    V: np.ndarray        # [n_points, 3, 3]  V_0 = J_l^T J_l
    W: sp.csr_matrix     # [12 n_cams, 3 n_points]  J_p^T J_l
    b_p: np.ndarray      # [12 n_cams]  J_p^T r
    b_l: np.ndarray      # [3 n_points] J_l^T r
    r: np.ndarray        # [n_obs, 4]


def normal_equations(P, X, cam_idx, pt_idx, meas, eta, n_cams, n_points):
    """U = J_p^T J_p, V_0 = J_l^T J_l, W = J_p^T J_l, b_p = J_p^T r,
    b_l = J_l^T r, by explicit products of the sparse Jacobian (Sec. 4.1)."""
    r = pose_residuals(P, X, cam_idx, pt_idx, meas, eta)
    Jp, Jl = jacobian_blocks(P, X, cam_idx, pt_idx, meas, eta)
    J = assemble_jacobian(Jp, Jl, cam_idx, pt_idx, n_cams, n_points)
    npc = 12 * n_cams
    J_p = J[:, :npc]
    J_l = J[:, npc:]
    Upp = (J_p.T @ J_p).toarray()
    U = np.stack([Upp[12 * i:12 * i + 12, 12 * i:12 * i + 12] for i in range(n_cams)])
    Vll = (J_l.T @ J_l).tocsr()
    V = np.zeros((n_points, 3, 3))
    Vc = Vll.tocoo()
    V[Vc.row // 3, Vc.row % 3, Vc.col % 3] = Vc.data
    W = (J_p.T @ J_l).tocsr()
    rv = r.ravel()
    return NormalEquations(U=U, V=V, W=W, b_p=J_p.T @ rv, b_l=J_l.T @ rv, r=r)


# ---------------------------------------------------------------------------
# Tangent space of the unit-norm camera manifold (Sec. 4.3)
# ---------------------------------------------------------------------------

def tangent_bases(P, manifold):
    """Per-camera orthonormal basis Q_i of the tangent space at x~_p^i:
    (x~_p^{i,perp})^T x~_p^i = 0 with orthonormal columns, taken from the
    right singular vectors of the 1 x 12 row vec(P_i). EUCLID: Q_i = I_12."""
    P = np.asarray(P, dtype=np.float64)
    n = P.shape[0]
    if manifold == EUCLID:
        return np.broadcast_to(np.eye(12), (n, 12, 12)).copy()
    Q = np.empty((n, 12, 11))
    for i in range(n):
        _, _, Vt = np.linalg.svd(P[i][None, :])
        Q[i] = Vt[1:].T
    return Q


def blockdiag(blocks):
    return sp.csr_matrix(sp.block_diag([sp.coo_matrix(b) for b in blocks], format="csr"))


# ---------------------------------------------------------------------------
# Reduced camera system (Eq. pose_update, Eq. schur_varpro, Sec. 4.3)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class ReducedSystem:
    Ut: np.ndarray            # [n_cams, k, k]  Q^T U Q + lambda I
    Wt: sp.csr_matrix         # [k n_cams, 3 n_points]  Q^T W
    Vinv: sp.csr_matrix       # block-diagonal V_0^{-1} (pseudo-inverse if needed)
    S: np.ndarray             # dense Schur complement
    g: np.ndarray             # right-hand side -(b~_p - W~ V^-1 b_l)
    Q: np.ndarray             # tangent bases
    lam: float


def reduced_system(ne: NormalEquations, Q, lam):
    """S = U~_lambda - W~ V_0^{-1} W~^T formed explicitly (dense) and
    g = -(b~_p - W~ V_0^{-1} b_l), with U~ = Q^T U Q + lambda I,
    W~ = Q^T W, b~_p = Q^T b_p (projected normal equation of Sec. 4.3 with
    D_p = I; for EUCLID Q = I and this is Eq. pose_update)."""
    n_cams, _, k = Q.shape
    Ut = np.einsum("nai,nab,nbj->nij", Q, ne.U, Q) + lam * np.eye(k)[None]
    Qbd = blockdiag(Q)                       # [12 n, k n]
    Wt = (Qbd.T @ ne.W).tocsr()
    Vinv = blockdiag(sym_inverse_batch(ne.V)[0])
    WVW = (Wt @ Vinv @ Wt.T).toarray()
    S = sla.block_diag(*Ut) - WVW
    g = -(Qbd.T @ ne.b_p - Wt @ (Vinv @ ne.b_l))
    return ReducedSystem(Ut=Ut, Wt=Wt, Vinv=Vinv, S=S, g=g, Q=Q, lam=lam)


def exact_step(rs: ReducedSystem):
    """delta = S^{-1} g by dense Cholesky (S is SPD: S >= lambda I).

    When S is so ill-conditioned (cond ~ 1e16, e.g. a landmark drifting to
    infinity after the cost has converged) that rounding makes it
    numerically indefinite, the solve falls back to the eigen-decomposition
    of S with every eigenvalue floored at lambda, the bound S >= lambda I
    holds in exact arithmetic."""
    try:
        c = sla.cho_factor(rs.S, lower=True)
        return sla.cho_solve(c, rs.g)
    except np.linalg.LinAlgError:
        w, E = np.linalg.eigh(rs.S)
        w = np.maximum(w, rs.lam)
        return E @ ((E.T @ rs.g) / w)


def series_step(rs: ReducedSystem, m, eps=0.0):
    """PoVar series (Sec. 4.2; Proposition 1 applied to S):
    delta = sum_{i<m} M^i U~^{-1} g with M = U~^{-1} W~ V^{-1} W~^T.
    Stops early after term k >= 1 when ||x_k|| <= eps * ||delta_k||.
    Returns (delta, number of terms used)."""
    Uinv = sla.block_diag(*[np.linalg.inv(b) for b in rs.Ut])
    x = Uinv @ rs.g
    delta = x.copy()
    terms = 1
    for _ in range(1, m):
        x = Uinv @ (rs.Wt @ (rs.Vinv @ (rs.Wt.T @ x)))
        delta += x
        terms += 1
        if eps > 0 and np.linalg.norm(x) <= eps * np.linalg.norm(delta):
            break
    return delta, terms


def schur_jacobi_blocks(rs: ReducedSystem):
    """Diagonal blocks S_ii of the explicit Schur complement (the Schur-Jacobi
    preconditioner of the "iterative" baseline, Sec. 5.2)."""
    k = rs.Ut.shape[1]
    n = rs.Ut.shape[0]
    return np.stack([rs.S[k * i:k * i + k, k * i:k * i + k] for i in range(n)])


def pcg_step(rs: ReducedSystem, iters, tol=0.0):
    """Conjugate gradients on S delta = g from delta = 0, preconditioned by
    the inverse diagonal blocks of S (Schur-Jacobi): the "iterative" VarPro
    baseline of Sec. 5.2 (at most 500 inner iterations there). Stops after
    `iters` iterations, or when ||g - S delta|| <= tol ||g|| (tol > 0).
    Returns (delta, iterations)."""
    k = rs.Ut.shape[1]
    Minv = sla.block_diag(*[np.linalg.inv(b) for b in schur_jacobi_blocks(rs)])
    g = rs.g
    delta = np.zeros_like(g)
    r = g.copy()
    z = Minv @ r
    p = z.copy()
    rz = float(r @ z)
    gn = float(np.linalg.norm(g))
    it = 0
    for it in range(1, iters + 1):
        Sp = rs.S @ p
        alpha = rz / float(p @ Sp)
        delta += alpha * p
        r -= alpha * Sp
        if tol > 0 and np.linalg.norm(r) <= tol * gn:
            break
        z = Minv @ r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    assert k > 0
    return delta, it


def series_matrix(rs: ReducedSystem):
    """Dense M = U~^{-1} W~ V^{-1} W~^T (used by the Lemma 1 / 2 pins)."""
    Uinv = sla.block_diag(*[np.linalg.inv(b) for b in rs.Ut])
    return Uinv @ (rs.Wt @ rs.Vinv @ rs.Wt.T).toarray()


# ---------------------------------------------------------------------------
# One damped VarPro step and the solve loop
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Params:
    eta: float = 0.1
    lambda0: float = 1e-4
    m: int = 10                 # number of series terms
    series_eps: float = 0.0     # 0: exactly m terms
    manifold: int = SPHERE
    solver: str = "series"      # "series" | "exact" | "pcg"
    method: str = "varpro"      # "varpro" (PoVar) | "poba" (joint LM, Sec. 2 / PoBA)
    lambda_l: float = 1.0       # PoBA: landmark damping lambda_l * lambda
    pcg_iters: int = 500        # "pcg": inner iterations (Sec. 5.2)
    pcg_tol: float = 0.0        # "pcg": stop at ||res|| <= tol ||g|| (0: run pcg_iters)


@dataclasses.dataclass
class State:
    P: np.ndarray               # [n_cams, 12]
    X: np.ndarray               # [n_points, 3]
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
    delta: np.ndarray           # [n_cams, 12] step in the ambient space
    P_trial: np.ndarray         # [n_cams, 12]


class Problem:
    def __init__(self, n_cams, n_points, cam_idx, pt_idx, meas):
        self.n_cams = int(n_cams)
        self.n_points = int(n_points)
        self.cam_idx = np.asarray(cam_idx, dtype=np.int64)
        self.pt_idx = np.asarray(pt_idx, dtype=np.int64)
        self.meas = np.asarray(meas, dtype=np.float64)

    def landmarks(self, P, eta):
        return landmarks(P, self.cam_idx, self.pt_idx, self.meas, eta, self.n_points)

    def cost(self, P, X, eta):
        return cost(P, X, self.cam_idx, self.pt_idx, self.meas, eta)

    def normal_equations(self, P, X, eta):
        return normal_equations(P, X, self.cam_idx, self.pt_idx, self.meas, eta,
                                self.n_cams, self.n_points)

    def init_state(self, P0, params: Params):
        P = np.array(P0, dtype=np.float64).reshape(self.n_cams, 12)
        X = self.landmarks(P, params.eta)
        return State(P=P, X=X, F=self.cost(P, X, params.eta), lam=params.lambda0)

    def step(self, st: State, params: Params):
        """One damped VarPro iteration at (P, X*(P)), or one PoBA iteration
        at (P, X) when params.method == "poba"."""
        if params.method == "poba":
            return self.poba_step(st, params)
        ne = self.normal_equations(st.P, st.X, params.eta)
        Q = tangent_bases(st.P, params.manifold)
        rs = reduced_system(ne, Q, st.lam)
        if params.solver == "exact":
            d, terms = exact_step(rs), 0
        elif params.solver == "pcg":
            d, terms = pcg_step(rs, params.pcg_iters, params.pcg_tol)
        else:
            d, terms = series_step(rs, params.m, params.series_eps)
        k = Q.shape[2]
        dP = np.einsum("nab,nb->na", Q, d.reshape(self.n_cams, k))
        P_new = st.P + dP
        if params.manifold == SPHERE:
            P_new = P_new / np.linalg.norm(P_new, axis=1, keepdims=True)
        X_new = self.landmarks(P_new, params.eta)
        F_new = self.cost(P_new, X_new, params.eta)
        pred = float(2.0 * rs.g @ d - d @ (rs.S @ d - st.lam * d))
        rho = (st.F - F_new) / pred if pred > 0 else 0.0
        accepted = F_new < st.F
        lam_used = st.lam
        rep = StepReport(cost_before=st.F, cost_after=F_new, pred=pred, rho=rho,
                         lambda_used=lam_used, lambda_next=0.0,
                         accepted=bool(accepted), terms_used=terms, delta=dP,
                         P_trial=P_new)
        if accepted:
            lam = max(st.lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), LAMBDA_MIN)
            new = State(P=P_new, X=X_new, F=F_new, lam=lam, nu=2.0,
                        iteration=st.iteration + 1)
        else:
            new = State(P=st.P, X=st.X, F=st.F, lam=st.lam * st.nu,
                        nu=2.0 * st.nu, iteration=st.iteration + 1)
        rep.lambda_next = new.lam
        return new, rep

    def poba_step(self, st: State, params: Params):
        """One iteration of joint Levenberg-Marquardt on the pOSE cost with
        the power series on the damped Schur complement (PoBA, Sec. 2): at
        (P, X) -- X is not re-eliminated -- the joint normal equation
        [[U + lambda I, W], [W^T, V + lambda_l lambda I]] (dP, dX) =
        -(b_p, b_l) is reduced to S dP = -(b_p - W V_lambda^-1 b_l) with
        S = U_lambda - W V_lambda^-1 W^T (tangent-projected on the sphere as
        in Sec. 4.3), solved by the series (or exactly / by PCG), and the
        landmarks follow by back-substitution dX = -V_lambda^-1 (b_l + W^T dP).
        The trial cost is evaluated at (P + dP, X + dX) (retracted cameras);
        pred is the Gauss-Newton model decrease ||r||^2 - ||r + J (dP, dX)||^2."""
        eta, lam = params.eta, st.lam
        ne = self.normal_equations(st.P, st.X, eta)
        Q = tangent_bases(st.P, params.manifold)
        n_c, _, k = Q.shape
        Ut = np.einsum("nai,nab,nbj->nij", Q, ne.U, Q) + lam * np.eye(k)[None]
        Vd = ne.V + params.lambda_l * lam * np.eye(3)[None]
        Vinv = blockdiag(np.linalg.inv(Vd))
        Qbd = blockdiag(Q)
        Wt = (Qbd.T @ ne.W).tocsr()
        S = sla.block_diag(*Ut) - (Wt @ Vinv @ Wt.T).toarray()
        g = -(Qbd.T @ ne.b_p - Wt @ (Vinv @ ne.b_l))
        rs = ReducedSystem(Ut=Ut, Wt=Wt, Vinv=Vinv, S=S, g=g, Q=Q, lam=lam)
        if params.solver == "exact":
            d, terms = exact_step(rs), 0
        elif params.solver == "pcg":
            d, terms = pcg_step(rs, params.pcg_iters, params.pcg_tol)
        else:
            d, terms = series_step(rs, params.m, params.series_eps)
        dP = np.einsum("nab,nb->na", Q, d.reshape(n_c, k))
        dX = -(Vinv @ (ne.b_l + ne.W.T @ dP.ravel())).reshape(-1, 3)
        P_new = st.P + dP
        if params.manifold == SPHERE:
            P_new = P_new / np.linalg.norm(P_new, axis=1, keepdims=True)
        X_new = st.X + dX
        F_new = self.cost(P_new, X_new, eta)
        Jp, Jl = jacobian_blocks(st.P, st.X, self.cam_idx, self.pt_idx, self.meas, eta)
        J = assemble_jacobian(Jp, Jl, self.cam_idx, self.pt_idx, self.n_cams, self.n_points)
        r = ne.r.ravel()
        step = np.concatenate([dP.ravel(), dX.ravel()])
        pred = float(r @ r - np.sum((r + J @ step) ** 2))
        rho = (st.F - F_new) / pred if pred > 0 else 0.0
        accepted = F_new < st.F
        rep = StepReport(cost_before=st.F, cost_after=F_new, pred=pred, rho=rho,
                         lambda_used=lam, lambda_next=0.0, accepted=bool(accepted),
                         terms_used=terms, delta=dP, P_trial=P_new)
        if accepted:
            lam_n = max(lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), LAMBDA_MIN)
            new = State(P=P_new, X=X_new, F=F_new, lam=lam_n, nu=2.0,
                        iteration=st.iteration + 1)
        else:
            new = State(P=st.P, X=st.X, F=st.F, lam=lam * st.nu, nu=2.0 * st.nu,
                        iteration=st.iteration + 1)
        rep.lambda_next = new.lam
        return new, rep

    def solve(self, P0, params: Params, max_iters=50, ftol=1e-6, target_cost=0.0,
              callback=None):
        """LM / VarPro loop: stops on an accepted step whose relative decrease
        is below ``ftol`` (Sec. 5.2: 50 iterations, ftol 1e-6), when the cost
        reaches ``target_cost`` (> 0), or after ``max_iters``."""
        st = self.init_state(P0, params)
        reports = []
        for _ in range(max_iters):
            st, rep = self.step(st, params)
            reports.append(rep)
            if callback is not None:
                callback(st, rep)
            if rep.accepted:
                if target_cost > 0 and rep.cost_after <= target_cost:
                    break
                if (rep.cost_before - rep.cost_after) < ftol * rep.cost_before:
                    break
            if st.lam > LAMBDA_MAX:
                break
        return st, reports


# ---------------------------------------------------------------------------
# Matrix-free variant for scenes whose dense S does not fit (series mode only)
# ---------------------------------------------------------------------------

class MatrixFreeProblem(Problem):
    """The same damped VarPro step as ``Problem.step`` in series mode, with
    the camera-landmark block W applied observation by observation
    (W = sum_k J_p,k^T J_l,k placed at camera i(k), landmark j(k)) instead of
    through the sparse Jacobian and the dense Schur complement. U, V, b_p,
    b_l are the same per-observation sums J^T J and J^T r. Observation sums
    are formed with sparse 0/1 incidence matrices (a library product).
    Pinned against ``Problem.step`` on small scenes (tests/test_oracle_pins.py).
    """

    CHUNK = 250_000

    def __init__(self, n_cams, n_points, cam_idx, pt_idx, meas):
        super().__init__(n_cams, n_points, cam_idx, pt_idx, meas)
        n = len(self.cam_idx)
        ones = np.ones(n)
        self.A_cam = sp.csr_matrix((ones, (self.cam_idx, np.arange(n))), shape=(self.n_cams, n))
        self.A_pt = sp.csr_matrix((ones, (self.pt_idx, np.arange(n))), shape=(self.n_points, n))

    def blocks(self, P, X, eta):
        """U (n_cams,12,12), b_p (n_cams,12), V (n_points,3,3), b_l, J_p, J_l."""
        n = len(self.cam_idx)
        r = pose_residuals(P, X, self.cam_idx, self.pt_idx, self.meas, eta)
        Jp, Jl = jacobian_blocks(P, X, self.cam_idx, self.pt_idx, self.meas, eta)
        U = np.zeros((self.n_cams, 144))
        for a in range(0, n, self.CHUNK):
            b = min(n, a + self.CHUNK)
            outer = np.einsum("nra,nrb->nab", Jp[a:b], Jp[a:b]).reshape(b - a, 144)
            U += self.A_cam[:, a:b] @ outer
        b_p = self.A_cam @ np.einsum("nra,nr->na", Jp, r)
        V = (self.A_pt @ np.einsum("nra,nrb->nab", Jl, Jl).reshape(n, 9)).reshape(-1, 3, 3)
        b_l = self.A_pt @ np.einsum("nra,nr->na", Jl, r)
        return U.reshape(-1, 12, 12), b_p, V, b_l, Jp, Jl

    def step(self, st: State, params: Params):
        if params.solver != "series":
            raise ValueError("MatrixFreeProblem only runs the series solver")
        eta, lam = params.eta, st.lam
        U, b_p, V, b_l, Jp, Jl = self.blocks(st.P, st.X, eta)
        Vinv, _ = sym_inverse_batch(V)
        Q = tangent_bases(st.P, params.manifold)
        k = Q.shape[2]
        Ut = np.einsum("nai,nab,nbj->nij", Q, U, Q) + lam * np.eye(k)[None]
        Utinv = np.linalg.inv(Ut)
        ci, pj = self.cam_idx, self.pt_idx

        def Wt(xc):          # (n_cams, 12) ambient -> (n_points, 3)
            y = np.einsum("nra,na->nr", Jp, xc[ci])
            return self.A_pt @ np.einsum("nrb,nr->nb", Jl, y)

        def W(s):            # (n_points, 3) -> (n_cams, 12)
            y = np.einsum("nrb,nb->nr", Jl, s[pj])
            return self.A_cam @ np.einsum("nra,nr->na", Jp, y)

        def lift(xt):        # tangent coordinates -> ambient
            return np.einsum("nab,nb->na", Q, xt)

        def proj(xa):        # ambient -> tangent coordinates (Q^T)
            return np.einsum("nab,na->nb", Q, xa)

        def Vi(t):
            return np.einsum("nab,nb->na", Vinv, t)

        g = -(proj(b_p) - proj(W(Vi(b_l))))
        x = np.einsum("nab,nb->na", Utinv, g)
        delta = x.copy()
        terms = 1
        for _ in range(1, params.m):
            x = np.einsum("nab,nb->na", Utinv, proj(W(Vi(Wt(lift(x))))))
            delta += x
            terms += 1
            if params.series_eps > 0 and (np.linalg.norm(x) <=
                                          params.series_eps * np.linalg.norm(delta)):
                break
        dP = lift(delta)
        S0d = np.einsum("nab,nb->na", Ut, delta) - lam * delta - proj(W(Vi(Wt(dP))))
        pred = float(2.0 * np.sum(g * delta) - np.sum(delta * S0d))
        P_new = st.P + dP
        if params.manifold == SPHERE:
            P_new = P_new / np.linalg.norm(P_new, axis=1, keepdims=True)
        X_new = self.landmarks(P_new, eta)
        F_new = self.cost(P_new, X_new, eta)
        rho = (st.F - F_new) / pred if pred > 0 else 0.0
        accepted = F_new < st.F
        rep = StepReport(cost_before=st.F, cost_after=F_new, pred=pred, rho=rho,
                         lambda_used=lam, lambda_next=0.0, accepted=bool(accepted),
                         terms_used=terms, delta=dP, P_trial=P_new)
        if accepted:
            lam_n = max(lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), LAMBDA_MIN)
            new = State(P=P_new, X=X_new, F=F_new, lam=lam_n, nu=2.0,
                        iteration=st.iteration + 1)
        else:
            new = State(P=st.P, X=st.X, F=st.F, lam=lam * st.nu, nu=2.0 * st.nu,
                        iteration=st.iteration + 1)
        rep.lambda_next = new.lam
        return new, rep
