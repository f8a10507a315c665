"""FP64 CPU oracle for the metric upgrade (autocalibration) of the
stratified problem.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module. The
product path (the C-ABI CUDA library and its Python binding) never imports,
links or calls it, and this module imports nothing from the product.

What it computes (paper: Weber, Hong, Cremers, ECCV 2024, supplementary
section "Metric Upgrade"): a projective reconstruction with cameras P_i is
upgraded by H = [[A, 0], [c^T, 1]] so that K_i^-1 P_i H ~ [R_i t_i]. With
H~ the three left-most columns of H, the rotation constraint reads
(K_i^-1 P_i) H~ H~^T (K_i^-1 P_i)^T ~ I up to a scale alpha_i per camera, and
c and the alpha_i minimize

    sum_i || alpha_i M_i(c) - I ||_F^2,   M_i = B_i H~(c) H~(c)^T B_i^T,
    B_i = K_i^-1 P_i H_0,

by Variable Projection: every alpha_i is eliminated in closed form
(alpha_i = <M_i, I>_F / ||M_i||_F^2) and c is found by Levenberg-Marquardt on
the reduced residuals, whose Jacobian follows from the product rule
d(H~ H~^T) = dH~ H~^T + H~ dH~^T (the matrix derivative the paper quotes).

Readings where the paper is silent:

* A is not optimized (H~ depends on c alone in the paper's problem). The
  reconstruction is first brought to the frame where the calibrated
  reference camera K_0^-1 P_0 (camera 0) is [I | 0]:
  H_0 = [[K_0^-1 P_0], [C^T]]^-1 with C the null vector of P_0 (its centre). In that frame A = I, so H~(c) = [[I], [c^T]] and c^T is
  the plane at infinity up to sign, as the paper's comment on (c^T 1) says.
* The paper does not say where c starts; the cost is not convex in c (from
  c = 0 the iteration can stop at a stationary point away from the metric
  solution). The start is the linear estimate of the dual absolute quadric
  Q = H~ H~^T of the autocalibration literature the paper cites: every
  camera gives five equations linear in the ten entries of Q (the
  off-diagonal entries of B_i Q B_i^T vanish, its diagonal entries are
  equal); Q is their least-squares null vector, scaled so that its upper
  3x3 block has trace 3, and c is its last column.
* The Frobenius norm runs over all nine entries of the 3x3 residual.
* Damping and accept rule of the first stage (Madsen-Nielsen, accept iff
  the cost decreases), D = I, lambda0 = 1e-4; stop at a relative decrease
  below ftol on an accepted step or after max_iters iterations.

Parity status: pinned by tests/test_oracle_metric_pins.py except the
damping and stop conventions ("parity unpinned -- convention").
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .povar_oracle import LAMBDA_MAX, LAMBDA_MIN


def frame_to_reference(P0):
    """H_0 with P_0 H_0 = [I | 0]: the inverse of P_0 stacked on its
    centre C (P_0 C = 0, from the SVD)."""
    P0 = np.asarray(P0, dtype=np.float64).reshape(3, 4)
    _, _, Vt = np.linalg.svd(P0)
    C = Vt[-1]
    return np.linalg.inv(np.vstack([P0, C[None, :]]))


def upgrade_blocks(P, K, H0):
    """B_i = K_i^-1 P_i H_0, [n, 3, 4]."""
    Pm = np.asarray(P, dtype=np.float64).reshape(-1, 3, 4)
    Kinv = np.linalg.inv(np.asarray(K, dtype=np.float64).reshape(-1, 3, 3))
    return np.einsum("nab,nbc,cd->nad", Kinv, Pm, H0)


def h_tilde(c):
    """H~(c) = [[I], [c^T]] (4x3)."""
    return np.vstack([np.eye(3), np.asarray(c, dtype=np.float64)[None, :]])


def m_blocks(B, c):
    """M_i(c) = B_i H~ H~^T B_i^T, [n, 3, 3]."""
    Q = h_tilde(c) @ h_tilde(c).T
    return np.einsum("nab,bc,ndc->nad", B, Q, B)


def alphas(M):
    """The closed-form scale per camera: argmin_a ||a M - I||_F."""
    return np.einsum("naa->n", M) / np.einsum("nab,nab->n", M, M)


def residuals(B, c):
    """Reduced residuals alpha_i(c) M_i(c) - I, flattened: [n, 9]."""
    M = m_blocks(B, c)
    a = alphas(M)
    return (a[:, None, None] * M - np.eye(3)[None]).reshape(-1, 9)


def cost(B, c):
    r = residuals(B, c)
    return float(np.sum(r * r))


def jacobian(B, c):
    """d residual_i / d c, [n, 9, 3]: dM by the product rule on H~ H~^T,
    then the derivative of alpha(c) M(c) with alpha = <M, I> / <M, M>."""
    M = m_blocks(B, c)
    Ht = h_tilde(c)
    n = B.shape[0]
    J = np.empty((n, 9, 3))
    tr = np.einsum("naa->n", M)
    mm = np.einsum("nab,nab->n", M, M)
    a = tr / mm
    for k in range(3):
        dH = np.zeros((4, 3))
        dH[3, k] = 1.0
        dQ = dH @ Ht.T + Ht @ dH.T
        dM = np.einsum("nab,bc,ndc->nad", B, dQ, B)
        dtr = np.einsum("naa->n", dM)
        dmm = 2.0 * np.einsum("nab,nab->n", M, dM)
        da = (dtr * mm - tr * dmm) / (mm * mm)
        J[:, :, k] = (a[:, None, None] * dM + da[:, None, None] * M).reshape(n, 9)
    return J


# index pairs of the 10 free entries of a symmetric 4x4 matrix
_Q_PAIRS = [(a, b) for a in range(4) for b in range(a, 4)]


def linear_start(B):
    """c from the linear estimate of Q = H~ H~^T (see the module header)."""
    rows = []
    for Bi in B:
        def coeffs(r, s):
            # coefficient of each free entry of Q in (B Q B^T)_{rs}
            out = []
            for a, b in _Q_PAIRS:
                v = Bi[r, a] * Bi[s, b]
                if a != b:
                    v += Bi[r, b] * Bi[s, a]
                out.append(v)
            return np.array(out)
        rows += [coeffs(0, 1), coeffs(0, 2), coeffs(1, 2),
                 coeffs(0, 0) - coeffs(1, 1), coeffs(0, 0) - coeffs(2, 2)]
    _, _, Vt = np.linalg.svd(np.array(rows))
    q = Vt[-1]
    Q = np.zeros((4, 4))
    for v, (a, b) in zip(q, _Q_PAIRS):
        Q[a, b] = Q[b, a] = v
    Q *= 3.0 / np.trace(Q[:3, :3])
    return Q[:3, 3].copy()


@dataclasses.dataclass
class Result:
    c: np.ndarray
    H: np.ndarray          # H_0 [[I, 0], [c^T, 1]]
    alpha: np.ndarray
    cost: float
    iterations: int
    trace: list


def upgrade(P, K=None, c0=None, lambda0=1e-4, max_iters=100, ftol=1e-12):
    """Levenberg-Marquardt on the reduced residuals from c0 (default: the
    linear estimate)."""
    P = np.asarray(P, dtype=np.float64).reshape(-1, 12)
    n = P.shape[0]
    K = np.broadcast_to(np.eye(3), (n, 3, 3)) if K is None else K
    K = np.asarray(K, dtype=np.float64).reshape(n, 3, 3)
    H0 = frame_to_reference(np.linalg.solve(K[0], P[0].reshape(3, 4)))
    B = upgrade_blocks(P, K, H0)
    c = linear_start(B) if c0 is None else np.asarray(c0, dtype=np.float64).copy()
    F = cost(B, c)
    lam, nu = lambda0, 2.0
    trace = [F]
    it = 0
    for it in range(1, max_iters + 1):
        r = residuals(B, c).ravel()
        J = jacobian(B, c).reshape(-1, 3)
        g = J.T @ r
        Hn = J.T @ J
        d = np.linalg.solve(Hn + lam * np.eye(3), -g)
        Fn = cost(B, c + d)
        pred = float(-2.0 * g @ d - d @ Hn @ d)
        rho = (F - Fn) / pred if pred > 0 else 0.0
        if Fn < F:
            decrease = F - Fn
            c, F = c + d, Fn
            lam = max(lam * max(1.0 / 3.0, 1.0 - (2.0 * rho - 1.0) ** 3), LAMBDA_MIN)
            nu = 2.0
            trace.append(F)
            if decrease < ftol * (F + decrease):
                break
        else:
            lam *= nu
            nu *= 2.0
            trace.append(F)
            if lam > LAMBDA_MAX:
                break
    H = H0 @ np.block([[np.eye(3), np.zeros((3, 1))], [c[None, :], np.ones((1, 1))]])
    return Result(c=c, H=H, alpha=alphas(m_blocks(B, c)), cost=F, iterations=it, trace=trace)
