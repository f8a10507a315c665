// a2 + a3: closed-form VarPro landmarks and the pOSE cost, in FP64.
//
// Eq. update_landmark: with the cameras fixed, every landmark solves its own
// 3x3 linear least-squares problem. For observation (i, j, m = (u, v)) the
// pOSE residual (Eq. pose) is r = B(m) (P_i (X_j, 1)) - d(m), so landmark j's
// normal matrix and right-hand side are
//     V_j = sum P^T C P,   h_j = sum P^T (C p4 - (eta u, eta v, 0)),
// with P the left 3x3 of P_i, p4 its last column and C = B^T B =
//     [[1, 0, -a u], [0, 1, -a v], [-a u, -a v, a (u^2 + v^2)]], a = 1 - eta.
// Both are affine in (u, v, u^2 + v^2) with per-camera coefficients, so each
// camera carries a 48-double table (computed once per camera set) and one
// observation costs 38 FP64 operations. X_j = -V_j^-1 h_j through the
// Cholesky factor V = L L^T; the kernel also stores F = L^-1 (V^-1 = F^T F),
// which the series kernels use. A numerically rank-deficient V_j
// (cond > 1e12) falls back to the Moore-Penrose pseudo-inverse (footnote of
// Sec. 4.2) from a Jacobi eigen-decomposition.
// The cost is then evaluated directly, in a second pass over the landmark's
// observations: sum_k ||r_k||^2 at the solved X (17 FP64 operations per
// observation). The shortcut sum_k ||c_k||^2 + h^T X (c_k = B p4 - d, exact at
// the optimum) is not used: it cancels catastrophically when V_j is
// ill-conditioned and X_j large (a trial step towards degenerate cameras gave
// a negative cost that way), while the direct sum is always >= 0 and accurate.
// F = ||r||^2 (Eq. ba_first_stage) is summed into one FP64 partial per warp
// and a single block adds the partials in a fixed order (deterministic).
#include <mutex>

#include "df64.cuh"
#include "povar_internal.cuh"

namespace povar {
namespace {

struct SlotBufs {
  double* X[2];
  double* F[2];
  float4* A[2];
  float4* B[2];
  float* C[2];
};

// Ltab layout (48 doubles per camera):
//  [0,6) R, [6,12) E1, [12,18) E2, [18,24) Fm   (symmetric 3x3: 00 01 02 11 12 22)
//  [24,27) h0, [27,30) hu, [30,33) hv, [33,36) hw, [36,48) unused
// 64 threads per camera: thread e < 36 computes table entry e, threads
// 36 <= e < 48 copy P[e - 36] into the double-float block, threads e < 12
// also write the FP32 copy of P; consecutive threads write consecutive
// entries, so the stores of a warp coalesce.
__global__ void __launch_bounds__(256)
k_ltab(const DeviceState* __restrict__ st, int which_rel, double eta,
       const double* __restrict__ P0, const double* __restrict__ P1, int nc,
       double* __restrict__ Ltab, float2* __restrict__ Ldf, float* __restrict__ C0,
       float* __restrict__ C1) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int i = (int)(g >> 6), e = (int)(g & 63);
  if (i >= nc) return;
  if (which_rel == 1 && st->converged) return;
  const int t = which_rel ? 1 - st->cur : st->cur;
  const double* P = (t ? P1 : P0) + 12 * (size_t)i;
  if (e < 12) ((t ? C1 : C0) + 12 * (size_t)i)[e] = (float)P[e];  // for the FP32 kernels
  if (e >= 48) return;
  const double a = 1.0 - eta;
  double v;
  if (e < 24) {
    // symmetric 3x3 entry (x, y) of block R, E1, E2 or Fm
    const int k = e % 6, blk = e / 6;
    const int x = k < 3 ? 0 : (k < 5 ? 1 : 2);
    const int y = k < 3 ? k : (k < 5 ? k - 2 : 2);
    const double p0x = P[x], p0y = P[y], p1x = P[4 + x], p1y = P[4 + y];
    const double p2x = P[8 + x], p2y = P[8 + y];
    if (blk == 0) v = p0x * p0y + p1x * p1y;
    else if (blk == 1) v = -a * (p0x * p2y + p2x * p0y);
    else if (blk == 2) v = -a * (p1x * p2y + p2x * p1y);
    else v = a * p2x * p2y;
  } else if (e < 36) {
    const int c = (e - 24) % 3, blk = (e - 24) / 3;
    const double q0 = P[3], q1 = P[7], q2 = P[11];
    const double p0 = P[c], p1 = P[4 + c], p2 = P[8 + c];
    if (blk == 0) v = q0 * p0 + q1 * p1;
    else if (blk == 1) v = (-a * q2 - eta) * p0 - a * q0 * p2;
    else if (blk == 2) v = (-a * q2 - eta) * p1 - a * q1 * p2;
    else v = a * q2 * p2;
  } else {
    v = P[e - 36];
  }
  if (e < 36) Ltab[48 * (size_t)i + e] = v;
  // double-float copy: the 36 table entries, then P itself (12)
  const float hi = (float)v;
  Ldf[48 * (size_t)i + e] = make_float2(hi, (float)(v - (double)hi));
}

// Symmetric 3x3 packed as (00 01 02 11 12 22).
__device__ __forceinline__ double sym_at(const double* V, int r, int c) {
  const int lo = r < c ? r : c, hi = r < c ? c : r;
  const int idx = lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
  return V[idx];
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 (textbook rotation
// formulas, Golub & Van Loan Sec. 8.5). Returns eigenvalues w and
// eigenvectors as the columns of Q.
__device__ __forceinline__ void jacobi3(const double* V, double w[3], double Q[3][3]) {
  double A[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      A[r][c] = sym_at(V, r, c);
      Q[r][c] = r == c ? 1.0 : 0.0;
    }
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
    const double dia = fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]);
    if (off <= 1e-300 || off <= 1e-18 * dia) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int pp = pq == 2 ? 1 : 0, qq = pq == 0 ? 1 : 2;
      const double apq = A[pp][qq];
      if (apq == 0.0) continue;
      const double theta = (A[qq][qq] - A[pp][pp]) / (2.0 * apq);
      const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
      for (int k = 0; k < 3; ++k) {
        const double akp = A[k][pp], akq = A[k][qq];
        A[k][pp] = c * akp - s * akq;
        A[k][qq] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        const double apk = A[pp][k], aqk = A[qq][k];
        A[pp][k] = c * apk - s * aqk;
        A[qq][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        const double qkp = Q[k][pp], qkq = Q[k][qq];
        Q[k][pp] = c * qkp - s * qkq;
        Q[k][qq] = s * qkp + c * qkq;
      }
    }
  }
  w[0] = A[0][0];
  w[1] = A[1][1];
  w[2] = A[2][2];
}

struct Sym3 {
  double v[6];
};
struct Vec3 {
  double x[3];
};
struct PinvOut {
  double X[3];
  double F[6];
  bool deficient;
};

// Pseudo-inverse path: X = -V^+ h and a lower-triangular F with F^T F = V^+
// (Cholesky of the index-reversed V^+, zero pivots giving zero columns).
// `deficient` tells whether V was numerically rank-deficient. Arguments are
// passed by value so that the caller's accumulators stay in registers.
__device__ __forceinline__ PinvOut pinv_solve(Sym3 Vs, Vec3 hs) {
  const double* V = Vs.v;
  const double* h = hs.x;
  PinvOut out;
  double* X = out.X;
  double* F = out.F;
  double w[3], Q[3][3];
  jacobi3(V, w, Q);
  const double wmax = fmax(w[0], fmax(w[1], w[2]));
  const double wmin = fmin(w[0], fmin(w[1], w[2]));
  const bool deficient = !(wmax > 0.0) || wmin <= wmax / PINV_COND;
  double A[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k)
        if (w[k] > wmax / PINV_COND && w[k] > 0.0) acc += Q[r][k] * Q[c][k] / w[k];
      A[r][c] = acc;
    }
  for (int r = 0; r < 3; ++r) X[r] = -(A[r][0] * h[0] + A[r][1] * h[1] + A[r][2] * h[2]);
  // G = chol(J A J), lower; F = J G^T J, i.e. F[a][b] = G[2-b][2-a].
  double R[3][3], G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[r][c] = A[2 - r][2 - c];
  const double scale = fmax(fmax(fabs(R[0][0]), fabs(R[1][1])), fabs(R[2][2]));
  for (int k = 0; k < 3; ++k) {
    double d = R[k][k];
    for (int q = 0; q < k; ++q) d -= G[k][q] * G[k][q];
    if (d <= scale * 1e-14) continue;  // zero pivot: column stays zero
    G[k][k] = sqrt(d);
    for (int r = k + 1; r < 3; ++r) {
      double e = R[r][k];
      for (int q = 0; q < k; ++q) e -= G[r][q] * G[k][q];
      G[r][k] = e / G[k][k];
    }
  }
  F[0] = G[2][2];  // F00
  F[1] = G[2][1];  // F10
  F[2] = G[1][1];  // F11
  F[3] = G[2][0];  // F20
  F[4] = G[1][0];  // F21
  F[5] = G[0][0];  // F22
  out.deficient = deficient;
  return out;
}

__global__ void __launch_bounds__(BLOCK)
k_landmark(DeviceState* __restrict__ st, int which_rel, double eta,
           const uint32_t* __restrict__ slot_len, const uint32_t* __restrict__ sell_off,
           const int32_t* __restrict__ sell_cam, const double2* __restrict__ sell_m,
           const double* __restrict__ Ltab, const double* __restrict__ P0,
           const double* __restrict__ P1, int np, SlotBufs bufs,
           double* __restrict__ cost_part, int* __restrict__ pinv_part) {
  if (which_rel == 1 && st->converged) return;
  const int t = which_rel ? 1 - st->cur : st->cur;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  if (s == 0) st->x_df[t] = 0;
  double cost = 0.0;
  int npinv = 0;
  // padding slots (track length 0) sit between the slices of the layout
  if (s < np && slot_len[s] > 0) {
    const uint32_t len = slot_len[s];
    const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
    double V[6] = {0, 0, 0, 0, 0, 0}, h[3] = {0, 0, 0};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const double2 m = sell_m[pos];
      const double u = m.x, v = m.y, w = u * u + v * v;
      const double2* T = reinterpret_cast<const double2*>(Ltab + 48 * (size_t)i);
      double tb[36];
#pragma unroll
      for (int q = 0; q < 18; ++q) {
        const double2 x = __ldg(T + q);
        tb[2 * q] = x.x;
        tb[2 * q + 1] = x.y;
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) V[e] += tb[e] + u * tb[6 + e] + v * tb[12 + e] + w * tb[18 + e];
#pragma unroll
      for (int c = 0; c < 3; ++c) h[c] += tb[24 + c] + u * tb[27 + c] + v * tb[30 + c] + w * tb[33 + c];
    }
    // Cholesky V = L L^T through reciprocal square roots; F = L^-1
    double X[3], F[6];
    const double dmax = fmax(V[0], fmax(V[3], V[5]));
    const double f00 = rsqrt(V[0]);
    const double l10 = V[1] * f00, l20 = V[2] * f00;
    const double d1 = V[3] - l10 * l10;
    const double f11 = rsqrt(d1);
    const double l21 = (V[4] - l20 * l10) * f11;
    const double d2 = V[5] - l20 * l20 - l21 * l21;
    const double f22 = rsqrt(d2);
    const bool suspect = !(V[0] > 1e-9 * dmax) || !(d1 > 1e-9 * dmax) || !(d2 > 1e-9 * dmax) ||
                         !(dmax > 0.0);
    bool deficient = false;
    if (suspect) {
      Sym3 vs;
      Vec3 hs;
      for (int e = 0; e < 6; ++e) vs.v[e] = V[e];
      for (int e = 0; e < 3; ++e) hs.x[e] = h[e];
      const PinvOut o = pinv_solve(vs, hs);
      deficient = o.deficient;
      for (int e = 0; e < 3; ++e) X[e] = o.X[e];
      for (int e = 0; e < 6; ++e) F[e] = o.F[e];
    }
    if (!deficient) {
      const double f10 = -l10 * f00 * f11;
      const double f20 = -(l20 * f00 + l21 * f10) * f22;
      const double f21 = -l21 * f11 * f22;
      F[0] = f00; F[1] = f10; F[2] = f11; F[3] = f20; F[4] = f21; F[5] = f22;
      // z = F h, X = -F^T z
      const double z0 = f00 * h[0];
      const double z1 = f10 * h[0] + f11 * h[1];
      const double z2 = f20 * h[0] + f21 * h[1] + f22 * h[2];
      X[0] = -(f00 * z0 + f10 * z1 + f20 * z2);
      X[1] = -(f11 * z1 + f21 * z2);
      X[2] = -(f22 * z2);
    }
    npinv = deficient ? 1 : 0;
    double* Xo = bufs.X[t] + 3 * (size_t)s;
    Xo[0] = X[0]; Xo[1] = X[1]; Xo[2] = X[2];
    double* Fo = bufs.F[t] + 6 * (size_t)s;
#pragma unroll
    for (int e = 0; e < 6; ++e) Fo[e] = F[e];
    bufs.A[t][s] = make_float4((float)X[0], (float)X[1], (float)X[2], (float)F[0]);
    bufs.B[t][s] = make_float4((float)F[1], (float)F[2], (float)F[3], (float)F[4]);
    bufs.C[t][s] = (float)F[5];
    // r_k = B_k P_i (X, 1) - d_k: with y = P_i (X, 1),
    // ||r_k||^2 = (1 - eta) ((y0 - u y2)^2 + (y1 - v y2)^2) + eta ((y0 - u)^2 + (y1 - v)^2)
    const double* __restrict__ Pc = t ? P1 : P0;
    double e1 = 0.0, e2 = 0.0;
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const double2 m = sell_m[pos];
      const double2* Q = reinterpret_cast<const double2*>(Pc + 12 * (size_t)i);
      double q[12];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const double2 x = __ldg(Q + r);
        q[2 * r] = x.x;
        q[2 * r + 1] = x.y;
      }
      const double y0 = fma(q[0], X[0], fma(q[1], X[1], fma(q[2], X[2], q[3])));
      const double y1 = fma(q[4], X[0], fma(q[5], X[1], fma(q[6], X[2], q[7])));
      const double y2 = fma(q[8], X[0], fma(q[9], X[1], fma(q[10], X[2], q[11])));
      const double a0 = fma(-m.x, y2, y0), a1 = fma(-m.y, y2, y1);
      const double b0 = y0 - m.x, b1 = y1 - m.y;
      e1 = fma(a0, a0, fma(a1, a1, e1));
      e2 = fma(b0, b0, fma(b1, b1, e2));
    }
    cost = (1.0 - eta) * e1 + eta * e2;
  } else {
    // padding slot (the slot arrays are padded to a whole number of blocks)
    double* Xo = bufs.X[t] + 3 * (size_t)s;
    Xo[0] = Xo[1] = Xo[2] = 0.0;
    double* Fo = bufs.F[t] + 6 * (size_t)s;
    for (int e = 0; e < 6; ++e) Fo[e] = 0.0;
    bufs.A[t][s] = make_float4(0.f, 0.f, 0.f, 0.f);
    bufs.B[t][s] = make_float4(0.f, 0.f, 0.f, 0.f);
    bufs.C[t][s] = 0.f;
  }
  // one deterministic partial per warp (no block barrier: slices finish
  // independently)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cost += __shfl_xor_sync(0xffffffffu, cost, o);
    npinv += __shfl_xor_sync(0xffffffffu, npinv, o);
  }
  if ((threadIdx.x & 31) == 0) {
    cost_part[s / 32] = cost;
    pinv_part[s / 32] = npinv;
  }
}

// The same elimination and direct cost as k_landmark with the arithmetic of
// both per-observation passes and of the per-landmark Cholesky solve in
// double-float (about 48 bits; df64.cuh), for the mixed-precision solve:
// the FP64 pipe, which bounds k_landmark, is left almost idle. A landmark
// whose Cholesky pivots flag a near rank-deficient V_j takes the FP64
// pseudo-inverse path of k_landmark. Writes X (FP64), the FP32 copies used
// by the FP32 kernels and the cost partials; the FP64 factor F64 is not
// written (an FP64 step re-solves the landmarks with k_landmark first).
// The kernel is bound by FP32 issue; capping it at 64 registers (4 blocks
// per SM, a few spilled values) hides more latency than the spills cost.
__global__ void __launch_bounds__(BLOCK, 4)
k_landmark_df(DeviceState* __restrict__ st, int which_rel, df64 a, df64 eta,
              const uint32_t* __restrict__ slot_len, const uint32_t* __restrict__ sell_off,
              const int32_t* __restrict__ sell_cam, const float4* __restrict__ sell_mdf,
              const float2* __restrict__ Ldf, int np, SlotBufs bufs,
              double* __restrict__ cost_part, int* __restrict__ pinv_part) {
  if (which_rel == 1 && st->converged) return;
  const int t = which_rel ? 1 - st->cur : st->cur;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  if (s == 0) st->x_df[t] = 1;
  df64 cost = {0.f, 0.f};
  int npinv = 0;
  // padding slots (track length 0) sit between the slices of the layout
  if (s < np && slot_len[s] > 0) {
    const uint32_t len = slot_len[s];
    const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
    df64 V[6], h[3];
#pragma unroll
    for (int e = 0; e < 6; ++e) V[e] = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = {0.f, 0.f};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const float4 m = sell_mdf[pos];
      const df64 u = {m.x, m.y}, v = {m.z, m.w};
      df64 w = df_mul(v, v);
      df_acc_mul(w, u, u);
      w = df_norm(w);
      const float4* T4 = reinterpret_cast<const float4*>(Ldf + 48 * (size_t)i);
      df64 tb[36];
#pragma unroll
      for (int q = 0; q < 18; ++q) {
        const float4 x = __ldg(T4 + q);
        tb[2 * q] = {x.x, x.y};
        tb[2 * q + 1] = {x.z, x.w};
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        df_acc(V[e], tb[e]);
        df_acc_mul(V[e], u, tb[6 + e]);
        df_acc_mul(V[e], v, tb[12 + e]);
        df_acc_mul(V[e], w, tb[18 + e]);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        df_acc(h[c], tb[24 + c]);
        df_acc_mul(h[c], u, tb[27 + c]);
        df_acc_mul(h[c], v, tb[30 + c]);
        df_acc_mul(h[c], w, tb[33 + c]);
      }
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) V[e] = df_norm(V[e]);
#pragma unroll
    for (int c = 0; c < 3; ++c) h[c] = df_norm(h[c]);
    // Cholesky V = L L^T through reciprocal square roots; F = L^-1
    const df64 f00 = df_rsqrt(V[0]);
    const df64 l10 = df_mul(V[1], f00), l20 = df_mul(V[2], f00);
    const df64 d1 = df_sub(V[3], df_mul(l10, l10));
    const df64 f11 = df_rsqrt(d1);
    const df64 l21 = df_mul(df_sub(V[4], df_mul(l20, l10)), f11);
    const df64 d2 = df_sub(df_sub(V[5], df_mul(l20, l20)), df_mul(l21, l21));
    const df64 f22 = df_rsqrt(d2);
    const float dmax = fmaxf(V[0].hi, fmaxf(V[3].hi, V[5].hi));
    const bool suspect = !(V[0].hi > 1e-9f * dmax) || !(d1.hi > 1e-9f * dmax) ||
                         !(d2.hi > 1e-9f * dmax) || !(dmax > 0.f);
    df64 X[3];
    float F[6];
    double X64v[3], F64v[6];
    bool deficient = false;
    if (suspect) {
      Sym3 vs;
      Vec3 hs;
      for (int e = 0; e < 6; ++e) vs.v[e] = df_to_double(V[e]);
      for (int c = 0; c < 3; ++c) hs.x[c] = df_to_double(h[c]);
      const PinvOut o = pinv_solve(vs, hs);
      deficient = o.deficient;
      for (int c = 0; c < 3; ++c) X64v[c] = o.X[c];
      for (int e = 0; e < 6; ++e) F64v[e] = o.F[e];
    }
    if (!deficient) {
      const df64 f10 = df_neg(df_mul(df_mul(l10, f00), f11));
      const df64 f20 = df_neg(df_mul(df_add(df_mul(l20, f00), df_mul(l21, f10)), f22));
      const df64 f21 = df_neg(df_mul(df_mul(l21, f11), f22));
      // z = F h, X = -F^T z
      const df64 z0 = df_mul(f00, h[0]);
      const df64 z1 = df_add(df_mul(f10, h[0]), df_mul(f11, h[1]));
      const df64 z2 = df_add(df_add(df_mul(f20, h[0]), df_mul(f21, h[1])), df_mul(f22, h[2]));
      X[0] = df_neg(df_add(df_add(df_mul(f00, z0), df_mul(f10, z1)), df_mul(f20, z2)));
      X[1] = df_neg(df_add(df_mul(f11, z1), df_mul(f21, z2)));
      X[2] = df_neg(df_mul(f22, z2));
      F[0] = f00.hi; F[1] = f10.hi; F[2] = f11.hi; F[3] = f20.hi; F[4] = f21.hi; F[5] = f22.hi;
    } else {
      for (int c = 0; c < 3; ++c) X[c] = df_from_double(X64v[c]);
      for (int e = 0; e < 6; ++e) F[e] = (float)F64v[e];
    }
    npinv = deficient ? 1 : 0;
    // X as double-float pairs in the FP64 buffer (same 24 bytes; x_df[t] = 1)
    float2* Xo = reinterpret_cast<float2*>(bufs.X[t] + 3 * (size_t)s);
    Xo[0] = make_float2(X[0].hi, X[0].lo);
    Xo[1] = make_float2(X[1].hi, X[1].lo);
    Xo[2] = make_float2(X[2].hi, X[2].lo);
    bufs.A[t][s] = make_float4(X[0].hi, X[1].hi, X[2].hi, F[0]);
    bufs.B[t][s] = make_float4(F[1], F[2], F[3], F[4]);
    bufs.C[t][s] = F[5];
    // ||r_k||^2 = (1 - eta) ((y0 - u y2)^2 + (y1 - v y2)^2) + eta ((y0 - u)^2 + (y1 - v)^2)
    // with y = P_i (X, 1), summed in double-float
    df64 e1 = {0.f, 0.f}, e2 = {0.f, 0.f};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const float4 m = sell_mdf[pos];
      const df64 nu = {-m.x, -m.y}, nv = {-m.z, -m.w};
      const float4* Q4 = reinterpret_cast<const float4*>(Ldf + 48 * (size_t)i + 36);
      df64 q[12];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const float4 x = __ldg(Q4 + r);
        q[2 * r] = {x.x, x.y};
        q[2 * r + 1] = {x.z, x.w};
      }
      df64 y[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        df64 acc = q[4 * r + 3];
        df_acc_mul(acc, q[4 * r], X[0]);
        df_acc_mul(acc, q[4 * r + 1], X[1]);
        df_acc_mul(acc, q[4 * r + 2], X[2]);
        y[r] = df_norm(acc);
      }
      df64 a0 = y[0], a1 = y[1];
      df_acc_mul(a0, nu, y[2]);
      df_acc_mul(a1, nv, y[2]);
      a0 = df_norm(a0);
      a1 = df_norm(a1);
      df64 b0 = y[0], b1 = y[1];
      df_acc(b0, nu);
      df_acc(b1, nv);
      b0 = df_norm(b0);
      b1 = df_norm(b1);
      df_acc_mul(e1, a0, a0);
      df_acc_mul(e1, a1, a1);
      df_acc_mul(e2, b0, b0);
      df_acc_mul(e2, b1, b1);
    }
    cost = df_add(df_mul(a, df_norm(e1)), df_mul(eta, df_norm(e2)));
  } else {
    double* Xo = bufs.X[t] + 3 * (size_t)s;
    Xo[0] = Xo[1] = Xo[2] = 0.0;
    bufs.A[t][s] = make_float4(0.f, 0.f, 0.f, 0.f);
    bufs.B[t][s] = make_float4(0.f, 0.f, 0.f, 0.f);
    bufs.C[t][s] = 0.f;
  }
  // warp sum in double-float, one FP64 partial per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const df64 other = {__shfl_xor_sync(0xffffffffu, cost.hi, o),
                        __shfl_xor_sync(0xffffffffu, cost.lo, o)};
    cost = df_add(cost, other);
    npinv += __shfl_xor_sync(0xffffffffu, npinv, o);
  }
  if ((threadIdx.x & 31) == 0) {
    cost_part[s / 32] = df_to_double(cost);
    pinv_part[s / 32] = npinv;
  }
}

// F = sum of the per-warp cost partials (and the pseudo-inverse count):
// each of the FIN_BLOCKS blocks adds a fixed contiguous range of partials,
// the last block to finish (atomic ticket) adds the block sums in block
// order, so the result does not depend on the order the blocks ran in.
__global__ void __launch_bounds__(256)
k_cost_finish(DeviceState* __restrict__ st, int which_rel, const double* __restrict__ part,
              const int* __restrict__ pinv, int n, double* __restrict__ blk,
              int* __restrict__ blk_i, uint32_t* __restrict__ ticket) {
  if (which_rel == 1 && st->converged) return;
  __shared__ double red[256];
  __shared__ int redi[256];
  __shared__ int last;
  const int per = (n + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b0 = (int)blockIdx.x * per, b1 = min(n, b0 + per);
  double c = 0.0;
  int q = 0;
  for (int i = b0 + (int)threadIdx.x; i < b1; i += 256) {
    c += part[i];
    q += pinv[i];
  }
  red[threadIdx.x] = c;
  redi[threadIdx.x] = q;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      redi[threadIdx.x] += redi[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = red[0];
    blk_i[blockIdx.x] = redi[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  c = 0.0;
  q = 0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += 256) {
    c += __ldcg(blk + i);
    q += __ldcg(blk_i + i);
  }
  red[threadIdx.x] = c;
  redi[threadIdx.x] = q;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[threadIdx.x] += red[threadIdx.x + o];
      redi[threadIdx.x] += redi[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *ticket = 0u;
    if (which_rel == 0) {
      st->F = red[0];
      if (!isfinite(red[0])) st->error = POVAR_ENUMERIC;
    } else {
      st->F_new = red[0];
    }
    st->n_pinv = redi[0];
  }
}

}  // namespace

// double-float pair of a host double (kernel argument)
static df64 df_host(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

// Per-camera landmark tables of the current (0) or trial (1) cameras.
povar_status launch_ltab(Problem* p, int which_rel, double eta) {
  k_ltab<<<grid_for((int64_t)p->nc * 64, 256), 256, 0, p->stream>>>(
      p->state, which_rel, eta, p->P64[0], p->P64[1], p->nc, p->Ltab, p->Ltab_df, p->camP32[0],
      p->camP32[1]);
  ++p->launches;
  return check_launch(p, "ltab");
}

povar_status launch_landmarks(Problem* p, int which_rel, double eta, int precision) {
  povar_status s0;
  if ((s0 = launch_ltab(p, which_rel, eta)) != POVAR_OK) return s0;
  --p->launches;   // counted with the landmark launch below
  SlotBufs b;
  for (int t = 0; t < 2; ++t) {
    b.X[t] = p->X64[t];
    b.F[t] = p->F64[t];
    b.A[t] = p->pdA[t];
    b.B[t] = p->pdB[t];
    b.C[t] = p->pdC[t];
  }
  // trial landmarks of a mixed-precision step in double-float; every other
  // evaluation (and every FP64 step) in FP64
  if (which_rel == 1 && precision != POVAR_FP64)
    k_landmark_df<<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, which_rel, df_host(1.0 - eta), df_host(eta), p->slot_len, p->sell_off, p->sell_cam, p->sell_mdf,
        p->Ltab_df, p->np_pad, b, p->cost_part, p->pinv_part);
  else
    k_landmark<<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, which_rel, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->Ltab,
        p->P64[0], p->P64[1], p->np_pad, b, p->cost_part, p->pinv_part);
  p->launches += 2;
  return check_launch(p, "landmark");
}

povar_status launch_cost_finish(Problem* p, int which_rel) {
  k_cost_finish<<<FIN_BLOCKS, 256, 0, p->stream>>>(p->state, which_rel, p->cost_part,
                                                   p->pinv_part, p->np_pad / 32, p->fin_blk,
                                                   p->fin_blk_i, p->fin_ticket);
  ++p->launches;
  return check_launch(p, "cost_finish");
}

}  // namespace povar

// ---------------------------------------------------------------------------
// Allocation-free cost evaluation (povar_cost_noalloc).
//
// The same landmark elimination and cost as k_landmark + k_cost_finish, read
// from a caller-provided landmark-major CSR (one thread per landmark) instead
// of the handle's SELL slots. The per-block cost partials, the only working
// memory beyond the caller's inputs and outputs, live in the fixed array
// below; its device address is looked up once per device. Every partial the
// sum kernel reads is written first by its block in the same call, so the
// array needs no clearing between calls.
// ---------------------------------------------------------------------------
namespace povar {
namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_MAX_BLOCKS = POVAR_NOALLOC_MAX_POINTS / NA_BLOCK;
static_assert(NA_MAX_BLOCKS * NA_BLOCK == POVAR_NOALLOC_MAX_POINTS, "whole blocks");

static __device__ __align__(256) double na_partials[NA_MAX_BLOCKS];

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
double* na_ptr[NA_MAX_DEVICES] = {};

__global__ void __launch_bounds__(NA_BLOCK)
k_landmark_csr(const double* __restrict__ P, int nc, const uint32_t* __restrict__ off,
               const int32_t* __restrict__ cam, const double2* __restrict__ meas,
               int64_t nobs, int np, double eta, double* __restrict__ X_out,
               double* __restrict__ part) {
  __shared__ double red[NA_BLOCK / 32];
  const int j = blockIdx.x * NA_BLOCK + threadIdx.x;
  double cost = 0.0;
  if (j < np) {
    // observation range, clamped to the arrays; a malformed range or camera
    // index makes the cost NaN instead of being read out of bounds
    const int64_t b0 = off[j], e0 = off[j + 1];
    bool bad = e0 < b0 || e0 > nobs;
    const int64_t e = e0 < nobs ? e0 : nobs;
    const int64_t b = b0 < e ? b0 : e;
    const double a = 1.0 - eta;
    // V = sum Pbar^T C Pbar, h = sum Pbar^T (C p4 - (eta u, eta v, 0)) with
    // C = [[1, 0, -a u], [0, 1, -a v], [-a u, -a v, a (u^2 + v^2)]]; with
    // rows p_r of Pbar, V = sum_r p_r (C Pbar)_r^T and h = sum_r c_r p_r.
    double V[6] = {0, 0, 0, 0, 0, 0}, h[3] = {0, 0, 0};
    for (int64_t k = b; k < e; ++k) {
      const int i = cam[k];
      if ((unsigned)i >= (unsigned)nc) {
        bad = true;
        continue;
      }
      const double2 m = meas[k];
      const double u = m.x, v = m.y, w = u * u + v * v;
      const double2* Q = reinterpret_cast<const double2*>(P + 12 * (size_t)i);
      double q[12];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const double2 x = __ldg(Q + r);
        q[2 * r] = x.x;
        q[2 * r + 1] = x.y;
      }
      const double* p0 = q;
      const double* p1 = q + 4;
      const double* p2 = q + 8;
      double r0[3], r1[3], r2[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        r0[c] = p0[c] - a * u * p2[c];
        r1[c] = p1[c] - a * v * p2[c];
        r2[c] = a * (w * p2[c] - u * p0[c] - v * p1[c]);
      }
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int t = 0; t < 6; ++t)
        V[t] += p0[ia[t]] * r0[ib[t]] + p1[ia[t]] * r1[ib[t]] + p2[ia[t]] * r2[ib[t]];
      const double c0 = p0[3] - a * u * p2[3] - eta * u;
      const double c1 = p1[3] - a * v * p2[3] - eta * v;
      const double c2 = a * (w * p2[3] - u * p0[3] - v * p1[3]);
#pragma unroll
      for (int c = 0; c < 3; ++c) h[c] += c0 * p0[c] + c1 * p1[c] + c2 * p2[c];
    }
    // X = -V^-1 h by the Cholesky factor, pseudo-inverse when deficient
    double X[3];
    const double dmax = fmax(V[0], fmax(V[3], V[5]));
    const double f00 = rsqrt(V[0]);
    const double l10 = V[1] * f00, l20 = V[2] * f00;
    const double d1 = V[3] - l10 * l10;
    const double f11 = rsqrt(d1);
    const double l21 = (V[4] - l20 * l10) * f11;
    const double d2 = V[5] - l20 * l20 - l21 * l21;
    const double f22 = rsqrt(d2);
    const bool suspect = !(V[0] > 1e-9 * dmax) || !(d1 > 1e-9 * dmax) || !(d2 > 1e-9 * dmax) ||
                         !(dmax > 0.0);
    bool deficient = false;
    if (suspect) {
      Sym3 vs;
      Vec3 hs;
      for (int t = 0; t < 6; ++t) vs.v[t] = V[t];
      for (int c = 0; c < 3; ++c) hs.x[c] = h[c];
      const PinvOut o = pinv_solve(vs, hs);
      deficient = o.deficient;
      for (int c = 0; c < 3; ++c) X[c] = o.X[c];
    }
    if (!deficient) {
      const double f10 = -l10 * f00 * f11;
      const double f20 = -(l20 * f00 + l21 * f10) * f22;
      const double f21 = -l21 * f11 * f22;
      const double z0 = f00 * h[0];
      const double z1 = f10 * h[0] + f11 * h[1];
      const double z2 = f20 * h[0] + f21 * h[1] + f22 * h[2];
      X[0] = -(f00 * z0 + f10 * z1 + f20 * z2);
      X[1] = -(f11 * z1 + f21 * z2);
      X[2] = -(f22 * z2);
    }
    if (X_out) {
      X_out[3 * (size_t)j] = X[0];
      X_out[3 * (size_t)j + 1] = X[1];
      X_out[3 * (size_t)j + 2] = X[2];
    }
    // sum_k ||r_k||^2 at X, directly (Eq. pose, Eq. ba_first_stage)
    double s1 = 0.0, s2 = 0.0;
    for (int64_t k = b; k < e; ++k) {
      const int i = cam[k];
      if ((unsigned)i >= (unsigned)nc) continue;
      const double2 m = meas[k];
      const double2* Q = reinterpret_cast<const double2*>(P + 12 * (size_t)i);
      double q[12];
#pragma unroll
      for (int r = 0; r < 6; ++r) {
        const double2 x = __ldg(Q + r);
        q[2 * r] = x.x;
        q[2 * r + 1] = x.y;
      }
      const double y0 = fma(q[0], X[0], fma(q[1], X[1], fma(q[2], X[2], q[3])));
      const double y1 = fma(q[4], X[0], fma(q[5], X[1], fma(q[6], X[2], q[7])));
      const double y2 = fma(q[8], X[0], fma(q[9], X[1], fma(q[10], X[2], q[11])));
      const double a0 = fma(-m.x, y2, y0), a1 = fma(-m.y, y2, y1);
      const double g0 = y0 - m.x, g1 = y1 - m.y;
      s1 = fma(a0, a0, fma(a1, a1, s1));
      s2 = fma(g0, g0, fma(g1, g1, s2));
    }
    cost = bad ? __longlong_as_double(0x7ff8000000000000LL) : a * s1 + eta * s2;
  }
  // block partial in a fixed order: warp tree, then the warps in index order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cost;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NA_BLOCK / 32; ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

// Sum of the nb block partials in a fixed order into *cost_out.
__global__ void __launch_bounds__(256)
k_noalloc_sum(const double* __restrict__ part, int nb, double* __restrict__ cost_out) {
  __shared__ double red[256];
  double c = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) c += part[i];
  red[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *cost_out = red[0];
}

// Device address of the working array on the current device (looked up on
// the first call for that device).
cudaError_t na_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(na_mutex);
  if (!na_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, na_partials);
    if (e != cudaSuccess) return e;
    na_ptr[dev] = static_cast<double*>(ptr);
  }
  *out = na_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace povar

extern "C" povar_status povar_cost_noalloc(int32_t n_cams, int32_t n_points, int64_t n_obs,
                                           const double* P, const uint32_t* off_pt,
                                           const int32_t* cam, const double* meas, double eta,
                                           double* X_out, double* cost_out, void* cuda_stream) {
  using namespace povar;
  // argument checks first: they make no CUDA call
  if (!P || !off_pt || !cam || !meas || !cost_out) return POVAR_EINVAL;
  if (n_cams < 1 || n_points < 1 || n_obs < 1) return POVAR_EINVAL;
  if (n_points > POVAR_NOALLOC_MAX_POINTS) return POVAR_EINVAL;
  if (!(eta >= 0.0 && eta <= 1.0)) return POVAR_EINVAL;
  // the kernel reads P and meas as 16-byte pairs and the other arrays as
  // their own element type: a misaligned pointer is refused here instead of
  // faulting on the device
  const auto misaligned = [](const void* q, uintptr_t align) {
    return (reinterpret_cast<uintptr_t>(q) & (align - 1)) != 0;
  };
  if (misaligned(P, 16) || misaligned(meas, 16) || misaligned(off_pt, 4) ||
      misaligned(cam, 4) || misaligned(cost_out, 8) || (X_out && misaligned(X_out, 8)))
    return POVAR_EINVAL;
  // an error left pending by earlier, unrelated work belongs to its owner:
  // report it without consuming it, and launch nothing
  if (cudaPeekAtLastError() != cudaSuccess) return POVAR_ECUDA;
  double* part = nullptr;
  if (na_scratch(&part) != cudaSuccess) {
    cudaGetLastError();   // the error of this call's own look-up
    return POVAR_ECUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nb = (n_points + NA_BLOCK - 1) / NA_BLOCK;
  k_landmark_csr<<<nb, NA_BLOCK, 0, s>>>(P, n_cams, off_pt, cam,
                                         reinterpret_cast<const double2*>(meas), n_obs, n_points,
                                         eta, X_out, part);
  if (cudaGetLastError() != cudaSuccess) return POVAR_ECUDA;
  k_noalloc_sum<<<1, 256, 0, s>>>(part, nb, cost_out);
  if (cudaGetLastError() != cudaSuccess) return POVAR_ECUDA;
  return POVAR_OK;
}
