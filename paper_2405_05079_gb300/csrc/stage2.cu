// Second stage of the stratified problem: projective refinement (Eq.
// second_stage) by Riemannian PoBA (Sec. 4.3). Cameras P_i (3x4, vec on the
// unit sphere of R^12) and homogeneous landmarks X_j (unit sphere of R^4);
// per observation y = P_i X_j, r = (y1 / y3, y2 / y3) - m_ij, and with
// iz = 1 / y3, pi = (y1, y2) iz:
//   D  = d pi / d y = iz [[1, 0, -pi0], [0, 1, -pi1]]          (2x3)
//   J_p = D (I_3 (x) X^T) (2x12),  J_l = D P_i (2x4),
//   E  = D^T D = iz^2 [[1, 0, -pi0], [0, 1, -pi1], [-pi0, -pi1, pi0^2 + pi1^2]],
//   J_p^T J_p = E (x) X X^T,  J_p^T J_l = (I_3 (x) X) E P_i.
// Both tangent spaces are handled in projector form (Pi = I - x^ x^T), as
// the first stage's cameras: a damped block B restricted to the tangent
// space is inverted as (Pi B Pi + mu Pi + x^ x^T)^-1 - x^ x^T.
// Kernels (one LM iteration):
//   k_s2_prep        per landmark slot (FP64): V = sum (D P)^T (D P),
//                    b_l = sum (D P)^T r, the projected damped inverse G_l
//                    (mu = lambda_l lambda), s = G_l b_l; cost partials;
//   k_s2_linearize   camera-major chunks: the 60 moments E (x) XX^T of U and
//                    the reduced right-hand side J_p^T (r - J_l s) =
//                    b_p - W G_l b_l (projection and residual in FP64, sums
//                    in FP64, or FP32 in mixed precision);
//   k_s2_camera_prepare  per camera: damped projected 12x12 inverse G, the
//                    first series term x0 = -G (b_p - W s), FP32 copies;
//   per series term: k_s2_gather (per slot: s = G_l sum P^T E (Y X)) and
//                    k_s2_scatter (per chunk: sum (E P s) (x) X), then the
//                    first stage's per-camera apply (x = G z, delta += x);
//   k_s2_trial       per slot: back-substitution dX = -G_l (b_l + W^T dP),
//                    retraction X' = (X + dX) / |X + dX|, the trial cost at
//                    (P', X') and the Gauss-Newton model ||r + J dP + J dX||^2
//                    (projections, residuals and cost in FP64; W^T dP and the
//                    linearized model terms in FP32 in mixed precision).
// The per-camera update / retraction and the controller are the first
// stage's. Sums run in a fixed order (per thread, then fixed shuffles), so
// results do not depend on scheduling.
#include <algorithm>
#include <vector>

#include "block12.cuh"
#include "povar_internal.cuh"
#include "reproj.cuh"

namespace povar {
namespace {

using namespace b12;
using namespace rp;

constexpr int S2_LIN = 72;   // 60 moments of U + 12 right-hand-side entries

__device__ __forceinline__ double warp_total(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// G = (Pi V Pi + mu Pi + x x^T)^-1 - x x^T for the unit x, V symmetric
// (10 entries), by an unrolled 4x4 Cholesky in FP64. Returns false if a
// pivot is not positive (the block is then left as computed with floored
// pivots).
__device__ bool projected_inverse4(const double V[10], const double x[4], double mu,
                                   double G[10]) {
  double v[4];
  sym4_mul(V, x, v);
  const double c = v[0] * x[0] + v[1] * x[1] + v[2] * x[2] + v[3] * x[3];
  double A[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
      A[a][b] = V[sd_t10(a, b)] - v[a] * x[b] - x[a] * v[b] + (c - mu + 1.0) * x[a] * x[b] +
                (a == b ? mu : 0.0);
  bool ok = true;
  double L[4][4] = {};
  double rinv[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double d = A[k][k];
#pragma unroll
    for (int q = 0; q < k; ++q) d -= L[k][q] * L[k][q];
    if (!(d > 0.0)) ok = false;
    d = fmax(d, 1e-300);
    const double r = rsqrt(d);
    L[k][k] = d * r;
    rinv[k] = r;
#pragma unroll
    for (int a = k + 1; a < 4; ++a) {
      double s = A[a][k];
#pragma unroll
      for (int q = 0; q < k; ++q) s -= L[a][q] * L[k][q];
      L[a][k] = s * r;
    }
  }
  // Li = L^-1 (lower), then A^-1 = Li^T Li
  double Li[4][4] = {};
#pragma unroll
  for (int col = 0; col < 4; ++col) {
#pragma unroll
    for (int row = col; row < 4; ++row) {
      double s = row == col ? 1.0 : 0.0;
#pragma unroll
      for (int k = col; k < row; ++k) s -= L[row][k] * Li[k][col];
      Li[row][col] = s * rinv[row];
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      double s = 0.0;
#pragma unroll
      for (int k = b; k < 4; ++k) s += Li[k][a] * Li[k][b];
      G[sd_t10(a, b)] = s - x[a] * x[b];
    }
  return ok;
}

// Slot s's observation k (landmark-major SELL layout)
__device__ __forceinline__ uint32_t sell_pos(const uint32_t* __restrict__ sell_off, int s,
                                             uint32_t k) {
  return sell_off[s / SLICE] + (uint32_t)(s % SLICE) + k * SLICE;
}

// Warp partials of a per-slot value (slots of a warp = one SELL slice).
__device__ __forceinline__ void warp_partial(double v, double* __restrict__ out, int s) {
  v = warp_total(v);
  if ((threadIdx.x & 31) == 0) out[s / 32] = v;
}

// ---------------------------------------------------------------------------
// Set-up: normalized cameras and landmarks, cost
// ---------------------------------------------------------------------------

__global__ void k_s2_set_cameras(const DeviceState* __restrict__ st, int nc,
                                 const double* __restrict__ Pin, double* __restrict__ P0,
                                 double* __restrict__ P1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double* P = (st->cur ? P1 : P0) + 12 * (size_t)i;
  const double* src = Pin ? Pin + 12 * (size_t)i : P;
  double q[12], nn = 0.0;
  for (int e = 0; e < 12; ++e) {
    q[e] = src[e];
    nn += q[e] * q[e];
  }
  const double f = 1.0 / sqrt(nn);
  for (int e = 0; e < 12; ++e) P[e] = q[e] * f;
}

// Homogeneous landmarks per slot: from Xin (by landmark id, 4 each) or from
// the first stage's FP64 landmarks (X, 1); normalized. Padding slots get 0.
__global__ void k_s2_set_points(const DeviceState* __restrict__ st, int np_pad,
                                const uint32_t* __restrict__ slot_pt, const double* __restrict__ Xin,
                                const double* __restrict__ X3_0, const double* __restrict__ X3_1,
                                double* __restrict__ X4_0, double* __restrict__ X4_1,
                                float4* __restrict__ X4f) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np_pad) return;
  const int cur = st->cur;
  double* X4 = (cur ? X4_1 : X4_0) + 4 * (size_t)s;
  const uint32_t j = slot_pt[s];
  double x[4] = {0.0, 0.0, 0.0, 0.0};
  if (j != ~0u) {
    if (Xin) {
      for (int e = 0; e < 4; ++e) x[e] = Xin[4 * (size_t)j + e];
    } else {
      const double* X3 = (cur ? X3_1 : X3_0) + 3 * (size_t)s;
      x[0] = X3[0];
      x[1] = X3[1];
      x[2] = X3[2];
      x[3] = 1.0;
    }
    const double f = 1.0 / sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2] + x[3] * x[3]);
    for (int e = 0; e < 4; ++e) x[e] *= f;
  }
  for (int e = 0; e < 4; ++e) X4[e] = x[e];
  X4f[s] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)x[3]);
}

__global__ void __launch_bounds__(BLOCK)
k_s2_cost(const DeviceState* __restrict__ st, const uint32_t* __restrict__ slot_len,
          const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
          const double2* __restrict__ sell_m, const double* __restrict__ P0,
          const double* __restrict__ P1, const double* __restrict__ X4_0,
          const double* __restrict__ X4_1, double* __restrict__ cost_part,
          int* __restrict__ pinv_part) {
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int cur = st->cur;
  const double* Pb = cur ? P1 : P0;
  const double* Xs = (cur ? X4_1 : X4_0) + 4 * (size_t)s;
  const double X[4] = {Xs[0], Xs[1], Xs[2], Xs[3]};
  const uint32_t len = slot_len[s];
  double c = 0.0;
  for (uint32_t k = 0; k < len; ++k) {
    const uint32_t pos = sell_pos(sell_off, s, k);
    double P[12];
    load12(Pb + 12 * (size_t)sell_cam[pos], P);
    const double2 m = sell_m[pos];
    const Proj<double> q = project(P, X);
    const double r0 = q.p0 - m.x, r1 = q.p1 - m.y;
    c += r0 * r0 + r1 * r1;
  }
  warp_partial(c, cost_part, s);
  if ((threadIdx.x & 31) == 0) pinv_part[s / 32] = 0;
}

// ---------------------------------------------------------------------------
// Landmark side of one step
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(BLOCK)
k_s2_prep(DeviceState* __restrict__ st, double lambda_l, const uint32_t* __restrict__ slot_len,
          const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
          const double2* __restrict__ sell_m, const double* __restrict__ P0,
          const double* __restrict__ P1, const double* __restrict__ X4_0,
          const double* __restrict__ X4_1, double* __restrict__ Gl64, float4* __restrict__ Gl32,
          double* __restrict__ bl64, double* __restrict__ s64, float4* __restrict__ X4f) {
  if (st->converged) return;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int cur = st->cur;
  const double* Pb = cur ? P1 : P0;
  const double* Xs = (cur ? X4_1 : X4_0) + 4 * (size_t)s;
  const double X[4] = {Xs[0], Xs[1], Xs[2], Xs[3]};
  const uint32_t len = slot_len[s];
  double G[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, bl[4] = {0, 0, 0, 0}, sv[4] = {0, 0, 0, 0};
  bool ok = true;
  if (len > 0) {
    double V[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = sell_pos(sell_off, s, k);
      double P[12];
      load12(Pb + 12 * (size_t)sell_cam[pos], P);
      const double2 m = sell_m[pos];
      const Proj<double> q = project(P, X);
      const double r0 = q.p0 - m.x, r1 = q.p1 - m.y;
      // rows of J_l = D P: iz (P_r - pi_r P_2)
      double g0[4], g1[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        g0[c] = q.iz * (P[c] - q.p0 * P[8 + c]);
        g1[c] = q.iz * (P[4 + c] - q.p1 * P[8 + c]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = a; b < 4; ++b) V[sd_t10(a, b)] += g0[a] * g0[b] + g1[a] * g1[b];
        bl[a] += g0[a] * r0 + g1[a] * r1;
      }
    }
    // if rounding leaves the damped block indefinite (a landmark close to a
    // camera's principal plane makes V huge), its damping is raised as for
    // the camera blocks: to 1e-12 of the largest diagonal entry, then x100
    // per attempt, at most 8 attempts, counted in the device state
    const double vmax = fmax(fmax(V[0], V[4]), fmax(V[7], V[9]));
    double mu = lambda_l * st->lam;
    int attempt = 0;
    for (; attempt < 8; ++attempt) {
      if (attempt > 0) mu = fmax(mu * 100.0, 1e-12 * vmax);
      ok = projected_inverse4(V, X, mu, G);
      if (ok) break;
    }
    if (ok && attempt > 0) atomicAdd(&st->n_regularized, 1);
    sym4_mul(G, bl, sv);
  }
  if (!ok) st->error = POVAR_ENUMERIC;
#pragma unroll
  for (int e = 0; e < 10; ++e) Gl64[10 * (size_t)s + e] = G[e];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    bl64[4 * (size_t)s + e] = bl[e];
    s64[4 * (size_t)s + e] = sv[e];
  }
  Gl32[3 * (size_t)s] = make_float4((float)G[0], (float)G[1], (float)G[2], (float)G[3]);
  Gl32[3 * (size_t)s + 1] = make_float4((float)G[4], (float)G[5], (float)G[6], (float)G[7]);
  Gl32[3 * (size_t)s + 2] = make_float4((float)G[8], (float)G[9], 0.f, 0.f);
  X4f[s] = make_float4((float)X[0], (float)X[1], (float)X[2], (float)X[3]);
}

// ---------------------------------------------------------------------------
// Camera side of one step
// ---------------------------------------------------------------------------

// One warp per camera-major chunk: 60 moments E_e X_c X_d (e over the six
// entries of E, t10 order of the moments) and the right-hand side
// J_p^T (r - J_l s) = vec((D^T (r - D P s)) X^T) (12). The projection and
// the residual are FP64; the accumulation runs in TA (FP64, or FP32 in
// mixed precision: each lane sums at most 16 observations of the chunk, the
// chunk's lane sums are added by fixed shuffles, chunk totals in FP64).
template <typename TA>
__global__ void __launch_bounds__(256)
k_s2_linearize(const DeviceState* __restrict__ st, int nchunks,
               const int32_t* __restrict__ chunk_cam, const uint32_t* __restrict__ chunk_beg,
               const uint32_t* __restrict__ cm_slot, const double2* __restrict__ cm_m,
               const double* __restrict__ P0, const double* __restrict__ P1,
               const double* __restrict__ X4_0, const double* __restrict__ X4_1,
               const double* __restrict__ s64, double* __restrict__ part) {
  if (st->converged) return;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= nchunks) return;
  const int cur = st->cur;
  double P[12];
  load12((cur ? P1 : P0) + 12 * (size_t)chunk_cam[c], P);
  TA Pa[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) Pa[e] = (TA)P[e];
  const double* Xb = cur ? X4_1 : X4_0;
  TA acc[S2_LIN];
#pragma unroll
  for (int e = 0; e < S2_LIN; ++e) acc[e] = 0;
  const uint32_t b = chunk_beg[c], e_ = chunk_beg[c + 1];
  for (uint32_t r = b + lane; r < e_; r += 32) {
    const uint32_t slot = cm_slot[r];
    const double2 m = cm_m[r];
    const double X[4] = {Xb[4 * (size_t)slot], Xb[4 * (size_t)slot + 1],
                         Xb[4 * (size_t)slot + 2], Xb[4 * (size_t)slot + 3]};
    const Proj<double> q = project(P, X);
    const TA Xa[4] = {(TA)X[0], (TA)X[1], (TA)X[2], (TA)X[3]};
    const TA sv[4] = {(TA)s64[4 * (size_t)slot], (TA)s64[4 * (size_t)slot + 1],
                      (TA)s64[4 * (size_t)slot + 2], (TA)s64[4 * (size_t)slot + 3]};
    Proj<TA> qa;
    qa.y[0] = (TA)q.y[0];
    qa.y[1] = (TA)q.y[1];
    qa.y[2] = (TA)q.y[2];
    qa.iz = (TA)q.iz;
    qa.p0 = (TA)q.p0;
    qa.p1 = (TA)q.p1;
    const TA iz2 = qa.iz * qa.iz;
    const TA E[6] = {iz2, (TA)0, -qa.p0 * iz2, iz2, -qa.p1 * iz2,
                     (qa.p0 * qa.p0 + qa.p1 * qa.p1) * iz2};
    const TA t10[10] = {Xa[0] * Xa[0], Xa[0] * Xa[1], Xa[0] * Xa[2], Xa[0] * Xa[3],
                        Xa[1] * Xa[1], Xa[1] * Xa[2], Xa[1] * Xa[3], Xa[2] * Xa[2],
                        Xa[2] * Xa[3], Xa[3] * Xa[3]};
#pragma unroll
    for (int kk = 0; kk < 6; ++kk) {
      if (kk == 1) continue;   // E_01 = 0
#pragma unroll
      for (int t = 0; t < 10; ++t) acc[10 * kk + t] += E[kk] * t10[t];
    }
    TA ps[3], dps[2], t[3];
    apply_p(Pa, sv, ps);
    apply_d(qa, ps, dps);
    const TA a[2] = {(TA)(q.p0 - m.x) - dps[0], (TA)(q.p1 - m.y) - dps[1]};
    apply_dt(qa, a, t);
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc[60 + 4 * rr + d] += t[rr] * Xa[d];
  }
  double* out = part + (size_t)c * S2_LIN;
#pragma unroll
  for (int e = 0; e < S2_LIN; ++e) {
    TA v = acc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((e & 31) == lane) out[e] = (double)v;
  }
}

// One warp per camera: U = E (x) XX^T from the chunk sums, the right-hand
// side, the damped tangent-projected inverse G (as the first stage's camera
// preparation: raised damping if rounding leaves the block indefinite), the
// first series term, FP32 copies of P, G.
template <typename T>
__global__ void __launch_bounds__(128)
k_s2_camera_prepare(DeviceState* __restrict__ st, int nc, const int32_t* __restrict__ cam_nchunk,
                    const int32_t* __restrict__ cam_chunk0, const double* __restrict__ part,
                    double* __restrict__ P0, double* __restrict__ P1, float* __restrict__ Pf0,
                    float* __restrict__ Pf1, double* __restrict__ U64, double* __restrict__ bp64,
                    double* __restrict__ G64, float* __restrict__ G32, T* __restrict__ Y,
                    T* __restrict__ D, double* __restrict__ camnorm) {
  if (st->converged) return;
  __shared__ double smA[4][12][13], smL[4][12][13], smI[4][12][13];
  __shared__ double smK[4][S2_LIN];
  __shared__ double smR[4][12];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x * 4 + wl;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->stop_series = 0;
    st->terms_used = 1;
    st->lam_used = st->lam;
  }
  if (i >= nc) return;
  const int cur = st->cur;
  const double lam = st->lam;
  const double* Pc = (cur ? P1 : P0) + 12 * (size_t)i;
  if (lane < 12) (cur ? Pf1 : Pf0)[12 * (size_t)i + lane] = (float)Pc[lane];
  const int n = cam_nchunk[i], c0 = cam_chunk0[i];
  for (int e = lane; e < S2_LIN; e += 32) {
    double s = 0.0;
    for (int q = 0; q < n; ++q) s += part[(size_t)(c0 + q) * S2_LIN + e];
    smK[wl][e] = s;
  }
  __syncwarp();
  double (*A)[13] = smA[wl];
  const double ph = unit_camera(Pc, lane, POVAR_SPHERE);
  const double bpl = lane < 12 ? smK[wl][60 + lane] : 0.0;
  // U entry ((a,c),(b,d)) = E_ab X_c X_d summed
  if (lane < 12) {
    const int ra = lane >> 2, rc = lane & 3;
    for (int q = 0; q < 12; ++q) {
      const int cb = q >> 2, cd = q & 3;
      const double u = smK[wl][10 * sym3(ra, cb) + sd_t10(rc, cd)];
      U64[(size_t)i * 144 + lane * 12 + q] = u;
    }
    bp64[(size_t)i * 12 + lane] = bpl;
  }
  __syncwarp();
  double umax = lane < 12 ? U64[(size_t)i * 144 + lane * 13] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
  double lam_eff = lam;
  bool ok = false;
  int attempt = 0;
  for (; attempt < 8 && !ok; ++attempt) {
    if (attempt > 0) lam_eff = fmax(lam_eff * 100.0, 1e-12 * umax);
    if (lane < 12)
      for (int q = 0; q < 12; ++q)
        A[lane][q] = U64[(size_t)i * 144 + lane * 12 + q] + (lane == q ? lam_eff : 0.0);
    __syncwarp();
    // Pi (U + lam I) Pi + p^ p^T
    double bp = 0.0;
    for (int q = 0; q < 12; ++q) {
      const double pq = __shfl_sync(0xffffffffu, ph, q);
      if (lane < 12) bp += A[lane][q] * pq;
    }
    const double cc = warp_sum(ph * bp);
    __syncwarp();
    for (int q = 0; q < 12; ++q) {
      const double pq = __shfl_sync(0xffffffffu, ph, q);
      const double bq = __shfl_sync(0xffffffffu, bp, q);
      if (lane < 12) A[lane][q] += -bp * pq - ph * bq + (cc + 1.0) * ph * pq;
    }
    __syncwarp();
    ok = chol_inverse12(A, smL[wl], smI[wl], smR[wl], lane);
  }
  if (lane == 0) {
    if (!ok) st->error = POVAR_ENUMERIC;
    else if (attempt > 1) atomicAdd(&st->n_regularized, 1);
  }
  double x0 = 0.0;
  for (int q = 0; q < 12; ++q) {
    const double pq = __shfl_sync(0xffffffffu, ph, q);
    const double bq = __shfl_sync(0xffffffffu, bpl, q);
    if (lane < 12) {
      const double g = smI[wl][lane][q] - ph * pq;
      G64[(size_t)i * 144 + lane * 12 + q] = g;
      G32[(size_t)i * 144 + lane * 12 + q] = (float)g;
      x0 -= g * bq;
    }
  }
  if (lane < 12) {
    Y[(size_t)i * 12 + lane] = (T)x0;
    Y[((size_t)nc + i) * 12 + lane] = (T)0;
    D[(size_t)i * 12 + lane] = (T)x0;
  }
  if (lane < 2) camnorm[2 * (size_t)i + lane] = 0.0;
}

// ---------------------------------------------------------------------------
// Series product W~ V~^-1 W~^T y
// ---------------------------------------------------------------------------

// Per slot: s = G_l sum_k P_i^T E_k (Y_i X) (landmark-major pass).
template <typename T>
__global__ void __launch_bounds__(BLOCK)
k_s2_gather(const DeviceState* __restrict__ st, const uint32_t* __restrict__ slot_len,
            const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
            const T* __restrict__ Pa, const T* __restrict__ Pb, const T* __restrict__ Y,
            S2Land<T> land, T* __restrict__ rec) {
  if (st->converged || st->stop_series) return;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int cur = st->cur;
  const T* Pc = cur ? Pb : Pa;
  T X[4], g[10];
  land.load(cur, s, X, g);
  T acc[4] = {0, 0, 0, 0};
  const uint32_t len = slot_len[s];
  for (uint32_t k = 0; k < len; ++k) {
    const int i = sell_cam[sell_pos(sell_off, s, k)];
    T P[12], Yi[12];
    load12(Pc + 12 * (size_t)i, P);
    load12(Y + 12 * (size_t)i, Yi);
    const Proj<T> q = project(P, X);
    T w[3], ew[3], pt[4];
    apply_p(Yi, X, w);
    apply_e(q, w, ew);
    apply_pt(P, ew, pt);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += pt[e];
  }
  T sv[4];
  sym4_mul(g, acc, sv);
#pragma unroll
  for (int e = 0; e < 4; ++e) rec[4 * (size_t)s + e] = sv[e];
}

// One warp per camera-major chunk: sum_k vec((E_k P_i s_j) X_j^T), reduced
// over the warp in a fixed order into the chunk's partial (12).
template <typename T>
__global__ void __launch_bounds__(256)
k_s2_scatter(const DeviceState* __restrict__ st, int nchunks,
             const int32_t* __restrict__ chunk_cam, const uint32_t* __restrict__ chunk_beg,
             const uint32_t* __restrict__ cm_slot, const T* __restrict__ Pa,
             const T* __restrict__ Pb, S2Land<T> land, const T* __restrict__ rec,
             T* __restrict__ part) {
  if (st->converged || st->stop_series) return;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= nchunks) return;
  const int cur = st->cur;
  T P[12];
  load12((cur ? Pb : Pa) + 12 * (size_t)chunk_cam[c], P);
  T acc[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) acc[e] = 0;
  const uint32_t b = chunk_beg[c], e_ = chunk_beg[c + 1];
  for (uint32_t r = b + lane; r < e_; r += 32) {
    const uint32_t slot = cm_slot[r];
    T X[4];
    land.load_x(cur, (int)slot, X);
    const T sv[4] = {rec[4 * (size_t)slot], rec[4 * (size_t)slot + 1], rec[4 * (size_t)slot + 2],
                     rec[4 * (size_t)slot + 3]};
    const Proj<T> q = project(P, X);
    T v[3], ev[3];
    apply_p(P, sv, v);
    apply_e(q, v, ev);
#pragma unroll
    for (int rr = 0; rr < 3; ++rr)
#pragma unroll
      for (int d = 0; d < 4; ++d) acc[4 * rr + d] += ev[rr] * X[d];
  }
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    T v = acc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == e) part[(size_t)c * 12 + e] = v;
  }
}

// ---------------------------------------------------------------------------
// Back-substitution, retraction, trial cost and model decrease
// ---------------------------------------------------------------------------

// TD: the type of the camera step; TA: the arithmetic of the linearized
// parts (W^T dP for the back-substitution, J dP + J dX for the model): FP64,
// or FP32 in mixed precision. The trial projections and residuals, the
// residuals at the current point, the back-substitution with G_l and the
// retraction are FP64 in both.
template <typename TD, typename TA>
__global__ void __launch_bounds__(BLOCK)
k_s2_trial(const DeviceState* __restrict__ st, const uint32_t* __restrict__ slot_len,
           const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
           const double2* __restrict__ sell_m, const double* __restrict__ P0,
           const double* __restrict__ P1, const TD* __restrict__ Dp, double* __restrict__ X4_0,
           double* __restrict__ X4_1, const double* __restrict__ Gl64,
           const double* __restrict__ bl64, double* __restrict__ cost_part,
           double* __restrict__ model_part, int* __restrict__ pinv_part) {
  if (st->converged) return;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int cur = st->cur;
  const double* Pc = cur ? P1 : P0;
  const double* Pn = cur ? P0 : P1;
  const double* Xs = (cur ? X4_1 : X4_0) + 4 * (size_t)s;
  double* Xo = (cur ? X4_0 : X4_1) + 4 * (size_t)s;
  const double X[4] = {Xs[0], Xs[1], Xs[2], Xs[3]};
  const TA Xa[4] = {(TA)X[0], (TA)X[1], (TA)X[2], (TA)X[3]};
  const uint32_t len = slot_len[s];
  double cost = 0.0, model = 0.0;
  double Xn[4] = {0, 0, 0, 0};
  if (len > 0) {
    // W^T dP = sum J_l^T J_p dP = sum P^T E (dP X)
    TA a[4] = {0, 0, 0, 0};
    for (uint32_t k = 0; k < len; ++k) {
      const int i = sell_cam[sell_pos(sell_off, s, k)];
      TA P[12], dP[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        P[e] = (TA)Pc[12 * (size_t)i + e];
        dP[e] = (TA)Dp[12 * (size_t)i + e];
      }
      const Proj<TA> q = project(P, Xa);
      TA w[3], ew[3], pt[4];
      apply_p(dP, Xa, w);
      apply_e(q, w, ew);
      apply_pt(P, ew, pt);
#pragma unroll
      for (int e = 0; e < 4; ++e) a[e] += pt[e];
    }
    double g[10], dx[4], ad[4];
#pragma unroll
    for (int e = 0; e < 10; ++e) g[e] = Gl64[10 * (size_t)s + e];
#pragma unroll
    for (int e = 0; e < 4; ++e) ad[e] = (double)a[e] + bl64[4 * (size_t)s + e];
    sym4_mul(g, ad, dx);
    double nn = 0.0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      dx[e] = -dx[e];
      Xn[e] = X[e] + dx[e];
      nn += Xn[e] * Xn[e];
    }
    const double f = 1.0 / sqrt(nn);
#pragma unroll
    for (int e = 0; e < 4; ++e) Xn[e] *= f;
    const TA dxa[4] = {(TA)dx[0], (TA)dx[1], (TA)dx[2], (TA)dx[3]};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = sell_pos(sell_off, s, k);
      const int i = sell_cam[pos];
      const double2 m = sell_m[pos];
      double P[12], Pt[12];
      load12(Pc + 12 * (size_t)i, P);
      load12(Pn + 12 * (size_t)i, Pt);
      // trial cost
      const Proj<double> qt = project(Pt, Xn);
      const double t0 = qt.p0 - m.x, t1 = qt.p1 - m.y;
      cost += t0 * t0 + t1 * t1;
      // model: r + D (dP X + P dX) at the current point
      const Proj<double> q = project(P, X);
      Proj<TA> qa;
      qa.y[0] = (TA)q.y[0];
      qa.y[1] = (TA)q.y[1];
      qa.y[2] = (TA)q.y[2];
      qa.iz = (TA)q.iz;
      qa.p0 = (TA)q.p0;
      qa.p1 = (TA)q.p1;
      TA Pa[12], dP[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        Pa[e] = (TA)P[e];
        dP[e] = (TA)Dp[12 * (size_t)i + e];
      }
      TA w[3], pdx[3], dl[2];
      apply_p(dP, Xa, w);
      apply_p(Pa, dxa, pdx);
#pragma unroll
      for (int rr = 0; rr < 3; ++rr) w[rr] += pdx[rr];
      apply_d(qa, w, dl);
      const double l0 = q.p0 - m.x + (double)dl[0], l1 = q.p1 - m.y + (double)dl[1];
      model += l0 * l0 + l1 * l1;
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) Xo[e] = Xn[e];
  warp_partial(cost, cost_part, s);
  warp_partial(model, model_part, s);
  if ((threadIdx.x & 31) == 0) pinv_part[s / 32] = 0;
}

// Homogeneous landmarks by landmark id (current buffer).
__global__ void k_s2_gather_points(const DeviceState* __restrict__ st, const double* __restrict__ X0,
                                   const double* __restrict__ X1,
                                   const uint32_t* __restrict__ pt_slot, int np,
                                   double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const double* X = (st->cur ? X1 : X0) + 4 * (size_t)pt_slot[j];
  for (int e = 0; e < 4; ++e) out[4 * (size_t)j + e] = X[e];
}

__global__ void k_s2_chunk_lists(int nc, int nchunks, const int32_t* __restrict__ cam_chunk0,
                                 uint32_t* __restrict__ off, uint32_t* __restrict__ idx) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nc) off[k] = (uint32_t)cam_chunk0[k];
  if (k == nc) off[k] = (uint32_t)nchunks;
  if (k < nchunks) idx[k] = (uint32_t)k;
}

}  // namespace
}  // namespace povar

namespace povar {

povar_status ensure_stage2(Problem* p) {
  if (p->s2off) return POVAR_OK;
  povar_status s;
  const size_t npd = (size_t)p->np_pad, nch = (size_t)std::max(p->nchunks, 1);
  if ((s = dev_alloc(p, &p->s2X[0], npd * 4, "s2X0")) ||
      (s = dev_alloc(p, &p->s2X[1], npd * 4, "s2X1")) ||
      (s = dev_alloc(p, &p->s2Xf, npd, "s2Xf")) ||
      (s = dev_alloc(p, &p->s2Gl64, npd * 10, "s2Gl64")) ||
      (s = dev_alloc(p, &p->s2Gl32, npd * 3, "s2Gl32")) ||
      (s = dev_alloc(p, &p->s2bl, npd * 4, "s2bl")) ||
      (s = dev_alloc(p, &p->s2s, npd * 4, "s2s")) ||
      (s = dev_alloc(p, &p->s2rec, npd * 4, "s2rec")) ||
      (s = dev_alloc(p, &p->s2lin, nch * S2_LIN, "s2lin")) ||
      (s = dev_alloc(p, &p->s2part, nch * 12, "s2part")) ||
      (s = dev_alloc(p, &p->s2idx, nch, "s2idx")) ||
      (s = dev_alloc(p, &p->s2off, (size_t)p->nc + 1, "s2off")))
    return s;
  POVAR_CUDA(cudaMemsetAsync(p->s2X[0], 0, npd * 4 * sizeof(double), p->stream));
  POVAR_CUDA(cudaMemsetAsync(p->s2X[1], 0, npd * 4 * sizeof(double), p->stream));
  const int n = std::max(p->nc + 1, p->nchunks);
  k_s2_chunk_lists<<<grid_for(n, 256), 256, 0, p->stream>>>(p->nc, p->nchunks, p->cam_chunk0,
                                                            p->s2off, p->s2idx);
  ++p->launches;
  return check_launch(p, "s2_chunk_lists");
}

povar_status launch_s2_set(Problem* p, const double* d_P, const double* d_X) {
  povar_status s;
  if ((s = ensure_stage2(p)) != POVAR_OK) return s;
  k_s2_set_cameras<<<grid_for(p->nc, 128), 128, 0, p->stream>>>(p->state, p->nc, d_P, p->P64[0],
                                                                p->P64[1]);
  k_s2_set_points<<<grid_for(p->np_pad, 256), 256, 0, p->stream>>>(
      p->state, p->np_pad, p->slot_pt, d_X, p->X64[0], p->X64[1], p->s2X[0], p->s2X[1],
      p->s2Xf);
  p->launches += 2;
  return check_launch(p, "s2_set");
}

povar_status launch_s2_cost(Problem* p) {
  k_s2_cost<<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
      p->state, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
      p->s2X[0], p->s2X[1], p->cost_part, p->pinv_part);
  ++p->launches;
  povar_status s;
  if ((s = check_launch(p, "s2_cost")) != POVAR_OK) return s;
  return launch_cost_finish(p, 0);
}

povar_status launch_s2_prep(Problem* p, double lambda_l) {
  k_s2_prep<<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
      p->state, lambda_l, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0],
      p->P64[1], p->s2X[0], p->s2X[1], p->s2Gl64, p->s2Gl32, p->s2bl, p->s2s, p->s2Xf);
  ++p->launches;
  return check_launch(p, "s2_prep");
}

povar_status launch_s2_linearize(Problem* p, int precision) {
  const unsigned g = grid_for(p->nchunks, 8);
  if (g == 0) return POVAR_OK;
  if (precision == POVAR_FP64)
    k_s2_linearize<double><<<g, 256, 0, p->stream>>>(
        p->state, p->nchunks, p->chunk_cam, p->chunk_beg, p->cm_slot, p->cm_m64, p->P64[0],
        p->P64[1], p->s2X[0], p->s2X[1], p->s2s, p->s2lin);
  else
    k_s2_linearize<float><<<g, 256, 0, p->stream>>>(
        p->state, p->nchunks, p->chunk_cam, p->chunk_beg, p->cm_slot, p->cm_m64, p->P64[0],
        p->P64[1], p->s2X[0], p->s2X[1], p->s2s, p->s2lin);
  ++p->launches;
  return check_launch(p, "s2_linearize");
}

povar_status launch_s2_camera_prepare(Problem* p, int precision) {
  const unsigned g = grid_for(p->nc, 4);
  if (precision == POVAR_FP64)
    k_s2_camera_prepare<double><<<g, 128, 0, p->stream>>>(
        p->state, p->nc, p->cam_nchunk, p->cam_chunk0, p->s2lin, p->P64[0], p->P64[1],
        p->camP32[0], p->camP32[1], p->U64, p->bp64, p->G64, p->G32, p->Y64, p->D64,
        p->camnorm);
  else
    k_s2_camera_prepare<float><<<g, 128, 0, p->stream>>>(
        p->state, p->nc, p->cam_nchunk, p->cam_chunk0, p->s2lin, p->P64[0], p->P64[1],
        p->camP32[0], p->camP32[1], p->U64, p->bp64, p->G64, p->G32, p->Y32, p->D32,
        p->camnorm);
  ++p->launches;
  return check_launch(p, "s2_camera_prepare");
}

povar_status launch_s2_series_term(Problem* p, int precision, int term, double eps) {
  // the series vector is double-buffered by term parity, as in the first stage
  const size_t yoff_in = ((term - 1) & 1) * (size_t)p->nc * 12;
  const unsigned gs = grid_for(p->nchunks, 8);
  if (precision == POVAR_FP64) {
    S2Land<double> land{p->s2X[0], p->s2X[1], p->s2Gl64};
    k_s2_gather<double><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, p->slot_len, p->sell_off, p->sell_cam, p->P64[0], p->P64[1],
        p->Y64 + yoff_in, land, p->s2rec);
    if (gs > 0)
      k_s2_scatter<double><<<gs, 256, 0, p->stream>>>(p->state, p->nchunks, p->chunk_cam,
                                                      p->chunk_beg, p->cm_slot, p->P64[0],
                                                      p->P64[1], land, p->s2rec, p->s2part);
  } else {
    S2Land<float> land{p->s2Xf, p->s2Gl32};
    float* rec = reinterpret_cast<float*>(p->s2rec);
    float* part = reinterpret_cast<float*>(p->s2part);
    k_s2_gather<float><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, p->slot_len, p->sell_off, p->sell_cam, p->camP32[0], p->camP32[1],
        p->Y32 + yoff_in, land, rec);
    if (gs > 0)
      k_s2_scatter<float><<<gs, 256, 0, p->stream>>>(p->state, p->nchunks, p->chunk_cam,
                                                     p->chunk_beg, p->cm_slot, p->camP32[0],
                                                     p->camP32[1], land, rec, part);
  }
  p->launches += gs > 0 ? 2 : 1;
  povar_status s;
  if ((s = check_launch(p, "s2_series")) != POVAR_OK) return s;
  return launch_series_apply(p, precision, term, eps, p->s2off, p->s2idx, p->s2part);
}

povar_status launch_s2_trial(Problem* p, int precision, int m) {
  if (precision == POVAR_FP64)
    k_s2_trial<double, double><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
        p->D64, p->s2X[0], p->s2X[1], p->s2Gl64, p->s2bl, p->cost_part, p->pred_part,
        p->pinv_part);
  else
    k_s2_trial<float, float><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
        p->D32, p->s2X[0], p->s2X[1], p->s2Gl64, p->s2bl, p->cost_part, p->pred_part,
        p->pinv_part);
  ++p->launches;
  povar_status s;
  if ((s = check_launch(p, "s2_trial")) != POVAR_OK) return s;
  if ((s = launch_cost_finish(p, 1)) != POVAR_OK) return s;
  return launch_model_pred_finish(p, m);
}

povar_status launch_s2_gather_points(Problem* p, double* d_out) {
  k_s2_gather_points<<<grid_for(p->np, 256), 256, 0, p->stream>>>(p->state, p->s2X[0],
                                                                  p->s2X[1], p->pt_slot, p->np,
                                                                  d_out);
  ++p->launches;
  return check_launch(p, "s2_gather_points");
}

}  // namespace povar
