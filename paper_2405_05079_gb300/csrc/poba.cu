// PoBA (Sec. 2 of the paper; the power-series bundle adjustment its
// PoVar builds on): joint Levenberg-Marquardt on the pOSE cost, one of the
// comparison solvers of Sec. 5.2. Unlike the VarPro step, the landmarks are
// variables of the damped iteration: at (P, X) the joint normal equation
//   [[U + lambda I, W], [W^T, V + lambda_l lambda I]] (dP, dX) = -(b_p, b_l)
// is reduced to the damped Schur complement
//   S = U_lambda - W V_lambda^-1 W^T,   S dP = -(b_p - W V_lambda^-1 b_l),
// which the same series kernels invert (they read the factor of V_lambda
// instead of V), and the landmarks follow by back-substitution
//   dX = -V_lambda^-1 (b_l + W^T dP).
// Kernels of this file:
//   k_poba_prep   per landmark at (P, X): V_j, h_j from the camera tables,
//                 b_l = V X + h (the gradient J_l^T r at X), the factor of
//                 V + lambda_l lambda I and s_j = V_lambda^-1 b_l. The
//                 right-hand side needs no extra pass: W s = sum J_p^T J_l s
//                 and J_l s = B Pbar s, so b_p - W s is J_p^T r evaluated at
//                 the shifted landmark X - s (k_linearize with sbl);
//   k_poba_trial  after the camera update, per landmark: dX from W^T dP
//                 (one pass over its observations), X' = X + dX into the
//                 trial buffer, then the trial cost at (P', X') and the
//                 Gauss-Newton model sum ||r + J_p dP + J_l dX||^2 (one more
//                 pass), per-warp partials;
//   k_poba_pred_finish  pred = F - sum of the model partials (fixed order).
// Everything here is FP64; in POVAR_MIXED_FP32 the linearization and the
// series run in FP32 as for PoVar.
#include "povar_internal.cuh"

namespace povar {
namespace {

// 1 - eta weighted measurement block C = B^T B of Eq. pose, applied to y:
// (y0 - a u y2, y1 - a v y2, a (w y2 - u y0 - v y1)), a = 1 - eta.
__device__ __forceinline__ void apply_c(double a, double u, double v, const double y[3],
                                        double c[3]) {
  const double w = u * u + v * v;
  c[0] = y[0] - a * u * y[2];
  c[1] = y[1] - a * v * y[2];
  c[2] = a * (w * y[2] - u * y[0] - v * y[1]);
}

__global__ void __launch_bounds__(BLOCK)
k_poba_prep(DeviceState* __restrict__ st, double lambda_l, const uint32_t* __restrict__ slot_len,
            const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
            const double2* __restrict__ sell_m, const double* __restrict__ Ltab,
            double* __restrict__ X0, double* __restrict__ X1, double* __restrict__ F0,
            double* __restrict__ F1, float4* __restrict__ A0, float4* __restrict__ A1,
            float4* __restrict__ B0, float4* __restrict__ B1, float* __restrict__ C0,
            float* __restrict__ C1, double* __restrict__ sbl64, float4* __restrict__ sbl32) {
  if (st->converged) return;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int t = st->cur;
  const double* X = (t ? X1 : X0) + 3 * (size_t)s;
  double* Fo = (t ? F1 : F0) + 6 * (size_t)s;
  const uint32_t len = slot_len[s];
  double F[6] = {0, 0, 0, 0, 0, 0}, sb[3] = {0, 0, 0};
  const double x[3] = {X[0], X[1], X[2]};
  if (len > 0) {
    const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
    double V[6] = {0, 0, 0, 0, 0, 0}, h[3] = {0, 0, 0};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const double2 m = sell_m[pos];
      const double u = m.x, v = m.y, w = u * u + v * v;
      const double* tb = Ltab + 48 * (size_t)i;
#pragma unroll
      for (int e = 0; e < 6; ++e)
        V[e] += tb[e] + u * tb[6 + e] + v * tb[12 + e] + w * tb[18 + e];
#pragma unroll
      for (int c = 0; c < 3; ++c)
        h[c] += tb[24 + c] + u * tb[27 + c] + v * tb[30 + c] + w * tb[33 + c];
    }
    // b_l = V X + h (symmetric V: 00 01 02 11 12 22)
    const double bl[3] = {V[0] * x[0] + V[1] * x[1] + V[2] * x[2] + h[0],
                          V[1] * x[0] + V[3] * x[1] + V[4] * x[2] + h[1],
                          V[2] * x[0] + V[4] * x[1] + V[5] * x[2] + h[2]};
    // factor F = L^-1 of V + lambda_l lambda I (positive definite for a
    // positive damping; pivots floored against rounding)
    const double damp = lambda_l * st->lam;
    const double v0 = V[0] + damp, v3 = V[3] + damp, v5 = V[5] + damp;
    const double f00 = rsqrt(fmax(v0, 1e-300));
    const double l10 = V[1] * f00, l20 = V[2] * f00;
    const double f11 = rsqrt(fmax(v3 - l10 * l10, 1e-300));
    const double l21 = (V[4] - l20 * l10) * f11;
    const double f22 = rsqrt(fmax(v5 - l20 * l20 - l21 * l21, 1e-300));
    const double f10 = -l10 * f00 * f11;
    const double f20 = -(l20 * f00 + l21 * f10) * f22;
    const double f21 = -l21 * f11 * f22;
    F[0] = f00; F[1] = f10; F[2] = f11; F[3] = f20; F[4] = f21; F[5] = f22;
    // s = F^T F b_l
    const double z0 = f00 * bl[0];
    const double z1 = f10 * bl[0] + f11 * bl[1];
    const double z2 = f20 * bl[0] + f21 * bl[1] + f22 * bl[2];
    sb[0] = f00 * z0 + f10 * z1 + f20 * z2;
    sb[1] = f11 * z1 + f21 * z2;
    sb[2] = f22 * z2;
  }
#pragma unroll
  for (int e = 0; e < 6; ++e) Fo[e] = F[e];
  (t ? A1 : A0)[s] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)F[0]);
  (t ? B1 : B0)[s] = make_float4((float)F[1], (float)F[2], (float)F[3], (float)F[4]);
  (t ? C1 : C0)[s] = (float)F[5];
  sbl64[3 * (size_t)s] = sb[0];
  sbl64[3 * (size_t)s + 1] = sb[1];
  sbl64[3 * (size_t)s + 2] = sb[2];
  sbl32[s] = make_float4((float)sb[0], (float)sb[1], (float)sb[2], 0.f);
}

// ||r_k||^2 of Eq. pose for y = P_i (X, 1) and measurement (u, v).
__device__ __forceinline__ double pose_sq(double eta, double u, double v, const double y[3]) {
  const double a0 = y[0] - u * y[2], a1 = y[1] - v * y[2];
  const double b0 = y[0] - u, b1 = y[1] - v;
  return (1.0 - eta) * (a0 * a0 + a1 * a1) + eta * (b0 * b0 + b1 * b1);
}

// y = Q (x, 1) for a 3x4 row-major block Q
__device__ __forceinline__ void mat34(const double Q[12], const double x[3], double y[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    y[r] = fma(Q[4 * r], x[0], fma(Q[4 * r + 1], x[1], fma(Q[4 * r + 2], x[2], Q[4 * r + 3])));
}

template <typename TD>
__global__ void __launch_bounds__(BLOCK)
k_poba_trial(DeviceState* __restrict__ st, double eta, const uint32_t* __restrict__ slot_len,
             const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
             const double2* __restrict__ sell_m, const double* __restrict__ P0,
             const double* __restrict__ P1, const TD* __restrict__ D, double* __restrict__ X0,
             double* __restrict__ X1, const double* __restrict__ F0,
             const double* __restrict__ F1, const double* __restrict__ sbl64,
             double* __restrict__ cost_part, double* __restrict__ pred_part) {
  if (st->converged) return;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int t = st->cur, nt = 1 - t;
  if (s == 0) st->x_df[nt] = 0;
  const double a = 1.0 - eta;
  const double* Pc = t ? P1 : P0;   // current cameras
  const double* Pn = t ? P0 : P1;   // trial cameras (written by the update)
  const double* Xc = (t ? X1 : X0) + 3 * (size_t)s;
  const double* F = (t ? F1 : F0) + 6 * (size_t)s;
  const uint32_t len = slot_len[s];
  double Xn[3] = {0.0, 0.0, 0.0};
  double cost = 0.0, lin = 0.0;
  if (len > 0) {
    const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
    const double x[3] = {Xc[0], Xc[1], Xc[2]};
    // pass 1: W^T dP = sum_k Pbar_i^T C_k (dP_i x~)
    double tt[3] = {0.0, 0.0, 0.0};
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const double2 m = sell_m[pos];
      double Di[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) Di[e] = (double)D[12 * (size_t)i + e];
      double y[3], c[3];
      mat34(Di, x, y);
      apply_c(a, m.x, m.y, y, c);
      const double* Q = Pc + 12 * (size_t)i;
#pragma unroll
      for (int q = 0; q < 3; ++q) tt[q] += Q[q] * c[0] + Q[4 + q] * c[1] + Q[8 + q] * c[2];
    }
    // dX = -(s + F^T F t), X' = X + dX
    const double z0 = F[0] * tt[0];
    const double z1 = F[1] * tt[0] + F[2] * tt[1];
    const double z2 = F[3] * tt[0] + F[4] * tt[1] + F[5] * tt[2];
    const double* sb = sbl64 + 3 * (size_t)s;
    Xn[0] = x[0] - (sb[0] + F[0] * z0 + F[1] * z1 + F[3] * z2);
    Xn[1] = x[1] - (sb[1] + F[2] * z1 + F[4] * z2);
    Xn[2] = x[2] - (sb[2] + F[5] * z2);
    // pass 2: trial cost at (P', X') and the linear model
    // r + J_p dP + J_l dX = B (P (X', 1) + dP (X, 1)) - d
    for (uint32_t k = 0; k < len; ++k) {
      const uint32_t pos = base + k * SLICE;
      const int i = sell_cam[pos];
      const double2 m = sell_m[pos];
      double Q[12], Di[12];
#pragma unroll
      for (int e = 0; e < 12; ++e) {
        Q[e] = Pn[12 * (size_t)i + e];
        Di[e] = (double)D[12 * (size_t)i + e];
      }
      double yt[3];
      mat34(Q, Xn, yt);
      cost += pose_sq(eta, m.x, m.y, yt);
#pragma unroll
      for (int e = 0; e < 12; ++e) Q[e] = Pc[12 * (size_t)i + e];
      double yl[3], yd[3];
      mat34(Q, Xn, yl);
      mat34(Di, x, yd);
      yl[0] += yd[0];
      yl[1] += yd[1];
      yl[2] += yd[2];
      lin += pose_sq(eta, m.x, m.y, yl);
    }
  }
  double* Xo = (nt ? X1 : X0) + 3 * (size_t)s;
  Xo[0] = Xn[0];
  Xo[1] = Xn[1];
  Xo[2] = Xn[2];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    cost += __shfl_xor_sync(0xffffffffu, cost, o);
    lin += __shfl_xor_sync(0xffffffffu, lin, o);
  }
  if ((threadIdx.x & 31) == 0) {
    cost_part[s / 32] = cost;
    pred_part[s / 32] = lin;
  }
}

// pred = F - sum of the model partials, one block, fixed order.
__global__ void __launch_bounds__(256)
k_poba_pred_finish(DeviceState* __restrict__ st, const double* __restrict__ part, int n, int m) {
  if (st->converged) return;
  __shared__ double red[256];
  double c = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) c += part[i];
  red[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->pred = st->F - red[0];
    if (!st->stop_series) st->terms_used = m;   // the series ran all m terms
  }
}

}  // namespace

povar_status launch_model_pred_finish(Problem* p, int m) {
  k_poba_pred_finish<<<1, 256, 0, p->stream>>>(p->state, p->pred_part, p->np_pad / 32, m);
  ++p->launches;
  return check_launch(p, "model_pred_finish");
}

povar_status ensure_poba(Problem* p) {
  if (p->sbl64) return POVAR_OK;
  povar_status s;
  if ((s = dev_alloc(p, &p->sbl64, (size_t)p->np_pad * 3, "sbl64")) ||
      (s = dev_alloc(p, &p->sbl32, (size_t)p->np_pad, "sbl32")))
    return s;
  POVAR_CUDA(cudaMemsetAsync(p->sbl64, 0, (size_t)p->np_pad * 3 * sizeof(double), p->stream));
  POVAR_CUDA(cudaMemsetAsync(p->sbl32, 0, (size_t)p->np_pad * sizeof(float4), p->stream));
  return POVAR_OK;
}

povar_status launch_poba_prep(Problem* p, double eta, double lambda_l) {
  povar_status s;
  if ((s = launch_ltab(p, 0, eta)) != POVAR_OK) return s;
  k_poba_prep<<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
      p->state, lambda_l, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->Ltab,
      p->X64[0], p->X64[1], p->F64[0], p->F64[1], p->pdA[0], p->pdA[1], p->pdB[0], p->pdB[1],
      p->pdC[0], p->pdC[1], p->sbl64, p->sbl32);
  ++p->launches;
  return check_launch(p, "poba_prep");
}

povar_status launch_poba_trial(Problem* p, int precision, double eta, int m) {
  if (precision == POVAR_FP64)
    k_poba_trial<double><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
        p->D64, p->X64[0], p->X64[1], p->F64[0], p->F64[1], p->sbl64, p->cost_part,
        p->pred_part);
  else
    k_poba_trial<float><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
        p->D32, p->X64[0], p->X64[1], p->F64[0], p->F64[1], p->sbl64, p->cost_part,
        p->pred_part);
  ++p->launches;
  povar_status s;
  if ((s = check_launch(p, "poba_trial")) != POVAR_OK) return s;
  if ((s = launch_cost_finish(p, 1)) != POVAR_OK) return s;
  k_poba_pred_finish<<<1, 256, 0, p->stream>>>(p->state, p->pred_part, p->np_pad / 32, m);
  ++p->launches;
  return check_launch(p, "poba_pred_finish");
}

}  // namespace povar
