// Metric upgrade of a projective reconstruction (the third stage of the
// stratified problem; supplementary section "Metric Upgrade" of the paper).
// With B_i = K_i^-1 P_i H_0 (H_0 puts the calibrated camera 0 at [I | 0])
// and H~(c) = [[I], [c^T]], the upgrade minimizes
//   sum_i || alpha_i M_i(c) - I ||_F^2,   M_i = N_i N_i^T,  N_i = B_i H~(c)
//        = B_i[:, 0:3] + b_i c^T  (b_i the last column of B_i),
// by Variable Projection: alpha_i = tr(M_i) / ||M_i||_F^2 in closed form,
// Levenberg-Marquardt on c with the derivative of the reduced residual
//   d(alpha M) / dc_k = alpha dM_k + (d alpha / dc_k) M,
//   dM_k = b n_k^T + n_k b^T  (n_k the k-th column of N),
// from the linear estimate of the dual absolute quadric Q = H~ H~^T (five
// linear equations per camera in the ten entries of Q; the eigenvector of
// the smallest eigenvalue of their normal matrix, by inverse iteration).
// The problem has three unknowns and one 3x3 block per camera: one block of
// 256 threads runs the whole iteration (cameras strided over the threads,
// fixed-order shared-memory sums, thread 0 solves the 3x3 systems), so a
// call is one launch for the set-up and one for the iteration.
#include <algorithm>
#include <cmath>
#include <vector>

#include "povar_internal.cuh"

namespace povar {
namespace {

constexpr int MU_THREADS = 256;
constexpr int MU_SUMS = 55;   // normal matrix of the linear start (10 x 10 upper)

// 3x3 inverse by the adjugate; false if singular
__device__ bool inv3(const double A[9], double R[9]) {
  const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8],
               c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  if (!(fabs(det) > 0.0)) return false;
  const double id = 1.0 / det;
  R[0] = c00 * id;
  R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  R[3] = c01 * id;
  R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  R[6] = c02 * id;
  R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
  return true;
}

// C = K^-1 P (3x4) for camera i; K null means identity
__device__ bool calibrated(const double* __restrict__ K, const double* __restrict__ P, int i,
                           double C[12]) {
  const double* Pi = P + 12 * (size_t)i;
  if (!K) {
    for (int e = 0; e < 12; ++e) C[e] = Pi[e];
    return true;
  }
  double Ki[9];
  if (!inv3(K + 9 * (size_t)i, Ki)) return false;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 4; ++q)
      C[4 * r + q] = Ki[3 * r] * Pi[q] + Ki[3 * r + 1] * Pi[4 + q] + Ki[3 * r + 2] * Pi[8 + q];
  return true;
}

// 4x4 inverse by Gauss-Jordan elimination with partial pivoting
__device__ bool inv4(double A[16], double R[16]) {
  for (int e = 0; e < 16; ++e) R[e] = (e % 5 == 0) ? 1.0 : 0.0;
  for (int k = 0; k < 4; ++k) {
    int piv = k;
    for (int r = k + 1; r < 4; ++r)
      if (fabs(A[4 * r + k]) > fabs(A[4 * piv + k])) piv = r;
    if (!(fabs(A[4 * piv + k]) > 0.0)) return false;
    if (piv != k)
      for (int q = 0; q < 4; ++q) {
        double t = A[4 * k + q];
        A[4 * k + q] = A[4 * piv + q];
        A[4 * piv + q] = t;
        t = R[4 * k + q];
        R[4 * k + q] = R[4 * piv + q];
        R[4 * piv + q] = t;
      }
    const double d = 1.0 / A[4 * k + k];
    for (int q = 0; q < 4; ++q) {
      A[4 * k + q] *= d;
      R[4 * k + q] *= d;
    }
    for (int r = 0; r < 4; ++r) {
      if (r == k) continue;
      const double f = A[4 * r + k];
      for (int q = 0; q < 4; ++q) {
        A[4 * r + q] -= f * A[4 * k + q];
        R[4 * r + q] -= f * R[4 * k + q];
      }
    }
  }
  return true;
}

// index of the free entry (a, b), a <= b, of a symmetric 4x4 matrix
__device__ __forceinline__ int qpair(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? hi : (lo == 1 ? 3 + hi : (lo == 2 ? 5 + hi : 9));
}

// Fixed-order sum of n values per thread over the block: xor-butterfly
// within each warp, then thread 0 adds the warps' sums in warp order.
// red holds n x (MU_THREADS / 32) warp sums.
__device__ void block_sum(double* red, const double* v, int n, double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int NW = MU_THREADS / 32;
  for (int e = 0; e < n; ++e) {
    double x = v[e];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[e * NW + w] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int e = 0; e < n; ++e) {
      double x = 0.0;
      for (int q = 0; q < NW; ++q) x += red[e * NW + q];
      out[e] = x;
    }
  __syncthreads();
}

struct MuOut {
  double H[16];
  double c[3];
  double cost;
  int iterations;
  int status;   // POVAR_OK, POVAR_EINVAL (singular K or frame), POVAR_ENUMERIC
};

// One thread: H_0 from the calibrated camera 0 (its centre completes it to
// an invertible 4x4 matrix).
__global__ void k_mu_frame(const double* __restrict__ K, const double* __restrict__ P,
                           double* __restrict__ H0, MuOut* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double C[12];
  out->status = POVAR_OK;
  if (!calibrated(K, P, 0, C)) {
    out->status = POVAR_EINVAL;
    return;
  }
  // centre: signed 3x3 minors of C (C c = 0)
  double cen[4];
  for (int j = 0; j < 4; ++j) {
    int col[3], n = 0;
    for (int q = 0; q < 4; ++q)
      if (q != j) col[n++] = q;
    const double m = C[col[0]] * (C[4 + col[1]] * C[8 + col[2]] - C[4 + col[2]] * C[8 + col[1]]) -
                     C[col[1]] * (C[4 + col[0]] * C[8 + col[2]] - C[4 + col[2]] * C[8 + col[0]]) +
                     C[col[2]] * (C[4 + col[0]] * C[8 + col[1]] - C[4 + col[1]] * C[8 + col[0]]);
    cen[j] = (j & 1) ? -m : m;
  }
  double A[16];
  for (int e = 0; e < 12; ++e) A[e] = C[e];
  for (int q = 0; q < 4; ++q) A[12 + q] = cen[q];
  if (!inv4(A, H0)) out->status = POVAR_EINVAL;
}

// Per camera: B_i = K_i^-1 P_i H_0 (3x4)
__global__ void k_mu_blocks(int nc, const double* __restrict__ K, const double* __restrict__ P,
                            const double* __restrict__ H0, double* __restrict__ B,
                            MuOut* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double C[12];
  if (!calibrated(K, P, i, C)) {
    out->status = POVAR_EINVAL;
    return;
  }
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 4; ++q)
      B[12 * (size_t)i + 4 * r + q] = C[4 * r] * H0[q] + C[4 * r + 1] * H0[4 + q] +
                                      C[4 * r + 2] * H0[8 + q] + C[4 * r + 3] * H0[12 + q];
}

// residual, Jacobian (9 x 3) and its products for one camera at c;
// acc: J^T J (6: 00 01 02 11 12 22), J^T r (3), r^T r (1)
__device__ void mu_camera(const double* __restrict__ Bi, const double c[3], bool jac,
                          double acc[10], double* alpha_out) {
  double N[9], b[3];
  for (int r = 0; r < 3; ++r) {
    b[r] = Bi[4 * r + 3];
    for (int k = 0; k < 3; ++k) N[3 * r + k] = Bi[4 * r + k] + b[r] * c[k];
  }
  double M[9];
  for (int a = 0; a < 3; ++a)
    for (int q = 0; q < 3; ++q)
      M[3 * a + q] = N[3 * a] * N[3 * q] + N[3 * a + 1] * N[3 * q + 1] + N[3 * a + 2] * N[3 * q + 2];
  const double tr = M[0] + M[4] + M[8];
  double mm = 0.0;
  for (int e = 0; e < 9; ++e) mm += M[e] * M[e];
  const double al = tr / mm;
  if (alpha_out) *alpha_out = al;
  double r[9];
  for (int e = 0; e < 9; ++e) r[e] = al * M[e] - ((e % 4 == 0) ? 1.0 : 0.0);
  double rr = 0.0;
  for (int e = 0; e < 9; ++e) rr += r[e] * r[e];
  acc[9] += rr;
  if (!jac) return;
  double J[9][3];
  double Mb[3];
  for (int a = 0; a < 3; ++a) Mb[a] = M[3 * a] * b[0] + M[3 * a + 1] * b[1] + M[3 * a + 2] * b[2];
  for (int k = 0; k < 3; ++k) {
    const double n[3] = {N[k], N[3 + k], N[6 + k]};
    double dM[9];
    for (int a = 0; a < 3; ++a)
      for (int q = 0; q < 3; ++q) dM[3 * a + q] = b[a] * n[q] + n[a] * b[q];
    const double dtr = 2.0 * (b[0] * n[0] + b[1] * n[1] + b[2] * n[2]);
    const double dmm = 4.0 * (Mb[0] * n[0] + Mb[1] * n[1] + Mb[2] * n[2]);
    const double da = (dtr * mm - tr * dmm) / (mm * mm);
    for (int e = 0; e < 9; ++e) J[e][k] = al * dM[e] + da * M[e];
  }
  for (int e = 0; e < 9; ++e) {
    acc[0] += J[e][0] * J[e][0];
    acc[1] += J[e][0] * J[e][1];
    acc[2] += J[e][0] * J[e][2];
    acc[3] += J[e][1] * J[e][1];
    acc[4] += J[e][1] * J[e][2];
    acc[5] += J[e][2] * J[e][2];
    acc[6] += J[e][0] * r[e];
    acc[7] += J[e][1] * r[e];
    acc[8] += J[e][2] * r[e];
  }
}

// Eigenvector of the smallest eigenvalue of the symmetric positive
// semi-definite 10x10 S by inverse iteration: Cholesky factor of
// S + delta I (delta = 1e-10 of the mean diagonal entry, above the rounding
// of a zero eigenvalue), then 24 solves from a fixed start vector, each
// followed by normalization.
__device__ void smallest_eigvec10(double S[10][10], double v[10]) {
  double tr = 0.0;
  for (int a = 0; a < 10; ++a) tr += S[a][a];
  const double delta = 1e-10 * tr / 10.0 + 1e-300;
  double L[10][10];
  for (int a = 0; a < 10; ++a)
    for (int q = 0; q <= a; ++q) {
      double x = S[a][q] + (a == q ? delta : 0.0);
      for (int k = 0; k < q; ++k) x -= L[a][k] * L[q][k];
      L[a][q] = a == q ? sqrt(fmax(x, 1e-300)) : x / L[q][q];
    }
  for (int a = 0; a < 10; ++a) v[a] = 1.0 + 0.1 * a;
  for (int it = 0; it < 24; ++it) {
    double y[10];
    for (int a = 0; a < 10; ++a) {
      double x = v[a];
      for (int k = 0; k < a; ++k) x -= L[a][k] * y[k];
      y[a] = x / L[a][a];
    }
    for (int a = 9; a >= 0; --a) {
      double x = y[a];
      for (int k = a + 1; k < 10; ++k) x -= L[k][a] * v[k];
      v[a] = x / L[a][a];
    }
    double nn = 0.0;
    for (int a = 0; a < 10; ++a) nn += v[a] * v[a];
    const double f = 1.0 / sqrt(nn);
    for (int a = 0; a < 10; ++a) v[a] *= f;
  }
}

// 3x3 SPD solve (A + lam I) d = -g by Cholesky; false if not positive
__device__ bool solve3(const double A[6], double lam, const double g[3], double d[3]) {
  const double a00 = A[0] + lam, a01 = A[1], a02 = A[2], a11 = A[3] + lam, a12 = A[4],
               a22 = A[5] + lam;
  if (!(a00 > 0.0)) return false;
  const double l00 = sqrt(a00), l10 = a01 / l00, l20 = a02 / l00;
  const double t11 = a11 - l10 * l10;
  if (!(t11 > 0.0)) return false;
  const double l11 = sqrt(t11), l21 = (a12 - l20 * l10) / l11;
  const double t22 = a22 - l20 * l20 - l21 * l21;
  if (!(t22 > 0.0)) return false;
  const double l22 = sqrt(t22);
  const double y0 = -g[0] / l00, y1 = (-g[1] - l10 * y0) / l11,
               y2 = (-g[2] - l20 * y0 - l21 * y1) / l22;
  d[2] = y2 / l22;
  d[1] = (y1 - l21 * d[2]) / l11;
  d[0] = (y0 - l10 * d[1] - l20 * d[2]) / l00;
  return true;
}

// The whole upgrade in one block: linear start, then Levenberg-Marquardt
// (Madsen-Nielsen damping, accept iff the cost decreases, stop on a relative
// decrease below ftol or after max_iters), then the scales and H.
__global__ void __launch_bounds__(MU_THREADS)
k_mu_solve(int nc, const double* __restrict__ B, const double* __restrict__ H0,
           double lambda0, int max_iters, double ftol, double* __restrict__ alpha,
           MuOut* __restrict__ out) {
  __shared__ double red[MU_SUMS * (MU_THREADS / 32)];
  __shared__ double tot[MU_SUMS];
  __shared__ double c[3], d[3];
  __shared__ int go;
  const int t = threadIdx.x;
  if (out->status != POVAR_OK) return;
  // linear start: normal matrix of the five equations per camera
  {
    double acc[MU_SUMS];
    for (int e = 0; e < MU_SUMS; ++e) acc[e] = 0.0;
    for (int i = t; i < nc; i += MU_THREADS) {
      const double* Bi = B + 12 * (size_t)i;
      double row[5][10];
      const int rs[5][2] = {{0, 1}, {0, 2}, {1, 2}, {0, 0}, {0, 0}};
      for (int eq = 0; eq < 5; ++eq) {
        for (int a = 0; a < 4; ++a)
          for (int q = a; q < 4; ++q) {
            auto coef = [&](int r, int s) {
              double v = Bi[4 * r + a] * Bi[4 * s + q];
              if (a != q) v += Bi[4 * r + q] * Bi[4 * s + a];
              return v;
            };
            double v = coef(rs[eq][0], rs[eq][1]);
            if (eq == 3) v -= coef(1, 1);
            if (eq == 4) v -= coef(2, 2);
            row[eq][qpair(a, q)] = v;
          }
      }
      int e = 0;
      for (int a = 0; a < 10; ++a)
        for (int q = a; q < 10; ++q, ++e)
          for (int eq = 0; eq < 5; ++eq) acc[e] += row[eq][a] * row[eq][q];
    }
    block_sum(red, acc, MU_SUMS, tot);
  }
  if (t == 0) {
    double S[10][10];
    int e = 0;
    for (int a = 0; a < 10; ++a)
      for (int q = a; q < 10; ++q, ++e) S[a][q] = S[q][a] = tot[e];
    double v[10];
    smallest_eigvec10(S, v);
    const double trq = v[qpair(0, 0)] + v[qpair(1, 1)] + v[qpair(2, 2)];
    const double sc = trq != 0.0 ? 3.0 / trq : 0.0;
    for (int k = 0; k < 3; ++k) c[k] = v[qpair(k, 3)] * sc;
  }
  __syncthreads();
  // Levenberg-Marquardt on c
  double F = 0.0, lam = lambda0, nu = 2.0;
  {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = t; i < nc; i += MU_THREADS) mu_camera(B + 12 * (size_t)i, c, false, acc, nullptr);
    block_sum(red, acc, 10, tot);
    F = tot[9];
  }
  int it = 0;
  for (it = 1; it <= max_iters; ++it) {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = t; i < nc; i += MU_THREADS) mu_camera(B + 12 * (size_t)i, c, true, acc, nullptr);
    block_sum(red, acc, 10, tot);
    double JJ[6], g[3];
    for (int e = 0; e < 6; ++e) JJ[e] = tot[e];
    for (int e = 0; e < 3; ++e) g[e] = tot[6 + e];
    if (t == 0) {
      double dd[3];
      const bool ok = solve3(JJ, lam, g, dd);
      for (int k = 0; k < 3; ++k) d[k] = ok ? dd[k] : 0.0;
      go = ok ? 1 : 0;
    }
    __syncthreads();
    double ct[3] = {c[0] + d[0], c[1] + d[1], c[2] + d[2]};
    double acc2[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = t; i < nc; i += MU_THREADS) mu_camera(B + 12 * (size_t)i, ct, false, acc2, nullptr);
    block_sum(red, acc2, 10, tot);
    const double Fn = tot[9];
    // model decrease ||r||^2 - ||r + J d||^2
    const double pred = -2.0 * (g[0] * d[0] + g[1] * d[1] + g[2] * d[2]) -
                        (d[0] * (JJ[0] * d[0] + JJ[1] * d[1] + JJ[2] * d[2]) +
                         d[1] * (JJ[1] * d[0] + JJ[3] * d[1] + JJ[4] * d[2]) +
                         d[2] * (JJ[2] * d[0] + JJ[4] * d[1] + JJ[5] * d[2]));
    const double rho = pred > 0.0 ? (F - Fn) / pred : 0.0;
    bool stop = false;
    if (go && Fn < F) {
      const double decrease = F - Fn;
      F = Fn;
      const double x = 2.0 * rho - 1.0;
      lam = fmax(lam * fmax(1.0 / 3.0, 1.0 - x * x * x), LAMBDA_MIN);
      nu = 2.0;
      __syncthreads();
      if (t == 0)
        for (int k = 0; k < 3; ++k) c[k] = ct[k];
      stop = decrease < ftol * (F + decrease);
    } else {
      lam *= nu;
      nu *= 2.0;
      stop = !(lam < LAMBDA_MAX);
    }
    __syncthreads();
    if (stop) break;
  }
  if (it > max_iters) it = max_iters;
  // scales and H = H_0 [[I, 0], [c^T, 1]]
  {
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = t; i < nc; i += MU_THREADS) {
      double a;
      mu_camera(B + 12 * (size_t)i, c, false, acc, &a);
      if (alpha) alpha[i] = a;
    }
  }
  if (t == 0) {
    for (int r = 0; r < 4; ++r) {
      for (int q = 0; q < 3; ++q) out->H[4 * r + q] = H0[4 * r + q] + H0[4 * r + 3] * c[q];
      out->H[4 * r + 3] = H0[4 * r + 3];
    }
    for (int k = 0; k < 3; ++k) out->c[k] = c[k];
    out->cost = F;
    out->iterations = it;
    if (!isfinite(F)) out->status = POVAR_ENUMERIC;
  }
}

}  // namespace

povar_status launch_metric_upgrade(Problem* p, const double* d_K, double lambda0, int max_iters,
                                   double ftol, double* H_out, double* alpha_out,
                                   double* cost_out, int* iters_out) {
  povar_status s;
  if (!p->mu_B) {
    if ((s = dev_alloc(p, &p->mu_B, (size_t)p->nc * 12 + 16, "mu_B")) ||
        (s = dev_alloc(p, &p->mu_alpha, (size_t)p->nc, "mu_alpha")) ||
        (s = dev_alloc_bytes(p, &p->mu_out, sizeof(MuOut), "mu_out")))
      return s;
  }
  double* H0 = p->mu_B + (size_t)p->nc * 12;
  MuOut* out = static_cast<MuOut*>(p->mu_out);
  // the current cameras: the buffer the device state names
  POVAR_CUDA(cudaMemcpyAsync(p->h_state, p->state, sizeof(DeviceState), cudaMemcpyDeviceToHost,
                             p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  const double* P = p->P64[p->h_state->cur];
  k_mu_frame<<<1, 32, 0, p->stream>>>(d_K, P, H0, out);
  k_mu_blocks<<<grid_for(p->nc, 128), 128, 0, p->stream>>>(p->nc, d_K, P, H0, p->mu_B, out);
  k_mu_solve<<<1, MU_THREADS, 0, p->stream>>>(p->nc, p->mu_B, H0, lambda0, max_iters, ftol,
                                              p->mu_alpha, out);
  p->launches += 3;
  if ((s = check_launch(p, "metric_upgrade")) != POVAR_OK) return s;
  MuOut h;
  POVAR_CUDA(cudaMemcpyAsync(&h, out, sizeof(MuOut), cudaMemcpyDeviceToHost, p->stream));
  if (alpha_out)
    POVAR_CUDA(cudaMemcpyAsync(alpha_out, p->mu_alpha, (size_t)p->nc * sizeof(double),
                               cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  if (h.status != POVAR_OK)
    return fail(p, (povar_status)h.status,
                h.status == POVAR_EINVAL ? "singular intrinsics or reference camera"
                                         : "non-finite metric-upgrade cost");
  for (int e = 0; e < 16; ++e) H_out[e] = h.H[e];
  if (cost_out) *cost_out = h.cost;
  if (iters_out) *iters_out = h.iterations;
  return POVAR_OK;
}

}  // namespace povar
