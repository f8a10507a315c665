// a4: linearization of the pOSE residual at (P, X*(P)) per camera (Sec. 4.1)
// a5: damped tangent-space camera blocks and their inverses (Sec. 4.3)
// a6: right-hand side and the first series term x_0 = U~^-1 g (Sec. 4.2)
//
// With y = P_i x~_j, the residual of Eq. pose is r = B(m) y - d(m), so
// J_p = B (x) x~^T and U_i = sum_k C_k (x) x~ x~^T with C = B^T B =
//   [[1, 0, -a u], [0, 1, -a v], [-a u, -a v, a (u^2 + v^2)]],  a = 1 - eta.
// Hence U_i is fully determined by four symmetric 4x4 moment sums
//   S0 = sum x~x~^T, Su = sum u x~x~^T, Sv = sum v x~x~^T, Sw = sum w x~x~^T
// (w = u^2 + v^2): blocks (0,0) = (1,1) = S0, (0,1) = 0, (0,2) = -a Su,
// (1,2) = -a Sv, (2,2) = a Sw. b_p,i = sum_k (B^T r_k) (x) x~_j.
// One warp reduces one camera-major chunk of observations into these 52
// numbers with shuffles (no atomics); the per-camera kernel adds the chunk
// partials in chunk order, so the result is deterministic.
//
// Centring (FP32 accumulation only): landmarks far from the origin make U_i
// a cancellation-prone sum with a huge condition number, and FP32 rounding
// of its entries then spoils the damped inverse. Each chunk accumulates the
// moments of x~' = (X - c, 1) about its own centre c (the chunk's mean
// landmark) and the gradient sums g (x) x~' (the residuals themselves use
// X); the per-camera kernel maps every chunk's sums back in FP64 exactly
// (x~ = x~' + (c, 0): S_ab = S'_ab + c_a S'_3b + c_b S'_a3 + c_a c_b S'_33,
// b_p[r][q] = b'_p[r][q] + c_q b'_p[r][3], with c_3 = 0) before adding them.
// The FP32 rounding is then relative to a well-conditioned matrix.
//
// Tangent space (POVAR_SPHERE): with p^ = P_i / ||P_i|| and Pi = I - p^p^T,
//   A_i = Pi U_i Pi + lambda Pi + p^ p^T   is SPD and, for any tangent v,
//   A_i^-1 v = Q (Q^T U_i Q + lambda I)^-1 Q^T v  for every orthonormal basis
// Q of the tangent space, so G_i = A_i^-1 - p^p^T = Q U~_i^-1 Q^T applies the
// inverse damped tangent block of Sec. 4.3 in ambient 12-d coordinates.
// POVAR_EUCLID: G_i = (U_i + lambda I)^-1. The 12x12 Cholesky and inverse are
// FP64; G is also stored in FP32 for the mixed-precision series.
#include "povar_internal.cuh"

namespace povar {
namespace {

template <typename T> struct M2;
template <> struct M2<float> { using type = float2; };
template <> struct M2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ void load_x(const float4* __restrict__ pdA,
                                       const double* __restrict__ X64, uint32_t slot,
                                       T& x0, T& x1, T& x2);
template <>
__device__ __forceinline__ void load_x<float>(const float4* __restrict__ pdA,
                                              const double* __restrict__, uint32_t slot,
                                              float& x0, float& x1, float& x2) {
  const float4 a = __ldg(pdA + slot);
  x0 = a.x; x1 = a.y; x2 = a.z;
}
template <>
__device__ __forceinline__ void load_x<double>(const float4* __restrict__,
                                               const double* __restrict__ X64, uint32_t slot,
                                               double& x0, double& x1, double& x2) {
  const double* x = X64 + 3 * (size_t)slot;
  x0 = __ldg(x); x1 = __ldg(x + 1); x2 = __ldg(x + 2);
}

// Three blocks per SM in FP32 (at most 85 registers; the centring pass
// would otherwise raise the count from 80 to about 120).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
k_linearize(const DeviceState* __restrict__ st, T s1, T s2, int nchunks,
            const int32_t* __restrict__ chunk_cam, const uint32_t* __restrict__ chunk_beg,
            const uint32_t* __restrict__ cm_slot, const typename M2<T>::type* __restrict__ cm_m,
            const T* __restrict__ P0, const T* __restrict__ P1,
            const float4* __restrict__ pdA0, const float4* __restrict__ pdA1,
            const double* __restrict__ X0, const double* __restrict__ X1,
            const float4* __restrict__ sbl32, const double* __restrict__ sbl64, int force,
            T* __restrict__ part) {
  // PoBA (sbl given, linearized every step): the residual is evaluated at
  // the landmark shifted by s_j = V_lambda^-1 b_l, which turns b_p into the
  // reduced right-hand side b_p - W V_lambda^-1 b_l; U and the outer
  // products keep X
  if (st->converged || (!force && !st->need_lin)) return;
  constexpr bool CENTER = sizeof(T) == 4;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= nchunks) return;
  const int cur = st->cur;
  const T* Pd = (cur ? P1 : P0) + 12 * (size_t)chunk_cam[c];
  const float4* pdA = cur ? pdA1 : pdA0;
  const double* X64 = cur ? X1 : X0;
  T P[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) P[e] = Pd[e];
  T acc[LIN_ACC];
#pragma unroll
  for (int e = 0; e < LIN_ACC; ++e) acc[e] = (T)0;
  const uint32_t b = chunk_beg[c], e_ = chunk_beg[c + 1];
  T ctr[3] = {0, 0, 0};
  if constexpr (CENTER) {
    // chunk centre: the mean landmark of the chunk (the pass brings the
    // chunk's landmark records into the cache for the main loop)
    for (uint32_t r = b + lane; r < e_; r += 32) {
      const float4 xa = __ldg(pdA + cm_slot[r]);
      ctr[0] += xa.x;
      ctr[1] += xa.y;
      ctr[2] += xa.z;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ctr[q] += __shfl_xor_sync(0xffffffffu, ctr[q], o);
      ctr[q] /= (T)(e_ - b);
    }
  }
  for (uint32_t r = b + lane; r < e_; r += 32) {
    const uint32_t slot = cm_slot[r];
    const auto m = cm_m[r];
    const T u = m.x, v = m.y, w = u * u + v * v;
    T x0, x1, x2;
    load_x<T>(pdA, X64, slot, x0, x1, x2);
    T xr0 = x0, xr1 = x1, xr2 = x2;
    if (sbl32) {
      if constexpr (sizeof(T) == 4) {
        const float4 sv = __ldg(sbl32 + slot);
        xr0 -= sv.x;
        xr1 -= sv.y;
        xr2 -= sv.z;
      } else {
        xr0 -= sbl64[3 * (size_t)slot];
        xr1 -= sbl64[3 * (size_t)slot + 1];
        xr2 -= sbl64[3 * (size_t)slot + 2];
      }
    }
    const T y0 = P[0] * xr0 + P[1] * xr1 + P[2] * xr2 + P[3];
    const T y1 = P[4] * xr0 + P[5] * xr1 + P[6] * xr2 + P[7];
    const T y2 = P[8] * xr0 + P[9] * xr1 + P[10] * xr2 + P[11];
    const T r0 = s1 * (y0 - u * y2), r1 = s1 * (y1 - v * y2);
    const T r2 = s2 * (y0 - u), r3 = s2 * (y1 - v);
    const T g[3] = {s1 * r0 + s2 * r2, s1 * r1 + s2 * r3, -s1 * (u * r0 + v * r1)};
    // moments and gradient about the chunk centre (zero in FP64)
    x0 -= ctr[0];
    x1 -= ctr[1];
    x2 -= ctr[2];
    const T xt[4] = {x0, x1, x2, (T)1};
    const T t10[10] = {x0 * x0, x0 * x1, x0 * x2, x0, x1 * x1, x1 * x2, x1, x2 * x2, x2, (T)1};
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      acc[q] += t10[q];
      acc[10 + q] += u * t10[q];
      acc[20 + q] += v * t10[q];
      acc[30 + q] += w * t10[q];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int bb = 0; bb < 4; ++bb) acc[40 + 4 * a + bb] += g[a] * xt[bb];
  }
#pragma unroll
  for (int e = 0; e < LIN_ACC; ++e) {
    T v = acc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[e] = v;
  }
  T* out = part + (size_t)c * LIN_PART;
#pragma unroll
  for (int e = 0; e < LIN_ACC; ++e)
    if ((e & 31) == lane) out[e] = acc[e];
  if (lane < 3) out[LIN_ACC + lane] = lane == 0 ? ctr[0] : (lane == 1 ? ctr[1] : ctr[2]);
}

// index of the unique entry (b, d) of a symmetric 4x4 in the t10 order
__device__ __forceinline__ int t10_index(int b, int d) {
  const int lo = b < d ? b : d, hi = b < d ? d : b;
  // rows: (0,0..3) -> 0..3, (1,1..3) -> 4..6, (2,2..3) -> 7..8, (3,3) -> 9
  return lo == 0 ? hi : (lo == 1 ? 3 + hi : (lo == 2 ? 5 + hi : 9));
}

// Entry e of a chunk's sums in the global basis from its centred sums S'
// (t10 moments of the four weights, then b_p) and its centre c = S'[52..54]
// (see the centring note above; c_3 = 0).
__device__ __forceinline__ double uncentre(const double* Sp, int e) {
  const double* cc = Sp + LIN_ACC;
  if (e < 40) {
    const int blk = e / 10 * 10, t = e % 10;
    // (a, b) of t10 entry t: rows (0,0..3), (1,1..3), (2,2..3), (3,3)
    const int a = t < 4 ? 0 : t < 7 ? 1 : t < 9 ? 2 : 3;
    const int bb = t < 4 ? t : t < 7 ? t - 3 : t < 9 ? t - 5 : 3;
    const double ca = a < 3 ? cc[a] : 0.0, cb = bb < 3 ? cc[bb] : 0.0;
    return Sp[blk + t] + ca * Sp[blk + t10_index(3, bb)] + cb * Sp[blk + t10_index(a, 3)] +
           ca * cb * Sp[blk + 9];
  }
  const int q = (e - 40) & 3;
  return Sp[e] + (q < 3 ? cc[q] * Sp[e - q + 3] : 0.0);
}

template <typename T>
__global__ void __launch_bounds__(128)
k_camera_prepare(DeviceState* __restrict__ st, double eta, int manifold, int nc,
                 const int32_t* __restrict__ cam_nchunk, const int32_t* __restrict__ cam_chunk0,
                 const T* __restrict__ part, const double* __restrict__ P0,
                 const double* __restrict__ P1, double* __restrict__ U64,
                 double* __restrict__ bp64, double* __restrict__ G64, float* __restrict__ G32, T* __restrict__ Y,
                 T* __restrict__ D, double* __restrict__ camnorm, int force) {
  if (st->converged) return;
  __shared__ double smA[4][12][13];
  __shared__ double smL[4][12][13];
  __shared__ double smAcc[4][LIN_ACC];
  __shared__ double smChk[4][LIN_PART];
  __shared__ double smInv[4][12];  // reciprocals of the Cholesky diagonal
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x * 4 + wl;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->stop_series = 0;
    st->terms_used = 1;
    st->lam_used = st->lam;
  }
  if (i >= nc) return;
  const int cur = st->cur;
  const int need_lin = force || st->need_lin;
  const double lam = st->lam;
  const double a = 1.0 - eta;
  const double* Pc = (cur ? P1 : P0) + 12 * (size_t)i;
  double (*A)[13] = smA[wl];
  double (*L)[13] = smL[wl];
  double* inv = smInv[wl];
  const double Pl = lane < 12 ? Pc[lane] : 0.0;
  double bpl = 0.0;
  if (need_lin) {
    const int n = cam_nchunk[i], c0 = cam_chunk0[i];
    double s_lo = 0.0, s_hi = 0.0;   // entries lane and lane + 32
    for (int q = 0; q < n; ++q) {
      const T* pc = part + (size_t)(c0 + q) * LIN_PART;
      for (int e = lane; e < LIN_ACC + 3; e += 32) smChk[wl][e] = (double)pc[e];
      __syncwarp();
      s_lo += uncentre(smChk[wl], lane);
      if (lane + 32 < LIN_ACC) s_hi += uncentre(smChk[wl], lane + 32);
      __syncwarp();
    }
    smAcc[wl][lane] = s_lo;
    if (lane + 32 < LIN_ACC) smAcc[wl][lane + 32] = s_hi;
    __syncwarp();
    if (lane < 12) {
      const int ra = lane >> 2, rb = lane & 3;
      for (int q = 0; q < 12; ++q) {
        const int ca = q >> 2, cd = q & 3;
        const int t = t10_index(rb, cd);
        const int lo = ra < ca ? ra : ca, hi = ra < ca ? ca : ra;
        double val;
        if (lo == hi && lo < 2) val = smAcc[wl][t];
        else if (lo == 0 && hi == 1) val = 0.0;
        else if (lo == 0) val = -a * smAcc[wl][10 + t];
        else if (lo == 1) val = -a * smAcc[wl][20 + t];
        else val = a * smAcc[wl][30 + t];
        A[lane][q] = val;
        U64[(size_t)i * 144 + lane * 12 + q] = val;
      }
      bpl = smAcc[wl][40 + lane];
      bp64[(size_t)i * 12 + lane] = bpl;
    }
  } else if (lane < 12) {
    for (int q = 0; q < 12; ++q) A[lane][q] = U64[(size_t)i * 144 + lane * 12 + q];
    bpl = bp64[(size_t)i * 12 + lane];
  }
  __syncwarp();
  // The 78 entries (r, j), j <= r, of a 12 x 12 lower triangle ordered by
  // column j descending (rows ascending within a column): the entries right
  // of column k are the first (11 - k)(12 - k) / 2. Lane l owns entries l,
  // l + 32 and l + 64 (< 78), so the triangular loops below run on all 32
  // lanes; every entry keeps its own operations in their original order.
  int tr[3], tj[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int e = lane + 32 * u;
    int m = 0;
    while ((m + 1) * (m + 2) / 2 <= e) ++m;   // e in column 11 - m
    tj[u] = 11 - m;
    tr[u] = tj[u] + (e - m * (m + 1) / 2);
    if (e >= 78) tj[u] = -1;                  // no entry
  }
  // Damped block and its Cholesky factor. If rounding leaves the block not
  // numerically positive definite (an FP32-accumulated U with a huge
  // condition number), the damping of this camera is raised -- to at least
  // 1e-12 of its largest diagonal entry, then x100 per attempt, at most 8
  // attempts -- and the event is counted in the device state.
  double umax = lane < 12 ? A[lane][lane] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
  double lam_eff = lam;
  bool bad = true;
  int attempt = 0;
  double ph = 0.0;
  for (; attempt < 8 && bad; ++attempt) {
    if (attempt > 0) {
      lam_eff = fmax(lam_eff * 100.0, 1e-12 * umax);
      if (lane < 12)
        for (int q = 0; q < 12; ++q) A[lane][q] = U64[(size_t)i * 144 + lane * 12 + q];
      __syncwarp();
    }
    // tangent projection + damping
    if (manifold == POVAR_SPHERE) {
      double nn = Pl * Pl;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
      ph = lane < 12 ? Pl / sqrt(nn) : 0.0;
      double up = 0.0;
      for (int q = 0; q < 12; ++q) {
        const double pq = __shfl_sync(0xffffffffu, ph, q);
        if (lane < 12) up += A[lane][q] * pq;
      }
      double cc = ph * up;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cc += __shfl_xor_sync(0xffffffffu, cc, o);
      __syncwarp();
      for (int q = 0; q < 12; ++q) {
        const double pq = __shfl_sync(0xffffffffu, ph, q);
        const double uq = __shfl_sync(0xffffffffu, up, q);
        if (lane < 12)
          A[lane][q] += -up * pq - ph * uq + (cc - lam_eff + 1.0) * ph * pq +
                        (lane == q ? lam_eff : 0.0);
      }
    } else if (lane < 12) {
      A[lane][lane] += lam_eff;
    }
    __syncwarp();
    // Cholesky A = L L^T (lower, in place), lanes own rows; one reciprocal
    // square root per pivot gives the diagonal (d r) and its inverse (r), so
    // the column scaling and the later solve multiply instead of divide
    bool lbad = false;
    for (int k = 0; k < 12; ++k) {
      if (lane == k) {
        const double d = A[k][k];
        if (!(d > 0.0)) lbad = true;
        const double dd = fmax(d, 1e-300);
        const double r = rsqrt(dd);
        A[k][k] = dd * r;
        inv[k] = r;
      }
      __syncwarp();
      if (lane > k && lane < 12) A[lane][k] *= inv[k];
      __syncwarp();
      // trailing update A[r][j] -= A[r][k] A[j][k] for k < j <= r
#pragma unroll
      for (int u = 0; u < 3; ++u)
        if (tj[u] > k) A[tr[u]][tj[u]] -= A[tr[u]][k] * A[tj[u]][k];
      __syncwarp();
    }
    bad = __any_sync(0xffffffffu, lbad);
  }
  if (lane == 0) {
    if (bad) st->error = POVAR_ENUMERIC;
    else if (attempt > 1) atomicAdd(&st->n_regularized, 1);
  }
  // L^-1 by columns (lane c owns column c)
  if (lane < 12) {
    const int c = lane;
    for (int r = 0; r < 12; ++r) {
      if (r < c) {
        L[r][c] = 0.0;
        continue;
      }
      double s = (r == c) ? 1.0 : 0.0;
      for (int k = c; k < r; ++k) s -= A[r][k] * L[k][c];
      L[r][c] = s * inv[r];
    }
  }
  __syncwarp();
  // A^-1 = L^-T L^-1 (entry (r, j), j <= r: the sum over k >= r of
  // L^-1[k][r] L^-1[k][j], mirrored), minus p^p^T on the sphere; x0 = -G b_p
  double x0 = 0.0;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    if (tj[u] < 0) continue;
    const int r = tr[u], j = tj[u];
    double s = 0.0;
    for (int k = r; k < 12; ++k) s += L[k][r] * L[k][j];
    A[r][j] = s;
    A[j][r] = s;
  }
  __syncwarp();
  for (int q = 0; q < 12; ++q) {
    const double pq = __shfl_sync(0xffffffffu, ph, q);
    const double bq = __shfl_sync(0xffffffffu, bpl, q);
    if (lane < 12) {
      double g = A[lane][q];
      if (manifold == POVAR_SPHERE) g -= ph * pq;
      G64[(size_t)i * 144 + lane * 12 + q] = g;
      G32[(size_t)i * 144 + lane * 12 + q] = (float)g;
      x0 -= g * bq;
    }
  }
  if (lane < 12) {
    Y[(size_t)i * 12 + lane] = (T)x0;                    // term parity 0
    Y[((size_t)nc + i) * 12 + lane] = (T)0;              // term parity 1
    D[(size_t)i * 12 + lane] = (T)x0;
  }
  if (lane < 2) camnorm[2 * (size_t)i + lane] = 0.0;
}

}  // namespace

povar_status launch_linearize(Problem* p, int precision, double eta, bool poba) {
  const unsigned g = grid_for(p->nchunks, 8);
  if (g == 0) return POVAR_OK;
  const float4* s32 = poba ? p->sbl32 : nullptr;
  const double* s64 = poba ? p->sbl64 : nullptr;
  const int force = poba ? 1 : 0;
  if (precision == POVAR_FP64) {
    k_linearize<double><<<g, 256, 0, p->stream>>>(
        p->state, sqrt(1.0 - eta), sqrt(eta), p->nchunks, p->chunk_cam, p->chunk_beg, p->cm_slot,
        p->cm_m64, p->P64[0], p->P64[1], p->pdA[0], p->pdA[1], p->X64[0], p->X64[1],
        s64 ? s32 : nullptr, s64, force, static_cast<double*>(p->part_lin));
  } else {
    k_linearize<float><<<g, 256, 0, p->stream>>>(
        p->state, (float)sqrt(1.0 - eta), (float)sqrt(eta), p->nchunks, p->chunk_cam,
        p->chunk_beg, p->cm_slot, p->cm_m32, p->camP32[0], p->camP32[1], p->pdA[0], p->pdA[1],
        p->X64[0], p->X64[1], s32, s64, force, static_cast<float*>(p->part_lin));
  }
  ++p->launches;
  return check_launch(p, "linearize");
}

povar_status launch_camera_prepare(Problem* p, int precision, int manifold, double eta,
                                   bool poba) {
  const unsigned g = grid_for(p->nc, 4);
  if (precision == POVAR_FP64) {
    k_camera_prepare<double><<<g, 128, 0, p->stream>>>(
        p->state, eta, manifold, p->nc, p->cam_nchunk, p->cam_chunk0,
        static_cast<const double*>(p->part_lin), p->P64[0], p->P64[1], p->U64, p->bp64,
        p->G64, p->G32, p->Y64, p->D64, p->camnorm, poba ? 1 : 0);
  } else {
    k_camera_prepare<float><<<g, 128, 0, p->stream>>>(
        p->state, eta, manifold, p->nc, p->cam_nchunk, p->cam_chunk0,
        static_cast<const float*>(p->part_lin), p->P64[0], p->P64[1], p->U64, p->bp64,
        p->G64, p->G32, p->Y32, p->D32, p->camnorm, poba ? 1 : 0);
  }
  ++p->launches;
  return check_launch(p, "camera_prepare");
}

}  // namespace povar
