// a7: one term of the PoVar series  x_k = U~^-1 W~ V^-1 W~^T x_{k-1}  (Sec. 4.2,
//     Proposition 1 applied to the reduced camera system; Sec. 4.3 in the
//     tangent space), matrix-free:
//       gather  (one thread per landmark slot, SELL-32 order):
//           t_j = sum_k W_k^T y_i = sum_k Pbar_i^T C_k (Y_i x~_j)
//           s_j = V_j^-1 t_j = F_j^T (F_j t_j)
//       scatter (one warp per camera-major chunk, shuffle reduction):
//           z_i = sum_k W_k s_j = sum_k vec((C_k Pbar_i s_j) x~_j^T)
//       finish  (the last warp of camera i, by atomic ticket):
//           x_i = G_i z_i;  delta_i += x_i
//     where Y_i is x_{k-1} of camera i viewed as a 3x4 matrix, Pbar_i the
//     left 3x3 of camera i and C_k = B_k^T B_k. No Jacobian is stored: per
//     observation the passes read a camera/landmark index and the
//     measurement only.
// a8: predicted decrease pred = 2 g^T d - d^T (S - lambda I) d
//       = -2 b_p^T d - d^T U d + sum_j ||F_j W^T d||^2   (d tangent, b_l = 0)
//     with one more gather pass at d and FP64 reductions.
#include "povar_internal.cuh"

namespace povar {
namespace {

template <typename T> struct Vt;
template <> struct Vt<float> { using m2 = float2; };
template <> struct Vt<double> { using m2 = double2; };

// Camera row r (3x4 row-major, 12 values per camera) as 4 values.
template <typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ tab, int i, int r, T out[4]);
template <>
__device__ __forceinline__ void load_row<float>(const float* __restrict__ tab, int i, int r,
                                                float out[4]) {
  const float4 q = __ldg(reinterpret_cast<const float4*>(tab + 12 * (size_t)i) + r);
  out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
}
template <>
__device__ __forceinline__ void load_row<double>(const double* __restrict__ tab, int i, int r,
                                                 double out[4]) {
  const double2* q = reinterpret_cast<const double2*>(tab + 12 * (size_t)i) + 2 * r;
  const double2 a = __ldg(q), b = __ldg(q + 1);
  out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

template <typename T>
struct PointData {
  // FP32 path
  const float4* A;
  const float4* B;
  const float* C;
  // FP64 path
  const double* X;
  const double* F;
};

template <typename T>
__device__ __forceinline__ void load_point(const PointData<T>& pd, int s, T X[3], T F[6]);
template <>
__device__ __forceinline__ void load_point<float>(const PointData<float>& pd, int s,
                                                  float X[3], float F[6]) {
  const float4 a = __ldg(pd.A + s), b = __ldg(pd.B + s);
  X[0] = a.x; X[1] = a.y; X[2] = a.z;
  F[0] = a.w; F[1] = b.x; F[2] = b.y; F[3] = b.z; F[4] = b.w; F[5] = __ldg(pd.C + s);
}
template <>
__device__ __forceinline__ void load_point<double>(const PointData<double>& pd, int s,
                                                   double X[3], double F[6]) {
  const double* x = pd.X + 3 * (size_t)s;
  const double* f = pd.F + 6 * (size_t)s;
  X[0] = x[0]; X[1] = x[1]; X[2] = x[2];
#pragma unroll
  for (int e = 0; e < 6; ++e) F[e] = f[e];
}

__device__ __forceinline__ void store_rec(float4* rec32, double2*, int s, const float S[3],
                                          const float X[3]) {
  rec32[2 * (size_t)s] = make_float4(S[0], S[1], S[2], X[0]);
  rec32[2 * (size_t)s + 1] = make_float4(X[1], X[2], 0.f, 0.f);
}
__device__ __forceinline__ void store_rec(float4*, double2* rec64, int s, const double S[3],
                                          const double X[3]) {
  rec64[4 * (size_t)s] = make_double2(S[0], S[1]);
  rec64[4 * (size_t)s + 1] = make_double2(S[2], X[0]);
  rec64[4 * (size_t)s + 2] = make_double2(X[1], X[2]);
}
__device__ __forceinline__ void load_rec(const float4* rec32, const double2*, uint32_t s,
                                         float S[3], float X[3]) {
  const float4 a = __ldg(rec32 + 2 * (size_t)s), b = __ldg(rec32 + 2 * (size_t)s + 1);
  S[0] = a.x; S[1] = a.y; S[2] = a.z; X[0] = a.w; X[1] = b.x; X[2] = b.y;
}
__device__ __forceinline__ void load_rec(const float4*, const double2* rec64, uint32_t s,
                                         double S[3], double X[3]) {
  const double2 a = __ldg(rec64 + 4 * (size_t)s), b = __ldg(rec64 + 4 * (size_t)s + 1),
                c = __ldg(rec64 + 4 * (size_t)s + 2);
  S[0] = a.x; S[1] = a.y; S[2] = b.x; X[0] = b.y; X[1] = c.x; X[2] = c.y;
}

// gather: PRED = false writes s_j and X_j into rec; PRED = true accumulates
// ||F_j t_j||^2 into one FP64 partial per block.
template <typename T, bool PRED>
__global__ void __launch_bounds__(BLOCK)
k_series_gather(const DeviceState* __restrict__ st, double eta,
                const uint32_t* __restrict__ slot_len, const uint32_t* __restrict__ sell_off,
                const int32_t* __restrict__ sell_cam,
                const typename Vt<T>::m2* __restrict__ sell_m, const T* __restrict__ camPa,
                const T* __restrict__ camPb, const T* __restrict__ vec, PointData<T> pd0,
                PointData<T> pd1,
                float4* __restrict__ rec32, double2* __restrict__ rec64,
                double* __restrict__ pred_part) {
  if (st->converged) return;
  if (!PRED && st->stop_series) return;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const PointData<T>& pd = st->cur ? pd1 : pd0;
  const T* __restrict__ camP = st->cur ? camPb : camPa;
  const T a = (T)(1.0 - eta);
  const uint32_t len = slot_len[s];
  const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
  T X[3], F[6];
  load_point<T>(pd, s, X, F);
  T t0 = 0, t1 = 0, t2 = 0;
  for (uint32_t k = 0; k < len; ++k) {
    const uint32_t pos = base + k * SLICE;
    const int i = sell_cam[pos];
    const auto m = sell_m[pos];
    T Y0[4], Y1[4], Y2[4], P0[4], P1[4], P2[4];
    load_row<T>(vec, i, 0, Y0);
    load_row<T>(vec, i, 1, Y1);
    load_row<T>(vec, i, 2, Y2);
    load_row<T>(camP, i, 0, P0);
    load_row<T>(camP, i, 1, P1);
    load_row<T>(camP, i, 2, P2);
    const T e0 = Y0[0] * X[0] + Y0[1] * X[1] + Y0[2] * X[2] + Y0[3];
    const T e1 = Y1[0] * X[0] + Y1[1] * X[1] + Y1[2] * X[2] + Y1[3];
    const T e2 = Y2[0] * X[0] + Y2[1] * X[1] + Y2[2] * X[2] + Y2[3];
    const T au = a * (T)m.x, av = a * (T)m.y;
    const T aw = au * (T)m.x + av * (T)m.y;
    const T c0 = e0 - au * e2;
    const T c1 = e1 - av * e2;
    const T c2 = aw * e2 - au * e0 - av * e1;
    t0 += P0[0] * c0 + P1[0] * c1 + P2[0] * c2;
    t1 += P0[1] * c0 + P1[1] * c1 + P2[1] * c2;
    t2 += P0[2] * c0 + P1[2] * c1 + P2[2] * c2;
  }
  // z = F t (F lower-triangular, V^-1 = F^T F)
  const T z0 = F[0] * t0;
  const T z1 = F[1] * t0 + F[2] * t1;
  const T z2 = F[3] * t0 + F[4] * t1 + F[5] * t2;
  if (PRED) {
    double q = (double)z0 * z0 + (double)z1 * z1 + (double)z2 * z2;
    __shared__ double red[BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
      double c = 0.0;
      for (int w = 0; w < BLOCK / 32; ++w) c += red[w];
      pred_part[blockIdx.x] = c;
    }
  } else {
    T S[3];
    S[0] = F[0] * z0 + F[1] * z1 + F[3] * z2;
    S[1] = F[2] * z1 + F[4] * z2;
    S[2] = F[5] * z2;
    store_rec(rec32, rec64, s, S, X);
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_series_scatter(DeviceState* __restrict__ st, double eta, int term, double eps, int nchunks,
                 int nc, int nc_active, const int32_t* __restrict__ chunk_cam,
                 const uint32_t* __restrict__ chunk_beg, const int32_t* __restrict__ cam_nchunk,
                 const int32_t* __restrict__ cam_chunk0, const uint32_t* __restrict__ cm_slot,
                 const typename Vt<T>::m2* __restrict__ cm_m, const T* __restrict__ camPa,
                 const T* __restrict__ camPb, const float4* __restrict__ rec32, const double2* __restrict__ rec64,
                 const T* __restrict__ G, T* __restrict__ part, uint32_t* __restrict__ cam_ticket,
                 uint32_t* __restrict__ done_ticket, double* __restrict__ camnorm,
                 T* __restrict__ Y, T* __restrict__ D) {
  if (st->converged || st->stop_series) return;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= nchunks) return;
  const int i = chunk_cam[c];
  const T a = (T)(1.0 - eta);
  const T* __restrict__ camP = st->cur ? camPb : camPa;
  T P[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) P[r][q] = camP[12 * (size_t)i + 4 * r + q];
  T acc[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) acc[e] = 0;
  const uint32_t b = chunk_beg[c], e_ = chunk_beg[c + 1];
  for (uint32_t r = b + lane; r < e_; r += 32) {
    const uint32_t slot = cm_slot[r];
    const auto m = cm_m[r];
    T S[3], X[3];
    load_rec(rec32, rec64, slot, S, X);
    const T w0 = P[0][0] * S[0] + P[0][1] * S[1] + P[0][2] * S[2];
    const T w1 = P[1][0] * S[0] + P[1][1] * S[1] + P[1][2] * S[2];
    const T w2 = P[2][0] * S[0] + P[2][1] * S[1] + P[2][2] * S[2];
    const T au = a * (T)m.x, av = a * (T)m.y;
    const T aw = au * (T)m.x + av * (T)m.y;
    const T q0 = w0 - au * w2;
    const T q1 = w1 - av * w2;
    const T q2 = aw * w2 - au * w0 - av * w1;
    acc[0] += q0 * X[0]; acc[1] += q0 * X[1]; acc[2] += q0 * X[2]; acc[3] += q0;
    acc[4] += q1 * X[0]; acc[5] += q1 * X[1]; acc[6] += q1 * X[2]; acc[7] += q1;
    acc[8] += q2 * X[0]; acc[9] += q2 * X[1]; acc[10] += q2 * X[2]; acc[11] += q2;
  }
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    T v = acc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    acc[e] = v;
  }
  const int nch = cam_nchunk[i];
  T z = 0;  // lane l < 12 holds z_l
  if (nch == 1) {
#pragma unroll
    for (int e = 0; e < 12; ++e)
      if (lane == e) z = acc[e];
  } else {
    T* out = part + (size_t)c * 12;
#pragma unroll
    for (int e = 0; e < 12; ++e)
      if (lane == e) out[e] = acc[e];
    __threadfence();
    unsigned ticket = 0;
    if (lane == 0) ticket = atomicAdd(cam_ticket + i, 1u);
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    if (ticket != (unsigned)(nch - 1)) return;
    __threadfence();
    if (lane == 0) cam_ticket[i] = 0;
    const int c0 = cam_chunk0[i];
    if (lane < 12) {
      T s = 0;
      for (int q = 0; q < nch; ++q) s += __ldcg(part + (size_t)(c0 + q) * 12 + lane);
      z = s;
    }
  }
  // x_i = G_i z_i, delta_i += x_i
  T x = 0;
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    const T zq = __shfl_sync(0xffffffffu, z, q);
    if (lane < 12) x += G[144 * (size_t)i + 12 * lane + q] * zq;
  }
  double yy = 0.0, dd = 0.0;
  if (lane < 12) {
    const T d = D[12 * (size_t)i + lane] + x;
    D[12 * (size_t)i + lane] = d;
    Y[12 * (size_t)i + lane] = x;
    yy = (double)x * x;
    dd = (double)d * d;
  }
  if (eps > 0.0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      yy += __shfl_xor_sync(0xffffffffu, yy, o);
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
    }
    if (lane == 0) {
      camnorm[2 * (size_t)i] = yy;
      camnorm[2 * (size_t)i + 1] = dd;
    }
    __threadfence();
    unsigned t2 = 0;
    if (lane == 0) t2 = atomicAdd(done_ticket, 1u);
    t2 = __shfl_sync(0xffffffffu, t2, 0);
    if (t2 != (unsigned)(nc_active - 1)) return;
    __threadfence();
    double sy = 0.0, sd = 0.0;
    for (int q = lane; q < nc; q += 32) {
      sy += __ldcg(camnorm + 2 * (size_t)q);
      sd += __ldcg(camnorm + 2 * (size_t)q + 1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    if (lane == 0) {
      *done_ticket = 0;
      if (sy <= eps * eps * sd) {
        st->stop_series = 1;
        st->terms_used = term + 1;
      }
    }
  }
}

// delta <- Pi delta on the sphere (removes rounding drift out of the tangent
// space before the predicted decrease and the update use it).
template <typename T>
__global__ void k_project_delta(const DeviceState* __restrict__ st, int nc,
                                const double* __restrict__ P0, const double* __restrict__ P1,
                                T* __restrict__ D) {
  if (st->converged) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const double* P = (st->cur ? P1 : P0) + 12 * (size_t)i;
  double nn = 0.0, pd = 0.0;
  for (int e = 0; e < 12; ++e) {
    nn += P[e] * P[e];
    pd += P[e] * (double)D[12 * (size_t)i + e];
  }
  const double f = pd / nn;
  for (int e = 0; e < 12; ++e) D[12 * (size_t)i + e] = (T)((double)D[12 * (size_t)i + e] - f * P[e]);
}

template <typename T>
__global__ void k_pred_finish(DeviceState* __restrict__ st, int nc, int nparts, int m,
                              const double* __restrict__ pred_part,
                              const double* __restrict__ U64, const double* __restrict__ bp64,
                              const T* __restrict__ D) {
  if (st->converged) return;
  __shared__ double red[256];
  double tv = 0.0;
  for (int q = threadIdx.x; q < nparts; q += 256) tv += pred_part[q];
  double du = 0.0, bd = 0.0;
  for (int i = threadIdx.x; i < nc; i += 256) {
    double d[12];
    for (int e = 0; e < 12; ++e) d[e] = (double)D[12 * (size_t)i + e];
    const double* U = U64 + 144 * (size_t)i;
    for (int r = 0; r < 12; ++r) {
      double s = 0.0;
      for (int q = 0; q < 12; ++q) s += U[12 * r + q] * d[q];
      du += d[r] * s;
      bd += bp64[12 * (size_t)i + r] * d[r];
    }
  }
  double v = -2.0 * bd - du + tv;
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->pred = red[0];
    if (!st->stop_series) st->terms_used = m;
  }
}

template <typename T>
PointData<T> point_data(Problem* p, int t) {
  PointData<T> pd;
  pd.A = p->pdA[t];
  pd.B = p->pdB[t];
  pd.C = p->pdC[t];
  pd.X = p->X64[t];
  pd.F = p->F64[t];
  return pd;
}

}  // namespace

povar_status launch_series_term(Problem* p, int precision, double eta, int term, double eps) {
  const unsigned gs = grid_for(p->nchunks, 8);
  if (precision == POVAR_FP64) {
    k_series_gather<double, false><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1], p->Y64,
        point_data<double>(p, 0), point_data<double>(p, 1), p->rec32, p->rec64, nullptr);
  } else {
    k_series_gather<float, false><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32, p->camP32, p->Y32,
        point_data<float>(p, 0), point_data<float>(p, 1), p->rec32, p->rec64, nullptr);
  }
  ++p->launches;
  if (gs > 0) {
    if (precision == POVAR_FP64) {
      k_series_scatter<double><<<gs, 256, 0, p->stream>>>(
          p->state, eta, term, eps, p->nchunks, p->nc, p->nc_active, p->chunk_cam,
          p->chunk_beg, p->cam_nchunk, p->cam_chunk0, p->cm_slot, p->cm_m64, p->P64[0],
          p->P64[1], p->rec32, p->rec64, p->G64, static_cast<double*>(p->part_ser), p->cam_ticket,
          p->done_ticket, p->camnorm, p->Y64, p->D64);
    } else {
      k_series_scatter<float><<<gs, 256, 0, p->stream>>>(
          p->state, eta, term, eps, p->nchunks, p->nc, p->nc_active, p->chunk_cam,
          p->chunk_beg, p->cam_nchunk, p->cam_chunk0, p->cm_slot, p->cm_m32, p->camP32,
          p->camP32, p->rec32, p->rec64, p->G32, static_cast<float*>(p->part_ser), p->cam_ticket,
          p->done_ticket, p->camnorm, p->Y32, p->D32);
    }
    ++p->launches;
  }
  return check_launch(p, "series_term");
}

povar_status launch_pred(Problem* p, int precision, double eta, int manifold, int m) {
  const unsigned gc = grid_for(p->nc, 128);
  if (precision == POVAR_FP64) {
    if (manifold == POVAR_SPHERE)
      k_project_delta<double><<<gc, 128, 0, p->stream>>>(p->state, p->nc, p->P64[0],
                                                         p->P64[1], p->D64);
    k_series_gather<double, true><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1], p->D64,
        point_data<double>(p, 0), point_data<double>(p, 1), p->rec32, p->rec64, p->pred_part);
    k_pred_finish<double><<<1, 256, 0, p->stream>>>(p->state, p->nc, p->n_slot_blocks, m,
                                                    p->pred_part, p->U64, p->bp64, p->D64);
  } else {
    if (manifold == POVAR_SPHERE)
      k_project_delta<float><<<gc, 128, 0, p->stream>>>(p->state, p->nc, p->P64[0], p->P64[1],
                                                        p->D32);
    k_series_gather<float, true><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, eta, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32, p->camP32, p->D32,
        point_data<float>(p, 0), point_data<float>(p, 1), p->rec32, p->rec64, p->pred_part);
    k_pred_finish<float><<<1, 256, 0, p->stream>>>(p->state, p->nc, p->n_slot_blocks, m,
                                                   p->pred_part, p->U64, p->bp64, p->D32);
  }
  p->launches += manifold == POVAR_SPHERE ? 3 : 2;
  return check_launch(p, "pred");
}

}  // namespace povar
