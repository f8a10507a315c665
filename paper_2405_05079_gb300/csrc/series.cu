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
#include "reproj.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

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

// Warps per camera block of the camera-row schedule.
constexpr int CAMROW_WARPS = 4;

// Loads of data that each kernel streams through once (SELL camera indices
// and measurements, per-landmark records): read-only, not allocated in L1, so
// that L1 keeps the camera rows that every slice row re-reads.
__device__ __forceinline__ int ld_stream(const int32_t* p) {
  int v;
  asm("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p) {
  float2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_stream(const double2* p) {
  double2 v;
  asm("ld.global.nc.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ float ld_stream(const float* p) {
  float v;
  asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double ld_stream(const double* p) {
  double v;
  asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
  uint4 v;
  asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
      : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ unsigned short ld_stream(const unsigned short* p) {
  unsigned short v;
  asm("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
  return v;
}

// Stored observation blocks G_k = C_k Pbar_i (row-major 3x3, g[3r + q]),
// one per SELL entry, in planes of BlockPlanes (layout in
// povar_internal.cuh). Blk<TS> loads them as T and stores them from T.
struct Bf16 {};   // storage tag: bfloat16, round to nearest even
template <typename TS> struct Blk;
template <> struct Blk<float> {
  static __device__ __forceinline__ void load(const BlockPlanes& b, size_t e, float g[9]) {
    const float4 x = ld_stream(static_cast<const float4*>(b.p[0]) + e);
    const float4 y = ld_stream(static_cast<const float4*>(b.p[1]) + e);
    g[0] = x.x; g[1] = x.y; g[2] = x.z; g[3] = x.w;
    g[4] = y.x; g[5] = y.y; g[6] = y.z; g[7] = y.w;
    g[8] = ld_stream(static_cast<const float*>(b.p[2]) + e);
  }
  static __device__ __forceinline__ void store(const BlockPlanes& b, size_t e, const float g[9]) {
    static_cast<float4*>(b.p[0])[e] = make_float4(g[0], g[1], g[2], g[3]);
    static_cast<float4*>(b.p[1])[e] = make_float4(g[4], g[5], g[6], g[7]);
    static_cast<float*>(b.p[2])[e] = g[8];
  }
};
template <> struct Blk<double> {
  static __device__ __forceinline__ void load(const BlockPlanes& b, size_t e, double g[9]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double2 x = ld_stream(static_cast<const double2*>(b.p[k]) + e);
      g[2 * k] = x.x;
      g[2 * k + 1] = x.y;
    }
    g[8] = ld_stream(static_cast<const double*>(b.p[4]) + e);
  }
  static __device__ __forceinline__ void store(const BlockPlanes& b, size_t e, const double g[9]) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
      static_cast<double2*>(b.p[k])[e] = make_double2(g[2 * k], g[2 * k + 1]);
    static_cast<double*>(b.p[4])[e] = g[8];
  }
};
// A bfloat16 is the upper half of an FP32 word: widening is a shift.
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t bf16_bits(float x) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x));
}
template <> struct Blk<Bf16> {
  static __device__ __forceinline__ void load(const BlockPlanes& b, size_t e, float g[9]) {
    const uint4 x = ld_stream(static_cast<const uint4*>(b.p[0]) + e);
    g[0] = bf16_lo(x.x); g[1] = bf16_hi(x.x); g[2] = bf16_lo(x.y); g[3] = bf16_hi(x.y);
    g[4] = bf16_lo(x.z); g[5] = bf16_hi(x.z); g[6] = bf16_lo(x.w); g[7] = bf16_hi(x.w);
    g[8] = bf16_lo((uint32_t)ld_stream(static_cast<const unsigned short*>(b.p[1]) + e));
  }
  static __device__ __forceinline__ void store(const BlockPlanes& b, size_t e, const float g[9]) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = bf16_bits(g[2 * k]) | (bf16_bits(g[2 * k + 1]) << 16);
    static_cast<uint4*>(b.p[0])[e] = make_uint4(w[0], w[1], w[2], w[3]);
    static_cast<unsigned short*>(b.p[1])[e] = (unsigned short)bf16_bits(g[8]);
  }
};

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
  const float4 a = ld_stream(pd.A + s), b = ld_stream(pd.B + s);
  X[0] = a.x; X[1] = a.y; X[2] = a.z;
  F[0] = a.w; F[1] = b.x; F[2] = b.y; F[3] = b.z; F[4] = b.w; F[5] = ld_stream(pd.C + s);
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
k_series_gather(const DeviceState* __restrict__ st, T a,
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
  const uint32_t len = slot_len[s];
  const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
  T X[3], F[6];
  load_point<T>(pd, s, X, F);
  T t0 = 0, t1 = 0, t2 = 0;
  // observations in chunks of RB: the chunk's camera indices and
  // measurements are loaded together so that RB rows are in flight per warp
  using M2 = typename Vt<T>::m2;
  constexpr int RB = 4;
  for (uint32_t k0 = 0; k0 < len; k0 += RB) {
    int ci[RB];
    M2 mi[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const bool in = k0 + u < len;
      ci[u] = in ? ld_stream(sell_cam + base + (k0 + u) * SLICE) : 0;
      mi[u] = in ? ld_stream(sell_m + base + (k0 + u) * SLICE) : M2{0, 0};
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      if (k0 + u >= len) break;
      const int i = ci[u];
      const auto m = mi[u];
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
  }
  // z = F t (F lower-triangular, V^-1 = F^T F)
  const T z0 = F[0] * t0;
  const T z1 = F[1] * t0 + F[2] * t1;
  const T z2 = F[3] * t0 + F[4] * t1 + F[5] * t2;
  if (PRED) {
    // per-warp sum in the series precision; partials are added in FP64
    T q = z0 * z0 + z1 * z1 + z2 * z2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0) pred_part[s / 32] = (double)q;
  } else {
    T S[3];
    S[0] = F[0] * z0 + F[1] * z1 + F[3] * z2;
    S[1] = F[2] * z1 + F[4] * z2;
    S[2] = F[5] * z2;
    store_rec(rec32, rec64, s, S, X);
  }
}

// Per-camera end of a series term, run by one warp whose lanes 0..11 hold
// z_i: x_i = G_i z_i, delta_i += x_i, Y_i = x_i; with the threshold rule
// (eps > 0) the last camera to finish (atomic ticket over `n_tickets`
// cameras) adds the per-camera norms in camera order and sets the stop flag.
template <typename T> struct Row12;
template <> struct Row12<float> {
  static __device__ __forceinline__ void load(const float* src, float r[12]) {
    const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 x = __ldg(q + k);
      r[4 * k] = x.x; r[4 * k + 1] = x.y; r[4 * k + 2] = x.z; r[4 * k + 3] = x.w;
    }
  }
};
template <> struct Row12<double> {
  static __device__ __forceinline__ void load(const double* src, double r[12]) {
    const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const double2 x = __ldg(q + k);
      r[2 * k] = x.x; r[2 * k + 1] = x.y;
    }
  }
};

template <typename T>
__device__ __forceinline__ void camera_update(int i, int lane, T z, const T* __restrict__ G,
                                              T* __restrict__ Y, T* __restrict__ D, double& yy,
                                              double& dd) {
  T g[12];
  Row12<T>::load(G + 144 * (size_t)i + 12 * (lane < 12 ? lane : 0), g);
  T x = 0;
#pragma unroll
  for (int q = 0; q < 12; ++q) x += g[q] * __shfl_sync(0xffffffffu, z, q);
  T y2 = 0, d2 = 0;
  if (lane < 12) {
    const T d = D[12 * (size_t)i + lane] + x;
    D[12 * (size_t)i + lane] = d;
    Y[12 * (size_t)i + lane] = x;
    y2 = x * x;
    d2 = d * d;
  }
  // warp sums in the series precision, converted once
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
  }
  yy = (double)y2;
  dd = (double)d2;
}

template <typename T>
__device__ __forceinline__ void finish_camera(DeviceState* __restrict__ st, int i, int lane, T z,
                                              int term, double eps, int n_tickets,
                                              const T* __restrict__ G,
                                              double* __restrict__ camnorm,
                                              uint32_t* __restrict__ done_ticket,
                                              T* __restrict__ Y, T* __restrict__ D, int nc) {
  double yy, dd;
  camera_update<T>(i, lane, z, G, Y, D, yy, dd);
  if (eps > 0.0) {
    if (lane == 0) {
      camnorm[2 * (size_t)i] = yy;
      camnorm[2 * (size_t)i + 1] = dd;
    }
    __threadfence();
    unsigned t2 = 0;
    if (lane == 0) t2 = atomicAdd(done_ticket, 1u);
    t2 = __shfl_sync(0xffffffffu, t2, 0);
    if (t2 != (unsigned)(n_tickets - 1)) return;
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

template <typename T>
__global__ void __launch_bounds__(256)
k_series_scatter(DeviceState* __restrict__ st, T a, int term, double eps, int nchunks,
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
  finish_camera<T>(st, i, lane, z, term, eps, nc_active, G, camnorm, done_ticket, Y, D, nc);
}


// ---------------------------------------------------------------------------
// Fused schedule: one pass over the SELL slices per series term.
//   pass 1 (lane = landmark j): t_j = sum_k Pbar_i^T C_k (Y_i x~_j),
//                               s_j = F_j^T F_j t_j
//   pass 2 (lanes in lockstep over track positions k): the contribution
//       vec((C_k Pbar_i s_j) x~_j^T) of every lane is reduced over the lanes
//       that share its camera -- the whole warp for a uniform slice row, a
//       run of consecutive lanes otherwise -- and written as one partial
//       per run. The run layout is fixed at creation, so every partial has a
//       fixed slot and the per-camera sums below are deterministic.
// ---------------------------------------------------------------------------

// Sum of v[0..11] over the 32 lanes by recursive halving (18 shuffles).
// Afterwards lanes 0, 8, 16, 24 hold totals (vbase .. vbase + 2) in r[0..2].
template <typename T>
__device__ __forceinline__ void warp_reduce12(const T v[12], int lane, T r[3], int& vbase) {
  const bool hiA = lane & 16, hiB = lane & 8;
  T r6[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const T send = hiA ? v[j] : v[j + 6];
    const T keep = hiA ? v[j + 6] : v[j];
    r6[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T send = hiB ? r6[j] : r6[j + 3];
    const T keep = hiB ? r6[j + 3] : r6[j];
    r[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r[j] += __shfl_xor_sync(0xffffffffu, r[j], 4);
    r[j] += __shfl_xor_sync(0xffffffffu, r[j], 2);
    r[j] += __shfl_xor_sync(0xffffffffu, r[j], 1);
  }
  vbase = (hiA ? 6 : 0) + (hiB ? 3 : 0);
}

// t += Pbar^T C (Y x~) for one observation (W^T-gather)
template <typename T>
__device__ __forceinline__ void gather_obs(const T Y0[4], const T Y1[4], const T Y2[4],
                                           const T P0[4], const T P1[4], const T P2[4], T a,
                                           T mu, T mv, const T X[3], T t[3]) {
  const T e0 = Y0[0] * X[0] + Y0[1] * X[1] + Y0[2] * X[2] + Y0[3];
  const T e1 = Y1[0] * X[0] + Y1[1] * X[1] + Y1[2] * X[2] + Y1[3];
  const T e2 = Y2[0] * X[0] + Y2[1] * X[1] + Y2[2] * X[2] + Y2[3];
  const T au = a * mu, av = a * mv;
  const T aw = au * mu + av * mv;
  const T c0 = e0 - au * e2;
  const T c1 = e1 - av * e2;
  const T c2 = aw * e2 - au * e0 - av * e1;
  t[0] += P0[0] * c0 + P1[0] * c1 + P2[0] * c2;
  t[1] += P0[1] * c0 + P1[1] * c1 + P2[1] * c2;
  t[2] += P0[2] * c0 + P1[2] * c1 + P2[2] * c2;
}

// v += vec((C Pbar s) x~^T) for one observation (W-scatter)
template <typename T>
__device__ __forceinline__ void scatter_obs(const T P0[4], const T P1[4], const T P2[4], T a,
                                            T mu, T mv, const T S[3], const T X[3], T v[12]) {
  const T w0 = P0[0] * S[0] + P0[1] * S[1] + P0[2] * S[2];
  const T w1 = P1[0] * S[0] + P1[1] * S[1] + P1[2] * S[2];
  const T w2 = P2[0] * S[0] + P2[1] * S[1] + P2[2] * S[2];
  const T au = a * mu, av = a * mv;
  const T aw = au * mu + av * mv;
  const T q0 = w0 - au * w2;
  const T q1 = w1 - av * w2;
  const T q2 = aw * w2 - au * w0 - av * w1;
  v[0] += q0 * X[0]; v[1] += q0 * X[1]; v[2] += q0 * X[2]; v[3] += q0;
  v[4] += q1 * X[0]; v[5] += q1 * X[1]; v[6] += q1 * X[2]; v[7] += q1;
  v[8] += q2 * X[0]; v[9] += q2 * X[1]; v[10] += q2 * X[2]; v[11] += q2;
}

// v += vec((G s) x~^T) for one observation with its stored block G = C Pbar
template <typename T>
__device__ __forceinline__ void stored_obs(const T g[9], const T S[3], const T X[3], T v[12]) {
  const T q0 = g[0] * S[0] + g[1] * S[1] + g[2] * S[2];
  const T q1 = g[3] * S[0] + g[4] * S[1] + g[5] * S[2];
  const T q2 = g[6] * S[0] + g[7] * S[1] + g[8] * S[2];
  v[0] += q0 * X[0]; v[1] += q0 * X[1]; v[2] += q0 * X[2]; v[3] += q0;
  v[4] += q1 * X[0]; v[5] += q1 * X[1]; v[6] += q1 * X[2]; v[7] += q1;
  v[8] += q2 * X[0]; v[9] += q2 * X[1]; v[10] += q2 * X[2]; v[11] += q2;
}

// q = C Pbar s for one observation: its W-scatter contribution is vec(q x~^T)
template <typename T>
__device__ __forceinline__ void scatter_q(const T P0[4], const T P1[4], const T P2[4], T a,
                                          T mu, T mv, const T S[3], T q[3]) {
  const T w0 = P0[0] * S[0] + P0[1] * S[1] + P0[2] * S[2];
  const T w1 = P1[0] * S[0] + P1[1] * S[1] + P1[2] * S[2];
  const T w2 = P2[0] * S[0] + P2[1] * S[1] + P2[2] * S[2];
  const T au = a * mu, av = a * mv;
  const T aw = au * mu + av * mv;
  q[0] = w0 - au * w2;
  q[1] = w1 - av * w2;
  q[2] = aw * w2 - au * w0 - av * w1;
}

// q = G s for one observation with its stored block G = C Pbar
template <typename T>
__device__ __forceinline__ void stored_q(const T g[9], const T S[3], T q[3]) {
  q[0] = g[0] * S[0] + g[1] * S[1] + g[2] * S[2];
  q[1] = g[3] * S[0] + g[4] * S[1] + g[5] * S[2];
  q[2] = g[6] * S[0] + g[7] * S[1] + g[8] * S[2];
}

// The columns of x~ = (X, 1) in the order in which reduce_rows halves them on
// this lane: lane bit 8 puts the pair {2, 3} first, lane bit 4 swaps within
// each pair, so that every halving stage keeps its first half. cfin is the
// column the lane holds at the end.
template <typename T>
__device__ __forceinline__ void stage_columns(const T X[3], int lane, T xp[4], int& cfin) {
  const bool hB = lane & 8, hC = lane & 4;
  const T one = 1;
  const T lo0 = hC ? X[1] : X[0], lo1 = hC ? X[0] : X[1];
  const T hi0 = hC ? one : X[2], hi1 = hC ? X[2] : one;
  xp[0] = hB ? hi0 : lo0;
  xp[1] = hB ? hi1 : lo1;
  xp[2] = hB ? lo0 : hi0;
  xp[3] = hB ? lo1 : hi1;
  cfin = (hB ? 2 : 0) + (hC ? 1 : 0);
}

// Sums over the 32 lanes of vec(q x~^T) for two consecutive warp-uniform
// slice rows (row A from every lane's qa, row B from qb); a single uniform
// row keeps warp_reduce12, whose cost this does not beat with an empty row B. Lanes with bit 16 own row B: in the
// first stage each lane keeps its row's q and sends the other row's q (3
// values instead of 12 products), and adds the partner's outer product with
// the partner's columns xq. The 12 sums are held column-major (3c + r) in the
// lane's stage order xp, so the stages over lane bits 8 and 4 keep the first
// half with no select; bits 2 and 1 finish the sums. Lanes with (lane & 3) ==
// 0 store entries cfin, 4 + cfin, 8 + cfin of their row's partial (outA /
// outB; a null pointer skips the row).
template <typename T>
__device__ __forceinline__ void reduce_rows(const T qa[3], const T qb[3], const T xp[4],
                                            const T xq[4], int lane, int cfin, T* outA,
                                            T* outB) {
  const bool hA = lane & 16;
  T qk[3], qo[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const T keep = hA ? qb[r] : qa[r];
    const T send = hA ? qa[r] : qb[r];
    qk[r] = keep;
    qo[r] = __shfl_xor_sync(0xffffffffu, send, 16);
  }
  T r12[12];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int r = 0; r < 3; ++r) r12[3 * c + r] = qk[r] * xp[c] + qo[r] * xq[c];
  T r6[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) r6[j] = r12[j] + __shfl_xor_sync(0xffffffffu, r12[6 + j], 8);
  T r3[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r3[j] = r6[j] + __shfl_xor_sync(0xffffffffu, r6[3 + j], 4);
    r3[j] += __shfl_xor_sync(0xffffffffu, r3[j], 2);
    r3[j] += __shfl_xor_sync(0xffffffffu, r3[j], 1);
  }
  T* out = hA ? outB : outA;
  if ((lane & 3) == 0 && out) {
    out[cfin] = r3[0];
    out[4 + cfin] = r3[1];
    out[8 + cfin] = r3[2];
  }
}

// Segmented sum of v over the runs of equal camera that start at the set
// bits of mask; the run starting at a valid lane stores its sum as the next
// partial from pbase (valid run starts in lane order).
template <typename T>
__device__ __forceinline__ void store_runs(T v[12], uint32_t mask, bool valid, uint32_t pbase,
                                           int lane, T* __restrict__ part) {
  const uint32_t nb = lane < 31 ? (mask >> (lane + 1)) : 0u;
  bool ok[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int o = 1 << q;
    ok[q] = (lane + o < 32) && ((nb & ((1u << o) - 1u)) == 0u);
  }
#pragma unroll
  for (int e = 0; e < 12; ++e) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const T other = __shfl_down_sync(0xffffffffu, v[e], 1 << q);
      if (ok[q]) v[e] += other;
    }
  }
  const uint32_t starts = mask & __ballot_sync(0xffffffffu, valid);
  if ((starts >> lane) & 1u) {
    T* out = part + ((size_t)pbase + __popc(starts & ((1u << lane) - 1u))) * 12;
#pragma unroll
    for (int e = 0; e < 12; ++e) out[e] = v[e];
  }
}

// Reduction of two rows of 12 values across the warp (transposed butterfly):
// lanes with (lane & 3) == 0 end with three totals of row `row_b`, entries
// vbase .. vbase + 2.
template <typename T>
__device__ __forceinline__ void warp_reduce24(const T vA[12], const T vB[12], int lane, T r[3],
                                              int& row_b, int& vbase) {
  // xor 16: keep one row, send the other
  const bool hiA = lane & 16, hiB = lane & 8, hiC = lane & 4;
  T r12[12];
#pragma unroll
  for (int j = 0; j < 12; ++j) {
    const T send = hiA ? vA[j] : vB[j];
    const T keep = hiA ? vB[j] : vA[j];
    r12[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  T r6[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const T send = hiB ? r12[j] : r12[j + 6];
    const T keep = hiB ? r12[j + 6] : r12[j];
    r6[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const T send = hiC ? r6[j] : r6[j + 3];
    const T keep = hiC ? r6[j + 3] : r6[j];
    r[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    r[j] += __shfl_xor_sync(0xffffffffu, r[j], 2);
    r[j] += __shfl_xor_sync(0xffffffffu, r[j], 1);
  }
  row_b = hiA ? 1 : 0;
  vbase = (hiB ? 6 : 0) + (hiC ? 3 : 0);
}

// Stored schedule: the blocks G_k = C_k Pbar_i of every SELL entry at the
// current cameras (zero for padding entries), written once per step before
// the series terms, which then read G_k instead of the camera's Pbar and the
// measurement: t_j += G_k^T (Y_i x~_j) and z_i += vec((G_k s_j) x~_j^T).
template <typename T, typename TS>
__global__ void __launch_bounds__(256)
k_build_blocks(const DeviceState* __restrict__ st, T a, int64_t nsell,
               const int32_t* __restrict__ sell_cam,
               const typename Vt<T>::m2* __restrict__ sell_m, const T* __restrict__ camPa,
               const T* __restrict__ camPb, BlockPlanes bp) {
  if (st->converged) return;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nsell) return;
  const int i = ld_stream(sell_cam + e);
  T g[9];
  if (i < 0) {
#pragma unroll
    for (int k = 0; k < 9; ++k) g[k] = 0;
  } else {
    const T* __restrict__ camP = st->cur ? camPb : camPa;
    T P0[4], P1[4], P2[4];
    load_row<T>(camP, i, 0, P0);
    load_row<T>(camP, i, 1, P1);
    load_row<T>(camP, i, 2, P2);
    const auto m = ld_stream(sell_m + e);
    const T au = a * (T)m.x, av = a * (T)m.y;
    const T aw = au * (T)m.x + av * (T)m.y;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      g[q] = P0[q] - au * P2[q];
      g[3 + q] = P1[q] - av * P2[q];
      g[6 + q] = aw * P2[q] - au * P0[q] - av * P1[q];
    }
  }
  Blk<TS>::store(bp, (size_t)e, g);
}

// TS = void: factored (schedule 1); otherwise the stored blocks of storage TS
// (schedule 4 / the BF16 precision). Both write the same run partials.
// Blocks per SM: four in FP32 (64 registers; the pass-1 chunk kept for pass
// 2 would otherwise raise it to 80 and cut the occupancy by a quarter), two
// in FP64.
template <typename T, typename TS>
__global__ void __launch_bounds__(BLOCK, sizeof(T) == 4 ? 4 : 2)
k_series_fused(const DeviceState* __restrict__ st, T a,
               const uint32_t* __restrict__ slot_len, const uint32_t* __restrict__ sell_off,
               const int32_t* __restrict__ sell_cam,
               const typename Vt<T>::m2* __restrict__ sell_m, const T* __restrict__ camPa,
               const T* __restrict__ camPb, const T* __restrict__ vec, PointData<T> pd0,
               PointData<T> pd1, const uint32_t* __restrict__ row_mask,
               const uint32_t* __restrict__ row_base, T* __restrict__ part, BlockPlanes bp,
               const uint32_t* __restrict__ slist = nullptr, int nslist = 0) {
  constexpr bool STORED = !std::is_void<TS>::value;
  using BS = typename std::conditional<STORED, TS, float>::type;
  if (st->converged || st->stop_series) return;
  const int lane = threadIdx.x & 31;
  // one warp per slice: the slice of the warp's index, or the warp's entry
  // of a slice list (the slices outside the groups of schedule 5)
  int s = blockIdx.x * BLOCK + threadIdx.x;
  if (slist) {
    const int wg = s >> 5;
    if (wg >= nslist) return;
    s = (int)__ldg(slist + wg) * SLICE + lane;
  }
  const PointData<T>& pd = st->cur ? pd1 : pd0;
  const T* __restrict__ camP = st->cur ? camPb : camPa;
  const uint32_t sbeg = sell_off[s / SLICE];
  const uint32_t width = (sell_off[s / SLICE + 1] - sbeg) / SLICE;
  const uint32_t len = slot_len[s];
  const uint32_t base = sbeg + (uint32_t)lane;
  T X[3], F[6];
  load_point<T>(pd, s, X, F);
  T t0 = 0, t1 = 0, t2 = 0;
  // pass 1 in chunks of RB observations: the chunk's camera indices and
  // measurements are loaded together so that RB rows are in flight per warp
  using M2 = typename Vt<T>::m2;
  constexpr int RB = 4;
  // the chunk loaded last stays in ci / mi: it is the first chunk of pass 2
  int ci[RB] = {0, 0, 0, 0};
  M2 mi[RB] = {M2{0, 0}, M2{0, 0}, M2{0, 0}, M2{0, 0}};
  for (uint32_t k0 = 0; k0 < len; k0 += RB) {
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const bool in = k0 + u < len;
      ci[u] = in ? ld_stream(sell_cam + base + (k0 + u) * SLICE) : 0;
      if constexpr (STORED)
        mi[u] = M2{0, 0};   // unused
      else
        mi[u] = in ? ld_stream(sell_m + base + (k0 + u) * SLICE) : M2{0, 0};
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      if (k0 + u >= len) break;
      const int i = ci[u];
      if constexpr (STORED) {
        T g[9];
        Blk<BS>::load(bp, base + (size_t)(k0 + u) * SLICE, g);
        T Y0[4], Y1[4], Y2[4];
        load_row<T>(vec, i, 0, Y0);
        load_row<T>(vec, i, 1, Y1);
        load_row<T>(vec, i, 2, Y2);
        const T e0 = Y0[0] * X[0] + Y0[1] * X[1] + Y0[2] * X[2] + Y0[3];
        const T e1 = Y1[0] * X[0] + Y1[1] * X[1] + Y1[2] * X[2] + Y1[3];
        const T e2 = Y2[0] * X[0] + Y2[1] * X[1] + Y2[2] * X[2] + Y2[3];
        t0 += g[0] * e0 + g[3] * e1 + g[6] * e2;
        t1 += g[1] * e0 + g[4] * e1 + g[7] * e2;
        t2 += g[2] * e0 + g[5] * e1 + g[8] * e2;
        continue;
      }
      const auto m = mi[u];
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
  }
  const T z0 = F[0] * t0;
  const T z1 = F[1] * t0 + F[2] * t1;
  const T z2 = F[3] * t0 + F[4] * t1 + F[5] * t2;
  const T S0 = F[0] * z0 + F[1] * z1 + F[3] * z2;
  const T S1 = F[2] * z1 + F[4] * z2;
  const T S2 = F[5] * z2;
  const uint32_t row0 = sbeg / SLICE;
  // pass 2 in chunks of RB slice rows, last chunk first: the rows' camera
  // indices, measurements and run metadata are loaded together, except (FP32)
  // for the last chunk, whose indices and measurements pass 1 loaded last (a
  // lane whose track reaches that chunk loaded it; every other lane has no
  // observation there); in FP64 the registers are scarcer than the reload.
  // Each row writes its own partial slots, so the order of the rows does not
  // change any result.
  const uint32_t klast = width > 0 ? (width - 1) / RB * RB : 0;
  for (int64_t kr = width > 0 ? (int64_t)klast : -1; kr >= 0; kr -= RB) {
    const uint32_t k0 = (uint32_t)kr;
    uint32_t mk[RB], bk[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const bool rin = k0 + u < width;
      const bool in = k0 + u < len;
      if constexpr (STORED) {
        ci[u] = in ? 0 : -1;   // only validity is needed
        mi[u] = M2{0, 0};
      } else if (sizeof(T) == 4 && k0 == klast) {
        if (!in) {
          ci[u] = -1;
          mi[u] = M2{0, 0};
        }
      } else {
        ci[u] = in ? ld_stream(sell_cam + base + (k0 + u) * SLICE) : -1;
        mi[u] = in ? ld_stream(sell_m + base + (k0 + u) * SLICE) : M2{0, 0};
      }
      mk[u] = rin ? __ldg(row_mask + row0 + k0 + u) : 0u;
      bk[u] = rin ? __ldg(row_base + row0 + k0 + u) : 0u;
    }
#pragma unroll
    for (int up = 0; up < RB; up += 2) {
    if (k0 + up >= width) break;
    // two consecutive uniform rows are reduced across the warp together
    if (k0 + up + 1 < width && mk[up] == 0u && mk[up + 1] == 0u) {
      T qA[3] = {0, 0, 0}, qB[3] = {0, 0, 0};
      const T Sv[3] = {S0, S1, S2};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = ci[up + h];
        if (i >= 0) {
          if constexpr (STORED) {
            T g[9];
            Blk<BS>::load(bp, base + (size_t)(k0 + up + h) * SLICE, g);
            stored_q<T>(g, Sv, h ? qB : qA);
          } else {
            T P0[4], P1[4], P2[4];
            load_row<T>(camP, i, 0, P0);
            load_row<T>(camP, i, 1, P1);
            load_row<T>(camP, i, 2, P2);
            scatter_q<T>(P0, P1, P2, a, (T)mi[up + h].x, (T)mi[up + h].y, Sv, h ? qB : qA);
          }
        }
      }
      T xp[4], xq[4];
      int cfin;
      stage_columns<T>(X, lane, xp, cfin);
#pragma unroll
      for (int c = 0; c < 4; ++c) xq[c] = __shfl_xor_sync(0xffffffffu, xp[c], 16);
      reduce_rows<T>(qA, qB, xp, xq, lane, cfin, part + (size_t)bk[up] * 12,
                     part + (size_t)bk[up + 1] * 12);
      continue;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
    const int u = up + h;
    if (k0 + u >= width) break;
    const int i = ci[u];
    const auto m = mi[u];
    const uint32_t mask = mk[u], pbase = bk[u];
    T v[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) v[e] = 0;
    if (i >= 0) {
      const T Sv[3] = {S0, S1, S2};
      if constexpr (STORED) {
        T g[9];
        Blk<BS>::load(bp, base + (size_t)(k0 + u) * SLICE, g);
        stored_obs<T>(g, Sv, X, v);
      } else {
        T P0[4], P1[4], P2[4];
        load_row<T>(camP, i, 0, P0);
        load_row<T>(camP, i, 1, P1);
        load_row<T>(camP, i, 2, P2);
        scatter_obs<T>(P0, P1, P2, a, (T)m.x, (T)m.y, Sv, X, v);
      }
    }
    if (mask == 0u) {
      T r[3];
      int vb;
      warp_reduce12<T>(v, lane, r, vb);
      if ((lane & 7) == 0) {
        T* out = part + (size_t)pbase * 12 + vb;
        out[0] = r[0]; out[1] = r[1]; out[2] = r[2];
      }
    } else {
      store_runs<T>(v, mask, i >= 0, pbase, lane, part);
    }
    }
    }
  }
}

// ---------------------------------------------------------------------------
// Second stage (projective reprojection error): one series product
// W~ V~^-1 W~^T y in one landmark-major pass over the SELL slices, with the
// first stage's run tables. Pass 1: lane = landmark j of the warp's slice,
// t_j = sum_k P_i^T E_k (Y_i X_j) over its observations, s_j = G_l,j t_j
// (G_l the projected damped inverse of V_j). Pass 2: every slice row's
// contributions vec((E_k P_i s_j) X_j^T) are summed over the lanes that see
// the same camera (one warp reduction for a warp-uniform row, a segmented
// sum over the runs otherwise) into the row's run partials, which
// k_series_apply adds per camera.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(BLOCK)
k_s2_fused(const DeviceState* __restrict__ st, const uint32_t* __restrict__ slot_len,
           const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
           const T* __restrict__ camPa, const T* __restrict__ camPb, const T* __restrict__ vec,
           rp::S2Land<T> land, const uint32_t* __restrict__ row_mask,
           const uint32_t* __restrict__ row_base, T* __restrict__ part) {
  if (st->converged || st->stop_series) return;
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * BLOCK + threadIdx.x;
  const int cur = st->cur;
  const T* __restrict__ camP = cur ? camPb : camPa;
  const uint32_t sbeg = sell_off[s / SLICE];
  const uint32_t width = (sell_off[s / SLICE + 1] - sbeg) / SLICE;
  const uint32_t len = slot_len[s];
  const uint32_t base = sbeg + (uint32_t)lane;
  T X[4], g[10];
  land.load(cur, s, X, g);
  T acc[4] = {0, 0, 0, 0};
  for (uint32_t k = 0; k < len; ++k) {
    const int i = ld_stream(sell_cam + base + k * SLICE);
    T P[12], Y[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      load_row<T>(camP, i, r, P + 4 * r);
      load_row<T>(vec, i, r, Y + 4 * r);
    }
    const rp::Proj<T> q = rp::project(P, X);
    T w[3], ew[3], pt[4];
    rp::apply_p(Y, X, w);
    rp::apply_e(q, w, ew);
    rp::apply_pt(P, ew, pt);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += pt[e];
  }
  T sv[4];
  rp::sym4_mul(g, acc, sv);
  const uint32_t row0 = sbeg / SLICE;
  for (uint32_t k = 0; k < width; ++k) {
    const bool in = k < len;
    const int i = in ? ld_stream(sell_cam + base + k * SLICE) : -1;
    const uint32_t mask = __ldg(row_mask + row0 + k), pbase = __ldg(row_base + row0 + k);
    T v[12];
#pragma unroll
    for (int e = 0; e < 12; ++e) v[e] = 0;
    if (in) {
      T P[12];
#pragma unroll
      for (int r = 0; r < 3; ++r) load_row<T>(camP, i, r, P + 4 * r);
      const rp::Proj<T> q = rp::project(P, X);
      T u[3], eu[3];
      rp::apply_p(P, sv, u);
      rp::apply_e(q, u, eu);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int d = 0; d < 4; ++d) v[4 * r + d] = eu[r] * X[d];
    }
    if (mask == 0u) {
      T r3[3];
      int vb;
      warp_reduce12<T>(v, lane, r3, vb);
      if ((lane & 7) == 0) {
        T* out = part + (size_t)pbase * 12 + vb;
        out[0] = r3[0]; out[1] = r3[1]; out[2] = r3[2];
      }
    } else {
      store_runs<T>(v, mask, in, pbase, lane, part);
    }
  }
}

// ---------------------------------------------------------------------------
// Group schedule (5). A group is a set of slices whose rows are all
// warp-uniform and whose row k sees the same camera in every slice of the
// group (landmarks whose tracks start at the same camera and run over the
// same cameras, as in video or trajectory capture; the layout starts a new
// slice at every smallest camera). One block per group:
//   staging: one thread issues bulk asynchronous copies (cp.async.bulk,
//            completion counted on an mbarrier) of every slice's
//            measurements, track lengths and landmark records (X, factor of
//            V^-1) into shared memory, while the block loads the P and Y
//            rows of the group's row cameras (the camera of a row comes from
//            the group's row table: no camera index is read per
//            observation);
//   phase 1: warp w takes slices w, w + 8, ... of the group; lane = landmark
//            j: t_j = sum_k Pbar_k^T C_k (Y_k x~_j), s_j = F_j^T F_j t_j,
//            all operands in shared memory;
//   phase 2: work items (row k, up to G5_ITEM slices of the group) strided
//            over the warps: each lane adds vec((C_k Pbar_k s_j) x~_j^T) of
//            its landmark in every slice of the item in registers, the warp
//            reduces once per item and writes the item's partial.
// Slices outside groups (a row whose lanes see several cameras) get blocks
// of their own in the same launch, whose 8 warps split the slice's rows: the
// per-lane track sums t_j of the warps are added in warp order, and every
// row writes its run partials as in the fused schedule. k_series_apply adds
// both kinds of partials per camera in a fixed order.
// ---------------------------------------------------------------------------

// All cameras' squared norms summed by threads [0, 32 NW) of the block in a
// fixed order (thread t takes cameras t, t + 32 NW, ...; the warps are
// combined in index order); the sums are valid in thread 0. Every thread of
// the block calls it (it holds a block barrier).
template <int NW>
__device__ __forceinline__ void camera_norm_sums(const double* __restrict__ camnorm, int nc,
                                                 double (*shn)[2], double& sy_out,
                                                 double& sd_out) {
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  double sy = 0.0, sd = 0.0;
  if (wl < NW) {
    for (int c0 = (int)threadIdx.x; c0 < nc; c0 += 4 * NW * 32) {
      double vy[4], vd[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * NW * 32;
        vy[u] = c < nc ? __ldcg(camnorm + 2 * (size_t)c) : 0.0;
        vd[u] = c < nc ? __ldcg(camnorm + 2 * (size_t)c + 1) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        sy += vy[u];
        sd += vd[u];
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    if (lane == 0) {
      shn[wl][0] = sy;
      shn[wl][1] = sd;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    sy = 0.0;
    sd = 0.0;
    for (int w = 0; w < NW; ++w) {
      sy += shn[w][0];
      sd += shn[w][1];
    }
  }
  sy_out = sy;
  sd_out = sd;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Wait for phase `parity` of `bar` with a bounded number of attempts (each
// attempt suspends the thread for a hardware-defined time); false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 22); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Landmark records of a group's slices staged in shared memory, in planes of
// G5_SLICES * 32 slots: FP32 (X0 X1 X2 F00)(F10 F11 F20 F21) as float4 and
// F22 as float; FP64 X (3 doubles) and F (6 doubles).
template <typename T> struct G5Pd;
template <> struct G5Pd<float> {
  static constexpr size_t N = (size_t)G5_SLICES * SLICE;
  static constexpr size_t BYTES = N * (16 + 16 + 4);
  static constexpr uint32_t SLICE_BYTES = SLICE * (16 + 16 + 4);
  static __device__ __forceinline__ void copy(unsigned char* base, int j,
                                              const PointData<float>& pd, uint32_t slot0,
                                              uint64_t* bar) {
    bulk_g2s(base + (size_t)j * SLICE * 16, pd.A + slot0, SLICE * 16, bar);
    bulk_g2s(base + N * 16 + (size_t)j * SLICE * 16, pd.B + slot0, SLICE * 16, bar);
    bulk_g2s(base + N * 32 + (size_t)j * SLICE * 4, pd.C + slot0, SLICE * 4, bar);
  }
  static __device__ __forceinline__ void load(const unsigned char* base, int e, float X[3],
                                              float F[6]) {
    const float4 p = reinterpret_cast<const float4*>(base)[e];
    const float4 q = reinterpret_cast<const float4*>(base + N * 16)[e];
    X[0] = p.x; X[1] = p.y; X[2] = p.z;
    F[0] = p.w; F[1] = q.x; F[2] = q.y; F[3] = q.z; F[4] = q.w;
    F[5] = reinterpret_cast<const float*>(base + N * 32)[e];
  }
  static __device__ __forceinline__ void loadX(const unsigned char* base, int e, float X[3]) {
    const float4 p = reinterpret_cast<const float4*>(base)[e];
    X[0] = p.x; X[1] = p.y; X[2] = p.z;
  }
};
template <> struct G5Pd<double> {
  static constexpr size_t N = (size_t)G5_SLICES * SLICE;
  static constexpr size_t BYTES = N * (24 + 48);
  static constexpr uint32_t SLICE_BYTES = SLICE * (24 + 48);
  static __device__ __forceinline__ void copy(unsigned char* base, int j,
                                              const PointData<double>& pd, uint32_t slot0,
                                              uint64_t* bar) {
    bulk_g2s(base + (size_t)j * SLICE * 24, pd.X + 3 * (size_t)slot0, SLICE * 24, bar);
    bulk_g2s(base + N * 24 + (size_t)j * SLICE * 48, pd.F + 6 * (size_t)slot0, SLICE * 48, bar);
  }
  static __device__ __forceinline__ void load(const unsigned char* base, int e, double X[3],
                                              double F[6]) {
    const double* x = reinterpret_cast<const double*>(base) + 3 * (size_t)e;
    const double* f = reinterpret_cast<const double*>(base + N * 24) + 6 * (size_t)e;
    X[0] = x[0]; X[1] = x[1]; X[2] = x[2];
#pragma unroll
    for (int k = 0; k < 6; ++k) F[k] = f[k];
  }
  static __device__ __forceinline__ void loadX(const unsigned char* base, int e, double X[3]) {
    const double* x = reinterpret_cast<const double*>(base) + 3 * (size_t)e;
    X[0] = x[0]; X[1] = x[1]; X[2] = x[2];
  }
};

// Row r (4 values) of the 3x4 camera block k staged in shared memory.
template <typename T>
__device__ __forceinline__ void srow(const T* tab, uint32_t k, int r, T out[4]);
template <>
__device__ __forceinline__ void srow<float>(const float* tab, uint32_t k, int r, float out[4]) {
  const float4 q = reinterpret_cast<const float4*>(tab + 12 * (size_t)k)[r];
  out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
}
template <>
__device__ __forceinline__ void srow<double>(const double* tab, uint32_t k, int r,
                                             double out[4]) {
  const double2* q = reinterpret_cast<const double2*>(tab + 12 * (size_t)k) + 2 * r;
  const double2 x = q[0], y = q[1];
  out[0] = x.x; out[1] = x.y; out[2] = y.x; out[3] = y.y;
}

// Dynamic shared memory of k_series_group (all offsets multiples of 16):
// mbarrier; camera rows P and Y per group row; staged measurements
// (G5_MROWS rows of 32); staged landmark records; s_j (3 planes); staged
// track lengths; per slice its index, first SELL entry, width and first
// staged measurement row; the group's work items and their partials'
// positions.
template <typename T> struct G5Layout {
  using M2 = typename Vt<T>::m2;
  static constexpr size_t BAR = 0;
  static constexpr size_t CP = 16;
  static constexpr size_t CY = CP + (size_t)G5_ROWS * 12 * sizeof(T);
  static constexpr size_t MEAS = CY + (size_t)G5_ROWS * 12 * sizeof(T);
  static constexpr size_t PD = MEAS + (size_t)G5_MROWS * SLICE * sizeof(M2);
  static constexpr size_t S = PD + G5Pd<T>::BYTES;
  static constexpr size_t LEN = S + 3 * (size_t)G5_SLICES * SLICE * sizeof(T);
  static constexpr size_t INFO = LEN + (size_t)G5_SLICES * SLICE * sizeof(uint32_t);
  static constexpr size_t ITEMS = INFO + 4 * (size_t)G5_SLICES * sizeof(uint32_t);
  static constexpr size_t IDEST = ITEMS + (size_t)G5_ROWS * sizeof(uint32_t);
  static constexpr size_t BYTES = IDEST + (size_t)G5_ROWS * sizeof(uint32_t);
};
// one item per group row: a row's slices (at most G5_SLICES) fit one item
static_assert(G5_SLICES <= G5_ITEM, "at most G5_ROWS items per group");
template <typename T>
constexpr size_t g5_smem_bytes() {
  return G5Layout<T>::BYTES;
}

// Tables of the group schedule passed to k_series_group.
struct G5Tables {
  const uint32_t* off;     // [ngroups + 1] slices of group g in slices
  const uint32_t* slices;  // slice indices, widest first
  const uint32_t* roff;    // [ngroups + 1] rows of group g in rowcam
  const int32_t* rowcam;   // camera of each group row
  const uint32_t* ioff;    // [ngroups + 1] items of group g
  const uint32_t* items;   // (row << 16) | (first slice << 8) | end slice
  const uint32_t* idest;   // per item: position of its partial (camera order)
  const uint32_t* rest;    // slices outside groups
  const uint4* sinfo;      // per group G5_SLICES entries (zero past its slices): slice,
                           // first SELL entry, width, first staged measurement row
  const int2* ghdr;        // per group: staged measurement rows, first row camera if the
                           // rows' cameras are consecutive (else -1)
  int ngroups;
};

template <typename T>
__device__ __forceinline__ void g5_group_block(
    DeviceState* __restrict__ st, T a, const uint32_t* __restrict__ slot_len,
    const uint32_t* __restrict__ sell_off, const typename Vt<T>::m2* __restrict__ sell_m,
    const T* __restrict__ camPa, const T* __restrict__ camPb, const T* __restrict__ vec,
    const PointData<T>& pd0, const PointData<T>& pd1, const G5Tables& tb, T* __restrict__ part,
    unsigned char* sm) {
  using L = G5Layout<T>;
  using M2 = typename Vt<T>::m2;
  constexpr int NW = G5_THREADS / 32;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + L::BAR);
  T* cP = reinterpret_cast<T*>(sm + L::CP);
  T* cY = reinterpret_cast<T*>(sm + L::CY);
  const M2* sm_m = reinterpret_cast<const M2*>(sm + L::MEAS);
  unsigned char* sm_pd = sm + L::PD;
  T* sS = reinterpret_cast<T*>(sm + L::S);
  const uint32_t* slen = reinterpret_cast<const uint32_t*>(sm + L::LEN);
  uint32_t* s_idx = reinterpret_cast<uint32_t*>(sm + L::INFO);
  uint32_t* s_off = s_idx + G5_SLICES;
  uint32_t* s_w = s_off + G5_SLICES;
  uint32_t* s_mrow = s_w + G5_SLICES;
  uint32_t* s_items = reinterpret_cast<uint32_t*>(sm + L::ITEMS);
  uint32_t* s_dest = reinterpret_cast<uint32_t*>(sm + L::IDEST);
  const int g = blockIdx.x, lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  // the group's table entries are at fixed offsets from g, so they load in
  // one round together with the state flags, before the copies are issued
  const uint32_t ns = __ldg(tb.off + g + 1) - __ldg(tb.off + g);
  const uint32_t rb = __ldg(tb.roff + g), nr = __ldg(tb.roff + g + 1) - rb;
  const uint32_t ib = __ldg(tb.ioff + g), ni = __ldg(tb.ioff + g + 1) - ib;
  const int2 hdr = __ldg(tb.ghdr + g);   // staged measurement rows, first row camera
  const uint4 info = wl == 0 && lane < G5_SLICES
                         ? __ldg(tb.sinfo + (size_t)g * G5_SLICES + lane)
                         : make_uint4(0, 0, 0, 0);
  if (st->converged || st->stop_series) return;
  const bool cur = st->cur != 0;
  const T* __restrict__ camP = cur ? camPb : camPa;
  const PointData<T>& pd = cur ? pd1 : pd0;

  if (wl == 0) {
    // lane j < ns: slice j's table entry (slice, first SELL entry, width,
    // first staged measurement row; the host keeps the rows within
    // G5_MROWS); lane 0 sets the expected byte count, then lane j issues the
    // bulk copies of slice j, and lane 0 those of the group's camera rows
    // when their cameras are consecutive
    if ((uint32_t)lane < ns) {
      s_idx[lane] = info.x;
      s_off[lane] = info.y;
      s_w[lane] = info.z;
      s_mrow[lane] = info.w;
    }
    if (lane == 0) {
      mbar_init(bar, 1);
      mbar_arrive_expect_tx(bar, (uint32_t)hdr.x * SLICE * (uint32_t)sizeof(M2) +
                                     ns * (G5Pd<T>::SLICE_BYTES + SLICE * 4u) +
                                     (hdr.y >= 0 ? 2u * nr * 12u * (uint32_t)sizeof(T) : 0u));
    }
    __syncwarp();
    if ((uint32_t)lane < ns) {
      const uint32_t j = (uint32_t)lane, slot0 = info.x * SLICE;
      bulk_g2s(sm + L::MEAS + (size_t)info.w * SLICE * sizeof(M2), sell_m + info.y,
               info.z * SLICE * (uint32_t)sizeof(M2), bar);
      bulk_g2s(sm + L::LEN + (size_t)j * SLICE * 4, slot_len + slot0, SLICE * 4, bar);
      G5Pd<T>::copy(sm_pd, (int)j, pd, slot0, bar);
    }
    if (lane == 0 && hdr.y >= 0) {
      bulk_g2s(cP, camP + 12 * (size_t)hdr.y, nr * 12u * (uint32_t)sizeof(T), bar);
      bulk_g2s(cY, vec + 12 * (size_t)hdr.y, nr * 12u * (uint32_t)sizeof(T), bar);
    }
  }
  // the group's work items while the copies are in flight
  for (uint32_t q = threadIdx.x; q < ni; q += G5_THREADS) {
    s_items[q] = __ldg(tb.items + ib + q);
    s_dest[q] = __ldg(tb.idest + ib + q);
  }
  if (hdr.y < 0) {
    // camera rows of the group rows (not consecutive cameras) while the
    // copies are in flight
    for (uint32_t q = threadIdx.x; q < nr * 24; q += G5_THREADS) {
      const uint32_t r = q / 24, e = q % 24;
      const size_t c = (size_t)__ldg(tb.rowcam + rb + r);
      if (e < 12)
        cP[12 * r + e] = camP[12 * c + e];
      else
        cY[12 * r + e - 12] = vec[12 * c + e - 12];
    }
  }
  __syncthreads();
  const bool arrived = mbar_wait_bounded(bar, 0);
  if (__syncthreads_or(!arrived)) {
    // the copies did not complete in time (in any thread's view): report
    // it, wait once more for them (bounded) so that none lands after the
    // block has exited, and skip the group
    if (threadIdx.x == 0) st->error = POVAR_ETIMEOUT;
    mbar_wait_bounded(bar, 0);
    return;
  }

  // phase 1: s_j of every landmark of the group
  for (uint32_t j = wl; j < ns; j += NW) {
    const int e = (int)(j * SLICE) + lane;
    const uint32_t width = s_w[j], len = slen[e];
    const M2* mrow = sm_m + (size_t)s_mrow[j] * SLICE + lane;
    T X[3], F[6];
    G5Pd<T>::load(sm_pd, e, X, F);
    T t[3] = {0, 0, 0};
    // branch-free over the rows: a lane past its track length adds its
    // contribution scaled by 0 (its staged measurement is the zero padding)
    for (uint32_t k = 0; k < width; ++k) {
      const M2 m = mrow[k * SLICE];
      const T f = k < len ? (T)1 : (T)0;
      const T Xf[3] = {f * X[0], f * X[1], f * X[2]};
      T Y0[4], Y1[4], Y2[4], P0[4], P1[4], P2[4];
      srow<T>(cY, k, 0, Y0);
      srow<T>(cY, k, 1, Y1);
      srow<T>(cY, k, 2, Y2);
      srow<T>(cP, k, 0, P0);
      srow<T>(cP, k, 1, P1);
      srow<T>(cP, k, 2, P2);
      // e = Y (f x~): the homogeneous 1 of x~ is scaled by f as well
      Y0[3] *= f;
      Y1[3] *= f;
      Y2[3] *= f;
      gather_obs<T>(Y0, Y1, Y2, P0, P1, P2, a, (T)m.x, (T)m.y, Xf, t);
    }
    const T z0 = F[0] * t[0];
    const T z1 = F[1] * t[0] + F[2] * t[1];
    const T z2 = F[3] * t[0] + F[4] * t[1] + F[5] * t[2];
    sS[e] = F[0] * z0 + F[1] * z1 + F[3] * z2;
    sS[G5_SLICES * SLICE + e] = F[2] * z1 + F[4] * z2;
    sS[2 * G5_SLICES * SLICE + e] = F[5] * z2;
  }
  __syncthreads();

  // phase 2: one partial per work item
  for (uint32_t it = wl; it < ni; it += NW) {
    const uint32_t item = s_items[it];
    const uint32_t k = item >> 16, j0 = (item >> 8) & 0xffu, j1 = item & 0xffu;
    T P0[4], P1[4], P2[4];
    srow<T>(cP, k, 0, P0);
    srow<T>(cP, k, 1, P1);
    srow<T>(cP, k, 2, P2);
    T v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = 0;
    for (uint32_t j = j0; j < j1; ++j) {
      // branch-free: a lane past its track length adds its contribution
      // scaled by 0 (s_j scaled; its staged measurement is zero padding)
      const int e = (int)(j * SLICE) + lane;
      const T f = k < slen[e] ? (T)1 : (T)0;
      const M2 m = sm_m[((size_t)s_mrow[j] + k) * SLICE + lane];
      T X[3];
      G5Pd<T>::loadX(sm_pd, e, X);
      const T S[3] = {f * sS[e], f * sS[G5_SLICES * SLICE + e],
                      f * sS[2 * G5_SLICES * SLICE + e]};
      scatter_obs<T>(P0, P1, P2, a, (T)m.x, (T)m.y, S, X, v);
    }
    T r[3];
    int vb;
    warp_reduce12<T>(v, lane, r, vb);
    if ((lane & 7) == 0) {
      T* out = part + (size_t)s_dest[it] * 12 + vb;
      out[0] = r[0];
      out[1] = r[1];
      out[2] = r[2];
    }
  }
}

// A slice outside the groups (some row's lanes see several cameras), one
// block: warp w takes rows w, w + 8, ... In the first pass each warp sums
// its rows' part of t_j per lane; the 8 warp sums are added in warp order,
// s_j = F_j^T F_j t_j. In the second pass every row writes its run partials
// (one per run of equal cameras, as the fused schedule).
template <typename T>
__device__ __forceinline__ void g5_rest_block(
    T a, const uint32_t* __restrict__ slot_len, const uint32_t* __restrict__ sell_off,
    const int32_t* __restrict__ sell_cam, const typename Vt<T>::m2* __restrict__ sell_m,
    const T* __restrict__ camP, const T* __restrict__ vec, const PointData<T>& pd,
    const uint32_t* __restrict__ row_mask, const uint32_t* __restrict__ row_base,
    uint32_t slice, T* __restrict__ part_run, unsigned char* sm) {
  using M2 = typename Vt<T>::m2;
  constexpr int NW = G5_THREADS / 32;
  T* tp = reinterpret_cast<T*>(sm + G5Layout<T>::MEAS);   // [NW][3][32]
  T* sS = tp + NW * 3 * SLICE;                              // [3][32]
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const uint32_t slot = slice * SLICE + (uint32_t)lane;
  const uint32_t sbeg = sell_off[slice];
  const uint32_t width = (sell_off[slice + 1] - sbeg) / SLICE;
  const uint32_t len = slot_len[slot];
  const uint32_t base = sbeg + (uint32_t)lane;
  T X[3], F[6];
  load_point<T>(pd, (int)slot, X, F);
  T t[3] = {0, 0, 0};
  for (uint32_t k = (uint32_t)wl; k < width; k += NW) {
    if (k < len) {
      const int i = ld_stream(sell_cam + base + k * SLICE);
      const M2 m = ld_stream(sell_m + base + k * SLICE);
      T Y0[4], Y1[4], Y2[4], P0[4], P1[4], P2[4];
      load_row<T>(vec, i, 0, Y0);
      load_row<T>(vec, i, 1, Y1);
      load_row<T>(vec, i, 2, Y2);
      load_row<T>(camP, i, 0, P0);
      load_row<T>(camP, i, 1, P1);
      load_row<T>(camP, i, 2, P2);
      gather_obs<T>(Y0, Y1, Y2, P0, P1, P2, a, (T)m.x, (T)m.y, X, t);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) tp[(wl * 3 + c) * SLICE + lane] = t[c];
  __syncthreads();
  if (wl == 0) {
    T u[3] = {0, 0, 0};
    for (int w = 0; w < NW; ++w)
#pragma unroll
      for (int c = 0; c < 3; ++c) u[c] += tp[(w * 3 + c) * SLICE + lane];
    const T z0 = F[0] * u[0];
    const T z1 = F[1] * u[0] + F[2] * u[1];
    const T z2 = F[3] * u[0] + F[4] * u[1] + F[5] * u[2];
    sS[lane] = F[0] * z0 + F[1] * z1 + F[3] * z2;
    sS[SLICE + lane] = F[2] * z1 + F[4] * z2;
    sS[2 * SLICE + lane] = F[5] * z2;
  }
  __syncthreads();
  const T S[3] = {sS[lane], sS[SLICE + lane], sS[2 * SLICE + lane]};
  const uint32_t row0 = sbeg / SLICE;
  for (uint32_t k = (uint32_t)wl; k < width; k += NW) {
    const uint32_t mask = __ldg(row_mask + row0 + k), pbase = __ldg(row_base + row0 + k);
    const int i = k < len ? ld_stream(sell_cam + base + k * SLICE) : -1;
    T v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = 0;
    if (i >= 0) {
      const M2 m = ld_stream(sell_m + base + k * SLICE);
      T P0[4], P1[4], P2[4];
      load_row<T>(camP, i, 0, P0);
      load_row<T>(camP, i, 1, P1);
      load_row<T>(camP, i, 2, P2);
      scatter_obs<T>(P0, P1, P2, a, (T)m.x, (T)m.y, S, X, v);
    }
    if (mask == 0u) {
      T r[3];
      int vb;
      warp_reduce12<T>(v, lane, r, vb);
      if ((lane & 7) == 0) {
        T* out = part_run + (size_t)pbase * 12 + vb;
        out[0] = r[0];
        out[1] = r[1];
        out[2] = r[2];
      }
    } else {
      store_runs<T>(v, mask, i >= 0, pbase, lane, part_run);
    }
  }
}

// The threshold rule of the series for the previous term (term - 1 >= 1),
// checked by block 0 of the term's group launch: the same sums in the same
// order as the last camera block of a per-camera finish would take them
// (camera_norm_sums over 4 warps); sets series_halt, which the term's
// camera finish reads. The finish kernels then need no ticket.
__device__ __forceinline__ void series_halt_check(DeviceState* __restrict__ st, int term,
                                                  double eps,
                                                  const double* __restrict__ camnorm, int nc) {
  __shared__ double shn[4][2];
  const bool check = term >= 2 && eps > 0.0 && !(st->converged || st->stop_series);
  double sy = 0.0, sd = 0.0;
  if (check) camera_norm_sums<4>(camnorm, nc, shn, sy, sd);
  if (threadIdx.x == 0) st->series_halt = check && sy <= eps * eps * sd ? 1 : 0;
}

// Blocks [0, ngroups) run the groups, the next ones the slices outside
// groups. part holds the item partials at their positions in the per-camera
// lists; the run partials of the slices outside groups go to part_run.
template <typename T>
__global__ void __launch_bounds__(G5_THREADS, sizeof(T) == 4 ? 3 : 1)
k_series_group(DeviceState* __restrict__ st, T a, const uint32_t* __restrict__ slot_len,
               const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
               const typename Vt<T>::m2* __restrict__ sell_m, const T* __restrict__ camPa,
               const T* __restrict__ camPb, const T* __restrict__ vec, PointData<T> pd0,
               PointData<T> pd1, G5Tables tb, const uint32_t* __restrict__ row_mask,
               const uint32_t* __restrict__ row_base, T* __restrict__ part,
               T* __restrict__ part_run, int term, double eps,
               const double* __restrict__ camnorm, int nc) {
  extern __shared__ __align__(16) unsigned char g5_smem[];
  if (blockIdx.x == 0) series_halt_check(st, term, eps, camnorm, nc);
  if ((int)blockIdx.x < tb.ngroups) {
    g5_group_block<T>(st, a, slot_len, sell_off, sell_m, camPa, camPb, vec, pd0, pd1, tb, part,
                      g5_smem);
  } else {
    if (st->converged || st->stop_series) return;
    const T* __restrict__ camP = st->cur ? camPb : camPa;
    const PointData<T>& pd = st->cur ? pd1 : pd0;
    g5_rest_block<T>(a, slot_len, sell_off, sell_cam, sell_m, camP, vec, pd, row_mask, row_base,
                     __ldg(tb.rest + (blockIdx.x - tb.ngroups)), part_run, g5_smem);
  }
}

// Per camera (k_series_apply, one block of 4 warps): z_i = sum of its
// partials in list order, then the camera update. With the threshold rule,
// the block that finishes last (atomic ticket) adds all cameras' norms and
// sets the stop flag (stop_check); in the group schedule the next term's
// group launch adds them instead (series_halt_check) and the block only
// stores its camera's norms.
template <typename T> struct Rec12;
template <> struct Rec12<float> {
  static __device__ __forceinline__ void add(const float* src, float acc[12]) {
    const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float4 x = __ldcg(q + r);
      acc[4 * r] += x.x; acc[4 * r + 1] += x.y; acc[4 * r + 2] += x.z; acc[4 * r + 3] += x.w;
    }
  }
};
template <> struct Rec12<double> {
  static __device__ __forceinline__ void add(const double* src, double acc[12]) {
    const double2* q = reinterpret_cast<const double2*>(src);
#pragma unroll
    for (int r = 0; r < 6; ++r) {
      const double2 x = __ldcg(q + r);
      acc[2 * r] += x.x; acc[2 * r + 1] += x.y;
    }
  }
};

// Threshold rule of the series (stop after term k when ||x_k|| <= eps
// ||delta_k||): every camera block stores the two squared norms of its
// camera; the block that arrives last on the ticket adds all cameras'
// norms (camera_norm_sums) and sets the stop flag. Thread 0 of the block
// holds the camera's norms on entry.
template <int NW>
__device__ __forceinline__ void stop_check(DeviceState* __restrict__ st, int term, double eps,
                                           int nc, int i, double yy, double dd,
                                           double* __restrict__ camnorm,
                                           uint32_t* __restrict__ done_ticket, int* sh_last,
                                           double (*shn)[2]) {
  if (threadIdx.x == 0) {
    camnorm[2 * (size_t)i] = yy;
    camnorm[2 * (size_t)i + 1] = dd;
    __threadfence();
    *sh_last = atomicAdd(done_ticket, 1u) == (unsigned)(nc - 1);
  }
  __syncthreads();
  if (!*sh_last) return;
  __threadfence();
  double sy, sd;
  camera_norm_sums<NW>(camnorm, nc, shn, sy, sd);
  if (threadIdx.x == 0) {
    *done_ticket = 0;
    if (sy <= eps * eps * sd) {
      st->stop_series = 1;
      st->terms_used = term + 1;
    }
  }
}

// Blocks per SM: twelve in FP32 (40 registers, a few spilled), so that a
// camera count up to 12 x the SM count (1,824 on 152 SMs) runs in one wave
// instead of 1.3; six in FP64 (80 registers, as without a bound).
//
// With cam_ndirect (group schedule), the first cam_ndirect[i] entries of
// camera i's list are partials stored at their own list position (entry q
// reads part[q], the index table holds q there), so they are read without
// the index load; the others through the index table.
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 12 : 6)
k_series_apply(DeviceState* __restrict__ st, int term, double eps, int nc,
               const uint32_t* __restrict__ cam_part_off, const uint32_t* __restrict__ cam_part_idx,
               const uint32_t* __restrict__ cam_ndirect, const T* __restrict__ part,
               const T* __restrict__ G, double* __restrict__ camnorm,
               uint32_t* __restrict__ done_ticket, T* __restrict__ Y, T* __restrict__ D,
               int late_check) {
  // one block of 4 warps per camera: each warp adds a strided quarter of the
  // camera's partials, the four warp sums are combined in a fixed order;
  // warp 0 loads the camera's row of G and of delta before the partials
  // arrive, so the update waits on no further load
  __shared__ T sh[4][12];
  __shared__ int sh_last;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x;
  const uint32_t b = __ldg(cam_part_off + i), e_ = __ldg(cam_part_off + i + 1);
  const uint32_t bd = cam_ndirect ? b + __ldg(cam_ndirect + i) : b;
  if (st->converged || st->stop_series) return;
  if (late_check && st->series_halt) {
    // the threshold rule held after the previous term (checked by this
    // term's group launch): the series ends with that term
    if (i == 0 && threadIdx.x == 0) {
      st->stop_series = 1;
      st->terms_used = term;
    }
    return;
  }
  T g[12], dprev = 0;
  if (wl == 0) {
    Row12<T>::load(G + 144 * (size_t)i + 12 * (lane < 12 ? lane : 0), g);
    if (lane < 12) dprev = D[12 * (size_t)i + lane];
  }
  T acc[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) acc[e] = 0;
  uint32_t q = b + threadIdx.x;
  for (; q + 128 < e_; q += 256) {
    const uint32_t i0 = q < bd ? q : __ldg(cam_part_idx + q);
    const uint32_t i1 = q + 128 < bd ? q + 128 : __ldg(cam_part_idx + q + 128);
    Rec12<T>::add(part + (size_t)i0 * 12, acc);
    Rec12<T>::add(part + (size_t)i1 * 12, acc);
  }
  if (q < e_) Rec12<T>::add(part + (size_t)(q < bd ? q : __ldg(cam_part_idx + q)) * 12, acc);
  {
    T r[3];
    int vb;
    warp_reduce12<T>(acc, lane, r, vb);
    if ((lane & 7) == 0) {
      sh[wl][vb] = r[0];
      sh[wl][vb + 1] = r[1];
      sh[wl][vb + 2] = r[2];
    }
  }
  __syncthreads();
  constexpr int NWARPS = 4;
  __shared__ double shn[NWARPS][2];
  double yy = 0.0, dd = 0.0;
  if (wl == 0) {
    T z = 0;
    if (lane < 12) z = ((sh[0][lane] + sh[1][lane]) + sh[2][lane]) + sh[3][lane];
    // x_i = G_i z_i, delta_i += x_i, Y_i = x_i
    T x = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) x += g[c] * __shfl_sync(0xffffffffu, z, c);
    T y2 = 0, d2 = 0;
    if (lane < 12) {
      const T d = dprev + x;
      D[12 * (size_t)i + lane] = d;
      Y[12 * (size_t)i + lane] = x;
      y2 = x * x;
      d2 = d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      y2 += __shfl_xor_sync(0xffffffffu, y2, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
    }
    yy = (double)y2;
    dd = (double)d2;
  }
  if (eps <= 0.0) return;
  if (late_check) {
    // the next term's group launch adds the norms (camera_norm_sums)
    if (threadIdx.x == 0) {
      camnorm[2 * (size_t)i] = yy;
      camnorm[2 * (size_t)i + 1] = dd;
    }
    return;
  }
  stop_check<NWARPS>(st, term, eps, nc, i, yy, dd, camnorm, done_ticket, &sh_last, shn);
}

// ---------------------------------------------------------------------------
// Camera-row schedule (2): after the landmark-major gather has written every
// landmark's record (s_j, X_j), one block per camera walks the slice rows
// that contain the camera (rows in index order, strided over the NW warps).
// Each lane adds the contribution vec((C_k Pbar_i s_j) x~_j^T) of its own
// landmark when that landmark's observation in the row is of this camera, so
// contributions accumulate in registers across rows; the block reduces once
// per camera, in a fixed order, and applies the camera update.
// ---------------------------------------------------------------------------
template <typename T, int NW>
__global__ void __launch_bounds__(NW * 32)
k_series_camrows(DeviceState* __restrict__ st, T a, int term, double eps, int nc,
                 const uint32_t* __restrict__ cam_row_off,
                 const uint32_t* __restrict__ cam_row_pos0,
                 const uint32_t* __restrict__ cam_row_slot0, const int32_t* __restrict__ sell_cam,
                 const typename Vt<T>::m2* __restrict__ sell_m, const T* __restrict__ camPa,
                 const T* __restrict__ camPb, const float4* __restrict__ rec32,
                 const double2* __restrict__ rec64, const T* __restrict__ G,
                 double* __restrict__ camnorm, uint32_t* __restrict__ done_ticket,
                 T* __restrict__ Y, T* __restrict__ D) {
  if (st->converged || st->stop_series) return;
  __shared__ T sh[NW][12];
  __shared__ int sh_last;
  using M2 = typename Vt<T>::m2;
  constexpr int RB = 4;
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x;
  const T* __restrict__ camP = st->cur ? camPb : camPa;
  T P0[4], P1[4], P2[4];
  load_row<T>(camP, i, 0, P0);
  load_row<T>(camP, i, 1, P1);
  load_row<T>(camP, i, 2, P2);
  T acc[12];
#pragma unroll
  for (int e = 0; e < 12; ++e) acc[e] = 0;
  const uint32_t b = cam_row_off[i], e_ = cam_row_off[i + 1];
  for (uint32_t q0 = b + wl; q0 < e_; q0 += NW * RB) {
    uint32_t pos[RB], slot[RB];
    int cv[RB];
    M2 mv[RB];
    T S[RB][3], X[RB][3];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const uint32_t q = q0 + NW * u;
      const bool in = q < e_;
      pos[u] = in ? __ldg(cam_row_pos0 + q) + lane : 0u;
      slot[u] = in ? __ldg(cam_row_slot0 + q) + lane : 0u;
      cv[u] = in ? ld_stream(sell_cam + pos[u]) : -1;
      mv[u] = in ? ld_stream(sell_m + pos[u]) : M2{0, 0};
      if (in) load_rec(rec32, rec64, slot[u], S[u], X[u]);
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      if (cv[u] != i) continue;
      const T w0 = P0[0] * S[u][0] + P0[1] * S[u][1] + P0[2] * S[u][2];
      const T w1 = P1[0] * S[u][0] + P1[1] * S[u][1] + P1[2] * S[u][2];
      const T w2 = P2[0] * S[u][0] + P2[1] * S[u][1] + P2[2] * S[u][2];
      const T au = a * (T)mv[u].x, av = a * (T)mv[u].y;
      const T aw = au * (T)mv[u].x + av * (T)mv[u].y;
      const T q0v = w0 - au * w2;
      const T q1v = w1 - av * w2;
      const T q2v = aw * w2 - au * w0 - av * w1;
      acc[0] += q0v * X[u][0]; acc[1] += q0v * X[u][1]; acc[2] += q0v * X[u][2]; acc[3] += q0v;
      acc[4] += q1v * X[u][0]; acc[5] += q1v * X[u][1]; acc[6] += q1v * X[u][2]; acc[7] += q1v;
      acc[8] += q2v * X[u][0]; acc[9] += q2v * X[u][1]; acc[10] += q2v * X[u][2]; acc[11] += q2v;
    }
  }
  T r[3];
  int vb;
  warp_reduce12<T>(acc, lane, r, vb);
  if ((lane & 7) == 0) {
    sh[wl][vb] = r[0];
    sh[wl][vb + 1] = r[1];
    sh[wl][vb + 2] = r[2];
  }
  __syncthreads();
  constexpr int NWARPS = NW;
  __shared__ double shn[NWARPS][2];
  double yy = 0.0, dd = 0.0;
  if (wl == 0) {
    T z = 0;
    if (lane < 12) {
#pragma unroll
      for (int w = 0; w < NW; ++w) z += sh[w][lane];
    }
    camera_update<T>(i, lane, z, G, Y, D, yy, dd);
  }
  if (eps <= 0.0) return;
  stop_check<NWARPS>(st, term, eps, nc, i, yy, dd, camnorm, done_ticket, &sh_last, shn);
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

// Per camera (one warp): d^T U d and b_p^T d in FP64 into camnorm[2i], [2i+1].
template <typename T>
__global__ void __launch_bounds__(256)
k_pred_cam(const DeviceState* __restrict__ st, int nc, const double* __restrict__ U64,
           const double* __restrict__ bp64, const T* __restrict__ D,
           double* __restrict__ camsum) {
  if (st->converged) return;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= nc) return;
  const double d = lane < 12 ? (double)D[12 * (size_t)i + lane] : 0.0;
  double su = 0.0;
  for (int q = 0; q < 12; ++q) {
    const double dq = __shfl_sync(0xffffffffu, d, q);
    if (lane < 12) su += U64[144 * (size_t)i + 12 * lane + q] * dq;
  }
  double du = d * su;
  double bd = lane < 12 ? bp64[12 * (size_t)i + lane] * d : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    du += __shfl_xor_sync(0xffffffffu, du, o);
    bd += __shfl_xor_sync(0xffffffffu, bd, o);
  }
  if (lane == 0) {
    camsum[2 * (size_t)i] = du;
    camsum[2 * (size_t)i + 1] = bd;
  }
}

// pred = -2 b_p^T d - d^T U d + sum_j ||F_j W^T d||^2, fixed-order sums.
// pred = sum of the per-warp partials ||F_j W^T d||^2 minus the camera terms
// d^T U d + 2 b_p^T d, over FIN_BLOCKS blocks with a fixed-order last-block
// finish (as k_cost_finish).
__global__ void __launch_bounds__(256)
k_pred_finish(DeviceState* __restrict__ st, int nc, int nparts, int m,
              const double* __restrict__ pred_part, const double* __restrict__ camsum,
              double* __restrict__ blk, uint32_t* __restrict__ ticket) {
  if (st->converged) return;
  __shared__ double red[256];
  __shared__ int last;
  const int per = (nparts + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b0 = (int)blockIdx.x * per, b1 = min(nparts, b0 + per);
  double v = 0.0;
  for (int q = b0 + (int)threadIdx.x; q < b1; q += 256) v += pred_part[q];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    blk[blockIdx.x] = red[0];
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  v = 0.0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += 256) v += __ldcg(blk + q);
  for (int i = threadIdx.x; i < nc; i += 256)
    v -= camsum[2 * (size_t)i] + 2.0 * camsum[2 * (size_t)i + 1];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *ticket = 0u;
    st->pred = red[0];
    if (!st->stop_series) st->terms_used = m;
  }
}

// ---------------------------------------------------------------------------
// Schedule 3 (row table). Creation groups slices (GROUP per warp, see
// povar_internal.cuh) and gives every group row whose valid lanes all see
// one camera that camera and its partial; other rows keep the run
// description of the fused schedule. Helpers shared with its kernel below.
// ---------------------------------------------------------------------------
// Per warp, 32 group rows at a time: the rows' cameras are read with one
// coalesced load (lane r holds the camera of row r0 + r) and the rows Y_i, P_i
// of every uniform row's camera are staged in shared memory by the lanes in
// parallel, so the row loop waits on no dependent global load; the
// measurements of the next row are loaded while the current one is computed.
template <typename T>
struct GroupStage {
  T cam[BLOCK / SLICE][SLICE][24];  // per warp, per staged row: Y rows (12) then P rows (12)
};

template <typename T>
__device__ __forceinline__ void stage_rows(T (*dst)[24], const int32_t* __restrict__ grow_cam,
                                           uint32_t rbeg, uint32_t nrow, const T* __restrict__ vec,
                                           const T* __restrict__ camP, bool with_y, int lane,
                                           int& gc) {
  __syncwarp();  // every lane is done with the previously staged rows
  gc = lane < (int)nrow ? __ldg(grow_cam + rbeg + lane) : -1;
  if (gc >= 0) {
    T row[4];
    if (with_y) {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        load_row<T>(vec, gc, q, row);
#pragma unroll
        for (int e = 0; e < 4; ++e) dst[lane][4 * q + e] = row[e];
      }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      load_row<T>(camP, gc, q, row);
#pragma unroll
      for (int e = 0; e < 4; ++e) dst[lane][12 + 4 * q + e] = row[e];
    }
  }
  __syncwarp();
}

static_assert(GROUP == 1, "k_series_rows takes one slice per group");

// Row-pair schedule (3) with one slice per warp: the per-row camera table
// of the grouped layout (GROUP = 1) gives every uniform slice row its camera
// without a dependent load, the rows of those cameras are staged in shared
// memory 32 rows at a time, the measurements of RB rows are loaded together,
// and in pass 2 two consecutive uniform rows are reduced across the warp
// together (27 shuffles for the pair instead of 18 per row). The row loops
// run over the slice width for all lanes (a lane past its track length
// contributes nothing), so every shuffle is executed by the whole warp.
// Rows that are not uniform take the per-lane camera and run path of the
// fused schedule.
template <typename T>
__global__ void __launch_bounds__(BLOCK)
k_series_rows(const DeviceState* __restrict__ st, T a, const uint32_t* __restrict__ slot_len,
              const uint32_t* __restrict__ sell_off, const int32_t* __restrict__ sell_cam,
              const typename Vt<T>::m2* __restrict__ sell_m, const T* __restrict__ camPa,
              const T* __restrict__ camPb, const T* __restrict__ vec, PointData<T> pd0,
              PointData<T> pd1, const uint32_t* __restrict__ grp_slice0,
              const uint32_t* __restrict__ grp_row0, int ngroups,
              const int32_t* __restrict__ grow_cam, const uint32_t* __restrict__ grow_base,
              const uint32_t* __restrict__ srow_mask, const uint32_t* __restrict__ srow_base,
              T* __restrict__ part) {
  __shared__ __align__(16) GroupStage<T> stage;
  if (st->converged || st->stop_series) return;
  const int wl = (int)(threadIdx.x >> 5);
  const int g = blockIdx.x * (BLOCK / SLICE) + wl;
  if (g >= ngroups) return;  // whole warp (no block-level barrier below)
  const int lane = threadIdx.x & 31;
  using M2 = typename Vt<T>::m2;
  constexpr int RB = 4;
  T (*sm)[24] = stage.cam[wl];
  const PointData<T>& pd = st->cur ? pd1 : pd0;
  const T* __restrict__ camP = st->cur ? camPb : camPa;
  const uint32_t s = grp_slice0[g];  // one slice per group
  const uint32_t r0 = grp_row0[g], W = grp_row0[g + 1] - r0;
  const uint32_t sb = sell_off[s];
  const uint32_t len = slot_len[s * SLICE + lane];
  const uint32_t base = sb + (uint32_t)lane;
  T X[3];
  {
    T F0[6];
    load_point<T>(pd, (int)(s * SLICE) + lane, X, F0);
  }
  T t[3] = {0, 0, 0};
  int gc = -1;
  // pass 1: t_j = sum over the landmark's observations of Pbar^T C (Y x~_j)
  for (uint32_t c0 = 0; c0 < W; c0 += SLICE) {
    const uint32_t nr = min(W - c0, (uint32_t)SLICE);
    stage_rows<T>(sm, grow_cam, r0 + c0, nr, vec, camP, true, lane, gc);
    for (uint32_t k0 = 0; k0 < nr; k0 += RB) {
      M2 m[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        const uint32_t r = c0 + k0 + u;
        m[u] = (k0 + u < nr && r < len) ? ld_stream(sell_m + base + r * SLICE) : M2{0, 0};
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        if (k0 + u >= nr) break;  // warp-uniform
        const uint32_t r = c0 + k0 + u;
        const int c = __shfl_sync(0xffffffffu, gc, (int)(k0 + u));
        if (c >= 0) {
          if (r < len) {
            const T* q = sm[k0 + u];
            T Y0[4], Y1[4], Y2[4], P0[4], P1[4], P2[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              Y0[e] = q[e]; Y1[e] = q[4 + e]; Y2[e] = q[8 + e];
              P0[e] = q[12 + e]; P1[e] = q[16 + e]; P2[e] = q[20 + e];
            }
            gather_obs<T>(Y0, Y1, Y2, P0, P1, P2, a, (T)m[u].x, (T)m[u].y, X, t);
          }
        } else if (r < len) {
          const int i = ld_stream(sell_cam + base + r * SLICE);
          T Y0[4], Y1[4], Y2[4], P0[4], P1[4], P2[4];
          load_row<T>(vec, i, 0, Y0);
          load_row<T>(vec, i, 1, Y1);
          load_row<T>(vec, i, 2, Y2);
          load_row<T>(camP, i, 0, P0);
          load_row<T>(camP, i, 1, P1);
          load_row<T>(camP, i, 2, P2);
          gather_obs<T>(Y0, Y1, Y2, P0, P1, P2, a, (T)m[u].x, (T)m[u].y, X, t);
        }
      }
    }
  }
  // s_j = V_j^-1 t_j = F^T (F t_j)
  T S[3];
  {
    T Xk[3], F[6];
    load_point<T>(pd, (int)(s * SLICE) + lane, Xk, F);
    const T z0 = F[0] * t[0];
    const T z1 = F[1] * t[0] + F[2] * t[1];
    const T z2 = F[3] * t[0] + F[4] * t[1] + F[5] * t[2];
    S[0] = F[0] * z0 + F[1] * z1 + F[3] * z2;
    S[1] = F[2] * z1 + F[4] * z2;
    S[2] = F[5] * z2;
  }
  // pass 2: camera contributions vec((C Pbar s_j) x~_j^T); the staged rows of
  // the first 32 rows are still in place when W <= 32
  for (uint32_t c0 = 0; c0 < W; c0 += SLICE) {
    const uint32_t nr = min(W - c0, (uint32_t)SLICE);
    if (W > (uint32_t)SLICE)
      stage_rows<T>(sm, grow_cam, r0 + c0, nr, vec, camP, false, lane, gc);
    for (uint32_t k4 = 0; k4 < nr; k4 += 4) {
      // the measurements of up to four rows are loaded together
      M2 m4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t r = c0 + k4 + u;
        m4[u] = (k4 + u < nr && r < len) ? ld_stream(sell_m + base + r * SLICE) : M2{0, 0};
      }
#pragma unroll
      for (int pr = 0; pr < 2; ++pr) {
      const uint32_t k0 = k4 + 2 * pr;
      if (k0 >= nr) break;  // warp-uniform
      const bool two = k0 + 1 < nr;
      const uint32_t rA = c0 + k0, rB = rA + 1;
      const int cA = __shfl_sync(0xffffffffu, gc, (int)k0);
      const int cB = __shfl_sync(0xffffffffu, gc, two ? (int)k0 + 1 : (int)k0);
      const M2 mA = m4[2 * pr], mB = m4[2 * pr + 1];
      if (two && cA >= 0 && cB >= 0) {
        T vA[12], vB[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) vA[e] = vB[e] = 0;
        if (rA < len) {
          const T* q = sm[k0];
          const T P0[4] = {q[12], q[13], q[14], q[15]}, P1[4] = {q[16], q[17], q[18], q[19]},
                  P2[4] = {q[20], q[21], q[22], q[23]};
          scatter_obs<T>(P0, P1, P2, a, (T)mA.x, (T)mA.y, S, X, vA);
        }
        if (rB < len) {
          const T* q = sm[k0 + 1];
          const T P0[4] = {q[12], q[13], q[14], q[15]}, P1[4] = {q[16], q[17], q[18], q[19]},
                  P2[4] = {q[20], q[21], q[22], q[23]};
          scatter_obs<T>(P0, P1, P2, a, (T)mB.x, (T)mB.y, S, X, vB);
        }
        T red[3];
        int rowb, vb;
        warp_reduce24<T>(vA, vB, lane, red, rowb, vb);
        if ((lane & 3) == 0) {
          T* out = part + (size_t)__ldg(grow_base + r0 + (rowb ? rB : rA)) * 12 + vb;
          out[0] = red[0];
          out[1] = red[1];
          out[2] = red[2];
        }
        continue;
      }
      // rows one at a time (an odd last row or a row that is not uniform)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;  // warp-uniform
        const uint32_t r = h ? rB : rA;
        const int c = h ? cB : cA;
        const M2 mr = h ? mB : mA;
        T v[12];
#pragma unroll
        for (int e = 0; e < 12; ++e) v[e] = 0;
        if (c >= 0) {
          if (r < len) {
            const T* q = sm[k0 + h];
            const T P0[4] = {q[12], q[13], q[14], q[15]}, P1[4] = {q[16], q[17], q[18], q[19]},
                    P2[4] = {q[20], q[21], q[22], q[23]};
            scatter_obs<T>(P0, P1, P2, a, (T)mr.x, (T)mr.y, S, X, v);
          }
          T red[3];
          int vb;
          warp_reduce12<T>(v, lane, red, vb);
          if ((lane & 7) == 0) {
            T* out = part + (size_t)__ldg(grow_base + r0 + r) * 12 + vb;
            out[0] = red[0];
            out[1] = red[1];
            out[2] = red[2];
          }
        } else {
          const uint32_t row = sb / SLICE + r;
          const uint32_t mask = __ldg(srow_mask + row), pbase = __ldg(srow_base + row);
          const int i = r < len ? ld_stream(sell_cam + base + r * SLICE) : -1;
          if (i >= 0) {
            T P0[4], P1[4], P2[4];
            load_row<T>(camP, i, 0, P0);
            load_row<T>(camP, i, 1, P1);
            load_row<T>(camP, i, 2, P2);
            scatter_obs<T>(P0, P1, P2, a, (T)mr.x, (T)mr.y, S, X, v);
          }
          if (mask == 0u) {
            T red[3];
            int vb;
            warp_reduce12<T>(v, lane, red, vb);
            if ((lane & 7) == 0) {
              T* out = part + (size_t)pbase * 12 + vb;
              out[0] = red[0];
              out[1] = red[1];
              out[2] = red[2];
            }
          } else {
            store_runs<T>(v, mask, i >= 0, pbase, lane, part);
          }
        }
      }
      }
    }
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

povar_status launch_series_term(Problem* p, int precision, double eta, int term, double eps,
                                int schedule) {
  const double a64 = 1.0 - eta;   // C_k = B_k^T B_k coefficient, 1 - eta
  const float a32 = (float)a64;
  // the series vector is double-buffered by term parity
  const size_t yoff_in = ((term - 1) & 1) * (size_t)p->nc * 12;
  const size_t yoff_out = (term & 1) * (size_t)p->nc * 12;
  if (schedule == 4 || precision == POVAR_MIXED_BF16) {
    const unsigned ga = (unsigned)p->nc;
    const BlockPlanes bp = block_planes(p, block_kind(precision));
    if (!bp.p[0]) return fail(p, POVAR_EINVAL, "stored blocks were not allocated");
    if (precision == POVAR_FP64) {
      k_series_fused<double, double><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
          p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0],
          p->P64[1], p->Y64 + yoff_in, point_data<double>(p, 0), point_data<double>(p, 1),
          p->row_mask, p->row_base, static_cast<double*>(p->part_run), bp);
      k_series_apply<double><<<ga, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam_part_off, p->cam_part_idx, nullptr,
          static_cast<const double*>(p->part_run), p->G64, p->camnorm, p->done_ticket,
          p->Y64 + yoff_out, p->D64, 0);
    } else {
      if (precision == POVAR_MIXED_BF16)
        k_series_fused<float, Bf16><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
            p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
            p->camP32[1], p->Y32 + yoff_in, point_data<float>(p, 0), point_data<float>(p, 1),
            p->row_mask, p->row_base, static_cast<float*>(p->part_run), bp);
      else
        k_series_fused<float, float><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
            p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
            p->camP32[1], p->Y32 + yoff_in, point_data<float>(p, 0), point_data<float>(p, 1),
            p->row_mask, p->row_base, static_cast<float*>(p->part_run), bp);
      k_series_apply<float><<<ga, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam_part_off, p->cam_part_idx, nullptr,
          static_cast<const float*>(p->part_run), p->G32, p->camnorm, p->done_ticket,
          p->Y32 + yoff_out, p->D32, 0);
    }
    p->launches += 2;
    return check_launch(p, "series_term (stored blocks)");
  }
  if (schedule == 5) {
    // one launch for the groups and the slices outside groups (run partials
    // after the item partials), then the per-camera sums
    const unsigned gb = (unsigned)(p->g5_ngroups + p->g5_nrest);
    const int64_t nit = p->g5_nlist;
    const G5Tables tb{p->g5_off,  p->g5_slices, p->g5_roff, p->g5_rowcam,
                      p->g5_ioff, p->g5_items,  p->g5_idest, p->g5_rest,
                      reinterpret_cast<const uint4*>(p->g5_sinfo),
                      reinterpret_cast<const int2*>(p->g5_ghdr), p->g5_ngroups};
    if (precision == POVAR_FP64) {
      double* part = static_cast<double*>(p->part5);
      if (gb > 0)
        k_series_group<double><<<gb, G5_THREADS, g5_smem_bytes<double>(), p->stream>>>(
            p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0],
            p->P64[1], p->Y64 + yoff_in, point_data<double>(p, 0), point_data<double>(p, 1), tb,
            p->row_mask, p->row_base, part, part + nit * 12, term, eps, p->camnorm, p->nc);
      k_series_apply<double><<<p->nc, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam5_off, p->cam5_idx, p->cam5_ndirect, part, p->G64, p->camnorm,
          p->done_ticket, p->Y64 + yoff_out, p->D64, gb > 0 ? 1 : 0);
    } else {
      float* part = static_cast<float*>(p->part5);
      if (gb > 0)
        k_series_group<float><<<gb, G5_THREADS, g5_smem_bytes<float>(), p->stream>>>(
            p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
            p->camP32[1], p->Y32 + yoff_in, point_data<float>(p, 0), point_data<float>(p, 1), tb,
            p->row_mask, p->row_base, part, part + nit * 12, term, eps, p->camnorm, p->nc);
      k_series_apply<float><<<p->nc, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam5_off, p->cam5_idx, p->cam5_ndirect, part, p->G32, p->camnorm,
          p->done_ticket, p->Y32 + yoff_out, p->D32, gb > 0 ? 1 : 0);
    }
    p->launches += 1 + (gb > 0);
    return check_launch(p, "series_term (groups)");
  }
  if (schedule == 2) {
    if (precision == POVAR_FP64) {
      k_series_gather<double, false><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
          p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
          p->Y64 + yoff_in, point_data<double>(p, 0), point_data<double>(p, 1), p->rec32,
          p->rec64, nullptr);
      k_series_camrows<double, CAMROW_WARPS><<<p->nc, CAMROW_WARPS * 32, 0, p->stream>>>(
          p->state, a64, term, eps, p->nc, p->cam_row_off, p->cam_row_pos0, p->cam_row_slot0,
          p->sell_cam, p->sell_m64, p->P64[0], p->P64[1], p->rec32, p->rec64, p->G64,
          p->camnorm, p->done_ticket, p->Y64 + yoff_out, p->D64);
    } else {
      k_series_gather<float, false><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
          p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
          p->camP32[1], p->Y32 + yoff_in, point_data<float>(p, 0), point_data<float>(p, 1),
          p->rec32, p->rec64, nullptr);
      k_series_camrows<float, CAMROW_WARPS><<<p->nc, CAMROW_WARPS * 32, 0, p->stream>>>(
          p->state, a32, term, eps, p->nc, p->cam_row_off, p->cam_row_pos0, p->cam_row_slot0,
          p->sell_cam, p->sell_m32, p->camP32[0], p->camP32[1], p->rec32, p->rec64, p->G32,
          p->camnorm, p->done_ticket, p->Y32 + yoff_out, p->D32);
    }
    p->launches += 2;
    return check_launch(p, "series_term (camera rows)");
  }
  if (schedule == 3) {
    const unsigned gg = (unsigned)((p->ngroups + BLOCK / SLICE - 1) / (BLOCK / SLICE));
    if (precision == POVAR_FP64) {
      if (gg > 0)
        k_series_rows<double><<<gg, BLOCK, 0, p->stream>>>(
            p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0],
            p->P64[1], p->Y64 + yoff_in, point_data<double>(p, 0), point_data<double>(p, 1),
            p->grp_slice0, p->grp_row0, p->ngroups, p->grow_cam, p->grow_base, p->srow_mask,
            p->srow_base, static_cast<double*>(p->part3));
      k_series_apply<double><<<p->nc, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam_part3_off, p->cam_part3_idx, nullptr,
          static_cast<const double*>(p->part3), p->G64, p->camnorm, p->done_ticket,
          p->Y64 + yoff_out, p->D64, 0);
    } else {
      if (gg > 0)
        k_series_rows<float><<<gg, BLOCK, 0, p->stream>>>(
            p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
            p->camP32[1], p->Y32 + yoff_in, point_data<float>(p, 0), point_data<float>(p, 1),
            p->grp_slice0, p->grp_row0, p->ngroups, p->grow_cam, p->grow_base, p->srow_mask,
            p->srow_base, static_cast<float*>(p->part3));
      k_series_apply<float><<<p->nc, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam_part3_off, p->cam_part3_idx, nullptr,
          static_cast<const float*>(p->part3), p->G32, p->camnorm, p->done_ticket,
          p->Y32 + yoff_out, p->D32, 0);
    }
    p->launches += gg > 0 ? 2 : 1;
    return check_launch(p, "series_term (grouped)");
  }
  if (schedule == 1) {
    const unsigned ga = (unsigned)p->nc;
    if (precision == POVAR_FP64) {
      k_series_fused<double, void><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
          p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0],
          p->P64[1], p->Y64 + yoff_in, point_data<double>(p, 0), point_data<double>(p, 1), p->row_mask,
          p->row_base, static_cast<double*>(p->part_run), BlockPlanes{});
      k_series_apply<double><<<ga, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam_part_off, p->cam_part_idx, nullptr,
          static_cast<const double*>(p->part_run), p->G64, p->camnorm, p->done_ticket, p->Y64 + yoff_out,
          p->D64, 0);
    } else {
      k_series_fused<float, void><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
          p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
          p->camP32[1], p->Y32 + yoff_in, point_data<float>(p, 0), point_data<float>(p, 1), p->row_mask,
          p->row_base, static_cast<float*>(p->part_run), BlockPlanes{});
      k_series_apply<float><<<ga, 128, 0, p->stream>>>(
          p->state, term, eps, p->nc, p->cam_part_off, p->cam_part_idx, nullptr,
          static_cast<const float*>(p->part_run), p->G32, p->camnorm, p->done_ticket, p->Y32 + yoff_out,
          p->D32, 0);
    }
    p->launches += 2;
    return check_launch(p, "series_term (fused)");
  }
  const unsigned gs = grid_for(p->nchunks, 8);
  if (precision == POVAR_FP64) {
    k_series_gather<double, false><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1], p->Y64 + yoff_in,
        point_data<double>(p, 0), point_data<double>(p, 1), p->rec32, p->rec64, nullptr);
  } else {
    k_series_gather<float, false><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0], p->camP32[1], p->Y32 + yoff_in,
        point_data<float>(p, 0), point_data<float>(p, 1), p->rec32, p->rec64, nullptr);
  }
  ++p->launches;
  if (gs > 0) {
    if (precision == POVAR_FP64) {
      k_series_scatter<double><<<gs, 256, 0, p->stream>>>(
          p->state, a64, term, eps, p->nchunks, p->nc, p->nc_active, p->chunk_cam,
          p->chunk_beg, p->cam_nchunk, p->cam_chunk0, p->cm_slot, p->cm_m64, p->P64[0],
          p->P64[1], p->rec32, p->rec64, p->G64, static_cast<double*>(p->part_ser), p->cam_ticket,
          p->done_ticket, p->camnorm, p->Y64 + yoff_out, p->D64);
    } else {
      k_series_scatter<float><<<gs, 256, 0, p->stream>>>(
          p->state, a32, term, eps, p->nchunks, p->nc, p->nc_active, p->chunk_cam,
          p->chunk_beg, p->cam_nchunk, p->cam_chunk0, p->cm_slot, p->cm_m32, p->camP32[0],
          p->camP32[1], p->rec32, p->rec64, p->G32, static_cast<float*>(p->part_ser), p->cam_ticket,
          p->done_ticket, p->camnorm, p->Y32 + yoff_out, p->D32);
    }
    ++p->launches;
  }
  return check_launch(p, "series_term");
}

int block_kind(int precision) {
  return precision == POVAR_FP64 ? 0 : precision == POVAR_MIXED_BF16 ? 2 : 1;
}

// Bytes of one SELL entry's stored block, per kind (FP64, FP32, BF16).
static const int64_t kBlockBytes[3] = {72, 36, 18};

povar_status ensure_blocks(Problem* p, int kind) {
  if (p->blk[kind]) return POVAR_OK;
  const int64_t E = std::max<int64_t>(p->nsell, 1);
  return dev_alloc_bytes(p, &p->blk[kind], (size_t)(E * kBlockBytes[kind]), "stored blocks");
}

BlockPlanes block_planes(const Problem* p, int kind) {
  BlockPlanes b{};
  char* base = static_cast<char*>(p->blk[kind]);
  if (!base) return b;
  const size_t E = (size_t)std::max<int64_t>(p->nsell, 1);
  if (kind == 0) {
    for (int k = 0; k < 4; ++k) b.p[k] = base + 16 * E * k;
    b.p[4] = base + 64 * E;
  } else if (kind == 1) {
    b.p[0] = base;
    b.p[1] = base + 16 * E;
    b.p[2] = base + 32 * E;
  } else {
    b.p[0] = base;
    b.p[1] = base + 16 * E;
  }
  return b;
}

povar_status launch_build_blocks(Problem* p, int precision, double eta) {
  const double a64 = 1.0 - eta;
  const float a32 = (float)a64;
  const BlockPlanes bp = block_planes(p, block_kind(precision));
  if (!bp.p[0]) return fail(p, POVAR_EINVAL, "stored blocks were not allocated");
  const unsigned g = grid_for(p->nsell, 256);
  if (g == 0) return POVAR_OK;
  if (precision == POVAR_FP64)
    k_build_blocks<double, double><<<g, 256, 0, p->stream>>>(
        p->state, a64, p->nsell, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1], bp);
  else if (precision == POVAR_MIXED_BF16)
    k_build_blocks<float, Bf16><<<g, 256, 0, p->stream>>>(
        p->state, a32, p->nsell, p->sell_cam, p->sell_m32, p->camP32[0], p->camP32[1], bp);
  else
    k_build_blocks<float, float><<<g, 256, 0, p->stream>>>(
        p->state, a32, p->nsell, p->sell_cam, p->sell_m32, p->camP32[0], p->camP32[1], bp);
  ++p->launches;
  return check_launch(p, "build_blocks");
}

povar_status launch_project_delta(Problem* p, int precision) {
  const unsigned gc = grid_for(p->nc, 128);
  if (precision == POVAR_FP64)
    k_project_delta<double><<<gc, 128, 0, p->stream>>>(p->state, p->nc, p->P64[0], p->P64[1],
                                                       p->D64);
  else
    k_project_delta<float><<<gc, 128, 0, p->stream>>>(p->state, p->nc, p->P64[0], p->P64[1],
                                                      p->D32);
  ++p->launches;
  return check_launch(p, "project_delta");
}

povar_status launch_pred(Problem* p, int precision, double eta, int manifold, int m) {
  const double a64 = 1.0 - eta;
  const float a32 = (float)a64;
  const unsigned gc = grid_for(p->nc, 128);
  if (precision == POVAR_FP64) {
    if (manifold == POVAR_SPHERE)
      k_project_delta<double><<<gc, 128, 0, p->stream>>>(p->state, p->nc, p->P64[0],
                                                         p->P64[1], p->D64);
    k_series_gather<double, true><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1], p->D64,
        point_data<double>(p, 0), point_data<double>(p, 1), p->rec32, p->rec64, p->pred_part);
    k_pred_cam<double><<<grid_for(p->nc, 8), 256, 0, p->stream>>>(p->state, p->nc, p->U64,
                                                                   p->bp64, p->D64, p->camnorm);
    k_pred_finish<<<FIN_BLOCKS, 256, 0, p->stream>>>(p->state, p->nc, p->np_pad / 32, m,
                                                     p->pred_part, p->camnorm,
                                                     p->fin_blk + FIN_BLOCKS, p->fin_ticket + 1);
  } else {
    if (manifold == POVAR_SPHERE)
      k_project_delta<float><<<gc, 128, 0, p->stream>>>(p->state, p->nc, p->P64[0], p->P64[1],
                                                        p->D32);
    k_series_gather<float, true><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, a32, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0], p->camP32[1], p->D32,
        point_data<float>(p, 0), point_data<float>(p, 1), p->rec32, p->rec64, p->pred_part);
    k_pred_cam<float><<<grid_for(p->nc, 8), 256, 0, p->stream>>>(p->state, p->nc, p->U64,
                                                                  p->bp64, p->D32, p->camnorm);
    k_pred_finish<<<FIN_BLOCKS, 256, 0, p->stream>>>(p->state, p->nc, p->np_pad / 32, m,
                                                     p->pred_part, p->camnorm,
                                                     p->fin_blk + FIN_BLOCKS, p->fin_ticket + 1);
  }
  p->launches += manifold == POVAR_SPHERE ? 4 : 3;
  return check_launch(p, "pred");
}

povar_status launch_series_apply(Problem* p, int precision, int term, double eps,
                                 const uint32_t* off, const uint32_t* idx, const void* part) {
  const size_t yoff_out = (term & 1) * (size_t)p->nc * 12;
  if (precision == POVAR_FP64)
    k_series_apply<double><<<p->nc, 128, 0, p->stream>>>(
        p->state, term, eps, p->nc, off, idx, nullptr, static_cast<const double*>(part), p->G64,
        p->camnorm, p->done_ticket, p->Y64 + yoff_out, p->D64, 0);
  else
    k_series_apply<float><<<p->nc, 128, 0, p->stream>>>(
        p->state, term, eps, p->nc, off, idx, nullptr, static_cast<const float*>(part), p->G32,
        p->camnorm, p->done_ticket, p->Y32 + yoff_out, p->D32, 0);
  ++p->launches;
  return check_launch(p, "series_apply");
}

povar_status launch_s2_fused_term(Problem* p, int precision, int term, double eps) {
  const size_t yoff_in = ((term - 1) & 1) * (size_t)p->nc * 12;
  if (precision == POVAR_FP64) {
    rp::S2Land<double> land{p->s2X[0], p->s2X[1], p->s2Gl64};
    k_s2_fused<double><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, p->slot_len, p->sell_off, p->sell_cam, p->P64[0], p->P64[1],
        p->Y64 + yoff_in, land, p->row_mask, p->row_base, static_cast<double*>(p->part_run));
  } else {
    rp::S2Land<float> land{p->s2Xf, p->s2Gl32};
    k_s2_fused<float><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, p->slot_len, p->sell_off, p->sell_cam, p->camP32[0], p->camP32[1],
        p->Y32 + yoff_in, land, p->row_mask, p->row_base, static_cast<float*>(p->part_run));
  }
  ++p->launches;
  povar_status s;
  if ((s = check_launch(p, "s2_fused")) != POVAR_OK) return s;
  return launch_series_apply(p, precision, term, eps, p->cam_part_off, p->cam_part_idx,
                             p->part_run);
}

povar_status launch_wvw(Problem* p, int precision, double eta, const void* vec) {
  const double a64 = 1.0 - eta;
  if (precision == POVAR_FP64) {
    k_series_fused<double, void><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m64, p->P64[0], p->P64[1],
        static_cast<const double*>(vec), point_data<double>(p, 0), point_data<double>(p, 1),
        p->row_mask, p->row_base, static_cast<double*>(p->part_run), BlockPlanes{});
  } else {
    k_series_fused<float, void><<<p->n_slot_blocks, BLOCK, 0, p->stream>>>(
        p->state, (float)a64, p->slot_len, p->sell_off, p->sell_cam, p->sell_m32, p->camP32[0],
        p->camP32[1], static_cast<const float*>(vec), point_data<float>(p, 0),
        point_data<float>(p, 1), p->row_mask, p->row_base, static_cast<float*>(p->part_run),
        BlockPlanes{});
  }
  ++p->launches;
  return check_launch(p, "wvw");
}

// The group kernel's dynamic shared memory exceeds the default 48 KB limit in
// FP64; raise the per-kernel limit once per problem (outside any capture).
povar_status setup_group_kernels(Problem* p) {
  POVAR_CUDA(cudaFuncSetAttribute(k_series_group<double>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)g5_smem_bytes<double>()));
  POVAR_CUDA(cudaFuncSetAttribute(k_series_group<float>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)g5_smem_bytes<float>()));
  return POVAR_OK;
}

}  // namespace povar
