// Per-observation arithmetic of the projective reprojection error (second
// stage): y = P X for a row-major 3x4 camera and a homogeneous 4-vector,
// D = d pi / d y, E = D^T D applied to vectors, and the landmark records the
// series passes read. Shared by the second stage's kernels and its fused
// series pass.
#pragma once

#include "povar_internal.cuh"

namespace povar {
namespace rp {

// y, iz, pi0, pi1 of one observation
template <typename T>
struct Proj {
  T y[3];
  T iz, p0, p1;
};

template <typename T>
__device__ __forceinline__ Proj<T> project(const T P[12], const T X[4]) {
  Proj<T> o;
#pragma unroll
  for (int r = 0; r < 3; ++r)
    o.y[r] = P[4 * r] * X[0] + P[4 * r + 1] * X[1] + P[4 * r + 2] * X[2] + P[4 * r + 3] * X[3];
  o.iz = (T)1 / o.y[2];
  o.p0 = o.y[0] * o.iz;
  o.p1 = o.y[1] * o.iz;
  return o;
}

// D w (2-vector)
template <typename T>
__device__ __forceinline__ void apply_d(const Proj<T>& q, const T w[3], T out[2]) {
  out[0] = q.iz * (w[0] - q.p0 * w[2]);
  out[1] = q.iz * (w[1] - q.p1 * w[2]);
}

// D^T a (3-vector)
template <typename T>
__device__ __forceinline__ void apply_dt(const Proj<T>& q, const T a[2], T out[3]) {
  out[0] = q.iz * a[0];
  out[1] = q.iz * a[1];
  out[2] = -q.iz * (q.p0 * a[0] + q.p1 * a[1]);
}

// E w = D^T D w
template <typename T>
__device__ __forceinline__ void apply_e(const Proj<T>& q, const T w[3], T out[3]) {
  T d[2];
  apply_d(q, w, d);
  apply_dt(q, d, out);
}

// P^T t (4-vector) for the row-major 3x4 P
template <typename T>
__device__ __forceinline__ void apply_pt(const T P[12], const T t[3], T out[4]) {
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = P[c] * t[0] + P[4 + c] * t[1] + P[8 + c] * t[2];
}

// P x (3-vector)
template <typename T>
__device__ __forceinline__ void apply_p(const T P[12], const T x[4], T out[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
    out[r] = P[4 * r] * x[0] + P[4 * r + 1] * x[1] + P[4 * r + 2] * x[2] + P[4 * r + 3] * x[3];
}

// symmetric 4x4 in 10 entries: 00 01 02 03 11 12 13 22 23 33 (sd_t10 order)
template <typename T>
__device__ __forceinline__ void sym4_mul(const T g[10], const T x[4], T out[4]) {
  out[0] = g[0] * x[0] + g[1] * x[1] + g[2] * x[2] + g[3] * x[3];
  out[1] = g[1] * x[0] + g[4] * x[1] + g[5] * x[2] + g[6] * x[3];
  out[2] = g[2] * x[0] + g[5] * x[1] + g[7] * x[2] + g[8] * x[3];
  out[3] = g[3] * x[0] + g[6] * x[1] + g[8] * x[2] + g[9] * x[3];
}

template <typename T>
__device__ __forceinline__ void load12(const T* __restrict__ src, T out[12]) {
#pragma unroll
  for (int e = 0; e < 12; ++e) out[e] = src[e];
}

template <typename T> struct S2Land;
template <> struct S2Land<double> {
  const double* X0;
  const double* X1;
  const double* G;
  __device__ void load(int cur, int s, double X[4], double g[10]) const {
    const double* x = (cur ? X1 : X0) + 4 * (size_t)s;
#pragma unroll
    for (int e = 0; e < 4; ++e) X[e] = x[e];
#pragma unroll
    for (int e = 0; e < 10; ++e) g[e] = G[10 * (size_t)s + e];
  }
  __device__ void load_x(int cur, int s, double X[4]) const {
    const double* x = (cur ? X1 : X0) + 4 * (size_t)s;
#pragma unroll
    for (int e = 0; e < 4; ++e) X[e] = x[e];
  }
};
template <> struct S2Land<float> {
  const float4* Xf;
  const float4* G;
  __device__ void load(int, int s, float X[4], float g[10]) const {
    load_x(0, s, X);
    const float4 a = __ldg(G + 3 * (size_t)s), b = __ldg(G + 3 * (size_t)s + 1),
                 c = __ldg(G + 3 * (size_t)s + 2);
    g[0] = a.x; g[1] = a.y; g[2] = a.z; g[3] = a.w;
    g[4] = b.x; g[5] = b.y; g[6] = b.z; g[7] = b.w;
    g[8] = c.x; g[9] = c.y;
  }
  __device__ void load_x(int, int s, float X[4]) const {
    const float4 x = __ldg(Xf + s);
    X[0] = x.x; X[1] = x.y; X[2] = x.z; X[3] = x.w;
  }
};

}  // namespace rp
}  // namespace povar
