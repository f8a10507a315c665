// Warp-level helpers for 12x12 camera blocks and 4x4 landmark moments,
// shared by the conjugate-gradient solver and the second stage. One warp
// owns one camera: lanes 0..11 hold the rows of a block or the entries of a
// 12-vector; the remaining lanes carry zeros through the shuffles.
#pragma once

#include "povar_internal.cuh"

namespace povar {
namespace b12 {

// t10 order of the symmetric 4x4 moments: (0,0..3) (1,1..3) (2,2..3) (3,3)
__device__ __forceinline__ int sd_t10(int b, int d) {
  const int lo = b < d ? b : d, hi = b < d ? d : b;
  return lo == 0 ? hi : (lo == 1 ? 3 + hi : (lo == 2 ? 5 + hi : 9));
}
// index of the symmetric 3x3 entry (a, b): 00 01 02 11 12 22
__device__ __forceinline__ int sym3(int a, int b) {
  const int lo = a < b ? a : b, hi = a < b ? b : a;
  return lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
}

// lanes 0..11 hold a 12-vector x; returns (M x)_lane for the row-major 12x12
// block M (lanes >= 12 get 0)
template <typename T>
__device__ __forceinline__ T matvec12(const T* __restrict__ M, T x, int lane) {
  T y = 0;
#pragma unroll
  for (int q = 0; q < 12; ++q) {
    const T xq = __shfl_sync(0xffffffffu, x, q);
    if (lane < 12) y += M[lane * 12 + q] * xq;
  }
  return y;
}

// lanes 0..11: the unit camera p^ (0 in EUCLID)
__device__ __forceinline__ double unit_camera(const double* Pc, int lane, int manifold) {
  if (manifold != POVAR_SPHERE) return 0.0;
  const double Pl = lane < 12 ? Pc[lane] : 0.0;
  double nn = Pl * Pl;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
  return lane < 12 ? Pl / sqrt(nn) : 0.0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// In-place Cholesky inverse of the SPD 12x12 block A (rows owned by lanes
// 0..11, shared row-major with stride 13) into Inv (same layout); returns
// false (warp-uniform) if a pivot is not positive.
__device__ inline bool chol_inverse12(double (*A)[13], double (*L)[13], double (*Inv)[13],
                               double* rinv, int lane) {
  bool bad = false;
  for (int k = 0; k < 12; ++k) {
    if (lane == k) {
      const double d = A[k][k];
      if (!(d > 0.0)) bad = true;
      const double r = rsqrt(fmax(d, 1e-300));
      A[k][k] = fmax(d, 1e-300) * r;
      rinv[k] = r;
    }
    __syncwarp();
    if (lane > k && lane < 12) A[lane][k] *= rinv[k];
    __syncwarp();
    if (lane > k && lane < 12)
      for (int j = k + 1; j <= lane; ++j) A[lane][j] -= A[lane][k] * A[j][k];
    __syncwarp();
  }
  bad = __any_sync(0xffffffffu, bad);
  if (lane < 12) {
    const int c = lane;
    for (int r = 0; r < 12; ++r) {
      if (r < c) {
        L[r][c] = 0.0;
        continue;
      }
      double s = (r == c) ? 1.0 : 0.0;
      for (int k = c; k < r; ++k) s -= A[r][k] * L[k][c];
      L[r][c] = s * rinv[r];
    }
  }
  __syncwarp();
  if (lane < 12)
    for (int q = 0; q < 12; ++q) {
      const int k0 = lane > q ? lane : q;
      double s = 0.0;
      for (int k = k0; k < 12; ++k) s += L[k][lane] * L[k][q];
      Inv[lane][q] = s;
    }
  __syncwarp();
  return !bad;
}

}  // namespace b12
}  // namespace povar
