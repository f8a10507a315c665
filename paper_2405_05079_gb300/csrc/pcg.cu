// The "iterative" VarPro baseline of Sec. 5.2 of the paper: the reduced
// camera system S delta = g solved by conjugate gradients preconditioned
// with the inverse diagonal blocks of S (Schur-Jacobi), at most m inner
// iterations, stopping when ||g - S delta|| <= eps ||g||.
//   S = U~ - W~ V^-1 W~^T (tangent-projected on the unit-norm manifold in
//   the projector form of k_camera_prepare), V damped for PoBA.
// Kernels:
//   k_schur_diag   camera-major chunks: per observation the block
//                  W_k V^-1 W_k^T = K_k (x) x~ x~^T with
//                  K_k = (C_k Pbar_i) V_j^-1 (C_k Pbar_i)^T (3x3), i.e. the
//                  six entries of K times the ten moments of x~: 60 sums per
//                  chunk (one warp per chunk, fixed-order shuffles);
//   k_pcg_precond  per camera (FP64): S_ii = Pi (U + lambda I) Pi
//                  - Pi (sum of the chunk blocks) Pi (+ p^ p^T on the
//                  sphere), Cholesky inverse, minus p^ p^T on the sphere;
//   k_pcg_init     r = g = -Pi b_p, z = M^-1 r, p = z, delta = 0;
//   per iteration: the fused landmark pass (schedule 1) computes the
//   partials of W V^-1 W^T p, then
//   k_pcg_q        q = S p = Pi (U p - z) + lambda p and p.q,
//   k_pcg_update   delta += alpha p, r -= alpha q, z = M^-1 r, r.z, r.r,
//   k_pcg_dir      p = z + beta p.
// The global dot products are added per camera in camera order by the last
// block to finish (atomic ticket), so results do not depend on scheduling.
// Assumes at most one observation per (camera, landmark) pair (W_ij is then
// a single W_k).
#include <algorithm>
#include <cstddef>

#include "block12.cuh"
#include "povar_internal.cuh"

namespace povar {
namespace {

using namespace b12;

constexpr int SD_ACC = 60;   // 6 entries of K x 10 moments of x~

// FP64: landmarks and factors from the FP64 buffers; otherwise (mixed
// precision, whose trial landmarks are double-float and whose FP64 factor
// is not kept) from their FP32 copies. Sums in FP64 either way.
template <bool FP64>
__global__ void __launch_bounds__(256)
k_schur_diag(const DeviceState* __restrict__ st, double a, int nchunks,
             const int32_t* __restrict__ chunk_cam, const uint32_t* __restrict__ chunk_beg,
             const uint32_t* __restrict__ cm_slot, const double2* __restrict__ cm_m,
             const double* __restrict__ P0, const double* __restrict__ P1,
             const double* __restrict__ X0, const double* __restrict__ X1,
             const double* __restrict__ F0, const double* __restrict__ F1,
             const float4* __restrict__ A0, const float4* __restrict__ A1,
             const float4* __restrict__ B0, const float4* __restrict__ B1,
             const float* __restrict__ C0, const float* __restrict__ C1,
             double* __restrict__ part) {
  if (st->converged) return;
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= nchunks) return;
  const int cur = st->cur;
  const double* Pc = (cur ? P1 : P0) + 12 * (size_t)chunk_cam[c];
  const double* Xb = cur ? X1 : X0;
  const double* Fb = cur ? F1 : F0;
  double Pb[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) Pb[3 * r + q] = Pc[4 * r + q];
  double acc[SD_ACC];
#pragma unroll
  for (int e = 0; e < SD_ACC; ++e) acc[e] = 0.0;
  const uint32_t b = chunk_beg[c], e_ = chunk_beg[c + 1];
  for (uint32_t r = b + lane; r < e_; r += 32) {
    const uint32_t slot = cm_slot[r];
    const double2 m = cm_m[r];
    const double u = m.x, v = m.y, w = u * u + v * v, aa = a;
    double x[3], f[6];
    if constexpr (FP64) {
#pragma unroll
      for (int q = 0; q < 3; ++q) x[q] = Xb[3 * (size_t)slot + q];
#pragma unroll
      for (int q = 0; q < 6; ++q) f[q] = Fb[6 * (size_t)slot + q];
    } else {
      const float4 pa = __ldg((cur ? A1 : A0) + slot), pb = __ldg((cur ? B1 : B0) + slot);
      x[0] = pa.x; x[1] = pa.y; x[2] = pa.z;
      f[0] = pa.w; f[1] = pb.x; f[2] = pb.y; f[3] = pb.z; f[4] = pb.w;
      f[5] = __ldg((cur ? C1 : C0) + slot);
    }
    // V^-1 = F^T F with F lower-triangular (f00 f10 f11 f20 f21 f22)
    const double Vi[6] = {f[0] * f[0] + f[1] * f[1] + f[3] * f[3], f[2] * f[1] + f[4] * f[3],
                          f[5] * f[3], f[2] * f[2] + f[4] * f[4], f[5] * f[4], f[5] * f[5]};
    // G = C Pbar (rows of C: (1, 0, -a u), (0, 1, -a v), (-a u, -a v, a w))
    double G[9];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      G[q] = Pb[q] - aa * u * Pb[6 + q];
      G[3 + q] = Pb[3 + q] - aa * v * Pb[6 + q];
      G[6 + q] = aa * (w * Pb[6 + q] - u * Pb[q] - v * Pb[3 + q]);
    }
    // H = G V^-1, K = H G^T (symmetric)
    double H[9];
#pragma unroll
    for (int r2 = 0; r2 < 3; ++r2)
#pragma unroll
      for (int q = 0; q < 3; ++q)
        H[3 * r2 + q] = G[3 * r2] * Vi[sym3(0, q)] + G[3 * r2 + 1] * Vi[sym3(1, q)] +
                        G[3 * r2 + 2] * Vi[sym3(2, q)];
    double K[6];
    K[0] = H[0] * G[0] + H[1] * G[1] + H[2] * G[2];
    K[1] = H[0] * G[3] + H[1] * G[4] + H[2] * G[5];
    K[2] = H[0] * G[6] + H[1] * G[7] + H[2] * G[8];
    K[3] = H[3] * G[3] + H[4] * G[4] + H[5] * G[5];
    K[4] = H[3] * G[6] + H[4] * G[7] + H[5] * G[8];
    K[5] = H[6] * G[6] + H[7] * G[7] + H[8] * G[8];
    const double t10[10] = {x[0] * x[0], x[0] * x[1], x[0] * x[2], x[0], x[1] * x[1],
                            x[1] * x[2], x[1], x[2] * x[2], x[2], 1.0};
#pragma unroll
    for (int kk = 0; kk < 6; ++kk)
#pragma unroll
      for (int q = 0; q < 10; ++q) acc[10 * kk + q] += K[kk] * t10[q];
  }
#pragma unroll
  for (int e = 0; e < SD_ACC; ++e) {
    double val = acc[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    acc[e] = val;
  }
  double* out = part + (size_t)c * SD_ACC;
#pragma unroll
  for (int e = 0; e < SD_ACC; ++e)
    if ((e & 31) == lane) out[e] = acc[e];
}

// One warp per camera: the Schur-Jacobi block and its inverse. If rounding
// leaves the block not numerically positive definite (FP32-accumulated U and
// FP32 landmarks in mixed precision), its damping is raised as in the camera
// preparation -- to at least 1e-12 of the largest diagonal entry, then x100
// per attempt, at most 8 attempts; the preconditioner only has to be SPD.
__global__ void __launch_bounds__(128)
k_pcg_precond(DeviceState* __restrict__ st, int manifold, int nc,
              const int32_t* __restrict__ cam_nchunk, const int32_t* __restrict__ cam_chunk0,
              const double* __restrict__ part, const double* __restrict__ U64,
              const double* __restrict__ P0, const double* __restrict__ P1,
              double* __restrict__ M64, float* __restrict__ M32) {
  if (st->converged) return;
  __shared__ double smA[4][12][13], smL[4][12][13], smI[4][12][13];
  __shared__ double smK[4][SD_ACC];
  __shared__ double smR[4][12];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int i = blockIdx.x * 4 + wl;
  if (i >= nc) return;
  const double lam = st->lam_used;
  const double* Pc = (st->cur ? P1 : P0) + 12 * (size_t)i;
  const int n = cam_nchunk[i], c0 = cam_chunk0[i];
  for (int e = lane; e < SD_ACC; e += 32) {
    double s = 0.0;
    for (int q = 0; q < n; ++q) s += part[(size_t)(c0 + q) * SD_ACC + e];
    smK[wl][e] = s;
  }
  __syncwarp();
  double (*A)[13] = smA[wl];
  const double ph = unit_camera(Pc, lane, manifold);
  double umax = lane < 12 ? U64[(size_t)i * 144 + lane * 13] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) umax = fmax(umax, __shfl_xor_sync(0xffffffffu, umax, o));
  double lam_eff = lam;
  bool ok = false;
  for (int attempt = 0; attempt < 8 && !ok; ++attempt) {
    if (attempt > 0) lam_eff = fmax(lam_eff * 100.0, 1e-12 * umax);
    // B = U + lambda I - K (x) x~x~^T, entry ((a,c),(b,d)) = K_ab M_cd
    if (lane < 12) {
      const int ra = lane >> 2, rc = lane & 3;
      for (int q = 0; q < 12; ++q) {
        const int cb = q >> 2, cd = q & 3;
        const double wvw = smK[wl][10 * sym3(ra, cb) + sd_t10(rc, cd)];
        A[lane][q] = U64[(size_t)i * 144 + lane * 12 + q] - wvw + (lane == q ? lam_eff : 0.0);
      }
    }
    __syncwarp();
    if (manifold == POVAR_SPHERE) {
      // Pi B Pi + p^ p^T with Pi = I - p^ p^T
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
    }
    ok = chol_inverse12(A, smL[wl], smI[wl], smR[wl], lane);
  }
  if (lane == 0 && !ok) st->error = POVAR_ENUMERIC;
  for (int q = 0; q < 12; ++q) {
    const double pq = __shfl_sync(0xffffffffu, ph, q);
    if (lane < 12) {
      double g = smI[wl][lane][q];
      if (manifold == POVAR_SPHERE) g -= ph * pq;
      M64[(size_t)i * 144 + lane * 12 + q] = g;
      M32[(size_t)i * 144 + lane * 12 + q] = (float)g;
    }
  }
}

// Two values per camera in vals[2i], vals[2i+1] (written and fenced by the
// block's warps); the last block to finish adds them in camera order.
// Returns true in that block, with the totals in tot[0], tot[1] for every
// thread. Call from every thread of every block.
__device__ bool cam_sum(int nc, const double* __restrict__ vals, uint32_t* __restrict__ ticket,
                        double* tot) {
  __shared__ int last;
  __shared__ double shw[32][2];
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double s0 = 0.0, s1 = 0.0;
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    s0 += __ldcg(vals + 2 * (size_t)c);
    s1 += __ldcg(vals + 2 * (size_t)c + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    shw[threadIdx.x >> 5][0] = s0;
    shw[threadIdx.x >> 5][1] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a0 += shw[w][0];
      a1 += shw[w][1];
    }
    shw[0][0] = a0;
    shw[0][1] = a1;
    *ticket = 0u;
  }
  __syncthreads();
  tot[0] = shw[0][0];
  tot[1] = shw[0][1];
  return true;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_pcg_init(DeviceState* __restrict__ st, int manifold, int nc, const double* __restrict__ bp64,
           const double* __restrict__ P0, const double* __restrict__ P1,
           const T* __restrict__ M, T* __restrict__ r, T* __restrict__ z, T* __restrict__ p,
           T* __restrict__ D, double* __restrict__ vals, uint32_t* __restrict__ ticket) {
  if (st->converged) return;
  const int lane = threadIdx.x & 31, i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i < nc) {
    const double* Pc = (st->cur ? P1 : P0) + 12 * (size_t)i;
    const double ph = unit_camera(Pc, lane, manifold);
    double g = lane < 12 ? -bp64[12 * (size_t)i + lane] : 0.0;
    g -= ph * warp_sum(ph * g);                       // tangent projection
    const T rl = (T)g;
    const T zl = matvec12<T>(M + 144 * (size_t)i, rl, lane);
    if (lane < 12) {
      r[12 * (size_t)i + lane] = rl;
      z[12 * (size_t)i + lane] = zl;
      p[12 * (size_t)i + lane] = zl;
      D[12 * (size_t)i + lane] = (T)0;
    }
    const double rz = warp_sum((double)rl * (double)zl), gg = warp_sum((double)rl * (double)rl);
    if (lane == 0) {
      vals[2 * (size_t)i] = rz;
      vals[2 * (size_t)i + 1] = gg;
      __threadfence();
    }
  }
  double tot[2];
  if (cam_sum(nc, vals, ticket, tot) && threadIdx.x == 0) {
    st->pcg_rz = tot[0];
    st->pcg_gg = tot[1];
    st->terms_used = 0;
    if (!(tot[1] > 0.0)) st->stop_series = 1;
  }
}

// q = S p = Pi (U p - z) + lambda p with z = W V^-1 W^T p from the run
// partials of the landmark pass. One block of 128 threads per camera: thread
// t < 120 adds element t % 12 of every tenth partial, the ten sums of an
// element are added in a fixed order.
template <typename T>
__global__ void __launch_bounds__(128)
k_pcg_q(DeviceState* __restrict__ st, int manifold, int nc,
        const uint32_t* __restrict__ cam_part_off, const uint32_t* __restrict__ cam_part_idx,
        const T* __restrict__ part, const double* __restrict__ U64,
        const double* __restrict__ P0, const double* __restrict__ P1, const T* __restrict__ p,
        T* __restrict__ q, double* __restrict__ vals, uint32_t* __restrict__ ticket) {
  if (st->converged || st->stop_series) return;
  __shared__ double red[128];
  const int lane = threadIdx.x & 31, i = blockIdx.x;
  double acc = 0.0;
  if (threadIdx.x < 120) {
    const int e = threadIdx.x % 12;
    const uint32_t b = cam_part_off[i], e_ = cam_part_off[i + 1];
    for (uint32_t k = b + threadIdx.x / 12; k < e_; k += 10)
      acc += (double)part[(size_t)__ldg(cam_part_idx + k) * 12 + e];
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double zl = 0.0;
    if (lane < 12)
      for (int k = 0; k < 10; ++k) zl += red[12 * k + lane];
    const double* Pc = (st->cur ? P1 : P0) + 12 * (size_t)i;
    const double ph = unit_camera(Pc, lane, manifold);
    const double pl = lane < 12 ? (double)p[12 * (size_t)i + lane] : 0.0;
    const double up = matvec12<double>(U64 + 144 * (size_t)i, pl, lane);
    double w = up - zl;
    w -= ph * warp_sum(ph * w);
    const T ql = (T)(w + st->lam_used * pl);
    if (lane < 12) q[12 * (size_t)i + lane] = ql;
    const double pq = warp_sum(pl * (double)ql);
    if (lane == 0) {
      vals[2 * (size_t)i] = pq;
      vals[2 * (size_t)i + 1] = 0.0;
      __threadfence();
    }
  }
  double tot[2];
  if (cam_sum(nc, vals, ticket, tot) && threadIdx.x == 0) {
    // p.Sp > 0 for p != 0 (S >= lambda I); a zero p means r = 0: stop
    if (tot[0] > 0.0) {
      st->pcg_alpha = st->pcg_rz / tot[0];
    } else {
      st->pcg_alpha = 0.0;
      st->stop_series = 1;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_pcg_update(DeviceState* __restrict__ st, int nc, const T* __restrict__ M,
             const T* __restrict__ p, const T* __restrict__ q, T* __restrict__ r,
             T* __restrict__ z, T* __restrict__ D, double* __restrict__ vals,
             uint32_t* __restrict__ ticket, double eps, int it) {
  if (st->converged || st->stop_series) return;
  const int lane = threadIdx.x & 31, i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i < nc) {
    const T alpha = (T)st->pcg_alpha;
    T rl = 0;
    if (lane < 12) {
      const size_t o = 12 * (size_t)i + lane;
      D[o] += alpha * p[o];
      rl = r[o] - alpha * q[o];
      r[o] = rl;
    }
    const T zl = matvec12<T>(M + 144 * (size_t)i, rl, lane);
    if (lane < 12) z[12 * (size_t)i + lane] = zl;
    const double rz = warp_sum((double)rl * (double)zl), rr = warp_sum((double)rl * (double)rl);
    if (lane == 0) {
      vals[2 * (size_t)i] = rz;
      vals[2 * (size_t)i + 1] = rr;
      __threadfence();
    }
  }
  double tot[2];
  if (cam_sum(nc, vals, ticket, tot) && threadIdx.x == 0) {
    st->terms_used = it;
    st->pcg_beta = st->pcg_rz != 0.0 ? tot[0] / st->pcg_rz : 0.0;
    st->pcg_rz = tot[0];
    if (eps > 0.0 && tot[1] <= eps * eps * st->pcg_gg) st->stop_series = 1;
  }
}

template <typename T>
__global__ void k_pcg_dir(const DeviceState* __restrict__ st, int n, const T* __restrict__ z,
                          T* __restrict__ p) {
  if (st->converged || st->stop_series) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  p[k] = z[k] + (T)st->pcg_beta * p[k];
}

}  // namespace

povar_status ensure_pcg(Problem* p) {
  if (p->pcg_vals) return POVAR_OK;
  povar_status s;
  if ((s = dev_alloc(p, &p->pcg_vec, (size_t)p->nc * 48, "pcg_vec")) ||
      (s = dev_alloc(p, &p->pcg_M64, (size_t)p->nc * 144, "pcg_M64")) ||
      (s = dev_alloc(p, &p->pcg_M32, (size_t)p->nc * 144, "pcg_M32")) ||
      (s = dev_alloc(p, &p->pcg_sd, (size_t)std::max(p->nchunks, 1) * SD_ACC, "pcg_sd")) ||
      (s = dev_alloc(p, &p->pcg_vals, (size_t)p->nc * 2, "pcg_vals")) ||
      (s = dev_alloc(p, &p->pcg_ticket, 1, "pcg_ticket")))
    return s;
  POVAR_CUDA(cudaMemsetAsync(p->pcg_ticket, 0, sizeof(uint32_t), p->stream));
  return POVAR_OK;
}

namespace {

template <typename T>
povar_status pcg_iterations(Problem* p, int precision, int manifold, double eta, int iters,
                            double eps, T* D, const T* M) {
  const size_t n12 = (size_t)p->nc * 12;
  T* base = reinterpret_cast<T*>(p->pcg_vec);
  T *r = base, *z = base + n12, *pv = base + 2 * n12, *q = base + 3 * n12;
  const unsigned g8 = grid_for(p->nc, 8);
  k_pcg_init<T><<<g8, 256, 0, p->stream>>>(p->state, manifold, p->nc, p->bp64, p->P64[0],
                                           p->P64[1], M, r, z, pv, D, p->pcg_vals,
                                           p->pcg_ticket);
  ++p->launches;
  povar_status s;
  if ((s = check_launch(p, "pcg_init")) != POVAR_OK) return s;
  // flags read back every kCheck iterations: converged and stop_series are
  // adjacent ints of the device state
  constexpr int kCheck = 8;
  const size_t flag_off = offsetof(DeviceState, converged);
  static_assert(offsetof(DeviceState, stop_series) == offsetof(DeviceState, converged) + sizeof(int),
                "converged and stop_series must be adjacent");
  for (int it = 1; it <= iters; ++it) {
    if ((s = launch_wvw(p, precision, eta, pv)) != POVAR_OK) return s;
    k_pcg_q<T><<<p->nc, 128, 0, p->stream>>>(
        p->state, manifold, p->nc, p->cam_part_off, p->cam_part_idx,
        static_cast<const T*>(p->part_run), p->U64, p->P64[0], p->P64[1], pv, q, p->pcg_vals,
        p->pcg_ticket);
    k_pcg_update<T><<<g8, 256, 0, p->stream>>>(p->state, p->nc, M, pv, q, r, z, D, p->pcg_vals,
                                               p->pcg_ticket, eps, it);
    if (it < iters)
      k_pcg_dir<T><<<grid_for((int64_t)n12, 256), 256, 0, p->stream>>>(p->state, (int)n12, z, pv);
    p->launches += it < iters ? 3 : 2;
    if ((s = check_launch(p, "pcg_iteration")) != POVAR_OK) return s;
    if (it % kCheck == 0 && it < iters) {
      char* h = reinterpret_cast<char*>(p->h_state) + flag_off;
      POVAR_CUDA(cudaMemcpyAsync(h, reinterpret_cast<char*>(p->state) + flag_off, 2 * sizeof(int),
                                 cudaMemcpyDeviceToHost, p->stream));
      POVAR_CUDA(cudaStreamSynchronize(p->stream));
      if (p->h_state->converged || p->h_state->stop_series) break;
    }
  }
  return POVAR_OK;
}

}  // namespace

povar_status launch_pcg(Problem* p, int precision, int manifold, double eta, int iters,
                        double eps) {
  povar_status s;
  if ((s = ensure_pcg(p)) != POVAR_OK) return s;
  const double a = 1.0 - eta;
  const unsigned gsd = grid_for(p->nchunks, 8);
  if (gsd > 0) {
    if (precision == POVAR_FP64)
      k_schur_diag<true><<<gsd, 256, 0, p->stream>>>(
          p->state, a, p->nchunks, p->chunk_cam, p->chunk_beg, p->cm_slot, p->cm_m64, p->P64[0],
          p->P64[1], p->X64[0], p->X64[1], p->F64[0], p->F64[1], p->pdA[0], p->pdA[1], p->pdB[0],
          p->pdB[1], p->pdC[0], p->pdC[1], p->pcg_sd);
    else
      k_schur_diag<false><<<gsd, 256, 0, p->stream>>>(
          p->state, a, p->nchunks, p->chunk_cam, p->chunk_beg, p->cm_slot, p->cm_m64, p->P64[0],
          p->P64[1], p->X64[0], p->X64[1], p->F64[0], p->F64[1], p->pdA[0], p->pdA[1], p->pdB[0],
          p->pdB[1], p->pdC[0], p->pdC[1], p->pcg_sd);
    ++p->launches;
  }
  k_pcg_precond<<<grid_for(p->nc, 4), 128, 0, p->stream>>>(
      p->state, manifold, p->nc, p->cam_nchunk, p->cam_chunk0, p->pcg_sd, p->U64, p->P64[0],
      p->P64[1], p->pcg_M64, p->pcg_M32);
  ++p->launches;
  if ((s = check_launch(p, "pcg_precond")) != POVAR_OK) return s;
  if (precision == POVAR_FP64)
    return pcg_iterations<double>(p, precision, manifold, eta, iters, eps, p->D64, p->pcg_M64);
  return pcg_iterations<float>(p, precision, manifold, eta, iters, eps, p->D32, p->pcg_M32);
}

}  // namespace povar
