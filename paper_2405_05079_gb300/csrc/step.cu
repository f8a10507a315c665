// a9: camera update and retraction (Sec. 4.3: back-projection of the tangent
//     step, then normalization of every camera to unit Frobenius norm).
// a10: gain ratio, accept / reject and damping update of the LM / VarPro
//     controller, on the device so that a whole solve runs without host
//     round-trips (Sec. 5.2 fixes lambda0 = 1e-4, 50 iterations, ftol 1e-6;
//     the damping rule is Madsen-Nielsen: on accept lambda *= max(1/3,
//     1 - (2 rho - 1)^3), nu = 2; on reject lambda *= nu, nu *= 2; lambda is
//     kept >= LAMBDA_MIN and a damping above LAMBDA_MAX stops the solve).
//     Mixed-precision safeguard (not in the paper): when fallback_after > 0
//     and that many mixed-precision steps in a row were rejected, or the
//     damping grew FALLBACK_LAMBDA_GROWTH times above its value at the start
//     of the solve (or diverged), the controller stops the solve with
//     `fallback` set, and the host continues
//     it in FP64 (FP32 cannot resolve the reduced camera system when it is a
//     strong cancellation of much larger terms, e.g. landmarks drifting
//     towards infinity at a small pOSE weight).
// Also: state initialization, device random cameras (Philox4x32-10 of
//     Salmon et al., SC'11, with the Box-Muller transform) and the landmark
//     gather back to the caller's numbering.
#include "povar_internal.cuh"

namespace povar {
namespace {

template <typename T>
__global__ void k_update(const DeviceState* __restrict__ st, int manifold, int nc,
                         double* __restrict__ P0, double* __restrict__ P1,
                         const T* __restrict__ D) {
  if (st->converged) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const int cur = st->cur;
  const double* P = (cur ? P1 : P0) + 12 * (size_t)i;
  double* Pn = (cur ? P0 : P1) + 12 * (size_t)i;
  double q[12], nn = 0.0;
  for (int e = 0; e < 12; ++e) {
    q[e] = P[e] + (double)D[12 * (size_t)i + e];
    nn += q[e] * q[e];
  }
  const double f = manifold == POVAR_SPHERE ? 1.0 / sqrt(nn) : 1.0;
  for (int e = 0; e < 12; ++e) Pn[e] = q[e] * f;
}

__global__ void k_controller(DeviceState* __restrict__ st, povar_step_report* __restrict__ rep,
                             int precision) {
  if (st->converged) return;
  const double F = st->F, Fn = st->F_new, pred = st->pred;
  const double rho = pred > 0.0 ? (F - Fn) / pred : 0.0;
  const bool accepted = isfinite(Fn) && Fn < F;
  rep->cost_before = F;
  rep->cost_after = Fn;
  rep->pred = pred;
  rep->rho = rho;
  rep->lambda_used = st->lam_used;
  rep->accepted = accepted ? 1 : 0;
  rep->terms_used = st->terms_used;
  rep->precision = precision;
  st->products += st->terms_used > 1 ? st->terms_used - 1 : 0;
  st->rho = rho;
  st->accepted = accepted ? 1 : 0;
  st->iteration += 1;
  rep->iteration = st->iteration;
  int conv = 0;
  if (accepted) {
    const double x = 2.0 * rho - 1.0;
    st->lam = fmax(st->lam * fmax(1.0 / 3.0, 1.0 - x * x * x), LAMBDA_MIN);
    st->nu = 2.0;
    st->cur = 1 - st->cur;
    st->F = Fn;
    st->need_lin = 1;
    st->rej_run = 0;
    if (st->ftol > 0.0 && (F - Fn) < st->ftol * F) conv = 1;
    if (st->target > 0.0 && Fn <= st->target) conv = 1;
  } else {
    st->lam = st->lam * st->nu;
    st->nu = 2.0 * st->nu;
    st->need_lin = 0;
    st->rej_run += 1;
  }
  // mixed-precision safeguard: rejections in a row, a damping grown far
  // above its value at the start of the solve, or a diverging damping mean that
  // the FP32 steps have stopped being useful; the FP64 continuation starts
  // from the smallest damping of the solve
  st->lam_low = fmin(st->lam_low, st->lam_used);
  if (precision != POVAR_FP64 && st->fallback_after > 0 &&
      (st->rej_run >= st->fallback_after || st->lam > FALLBACK_LAMBDA_GROWTH * st->lam_ref ||
       !(st->lam < LAMBDA_MAX))) {
    st->lam = st->lam_low;
    st->nu = 2.0;
    st->rej_run = 0;
    st->fallback = 1;
    conv = 1;
  }
  if (st->max_iters > 0 && st->iteration >= st->max_iters) conv = 1;
  if (!(st->lam < LAMBDA_MAX)) {
    st->error = POVAR_ENOTCONVERGED;
    conv = 1;
  }
  rep->lambda_next = st->lam;
  rep->converged = conv;
  if (conv) st->converged = 1;
}

__global__ void k_init_state(DeviceState* __restrict__ st, double lambda0, int reset_lm,
                             int reset_all) {
  if (reset_all) {
    st->cur = 0;
    st->iteration = 0;
    st->accepted = 0;
    st->converged = 0;
    st->error = 0;
    st->stop_series = 0;
    st->terms_used = 0;
    st->max_iters = 0;
    st->ftol = 0.0;
    st->target = 0.0;
    st->F_new = 0.0;
    st->pred = 0.0;
    st->rho = 0.0;
    st->fallback_after = 0;
    st->fallback = 0;
  }
  st->need_lin = 1;
  if (reset_lm) {
    st->lam = lambda0;
    st->nu = 2.0;
    st->rej_run = 0;
    // the damping references of the safeguard follow a reset (it is
    // enqueued after k_begin when a solve starts from new cameras)
    st->lam_low = lambda0;
    st->lam_ref = lambda0;
  }
}

__global__ void k_begin(DeviceState* __restrict__ st, double ftol, double target, int max_iters,
                        int fallback_after) {
  st->converged = 0;
  st->fallback = 0;
  st->fallback_after = fallback_after;
  st->lam_low = st->lam;
  st->lam_ref = st->lam;
  st->ftol = ftol;
  st->target = target;
  st->max_iters = max_iters > 0 ? st->iteration + max_iters : 0;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of the
// multiply-xor round function with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += W0;
    k.y += W1;
  }
  return c;
}

// Camera i uses counters (i, q, 0, 0), q = 0..2; each counter gives four
// 32-bit words -> two (0, 1] uniforms pairs -> four N(0, 1) via Box-Muller.
__global__ void k_random_cameras(double* __restrict__ P, int nc, uint64_t seed, int normalize) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  double z[12];
  for (int q = 0; q < 3; ++q) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)q, 0u, 0u), key);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
    for (int h = 0; h < 2; ++h) {
      const double u1 = ((double)w[2 * h] + 1.0) * 2.3283064365386963e-10;  // (0, 1]
      const double u2 = ((double)w[2 * h + 1] + 1.0) * 2.3283064365386963e-10;
      const double rad = sqrt(-2.0 * log(u1));
      const double th = 6.283185307179586 * u2;
      z[4 * q + 2 * h] = rad * cos(th);
      z[4 * q + 2 * h + 1] = rad * sin(th);
    }
  }
  double nn = 0.0;
  for (int e = 0; e < 12; ++e) nn += z[e] * z[e];
  const double f = normalize ? 1.0 / sqrt(nn) : 1.0;
  for (int e = 0; e < 12; ++e) P[12 * (size_t)i + e] = z[e] * f;
}

__global__ void k_gather_points(const DeviceState* __restrict__ st,
                                const double* __restrict__ X0, const double* __restrict__ X1,
                                const uint32_t* __restrict__ pt_slot, int np,
                                double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const double* X = (st->cur ? X1 : X0) + 3 * (size_t)pt_slot[j];
  if (st->x_df[st->cur]) {
    // double-float pairs (written by the mixed-precision landmark kernel)
    const float2* Xf = reinterpret_cast<const float2*>(X);
    for (int c = 0; c < 3; ++c) out[3 * (size_t)j + c] = (double)Xf[c].x + (double)Xf[c].y;
  } else {
    out[3 * (size_t)j] = X[0];
    out[3 * (size_t)j + 1] = X[1];
    out[3 * (size_t)j + 2] = X[2];
  }
}

}  // namespace

povar_status launch_update(Problem* p, int precision, int manifold) {
  const unsigned g = grid_for(p->nc, 128);
  if (precision == POVAR_FP64)
    k_update<double><<<g, 128, 0, p->stream>>>(p->state, manifold, p->nc, p->P64[0],
                                               p->P64[1], p->D64);
  else
    k_update<float><<<g, 128, 0, p->stream>>>(p->state, manifold, p->nc, p->P64[0],
                                              p->P64[1], p->D32);
  ++p->launches;
  return check_launch(p, "update");
}

povar_status launch_controller(Problem* p, int precision) {
  k_controller<<<1, 1, 0, p->stream>>>(p->state, p->d_report, precision);
  ++p->launches;
  return check_launch(p, "controller");
}

povar_status launch_init_state(Problem* p, double lambda0, int reset_lm, int reset_all) {
  k_init_state<<<1, 1, 0, p->stream>>>(p->state, lambda0, reset_lm, reset_all);
  ++p->launches;
  return check_launch(p, "init_state");
}

namespace {

// Loop condition of a batch solve's device-side while node: one more batch
// step while some problem has not converged and fewer than loops[1] steps
// ran (loops[0] counts them).
__global__ void k_batch_continue(cudaGraphConditionalHandle h,
                                 DeviceState* const* __restrict__ states, int n,
                                 int* __restrict__ loops) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int l = loops[0] + 1;
  loops[0] = l;
  int any = 0;
  for (int k = 0; k < n; ++k) any |= states[k]->converged ? 0 : 1;
  cudaGraphSetConditional(h, (any && l < loops[1]) ? 1u : 0u);
}

}  // namespace

cudaError_t add_batch_continue(cudaGraph_t body, const cudaGraphNode_t* deps, size_t ndeps,
                               cudaGraphConditionalHandle h, DeviceState** d_states, int n,
                               int* d_loops) {
  cudaKernelNodeParams kp = {};
  void* args[] = {&h, &d_states, &n, &d_loops};
  kp.func = reinterpret_cast<void*>(k_batch_continue);
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(32);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaGraphNode_t node;
  return cudaGraphAddKernelNode(&node, body, deps, ndeps, &kp);
}

povar_status launch_begin(Problem* p, double ftol, double target, int max_iters,
                          int fallback_after) {
  k_begin<<<1, 1, 0, p->stream>>>(p->state, ftol, target, max_iters, fallback_after);
  ++p->launches;
  return check_launch(p, "begin");
}

povar_status launch_random_cameras(Problem* p, uint64_t seed, int normalize) {
  k_random_cameras<<<grid_for(p->nc, 128), 128, 0, p->stream>>>(p->P64[0], p->nc, seed,
                                                                normalize);
  ++p->launches;
  return check_launch(p, "random_cameras");
}

povar_status launch_gather_points(Problem* p, double* d_out) {
  k_gather_points<<<grid_for(p->np, 256), 256, 0, p->stream>>>(p->state, p->X64[0], p->X64[1],
                                                               p->pt_slot, p->np, d_out);
  ++p->launches;
  return check_launch(p, "gather_points");
}

}  // namespace povar
