/*
 * povar.h -- C-ABI of libpovar, a GB300-native (sm_103a) implementation of
 * the Power Variable Projection (PoVar) inner solve for initialization-free
 * bundle adjustment (Weber, Hong, Cremers, ECCV 2024).
 *
 * The problem statement follows the paper's first stage: given only image
 * measurements m_ij of landmark j in camera i (Sec. 3, observation set
 * Omega), n_p projective 3x4 cameras and n_l landmarks (Eq. ba_first_stage),
 * minimize the pOSE cost (Eq. pose) with weight eta by damped Variable
 * Projection (Sec. 4.1) whose reduced camera system is inverted by the
 * truncated power series of Sec. 4.2 (PoVar), optionally restricted to the
 * tangent space of the unit-norm camera manifold (Sec. 4.3).
 *
 * Conventions shared by every call
 *  - All arrays passed in or out are HOST arrays owned by the caller; the
 *    library copies inputs and writes outputs into caller-allocated memory.
 *    The problem handle owns all device memory until povar_destroy.
 *  - Cameras are 3x4 matrices stored row-major, 12 doubles per camera
 *    (rows p1, p2, p3). Landmarks are 3 doubles (X, Y, Z); the homogeneous
 *    landmark is (X, Y, Z, 1).
 *  - Measurements are normalized image coordinates (pixel - pp) / f,
 *    2 doubles (u, v) per observation.
 *  - Every call returns a povar_status; nothing aborts or throws across the
 *    ABI. After an error, povar_last_error() describes it.
 *  - A handle is used by one host thread at a time; handles are independent.
 *  - Device work is issued on the CUDA stream given to povar_create (NULL =
 *    the legacy default stream). Calls that return host data synchronize that
 *    stream before returning.
 */
#ifndef POVAR_H
#define POVAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct povar_problem povar_problem; /* opaque; owns device memory */

typedef enum {
  POVAR_OK = 0,
  POVAR_EINVAL = 1,          /* invalid argument (sizes, indices, params) */
  POVAR_ENOMEM = 2,          /* device or host allocation failed */
  POVAR_ECUDA = 3,           /* a CUDA runtime call or kernel launch failed */
  POVAR_ENUMERIC = 4,        /* non-finite cost or step on the device */
  POVAR_ETIMEOUT = 5,        /* reserved: a bounded device wait gave up */
  POVAR_ENOTCONVERGED = 6    /* damping diverged (step rejected repeatedly) */
} povar_status;

enum { POVAR_EUCLID = 0, POVAR_SPHERE = 1 };
enum { POVAR_FP64 = 0, POVAR_MIXED_FP32 = 1, POVAR_MIXED_BF16 = 2 };
enum { POVAR_BF16_FP32_TERMS = 6 };  /* POVAR_MIXED_BF16: terms 1..5 in FP32 */

/* Solver parameters (Sec. 5.2 of the paper gives eta = 0.1, lambda0 = 1e-4,
 * series order 20 with threshold 0.01).
 *  eta        pOSE weight in [0, 1] (Eq. pose).
 *  lambda0    initial damping of the camera block (D_p = I); used by the
 *             first step after povar_create / povar_set_cameras /
 *             povar_init_random (later steps use the adapted damping).
 *  series_eps series threshold: after term k >= 1 the series stops when
 *             ||x_k||_2 <= series_eps * ||delta_k||_2; 0 runs exactly m terms.
 *  lambda_l   0: PoVar (Sec. 4: VarPro, landmarks eliminated in closed form,
 *             V_0 undamped). > 0: PoBA, the comparison solver of Sec. 2 /
 *             Sec. 5.2 -- joint Levenberg-Marquardt over cameras and
 *             landmarks with landmark damping lambda_l * lambda (1 = the
 *             joint damping of PoBA): the same series inverts the damped
 *             Schur complement U_lambda - W V_lambda^-1 W^T, the landmarks
 *             follow by back-substitution and are not re-eliminated, pred is
 *             the Gauss-Newton model decrease. Landmark blocks and
 *             back-substitution are FP64 in both precisions;
 *             POVAR_MIXED_BF16 is not available with PoBA (POVAR_EINVAL).
 *  m          number of series terms, >= 1 (delta = sum_{i<m} M^i U^-1 g; the
 *             paper's "order 20" is m = 21).
 *  manifold   POVAR_EUCLID (unconstrained cameras, Eq. ba_first_stage) or
 *             POVAR_SPHERE (unit-norm cameras, tangent-space step and
 *             retraction by normalization, Sec. 4.3).
 *  precision  POVAR_FP64: every kernel in FP64.
 *             POVAR_MIXED_FP32: series and linearization in FP32; landmark
 *             elimination, 12x12 inverses, cost and gain ratio in FP64.
 *             POVAR_MIXED_BF16: POVAR_MIXED_FP32 whose series terms from
 *             term POVAR_BF16_FP32_TERMS on read the stored blocks of
 *             schedule 4 in bfloat16 (18 bytes per observation) and
 *             accumulate in FP32; the leading terms x_1 .. x_5 read the
 *             FP32 factors (the fused pass of schedule 1), where the
 *             rounding of the blocks would weigh most. The blocks are
 *             rounded, so its steps differ from the FP32 ones by about the
 *             bfloat16 rounding (2^-9 relative per block entry) of the
 *             later terms. params->schedule must be -1 or 4. The
 *             predicted decrease is computed in FP32 from the unrounded
 *             factors.
 *  schedule   series schedule: 0 = landmark-major gather pass + camera-major
 *             scatter pass over observation chunks; 1 = one fused
 *             landmark-major pass whose camera contributions are reduced
 *             across the lanes of a warp that share a camera; 2 =
 *             landmark-major gather pass + camera-major pass over the
 *             landmark slice rows that contain each camera; 3 = the fused
 *             pass of 1 where the camera of every slice row whose lanes all
 *             see one camera comes from a per-row table, and the rows of
 *             those cameras are staged in shared memory before the row loop
 *             (no dependent global load per row); 4 = the fused pass of 1
 *             reading, per observation, the stored 3x3 block
 *             G_k = B_k^T B_k Pbar_i (B_k^T times the landmark Jacobian block
 *             of Eq. pose; Pbar_i the left 3x3 of camera i), written once
 *             per step at the current cameras (72 / 36 bytes per SELL entry
 *             in FP64 / FP32, allocated at first use) instead of the camera
 *             rows and the measurement; 5 = groups of slices whose
 *             rows are all warp-uniform and see the same camera at each row
 *             index (tracks over the same consecutive cameras): one block
 *             per group stages the rows' cameras and the landmarks' s_j in
 *             shared memory and reduces once per row (at most 20 slices
 *             and 128 slice rows per group);
 *             other slices run the fused pass of 1; -1 = autotuned (see
 *             povar_get_tuning). All schedules compute the same series (up
 *             to rounding order). */
enum { POVAR_NSCHEDULES = 6 };
/*  solver     POVAR_SOLVER_SERIES (0): the power series above.
 *             POVAR_SOLVER_PCG (1): the "iterative" baseline of Sec. 5.2 --
 *             conjugate gradients on the same (damped, tangent-projected)
 *             reduced camera system from delta = 0, preconditioned by the
 *             inverse 12x12 diagonal blocks of the Schur complement
 *             (Schur-Jacobi). Then m is the maximum number of inner
 *             iterations (500 in Sec. 5.2) and series_eps the relative
 *             residual tolerance: the iteration stops when
 *             ||g - S delta||_2 <= series_eps * ||g||_2 (0 runs exactly m
 *             iterations). One landmark pass of schedule 1 per iteration
 *             (params->schedule is not used). PCG steps are issued without
 *             a CUDA graph and read a device flag every 8 iterations; they
 *             are not available in a batch (POVAR_EINVAL there).
 *             POVAR_MIXED_BF16 is not available with PCG (POVAR_EINVAL). */
enum { POVAR_SOLVER_SERIES = 0, POVAR_SOLVER_PCG = 1 };
typedef struct {
  double eta;
  double lambda0;
  double series_eps;
  double lambda_l;
  int32_t m;
  int32_t manifold;
  int32_t precision;
  int32_t schedule;
  int32_t solver;
  int32_t reserved;    /* must be 0 */
} povar_params;

/* Report of one damped VarPro iteration. cost_before is F at the iterate the
 * step started from, cost_after is F at the trial cameras (with landmarks
 * re-solved in closed form), pred the predicted decrease
 * 2 g^T d - d^T (S - lambda I) d, rho = (cost_before - cost_after) / pred.
 * The step is accepted iff cost_after < cost_before. */
typedef struct {
  double cost_before;
  double cost_after;
  double pred;
  double rho;
  double lambda_used;
  double lambda_next;
  int32_t accepted;
  int32_t terms_used;
  int32_t iteration;
  int32_t converged;
  float ms;                  /* device time of the step (0 if not measured) */
  int32_t precision;         /* precision the step ran in (POVAR_FP64 after the
                                mixed-precision safeguard of povar_solve) */
  int32_t fp64_fallback_at;  /* povar_solve: iteration at which the safeguard
                                switched to FP64 (0: it did not) */
  float reserved[1];
} povar_step_report;

/* Create a problem from the observation set Omega (Sec. 3):
 *  n_cams, n_points  number of cameras (n_p) and landmarks (n_l), >= 1.
 *  n_obs             number of observations, >= 1.
 *  cam_idx[n_obs]    camera index of each observation, 0 <= . < n_cams.
 *  pt_idx[n_obs]     landmark index of each observation, 0 <= . < n_points.
 *  meas[2*n_obs]     normalized measurement (u, v) of each observation.
 *  cuda_stream       cudaStream_t to issue work on (NULL = default stream).
 * Every landmark must be observed at least once (else POVAR_EINVAL); a
 * camera without observations is allowed (its step is zero). Sizes are
 * checked on the host before anything is allocated; indices out of range and
 * non-finite measurements are found by a device check right after the copy
 * of the arrays, before any index is used (POVAR_EINVAL, nothing is kept).
 * Builds the camera-major and point-major observation orders, the landmark
 * layout and the run tables of the series on the device (stable integer
 * sorts, bit-exact) and allocates all device state. The arrays are only read
 * during the call.
 * Cameras start at zero: call povar_set_cameras or povar_init_random. */
povar_status povar_create(int32_t n_cams, int32_t n_points, int64_t n_obs,
                          const int32_t* cam_idx, const int32_t* pt_idx,
                          const double* meas, void* cuda_stream,
                          povar_problem** out);

/* Release all device and host memory of the handle (NULL is a no-op). */
void povar_destroy(povar_problem* p);

/* Text of the last error on this handle ("" if none). Owned by the handle. */
const char* povar_last_error(const povar_problem* p);

/* Set the cameras (n_cams x 12 row-major doubles) and re-solve every
 * landmark in closed form (Eq. update_landmark) at pOSE weight eta. Resets
 * the damping state: the next step starts from params->lambda0. P may be a
 * host pointer (checked for finite values) or a device pointer of the
 * handle's device (copied device to device, not checked). */
povar_status povar_set_cameras(povar_problem* p, const double* P, double eta);

/* Random initialization of the paper's experiments (Sec. 5.2): every camera
 * entry iid N(0, 1) from a counter-based Philox4x32-10 stream keyed by
 * seed, normalized to unit Frobenius norm when manifold == POVAR_SPHERE;
 * landmarks then follow in closed form. Resets the damping state. */
povar_status povar_init_random(povar_problem* p, uint64_t seed, int32_t manifold,
                               double eta);

/* Copy the current cameras (n_cams x 12) / landmarks (n_points x 3) out. */
povar_status povar_get_cameras(povar_problem* p, double* P_out);
povar_status povar_get_points(povar_problem* p, double* X_out);

/* ---- Second stage: projective refinement (Eq. second_stage) by Riemannian
 * PoBA (RiPoBA, Sec. 4.3), on the same observations and handle.
 * Cameras P_i are 3x4 with vec(P_i) on the unit sphere of R^12 (the same
 * camera buffers as the first stage, row-major); landmarks are homogeneous
 * 4-vectors on the unit sphere of R^4. The cost is
 *   F2 = sum over observations of ||(y1 / y3, y2 / y3) - m_ij||^2,
 *   y = P_i X_j,
 * with the normalized measurements given to povar_create. A step is joint
 * Levenberg-Marquardt on both tangent spaces (projected normal equation of
 * Sec. 4.3, damping lambda on the cameras and lambda_l * lambda on the
 * landmarks, D = I): the power series (Lemma 2) inverts the damped
 * Riemannian Schur complement, the landmarks follow by back-substitution,
 * cameras and landmarks are retracted by normalization, pred is the
 * Gauss-Newton model decrease, and accept/reject and the damping rule are
 * the first stage's.
 *
 * povar_s2_set: start the second stage. P (host, n_cams*12) and X (host,
 * n_points*4, by landmark id), both finite; rows are normalized by the
 * library. With P == X == NULL the start is the first stage's result:
 * the current cameras (normalized) and the homogeneous (X_j, 1) of the
 * first stage's closed-form landmarks at them (re-solved in FP64 when the
 * last step was mixed); POVAR_EINVAL if there is no first-stage state or
 * if only P is given. Computes the cost; the next povar_s2_step / solve
 * starts with damping params->lambda0. Synchronizes the stream.
 * povar_s2_cost: F2 at the current iterate.
 * povar_s2_step / povar_s2_solve: as povar_step / povar_solve (same
 * report, stop rules and mixed-precision safeguard) for the second stage.
 * params: m, series_eps, lambda0 as for the first stage; lambda_l > 0
 * (1 = the paper's joint damping); manifold must be POVAR_SPHERE;
 * precision POVAR_FP64 or POVAR_MIXED_FP32 (FP32 series terms, camera
 * vectors, sums of the camera linearization and the linearized terms of the
 * trial (W^T dP, J dP + J dX); landmark blocks and their inverses,
 * projections, residuals, back-substitution and cost in FP64); solver POVAR_SOLVER_SERIES; schedule 0 = a landmark-major pass
 * (s_j per landmark) and a camera-major pass over the observation chunks,
 * 1 or -1 = one landmark-major pass whose camera contributions are summed
 * over the runs of equal camera in each slice row (the first stage's
 * schedule 1); eta is not used. Steps are issued without a CUDA graph.
 * povar_s2_get_points: the current homogeneous landmarks (n_points*4, by
 * landmark id); the cameras come from povar_get_cameras.
 * A first-stage call after second-stage steps re-solves the first stage's
 * landmarks at the current cameras; a second-stage call after first-stage
 * steps recomputes F2 and restarts the damping. POVAR_EINVAL before the
 * first povar_s2_set. */
povar_status povar_s2_set(povar_problem* p, const double* P, const double* X);
povar_status povar_s2_cost(povar_problem* p, double* cost_out);
povar_status povar_s2_step(povar_problem* p, const povar_params* params,
                           povar_step_report* report);
povar_status povar_s2_solve(povar_problem* p, const povar_params* params, int32_t max_iters,
                            double ftol, double target_cost, povar_step_report* last,
                            int32_t* iters_out);
povar_status povar_s2_get_points(povar_problem* p, double* X_out);

/* ---- Metric upgrade (the third stage of the stratified problem;
 * supplementary section "Metric Upgrade"): finds H = H_0 [[I, 0], [c^T, 1]]
 * such that K_i^-1 P_i H ~ [R_i t_i] for the handle's current cameras P_i
 * (after either stage). H_0 puts the calibrated camera 0, K_0^-1 P_0, at
 * [I | 0]; c (the plane at infinity up to sign) and a scale alpha_i per
 * camera minimize sum_i ||alpha_i B_i H~ H~^T B_i^T - I||_F^2 with
 * B_i = K_i^-1 P_i H_0 and H~ = [[I], [c^T]], by Variable Projection: the
 * alpha_i in closed form, Levenberg-Marquardt on c (lambda0 = 1e-4, the
 * first stage's damping rule, stop on an accepted step whose relative
 * decrease is below ftol, or after max_iters iterations) from the linear
 * estimate of the dual absolute quadric H~ H~^T. All in FP64.
 * K: n_cams row-major 3x3 intrinsics on the host (invertible), or NULL for
 * the identity (measurements already normalized). H_out: 16 doubles,
 * row-major. alpha_out (n_cams, may be NULL): the scales; the metric camera
 * i is sqrt(|alpha_i|) K_i^-1 P_i H up to sign. cost_out, iters_out may be
 * NULL. POVAR_EINVAL for fewer than 3 cameras, a singular K_i or reference
 * camera, non-finite K; the cameras are not changed. Synchronizes the
 * stream. */
povar_status povar_metric_upgrade(povar_problem* p, const double* K, int32_t max_iters,
                                  double ftol, double* H_out, double* alpha_out,
                                  double* cost_out, int32_t* iters_out);

/* pOSE cost F = ||r||^2 (Eq. ba_first_stage) at the current cameras with
 * the landmarks at their closed-form optimum for this eta. */
povar_status povar_cost(povar_problem* p, double eta, double* cost_out);

/* One damped VarPro iteration (Sec. 4.1-4.3): linearize at (P, X*(P)),
 * damped tangent-space camera blocks, PoVar series for the reduced camera
 * system, predicted decrease, update + retraction, closed-form landmarks at
 * the trial cameras, cost, gain ratio, accept/reject, damping update.
 * report may be NULL. Synchronizes the stream. */
povar_status povar_step(povar_problem* p, const povar_params* params,
                        povar_step_report* report);

/* Iterate povar_step until an accepted step has relative decrease below
 * ftol, the cost reaches target_cost (if > 0), or max_iters steps ran.
 * last (may be NULL) receives the report of the last step, iters_out (may
 * be NULL) the number of steps taken. Steps are issued without a host
 * round-trip in between; the stream is synchronized every few steps.
 *
 * Mixed-precision safeguard (POVAR_MIXED_FP32 / POVAR_MIXED_BF16; not in
 * the paper): when POVAR_FALLBACK_REJECTIONS consecutive mixed steps are
 * rejected, or the damping grows 1e10 times above its value at the start
 * of the solve (or diverges), the remaining steps of this solve run in
 * POVAR_FP64 (same schedule rule, landmarks re-solved in FP64 first,
 * damping reset to the smallest one of the solve). FP32 series and
 * linearizations cannot resolve the reduced camera system where it is a
 * strong cancellation of much larger terms (e.g. landmarks drifting towards
 * infinity at a small pOSE weight); there every damping is rejected and a
 * pure mixed solve would stall. last->fp64_fallback_at reports the iteration
 * at which it switched. povar_step and the batch solves never switch. */
enum { POVAR_FALLBACK_REJECTIONS = 10 };
povar_status povar_solve(povar_problem* p, const povar_params* params,
                         int32_t max_iters, double ftol, double target_cost,
                         povar_step_report* last, int32_t* iters_out);

/* ---- diagnostics (inspection of intermediate results for testing) ---- */

/* Landmark layout and run tables built by povar_create (the SELL-32 layout
 * of the series and landmark kernels). sizes[6] receives np_pad (slots),
 * n_slices, n_sell (slice entries), n_rows (slice rows), n_part (run
 * partials), n_visits (camera-row visits); call with NULL arrays to get them.
 * slot_pt[np_pad]: landmark of each slot (0xffffffff for padding);
 * sell_off[n_slices + 1]: first entry of each slice; sell_cam[n_sell]: camera
 * of each entry (-1 for padding); row_mask[n_rows] / row_base[n_rows]: runs of
 * each slice row (0 = all valid lanes see one camera) and its first partial;
 * cam_part_off[n_cams + 1] / cam_part_idx[n_part]: partials of each camera in
 * increasing index. Any array may be NULL; arrays are host memory. */
povar_status povar_get_layout(povar_problem* p, int64_t* sizes, uint32_t* slot_pt,
                              uint32_t* sell_off, int32_t* sell_cam, uint32_t* row_mask,
                              uint32_t* row_base, uint32_t* cam_part_off,
                              uint32_t* cam_part_idx);

/* Observation orders built by povar_create: perm_pt[n_obs] lists the
 * observation ids sorted by (landmark, id), off_pt[n_points + 1] the segment
 * starts; perm_cam / off_cam the same by (camera, id). Any pointer may be
 * NULL. */
povar_status povar_get_orders(povar_problem* p, uint32_t* perm_pt, uint32_t* off_pt,
                              uint32_t* perm_cam, uint32_t* off_cam);

/* Linearization of the last step (undamped U_i = J_p^T J_p as n_cams x 144
 * row-major, and b_p = J_p^T r as n_cams x 12) and the step delta of the
 * last step in the ambient camera space (n_cams x 12, tangent to the
 * unit sphere in POVAR_SPHERE mode). Any pointer may be NULL. */
povar_status povar_get_last_step(povar_problem* p, double* U_out, double* bp_out,
                                 double* delta_out);

/* Phase timing with CUDA events recorded on the handle's stream around each
 * phase of every step (no extra host synchronization). Phases, in order:
 * 0 linearization, 1 damped camera blocks + first term, 2 series terms,
 * 3 predicted decrease, 4 camera update, 5 landmarks + cost at the trial
 * cameras, 6 controller. povar_get_profile writes, per phase, the summed
 * device milliseconds (ms_out[POVAR_NPHASES]), the number of timed steps
 * (steps_out) and the number of series products M y computed by those steps
 * (products_out: terms used minus one per step, so the per-product time of
 * phase 2 is ms_out[2] / products_out), and zeroes the counters when
 * reset != 0. Output pointers may be NULL. Timing applies to povar_step and
 * povar_solve issued while enabled; in povar_solve, which runs each step as
 * one CUDA graph, the phase events are part of the graph and the steps that
 * end at a host synchronization point (every fourth step and the last one)
 * are sampled, skipping a sampled launch that found the solve already
 * converged and did no work. */
enum { POVAR_NPHASES = 7 };
povar_status povar_set_profiling(povar_problem* p, int32_t enable);
povar_status povar_get_profile(povar_problem* p, double* ms_out, int64_t* steps_out,
                               int64_t* products_out, int32_t reset);

/* Series-schedule autotuner. The first povar_solve with params->schedule
 * = -1 times every schedule (0 .. POVAR_NSCHEDULES-1) on the live state
 * with CUDA events (one warm-up term, then three timed terms; a second
 * round re-times the schedules within 15% of the first round's fastest)
 * and keeps the fastest for that precision; the per-step build of the
 * stored blocks of schedule 4 is timed too and charged to that schedule
 * spread over the m - 1 terms of a step. Later solves and povar_step with
 * schedule -1 use it. povar_get_tuning returns the chosen schedule (-1
 * before tuning) and the measured milliseconds per series term
 * (ms_out[POVAR_NSCHEDULES], may be NULL) for POVAR_FP64 or
 * POVAR_MIXED_FP32 (POVAR_MIXED_BF16 is not tuned: POVAR_EINVAL). */
povar_status povar_get_tuning(povar_problem* p, int32_t precision, int32_t* schedule_out,
                              float* ms_out);

/* Device memory held by a handle (bytes), and an upper-bound estimate of
 * it from the problem sizes alone, for admission control before
 * povar_create. Handles take their device memory from a memory pool that the
 * library keeps per device; memory of destroyed handles stays in that pool
 * for later handles until povar_release_cached_memory returns it to the
 * device. */
int64_t povar_device_bytes(const povar_problem* p);
int64_t povar_estimate_bytes(int32_t n_cams, int32_t n_points, int64_t n_obs);
void povar_release_cached_memory(void);

/* Number of kernel launches this handle has issued so far. */
int64_t povar_launch_count(const povar_problem* p);

/* ---- batches of independent problems ----
 * Many independent problems of uneven sizes, given as concatenated arrays
 * with per-problem sizes: problem k has n_cams[k] cameras, n_points[k]
 * landmarks and n_obs[k] observations; its observations follow those of
 * problems 0..k-1 in cam_idx / pt_idx / meas (2 doubles each), with indices
 * local to the problem. Cameras of all problems are concatenated likewise
 * (12 doubles per camera). povar_batch_solve runs the whole solve as one
 * CUDA-graph launch: a device-side while loop (a conditional graph node)
 * whose body holds one step of every problem (the problems' step graphs as
 * child graphs, without dependencies between problems, so their kernels
 * overlap) followed by a one-thread kernel that repeats the body while some
 * problem has not converged and fewer than max_iters steps ran; each problem
 * stops on its own device-side convergence flag and the host waits once, at
 * the end. When the problems' phase profiling is on (povar_set_profiling),
 * or the loop cannot be built, every step is one launch and the host checks
 * the flags every fourth step. With schedule -1, a problem of at most
 * 262,144 observations runs schedule 0 in a batch (kernels that leave room
 * for the other problems' blocks; the 64-problem batched family runs 1.8x
 * faster than with each problem's own autotuned choice), a larger one
 * picks its own series schedule by the autotuner of povar_solve before the
 * first iteration. Results are identical to solving each problem alone with
 * the same parameters and schedule. target_costs, reports and iters_out
 * hold one entry per problem (each may be NULL). */
typedef struct povar_batch povar_batch;
povar_status povar_batch_create(int32_t n_problems, const int32_t* n_cams,
                                const int32_t* n_points, const int64_t* n_obs,
                                const int32_t* cam_idx, const int32_t* pt_idx,
                                const double* meas, void* cuda_stream, povar_batch** out);
void povar_batch_destroy(povar_batch* b);
const char* povar_batch_last_error(const povar_batch* b);
povar_problem* povar_batch_problem(povar_batch* b, int32_t k);
povar_status povar_batch_set_cameras(povar_batch* b, const double* P, double eta);
povar_status povar_batch_get_cameras(povar_batch* b, double* P_out);
povar_status povar_batch_cost(povar_batch* b, double eta, double* costs_out);
povar_status povar_batch_solve(povar_batch* b, const povar_params* params, int32_t max_iters,
                               double ftol, const double* target_costs,
                               povar_step_report* reports, int32_t* iters_out);
/* povar_batch_solve with one parameter set per problem: params[k] for
 * problem k (n_problems entries; e.g. a series length m per problem size from
 * a tuning table). Each problem's result equals solving it alone with
 * params[k]. */
povar_status povar_batch_solve_each(povar_batch* b, const povar_params* params,
                                    int32_t max_iters, double ftol, const double* target_costs,
                                    povar_step_report* reports, int32_t* iters_out);

/* ---- allocation-free cost evaluation ----
 * No counterpart in the paper: a library utility. It returns the pOSE cost
 * at the given cameras with every landmark eliminated in closed form (each
 * landmark is the least-squares point of its observations for those cameras,
 * a pseudo-inverse where its 3x3 normal block is rank-deficient), all in
 * FP64: the same value as povar_set_cameras + povar_cost + povar_get_points,
 * but without a problem handle and without allocating any memory.
 *
 * Who needs it: callers that must not allocate at the point of the call.
 * cudaMalloc and cudaFree synchronize the device, so a latency-critical loop
 * that evaluates a candidate camera set while other work is in flight cannot
 * afford them; a process whose device memory is fully reserved by another
 * allocator (a caching allocator holding the whole pool, a fixed arena)
 * cannot obtain more; and a caller that only needs the cost of a few camera
 * sets does not want to build and keep a handle (observation orders, series
 * buffers) for it. The working memory is one fixed array inside the library
 * (per-block cost partials, POVAR_NOALLOC_MAX_POINTS / 256 doubles = 128 KB),
 * which bounds the problem size.
 *
 * Inputs (all DEVICE pointers, caller-owned, only read): P = n_cams x 12
 * row-major FP64 cameras, 16-byte aligned; the observations in
 * landmark-major order: off_pt[n_points + 1] (u32, observations of landmark
 * j are off_pt[j] .. off_pt[j+1]-1), cam[n_obs] (i32 camera index) and
 * meas[n_obs x 2] (FP64 normalized coordinates, 16-byte aligned). Outputs
 * (DEVICE pointers, caller-owned, 8-byte aligned): cost_out[1] receives the
 * cost; X_out (n_points x 3 FP64, may be NULL) receives the landmarks. Work
 * is enqueued on cuda_stream (NULL = legacy default stream) and nothing is
 * synchronized: the outputs are ready when the stream reaches this point.
 *
 * Errors: POVAR_EINVAL for a NULL pointer, a size < 1, eta outside [0, 1],
 * n_points > POVAR_NOALLOC_MAX_POINTS (the fixed working array would be too
 * small), or a pointer that is not aligned as stated above (P and meas to 16
 * bytes, off_pt and cam to 4, cost_out and X_out to 8); these checks make no
 * CUDA call and nothing is launched. POVAR_ECUDA, with nothing launched, if
 * a CUDA error from earlier work is already pending on the calling thread
 * (it is left pending for its owner); POVAR_ECUDA also if the set-up or a
 * launch of this call fails. Index errors are detected on the device
 * without a host round trip: a camera index outside [0, n_cams) or an
 * offset table that is decreasing or points past n_obs makes *cost_out NaN
 * (the offending observations are skipped, never read out of bounds).
 *
 * Set-up and concurrency: the first call on each device (with that device
 * current) looks up the device address of the library's working array
 * (cudaGetSymbolAddress, which also loads the library's device code if it
 * is not yet loaded); make that first call before any stream capture. The
 * address is kept for the life of the process: after cudaDeviceReset on a
 * device this entry point must not be called on that device again (the kept
 * address belonged to the destroyed context).
 * All calls on one device share the same working array, so calls whose
 * executions overlap in time (on different streams or from different host
 * threads without ordering between them) race and may return a wrong cost;
 * order them on one stream or with events. */
enum { POVAR_NOALLOC_MAX_POINTS = 4194304 };
povar_status povar_cost_noalloc(int32_t n_cams, int32_t n_points, int64_t n_obs,
                                const double* P, const uint32_t* off_pt, const int32_t* cam,
                                const double* meas, double eta, double* X_out,
                                double* cost_out, void* cuda_stream);

/* Library version string. */
const char* povar_version(void);

#ifdef __cplusplus
}
#endif

#endif /* POVAR_H */
