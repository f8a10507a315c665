// Internal declarations shared by the libpovar translation units.
//
// Data layout in device memory (one problem):
//  * Observations are kept in two device orders built once by povar_create:
//    - point-major "SELL-32" slices: landmarks are renumbered into slots
//      sorted by their smallest camera, then by track length (descending);
//      32 consecutive slots form a slice, and the t-th observation (in
//      camera order) of the slot in lane l of slice s sits at
//      sell_off[s] + 32 t + l. One thread owns one landmark; the loads of a
//      warp are coalesced, and when tracks are contiguous camera windows the
//      lanes of a slice row share one camera (warp-broadcast camera loads).
//    - camera-major list cut into chunks of <= CHUNK observations that never
//      cross a camera boundary; one warp reduces one chunk with shuffles and
//      the last warp of a camera (an atomic ticket) finishes the camera.
//  * Per camera: P (FP64, double-buffered), the damped inverse G (FP64 and
//    FP32), U and b_p (FP64), series vectors Y and delta (FP32 and FP64).
//  * Per landmark slot: X (FP64, double-buffered), the lower-triangular
//    factor F with F^T F = V^-1 (FP64 and FP32 copies), and the series
//    record (s = V^-1 W^T y, X) written by the gather pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/povar.h"

namespace povar {

constexpr int SLICE = 32;        // landmarks per SELL slice (one warp)
constexpr int CHUNK = 512;       // observations per camera-major chunk
constexpr int LIN_ACC = 52;      // linearization accumulators per chunk
constexpr int LIN_PART = 56;     // per-chunk partial: the accumulators, the chunk's centre (3), pad
constexpr int BLOCK = 256;       // threads per block for slot kernels
// Slices per group of the schedule-3 row table (its kernel takes one slice
// per warp). Groups of two and four slices per warp were measured slower on
// the 5M-observation scene (78 and 104 us per series product against 71):
// they save warp reductions, but their registers halve the occupancy of a
// latency-bound loop, and ordering by group width unbalances the blocks of
// the slot kernels.
constexpr int GROUP = 1;
// Group schedule (5): at most G5_SLICES slices, G5_ROWS rows and G5_MROWS
// slice rows (staged measurement rows) per group (one block each, three
// blocks per SM in FP32: 71 KB of shared memory each), work items of at
// most G5_ITEM slices of one row.
constexpr int G5_THREADS = 256;
constexpr int G5_SLICES = 20;
constexpr int G5_ROWS = 64;
constexpr int G5_MROWS = 128;
constexpr int G5_ITEM = 20;
// Blocks of the final cost and predicted-decrease sums (each block adds a
// fixed range, the last block to finish adds the block sums in order).
constexpr int FIN_BLOCKS = 64;
constexpr double PINV_COND = 1e12;
constexpr double LAMBDA_MIN = 1e-8;   // damping floor
constexpr double LAMBDA_MAX = 1e30;   // damping ceiling (solve reported as diverged)
// mixed-precision safeguard: damping growth over its value at the start of a
// solve after which its FP32 steps are taken to have failed
constexpr double FALLBACK_LAMBDA_GROWTH = 1e10;

// Stored observation blocks G_k = C_k Pbar_i (3x3, row-major g[3r + q]) of
// the stored series schedule, one per SELL entry e (E = max(nsell, 1)
// entries per plane), in planes so that the loads of a slice row coalesce:
//   FP64 (72 B): p[0..3] double2 (g0 g1)(g2 g3)(g4 g5)(g6 g7), p[4] double g8
//   FP32 (36 B): p[0], p[1] float4 (g0..g3)(g4..g7), p[2] float g8
//   BF16 (18 B): p[0] 8 x bf16 (g0..g7, g[2k] in the low half of word k),
//                p[1] bf16 g8
struct BlockPlanes {
  void* p[5];
};

// Device-resident LM / VarPro controller state (one per problem).
struct DeviceState {
  double F;          // cost at the current iterate
  double F_new;      // cost at the trial iterate
  double pred;       // predicted decrease of the last step
  double rho;        // gain ratio of the last step
  double lam;        // damping for the next step
  double nu;         // damping growth factor (Madsen-Nielsen)
  double lam_used;   // damping of the last step
  double tvt;        // sum_j ||F_j W^T delta||^2 of the last step
  double ftol;       // relative-decrease stop threshold (0: none)
  double target;     // target cost (<= 0: none)
  int cur;           // index (0/1) of the current P / X buffers
  int iteration;     // steps taken
  int accepted;      // last step accepted
  int need_lin;      // linearization must be recomputed
  int converged;     // stop flag: every step kernel returns immediately
  int stop_series;   // series early-stop flag (per step)
  int terms_used;    // series terms used by the last step
  int error;         // povar_status of a device-detected error
  int max_iters;     // iteration cap for povar_solve (0: none)
  int n_pinv;        // landmarks solved by pseudo-inverse at the last solve
  int n_regularized; // camera blocks whose damping had to be raised (cumulative)
  long long products; // series products M y computed by all steps (never reset)
  int x_df[2];        // landmark buffer t holds X as double-float pairs (1) or FP64 (0)
  int rej_run;        // consecutive rejected steps
  double lam_low;     // smallest damping used by a step of the current solve
  double lam_ref;     // damping at the start of the current solve
  int fallback_after; // mixed-precision safeguard: rejections that trigger it (0: off)
  int fallback;       // set with `converged` when the safeguard triggered
  // conjugate-gradient solver (POVAR_SOLVER_PCG) of the current step
  double pcg_rz;      // r^T z of the current residual
  double pcg_gg;      // g^T g (stop test ||r|| <= eps ||g||)
  double pcg_alpha;   // step length of the current iteration
  double pcg_beta;    // direction update coefficient
  // series threshold rule checked one term late (group schedule): set by
  // the term-t group launch when the rule held after term t - 1, so that
  // term t's camera finish ends the series instead of updating
  int series_halt;
};

// Host-side handle.
struct Problem {
  int32_t nc = 0, np = 0;
  int64_t nobs = 0;
  int32_t np_pad = 0, nslices = 0, nchunks = 0, nc_active = 0;
  int64_t nsell = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t launches = 0;
  double eta_cur = -1.0;   // eta the landmarks / cost were solved for
  bool fresh = true;       // next step re-initializes the damping
  int last_precision = POVAR_MIXED_FP32;

  // inputs (device)
  int32_t* d_cam = nullptr;
  int32_t* d_pt = nullptr;
  double* d_meas = nullptr;
  // orders (a1)
  uint32_t* perm_pt = nullptr;
  uint32_t* off_pt = nullptr;
  uint32_t* perm_cam = nullptr;
  uint32_t* off_cam = nullptr;
  // SELL point-major layout
  uint32_t* slot_pt = nullptr;    // [np_pad] landmark id of a slot (~0u: pad)
  uint32_t* pt_slot = nullptr;    // [np]
  uint32_t* slot_len = nullptr;   // [np_pad]
  uint32_t* sell_off = nullptr;   // [nslices + 1]
  int32_t* sell_cam = nullptr;    // [nsell] (-1: padding)
  float2* sell_m32 = nullptr;
  double2* sell_m64 = nullptr;
  float4* sell_mdf = nullptr;     // [nsell] (u_hi, u_lo, v_hi, v_lo) double-float pairs
  // camera-major list
  uint32_t* cm_slot = nullptr;    // [nobs]
  float2* cm_m32 = nullptr;
  double2* cm_m64 = nullptr;
  uint32_t* chunk_beg = nullptr;  // [nchunks + 1]
  int32_t* chunk_cam = nullptr;   // [nchunks]
  int32_t* cam_nchunk = nullptr;  // [nc]
  int32_t* cam_chunk0 = nullptr;  // [nc]
  uint32_t* cam_ticket = nullptr; // [nc]
  uint32_t* done_ticket = nullptr;// [1]
  // fused-schedule run structure (see build_runs in csr.cu)
  int64_t nrows = 0, npart = 0;
  uint32_t* row_mask = nullptr;     // [nrows]
  uint32_t* row_base = nullptr;     // [nrows]
  uint32_t* cam_part_off = nullptr; // [nc + 1]
  uint32_t* cam_part_idx = nullptr; // [npart]
  void* part_run = nullptr;         // [npart * 12] float or double
  int32_t nc_parts = 0;             // cameras with at least one partial
  // camera-row schedule: for camera i, the slice rows that contain it, as the
  // SELL position and the slot of lane 0 of the row (rows in index order)
  int64_t nvisits = 0;
  uint32_t* cam_row_off = nullptr;  // [nc + 1]
  uint32_t* cam_row_pos0 = nullptr; // [nvisits]
  uint32_t* cam_row_slot0 = nullptr;// [nvisits]
  // grouped schedule (3): one warp handles up to GROUP consecutive slices
  // whose first landmarks share the smallest camera; a group row (row t of
  // all the group's slices) whose valid lanes all see one camera yields a
  // single partial; other group rows fall back to per-slice-row runs
  int32_t ngroups = 0;
  int64_t ngrows = 0, npart3 = 0;
  uint32_t* grp_slice0 = nullptr;       // [ngroups + 1] first slice of each group
  uint32_t* grp_row0 = nullptr;         // [ngroups + 1] first group row of each group
  int32_t* grow_cam = nullptr;          // [ngrows] camera of a group-uniform row, else -1
  uint32_t* grow_base = nullptr;        // [ngrows] partial of a group-uniform row
  uint32_t* srow_mask = nullptr;        // [nrows] runs of slice rows in non-uniform group rows
  uint32_t* srow_base = nullptr;        // [nrows]
  // with one slice per group (GROUP = 1) the grouped partials are the
  // fused ones: these alias cam_part_off, cam_part_idx and part_run
  uint32_t* cam_part3_off = nullptr;    // [nc + 1]
  uint32_t* cam_part3_idx = nullptr;    // [npart3]
  void* part3 = nullptr;                // [npart3 * 12] float or double
  // group schedule (5): groups of slices whose rows are all warp-uniform and
  // that see the same camera at every row index; work items (row, slice
  // range) of each group; slices outside groups (g5_rest) run the fused pass;
  // per camera the item partials, then the run partials of its rows outside
  // groups, in a fixed order; an item's partial is stored at its position
  // in these lists (g5_idest), the run partials after all lists (offset by
  // g5_nlist)
  int32_t g5_ngroups = 0, g5_nrest = 0;
  int64_t g5_nitems = 0, g5_nslices = 0, g5_obs = 0, g5_nlist = 0;
  uint32_t* g5_off = nullptr;        // [ngroups + 1] slices of group g in g5_slices
  uint32_t* g5_slices = nullptr;     // [grouped slices] slice indices, widest first
  uint32_t* g5_roff = nullptr;       // [ngroups + 1] rows of group g in g5_rowcam
  int32_t* g5_rowcam = nullptr;      // camera of each group row
  uint32_t* g5_ioff = nullptr;       // [ngroups + 1] items of group g
  uint32_t* g5_items = nullptr;      // (row << 16) | (first slice << 8) | end slice
  uint32_t* g5_idest = nullptr;      // [nitems] list position of each item's partial
  uint32_t* g5_rest = nullptr;       // [nrest] slices outside groups
  uint32_t* g5_sinfo = nullptr;      // [4 * G5_SLICES * ngroups] per group and slice: slice,
                                     // first SELL entry, width, first staged measurement
                                     // row (zero past the group's slices)
  int32_t* g5_ghdr = nullptr;        // [2 * ngroups] staged measurement rows, first row
                                     // camera when the rows' cameras are consecutive (else -1)
  uint32_t* cam5_off = nullptr;      // [nc + 1]
  uint32_t* cam5_idx = nullptr;      // [nlist] partial of each list entry (an item's own
                                     // position, or nlist + run partial index)
  uint32_t* cam5_ndirect = nullptr;  // [nc] item partials at the head of camera i's list
  void* part5 = nullptr;             // [(nlist + npart) * 12] float or double
  // stored series blocks per kind (0 FP64, 1 FP32, 2 BF16), allocated at
  // first use and rebuilt by every step that runs the stored schedule
  void* blk[3] = {nullptr, nullptr, nullptr};
  int schedule_default = 1;         // chosen at creation from the run statistics
  int tuned_schedule[2] = {-1, -1}; // autotuned series schedule per precision (-1: not yet)
  float tune_ms[2][POVAR_NSCHEDULES] = {};  // measured ms per series term, per schedule
  // cameras
  double* P64[2] = {nullptr, nullptr};  // [nc*12]
  double* Ltab = nullptr;               // [nc*48] landmark tables at trial P
  float2* Ltab_df = nullptr;            // [nc*48] the same tables (36) and P (12) as double-floats
  bool lm_df = false;                   // current landmark buffers come from the double-float kernel
  float* camP32[2] = {nullptr, nullptr};  // [nc*12] FP32 copies of P64[0], P64[1]
  double* U64 = nullptr;                // [nc*144]
  double* bp64 = nullptr;               // [nc*12]
  double* G64 = nullptr;                // [nc*144]
  float* G32 = nullptr;                 // [nc*144]
  float* Y32 = nullptr;                 // [2*nc*12] series vector, double-buffered by term parity
  float* D32 = nullptr;                 // [nc*12]
  double* Y64 = nullptr;                // [2*nc*12]
  double* D64 = nullptr;
  double* camnorm = nullptr;            // [nc*2]
  void* part_lin = nullptr;             // [nchunks*LIN_ACC] float or double
  void* part_ser = nullptr;             // [nchunks*12] float or double
  // landmark slots
  double* X64[2] = {nullptr, nullptr};  // [np_pad*3]
  double* F64[2] = {nullptr, nullptr};  // [np_pad*6] factor F (V^-1 = F^T F)
  float4* pdA[2] = {nullptr, nullptr};  // (X0, X1, X2, F00)
  float4* pdB[2] = {nullptr, nullptr};  // (F10, F11, F20, F21)
  float* pdC[2] = {nullptr, nullptr};   // F22
  float4* rec32 = nullptr;              // [np_pad*2] (s0 s1 s2 X0)(X1 X2 - -)
  // PoBA (allocated at first use): s_j = V_lambda^-1 b_l per slot
  double* sbl64 = nullptr;              // [np_pad*3]
  float4* sbl32 = nullptr;              // [np_pad] (s0 s1 s2 -)
  bool lm_poba = false;                 // landmarks are PoBA iterates, not X*(P)
  // second stage (allocated at first use): homogeneous landmarks per slot
  double* s2X[2] = {nullptr, nullptr};  // [np_pad*4] unit 4-vectors, double-buffered
  float4* s2Xf = nullptr;               // [np_pad] FP32 copy of the current ones
  double* s2Gl64 = nullptr;             // [np_pad*10] projected damped inverse of V
  float4* s2Gl32 = nullptr;             // [np_pad*3] its FP32 copy (10 of 12 floats)
  double* s2bl = nullptr;               // [np_pad*4] b_l
  double* s2s = nullptr;                // [np_pad*4] s = G_l b_l
  double* s2rec = nullptr;              // [np_pad*4] series record s_j (float or double)
  double* s2lin = nullptr;              // [nchunks*72] chunk sums of U and the RHS
  double* s2part = nullptr;             // [nchunks*12] series chunk partials (float or double)
  uint32_t* s2off = nullptr;            // [nc+1] first chunk of each camera
  uint32_t* s2idx = nullptr;            // [nchunks] chunk indices 0..nchunks-1
  bool s2_live = false;                 // second-stage landmarks were set
  bool s2_current = false;              // the device state's cost is the second stage's
  // metric upgrade (allocated at first use)
  double* mu_B = nullptr;               // [nc*12 + 16] B_i = K_i^-1 P_i H_0, then H_0
  double* mu_alpha = nullptr;           // [nc] scales
  void* mu_out = nullptr;               // result record
  double* mu_K = nullptr;               // [nc*9] intrinsics staged from the host
  // conjugate-gradient solver (allocated at first use)
  double* pcg_vec = nullptr;            // [4*nc*12] r, z, p, q (float or double)
  double* pcg_M64 = nullptr;            // [nc*144] inverse Schur-Jacobi blocks
  float* pcg_M32 = nullptr;             // [nc*144] their FP32 copies
  double* pcg_sd = nullptr;             // [nchunks*60] chunk sums of the diagonal blocks
  double* pcg_vals = nullptr;           // [nc*2] per-camera dot products
  uint32_t* pcg_ticket = nullptr;       // last-block ticket of the dot products
  double2* rec64 = nullptr;             // [np_pad*4] (s0 s1)(s2 X0)(X1 X2)(- -)
  double* cost_part = nullptr;          // [np_pad / 32] one per warp
  double* fin_blk = nullptr;            // [2 * FIN_BLOCKS] block sums of the final reductions
  int* fin_blk_i = nullptr;             // [FIN_BLOCKS]
  uint32_t* fin_ticket = nullptr;       // [2] last-block tickets (cost, predicted decrease)
  double* pred_part = nullptr;          // [np_pad / 32] one per warp
  int* pinv_part = nullptr;             // [np_pad / 32] one per warp
  int32_t n_slot_blocks = 0;
  // controller
  DeviceState* state = nullptr;
  DeviceState* h_state = nullptr;       // host mirror (read after a stream synchronization)
  povar_step_report* d_report = nullptr;
  povar_step_report* h_report = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // phase profiling: events recorded at phase boundaries of every step
  bool profiling = false;
  std::vector<cudaEvent_t> prof_events;   // pool
  size_t prof_next = 0;                   // next free event in the pool
  std::vector<std::vector<size_t>> prof_steps;  // event indices of pending steps
  double prof_ms[POVAR_NPHASES] = {0};
  int64_t prof_count = 0;
  int64_t prof_products = 0;             // series products of the timed steps
  long long prof_products_mark = 0;      // device product counter at the last sync
  // CUDA graph of one step (povar_solve): captured on a library stream that
  // joins the caller's stream through events; cached per parameter set
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;          // the captured step (kept for batch graphs)
  povar_params gkey{};
  int gkey_sched = -2;
  int64_t g_launches = 0;               // kernels per graph launch
  bool g_profiled = false;              // graph carries the phase events below
  cudaEvent_t gprof[POVAR_NPHASES + 1] = {};  // phase boundaries inside the graph
  bool use_graphs = true;
  std::vector<void*> allocs;            // every device allocation, freed by destroy
  int64_t device_bytes = 0;             // sum of the device allocations
};

// ------------------------------------------------------------------ helpers
#define POVAR_CUDA(call)                                                     \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      return ::povar::fail(p, POVAR_ECUDA,                                   \
                           std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                        \
  } while (0)

povar_status fail(Problem* p, povar_status s, const std::string& msg);
povar_status check_launch(Problem* p, const char* what);

// Device allocation tracked by the handle (freed by povar_destroy): stream
// ordered on the problem's stream, from the library's memory pool of the
// current device (library_pool).
cudaError_t library_pool(cudaMemPool_t* out);
povar_status dev_alloc_bytes(Problem* p, void** ptr, size_t bytes, const char* what);
povar_status alloc_slot_arrays(Problem* p);
template <class T>
inline povar_status dev_alloc(Problem* p, T** ptr, size_t count, const char* what) {
  return dev_alloc_bytes(p, reinterpret_cast<void**>(ptr), count * sizeof(T), what);
}

inline unsigned grid_for(int64_t n, int block) {
  return (unsigned)((n + block - 1) / block);
}

// --------------------------------------------------------- csr.cu (a1)
povar_status build_orders(Problem* p, const int32_t* h_cam, const int32_t* h_pt);

// ---------------------------------------------------- landmark.cu (a2,a3)
// Landmark tables of the cameras in buffer `which_rel` (0: current, 1: trial)
// and the closed-form landmarks + cost at those cameras.
povar_status launch_landmarks(Problem* p, int which_rel, double eta, int precision = POVAR_FP64);
// Reduce the cost partials into state.F (which_rel 0) or state.F_new (1).
povar_status launch_cost_finish(Problem* p, int which_rel);

// ------------------------------------------------- linearize.cu (a4,a5,a6)
povar_status launch_linearize(Problem* p, int precision, double eta, bool poba = false);
povar_status launch_ltab(Problem* p, int which_rel, double eta);
povar_status launch_project_delta(Problem* p, int precision);
povar_status ensure_poba(Problem* p);
povar_status launch_poba_prep(Problem* p, double eta, double lambda_l);
povar_status launch_poba_trial(Problem* p, int precision, double eta, int m);
povar_status launch_camera_prepare(Problem* p, int precision, int manifold,
                                   double eta, bool poba = false);

// ---------------------------------------------------- series.cu (a7,a8)
// schedule 0: point gather + camera-major scatter; 1: fused runs; 2: camera
// rows; 3: row table; 4 (and every POVAR_MIXED_BF16 term): stored blocks
povar_status launch_series_term(Problem* p, int precision, double eta,
                                int term, double eps, int schedule);
povar_status launch_pred(Problem* p, int precision, double eta, int manifold, int m);
// z = W V^-1 W^T vec as run partials (part_run, schedule 1's fused pass) for
// a camera vector vec of the precision's type.
povar_status launch_wvw(Problem* p, int precision, double eta, const void* vec);

// ---------------------------------------------------- stage2.cu
// Second stage (projective refinement by Riemannian PoBA). P / X are device
// arrays (n_cams*12 / n_points*4 by landmark id) or null (keep the current
// cameras; landmarks (X, 1) from the first stage's FP64 landmarks).
povar_status ensure_stage2(Problem* p);
povar_status launch_s2_set(Problem* p, const double* d_P, const double* d_X);
povar_status launch_s2_cost(Problem* p);
povar_status launch_s2_prep(Problem* p, double lambda_l);
povar_status launch_s2_linearize(Problem* p, int precision);
povar_status launch_s2_camera_prepare(Problem* p, int precision);
povar_status launch_s2_series_term(Problem* p, int precision, int term, double eps);
// the same product in one landmark-major pass with the run tables (series.cu)
povar_status launch_s2_fused_term(Problem* p, int precision, int term, double eps);
povar_status launch_s2_trial(Problem* p, int precision, int m);
povar_status launch_s2_gather_points(Problem* p, double* d_out);
// the first stage's per-camera series finish over given partial lists
povar_status launch_series_apply(Problem* p, int precision, int term, double eps,
                                 const uint32_t* off, const uint32_t* idx, const void* part);
// pred = F - sum of the model partials in pred_part (PoBA, second stage)
povar_status launch_model_pred_finish(Problem* p, int m);

// ---------------------------------------------------- metric.cu
// Metric upgrade of the current cameras (d_K: n_cams 3x3 row-major on the
// device, or null for identity); synchronizes the stream.
povar_status launch_metric_upgrade(Problem* p, const double* d_K, double lambda0, int max_iters,
                                   double ftol, double* H_out, double* alpha_out,
                                   double* cost_out, int* iters_out);

// ---------------------------------------------------- pcg.cu
// Conjugate-gradient solve of the reduced camera system into the step buffer
// (after launch_camera_prepare): at most `iters` iterations, relative
// residual tolerance eps. Synchronizes the stream every few iterations to
// stop early; never captured in a graph.
povar_status ensure_pcg(Problem* p);
povar_status launch_pcg(Problem* p, int precision, int manifold, double eta, int iters,
                        double eps);
// Stored schedule (4) and the BF16 precision: block kind of a precision,
// allocation (before any capture), plane pointers, and the per-step build of
// G_k at the current cameras.
int block_kind(int precision);
povar_status ensure_blocks(Problem* p, int kind);
povar_status setup_group_kernels(Problem* p);
BlockPlanes block_planes(const Problem* p, int kind);
povar_status launch_build_blocks(Problem* p, int precision, double eta);

// ---------------------------------------------------- step.cu (a9,a10)
povar_status launch_update(Problem* p, int precision, int manifold);
povar_status launch_controller(Problem* p, int precision);
povar_status launch_init_state(Problem* p, double lambda0, int reset_lm, int reset_all);
povar_status launch_begin(Problem* p, double ftol, double target, int max_iters,
                          int fallback_after = 0);
povar_status launch_random_cameras(Problem* p, uint64_t seed, int normalize);
// Kernel node of a batch's device-side loop: sets the while node's condition
// (some problem not converged and fewer than d_loops[1] steps; d_loops[0]
// counts the steps).
cudaError_t add_batch_continue(cudaGraph_t body, const cudaGraphNode_t* deps, size_t ndeps,
                               cudaGraphConditionalHandle h, DeviceState** d_states, int n,
                               int* d_loops);
povar_status launch_gather_points(Problem* p, double* d_out);

}  // namespace povar
