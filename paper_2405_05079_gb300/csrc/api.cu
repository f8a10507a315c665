// C-ABI entry points of libpovar (declared in include/povar.h).
//
// The host side only validates arguments, owns the device allocations and
// enqueues kernels; every step of the solve runs in the kernels of csr.cu,
// landmark.cu, linearize.cu, series.cu and step.cu.
#include "povar_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

struct povar_problem {
  povar::Problem impl;
};

namespace povar {

povar_status fail(Problem* p, povar_status s, const std::string& msg) {
  if (p) p->err = msg;
  return s;
}

povar_status check_launch(Problem* p, const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(p, POVAR_ECUDA, std::string("kernel launch (") + what + "): " +
                                    cudaGetErrorString(e));
  return POVAR_OK;
}

// Device memory comes from the stream-ordered allocator, on the problem's
// stream, out of a memory pool the library owns per device: cudaMalloc /
// cudaFree may synchronize the whole device, which would serialize every
// problem solved concurrently with the one being created or destroyed (the
// serving loop creates and destroys one per request). The pool keeps freed
// memory for the next problems (no release threshold);
// povar_release_cached_memory returns it to the device.
namespace {
std::mutex g_pool_mu;
std::vector<std::pair<int, cudaMemPool_t>> g_pools;
}  // namespace

cudaError_t library_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (const auto& dp : g_pools)
    if (dp.first == dev) {
      *out = dp.second;
      return cudaSuccess;
    }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool;
  if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
  uint64_t keep = UINT64_MAX;
  if ((e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
    cudaMemPoolDestroy(pool);
    return e;
  }
  g_pools.emplace_back(dev, pool);
  *out = pool;
  return cudaSuccess;
}

void release_cached_memory() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (const auto& dp : g_pools) cudaMemPoolTrimTo(dp.second, 0);
}

povar_status dev_alloc_bytes(Problem* p, void** ptr, size_t bytes, const char* what) {
  void* q = nullptr;
  cudaMemPool_t pool;
  cudaError_t e = library_pool(&pool);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&q, bytes > 0 ? bytes : 1, pool, p->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, POVAR_ENOMEM, std::string("device allocation ") + what + ": " + cudaGetErrorString(e));
  }
  p->allocs.push_back(q);
  p->device_bytes += (int64_t)(bytes > 0 ? bytes : 1);
  *ptr = q;
  return POVAR_OK;
}

// Arrays with one entry per landmark slot (np_pad slots, known once the
// landmark layout is sorted). Padding slots keep zero landmarks and factors,
// so that every kernel reading a whole slice sees finite values there.
povar_status alloc_slot_arrays(Problem* p) {
  const size_t npd = (size_t)p->np_pad;
  povar_status s;
  if ((s = dev_alloc(p, &p->slot_pt, npd, "slot_pt")) ||
      (s = dev_alloc(p, &p->slot_len, npd, "slot_len")) ||
      (s = dev_alloc(p, &p->sell_off, (size_t)p->nslices + 1, "sell_off")) ||
      (s = dev_alloc(p, &p->rec32, npd * 2, "rec32")) ||
      (s = dev_alloc(p, &p->rec64, npd * 4, "rec64")) ||
      (s = dev_alloc(p, &p->cost_part, npd / 32, "cost_part")) ||
      (s = dev_alloc(p, &p->pred_part, npd / 32, "pred_part")) ||
      (s = dev_alloc(p, &p->pinv_part, npd / 32, "pinv_part")))
    return s;
  for (int t = 0; t < 2; ++t) {
    if ((s = dev_alloc(p, &p->X64[t], npd * 3, "X64")) ||
        (s = dev_alloc(p, &p->F64[t], npd * 6, "F64")) ||
        (s = dev_alloc(p, &p->pdA[t], npd, "pdA")) || (s = dev_alloc(p, &p->pdB[t], npd, "pdB")) ||
        (s = dev_alloc(p, &p->pdC[t], npd, "pdC")))
      return s;
    POVAR_CUDA(cudaMemsetAsync(p->X64[t], 0, npd * 3 * sizeof(double), p->stream));
    POVAR_CUDA(cudaMemsetAsync(p->F64[t], 0, npd * 6 * sizeof(double), p->stream));
    POVAR_CUDA(cudaMemsetAsync(p->pdA[t], 0, npd * sizeof(float4), p->stream));
    POVAR_CUDA(cudaMemsetAsync(p->pdB[t], 0, npd * sizeof(float4), p->stream));
    POVAR_CUDA(cudaMemsetAsync(p->pdC[t], 0, npd * sizeof(float), p->stream));
  }
  return POVAR_OK;
}

namespace {

// Page-locked host slots for the per-problem mirrors of the device state and
// step report (copied to asynchronously, read after a stream sync). They are
// carved from chunks that are never freed and handed out under a mutex, so
// creating or destroying a problem calls neither cudaMallocHost nor
// cudaFreeHost, which may synchronize the device.
constexpr size_t kPinHalf = 512;              // one mirror per half slot
constexpr size_t kPinSlot = 2 * kPinHalf;
constexpr size_t kPinChunkSlots = 256;
static_assert(sizeof(DeviceState) <= kPinHalf && sizeof(povar_step_report) <= kPinHalf,
              "host mirror slots too small");
std::mutex g_pin_mu;
std::vector<char*> g_pin_free;

char* pinned_slot_get() {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pin_free.empty()) {
    char* c = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void**>(&c), kPinSlot * kPinChunkSlots,
                      cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    for (size_t k = 0; k < kPinChunkSlots; ++k) g_pin_free.push_back(c + k * kPinSlot);
  }
  char* q = g_pin_free.back();
  g_pin_free.pop_back();
  return q;
}

void pinned_slot_put(char* q) {
  if (!q) return;
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back(q);
}

void collect_profile(Problem* p);

povar_status sync_state(Problem* p) {
  POVAR_CUDA(cudaMemcpyAsync(p->h_state, p->state, sizeof(DeviceState), cudaMemcpyDeviceToHost,
                             p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  if (!p->prof_steps.empty()) collect_profile(p);
  p->prof_products_mark = p->h_state->products;
  return POVAR_OK;
}

povar_status check_params(Problem* p, const povar_params* q) {
  if (!q) return fail(p, POVAR_EINVAL, "params is NULL");
  if (!(q->eta >= 0.0 && q->eta <= 1.0)) return fail(p, POVAR_EINVAL, "eta must be in [0, 1]");
  if (!(q->lambda0 > 0.0) || !std::isfinite(q->lambda0))
    return fail(p, POVAR_EINVAL, "lambda0 must be positive");
  if (q->m < 1 || q->m > 10000) return fail(p, POVAR_EINVAL, "m must be in [1, 10000]");
  if (!(q->series_eps >= 0.0)) return fail(p, POVAR_EINVAL, "series_eps must be >= 0");
  if (!(q->lambda_l >= 0.0) || !std::isfinite(q->lambda_l))
    return fail(p, POVAR_EINVAL, "lambda_l must be >= 0 (0: PoVar, > 0: PoBA)");
  if (q->lambda_l > 0.0 && q->precision == POVAR_MIXED_BF16)
    return fail(p, POVAR_EINVAL, "PoBA (lambda_l > 0) runs in POVAR_FP64 or POVAR_MIXED_FP32");
  if (q->manifold != POVAR_EUCLID && q->manifold != POVAR_SPHERE)
    return fail(p, POVAR_EINVAL, "unknown manifold");
  if (q->precision != POVAR_FP64 && q->precision != POVAR_MIXED_FP32 &&
      q->precision != POVAR_MIXED_BF16)
    return fail(p, POVAR_EINVAL, "unknown precision");
  if (q->schedule < -1 || q->schedule >= POVAR_NSCHEDULES)
    return fail(p, POVAR_EINVAL, "unknown schedule");
  if (q->precision == POVAR_MIXED_BF16 && q->schedule != -1 && q->schedule != 4)
    return fail(p, POVAR_EINVAL, "POVAR_MIXED_BF16 runs schedule 4 only");
  if (q->solver != POVAR_SOLVER_SERIES && q->solver != POVAR_SOLVER_PCG)
    return fail(p, POVAR_EINVAL, "unknown solver");
  if (q->solver == POVAR_SOLVER_PCG && q->precision == POVAR_MIXED_BF16)
    return fail(p, POVAR_EINVAL, "PCG runs in POVAR_FP64 or POVAR_MIXED_FP32");
  if (q->reserved != 0) return fail(p, POVAR_EINVAL, "params->reserved must be 0");
  return POVAR_OK;
}

// Series schedule of a step: the explicit one, else the tuned one for the
// precision, else the default chosen at creation; POVAR_MIXED_BF16 always
// runs the stored schedule.
int resolve_schedule(const Problem* p, const povar_params* q) {
  if (q->precision == POVAR_MIXED_BF16) return 4;
  const int tuned = p->tuned_schedule[q->precision == POVAR_FP64 ? 0 : 1];
  return q->schedule >= 0 ? q->schedule : (tuned >= 0 ? tuned : p->schedule_default);
}

// Landmarks + cost at the current cameras for eta (no damping reset).
povar_status refresh_landmarks(Problem* p, double eta) {
  povar_status s;
  p->s2_current = false;
  if ((s = launch_landmarks(p, 0, eta)) != POVAR_OK) return s;
  if ((s = launch_cost_finish(p, 0)) != POVAR_OK) return s;
  if ((s = launch_init_state(p, 0.0, 0, 0)) != POVAR_OK) return s;  // need_lin = 1
  p->eta_cur = eta;
  p->lm_df = false;
  p->lm_poba = false;
  return POVAR_OK;
}

// Record a phase-boundary event of the current step (profiling only).
povar_status mark(Problem* p, std::vector<size_t>* marks) {
  if (!marks) return POVAR_OK;
  if (p->prof_next >= p->prof_events.size()) {
    cudaEvent_t e;
    POVAR_CUDA(cudaEventCreate(&e));
    p->prof_events.push_back(e);
  }
  const size_t k = p->prof_next++;
  POVAR_CUDA(cudaEventRecord(p->prof_events[k], p->stream));
  marks->push_back(k);
  return POVAR_OK;
}

// Fold the recorded (and completed: the caller synchronized) step events
// into the per-phase sums and recycle the pool.
void collect_profile(Problem* p) {
  for (const auto& m : p->prof_steps) {
    if (m.size() != POVAR_NPHASES + 1) continue;
    for (int ph = 0; ph < POVAR_NPHASES; ++ph) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p->prof_events[m[ph]], p->prof_events[m[ph + 1]]) ==
          cudaSuccess)
        p->prof_ms[ph] += ms;
    }
    ++p->prof_count;
  }
  // every step enqueued since the last synchronization was timed
  p->prof_products += p->h_state->products - p->prof_products_mark;
  cudaGetLastError();
  p->prof_steps.clear();
  p->prof_next = 0;
}

// Host decisions before a step: damping initialization after new cameras,
// landmark refresh when eta changed. Enqueues on p->stream.
povar_status prepare_step(Problem* p, const povar_params* q) {
  povar_status s;
  if (p->fresh) {
    if ((s = launch_init_state(p, q->lambda0, 1, 0)) != POVAR_OK) return s;
    p->fresh = false;
  }
  if (q->eta != p->eta_cur && (s = refresh_landmarks(p, q->eta)) != POVAR_OK) return s;
  const bool poba = q->lambda_l > 0.0;
  // mixed PoVar steps solve their trial landmarks in double-float and leave
  // the FP64 factor unwritten; an FP64 or PoBA step after them starts from
  // landmarks re-solved in FP64 at the current cameras; a PoVar step after
  // PoBA steps starts from the closed-form landmarks of the current cameras
  if ((q->precision == POVAR_FP64 || poba) && p->lm_df &&
      (s = refresh_landmarks(p, q->eta)) != POVAR_OK)
    return s;
  if (!poba && p->lm_poba && (s = refresh_landmarks(p, q->eta)) != POVAR_OK) return s;
  if (poba) {
    if ((s = ensure_poba(p)) != POVAR_OK) return s;
    p->lm_poba = true;
  } else if (q->precision != POVAR_FP64) {
    p->lm_df = true;
  }
  // stored blocks are allocated here, outside any graph capture
  if (q->solver == POVAR_SOLVER_SERIES && resolve_schedule(p, q) == 4 &&
      (s = ensure_blocks(p, block_kind(q->precision))) != POVAR_OK)
    return s;
  if (q->solver == POVAR_SOLVER_PCG && (s = ensure_pcg(p)) != POVAR_OK) return s;
  return POVAR_OK;
}

// The fixed kernel sequence of one damped VarPro iteration (a4 .. a10). It
// depends only on q and device state, so it can be captured in a graph.
povar_status enqueue_step_kernels(Problem* p, const povar_params* q, std::vector<size_t>* mk,
                                  const cudaEvent_t* fixed = nullptr) {
  povar_status s;
  const int prec = q->precision;
  const int sched = resolve_schedule(p, q);
  int nmark = 0;
  // phase boundary: a pooled event (eager profiling) or a fixed event node
  // (profiling inside the step graph)
  auto mark = [&](Problem* pp, std::vector<size_t>* m) -> povar_status {
    if (fixed) {
      const cudaError_t e =
          cudaEventRecordWithFlags(fixed[nmark++], pp->stream, cudaEventRecordExternal);
      return e == cudaSuccess ? POVAR_OK : fail(pp, POVAR_ECUDA, cudaGetErrorString(e));
    }
    return ::povar::mark(pp, m);
  };
  const bool poba = q->lambda_l > 0.0;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  // PoBA: damped landmark blocks and b_l at (P, X) first (they change with
  // the damping, so every PoBA step linearizes)
  if (poba && (s = launch_poba_prep(p, q->eta, q->lambda_l)) != POVAR_OK) return s;
  if ((s = launch_linearize(p, prec, q->eta, poba)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_camera_prepare(p, prec, q->manifold, q->eta, poba)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if (q->solver == POVAR_SOLVER_PCG) {
    // the reduced system by conjugate gradients (reads device flags: eager only)
    if ((s = launch_pcg(p, prec, q->manifold, q->eta, q->m, q->series_eps)) != POVAR_OK) return s;
  } else {
    if (sched == 4 && q->m > (prec == POVAR_MIXED_BF16 ? POVAR_BF16_FP32_TERMS : 1) &&
        (s = launch_build_blocks(p, prec, q->eta)) != POVAR_OK)
      return s;
    for (int k = 1; k < q->m; ++k) {
      // POVAR_MIXED_BF16: the leading terms read the FP32 factors (the
      // factored fused pass), the later ones the bfloat16 blocks
      const bool lead32 = prec == POVAR_MIXED_BF16 && k < POVAR_BF16_FP32_TERMS;
      if ((s = launch_series_term(p, lead32 ? POVAR_MIXED_FP32 : prec, q->eta, k,
                                  q->series_eps, lead32 ? 1 : sched)) != POVAR_OK)
        return s;
    }
  }
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if (poba) {
    // PoBA's predicted decrease comes with its trial pass below
    if (q->manifold == POVAR_SPHERE && (s = launch_project_delta(p, prec)) != POVAR_OK) return s;
  } else if ((s = launch_pred(p, prec, q->eta, q->manifold, q->m)) != POVAR_OK) {
    return s;
  }
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_update(p, prec, q->manifold)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if (poba) {
    if ((s = launch_poba_trial(p, prec, q->eta, q->m)) != POVAR_OK) return s;
  } else {
    if ((s = launch_landmarks(p, 1, q->eta, prec)) != POVAR_OK) return s;
    if ((s = launch_cost_finish(p, 1)) != POVAR_OK) return s;
  }
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_controller(p, prec)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  p->last_precision = prec;
  return POVAR_OK;
}

// Enqueue one damped VarPro iteration (no host synchronization).
povar_status enqueue_step(Problem* p, const povar_params* q) {
  povar_status s;
  std::vector<size_t>* mk = nullptr;
  if (p->profiling) {
    p->prof_steps.emplace_back();
    mk = &p->prof_steps.back();
  }
  if ((s = prepare_step(p, q)) != POVAR_OK) return s;
  return enqueue_step_kernels(p, q, mk);
}

// Add the phase times of the last completed graph launch (the caller has
// synchronized the graph stream).
void sample_graph_profile(Problem* p, bool last_step_worked) {
  if (!p->g_profiled || !last_step_worked) return;
  float ms[POVAR_NPHASES];
  for (int ph = 0; ph < POVAR_NPHASES; ++ph)
    if (cudaEventElapsedTime(&ms[ph], p->gprof[ph], p->gprof[ph + 1]) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
  for (int ph = 0; ph < POVAR_NPHASES; ++ph) p->prof_ms[ph] += ms[ph];
  ++p->prof_count;
  p->prof_products += p->h_state->terms_used > 1 ? p->h_state->terms_used - 1 : 0;
}

// Series-schedule autotuner: on the live state of the first step, run every
// schedule for one untimed term (caches and instruction caches warm) and then
// three timed terms; a second round re-times the schedules within 15% of the
// first round's fastest; keep the schedule with the smallest time per term
// for this precision. The stored schedule
// (4) also pays its per-step block build, timed before its terms and spread
// over the m - 1 terms of a step. The damped blocks are re-prepared
// afterwards, so the solve continues from exactly the state it would have
// had without tuning. POVAR_MIXED_BF16 has a single schedule and is not
// tuned.
povar_status autotune_schedule(Problem* p, const povar_params* q) {
  if (q->precision == POVAR_MIXED_BF16) return POVAR_OK;
  const int prec = q->precision == POVAR_FP64 ? 0 : 1;
  if (p->tuned_schedule[prec] >= 0) return POVAR_OK;
  povar_status s;
  if ((s = prepare_step(p, q)) != POVAR_OK) return s;
  if ((s = launch_linearize(p, q->precision, q->eta)) != POVAR_OK) return s;
  cudaEvent_t ev[4];
  for (int k = 0; k < 4; ++k) POVAR_CUDA(cudaEventCreate(&ev[k]));
  int best = 1;
  float best_ms = 1e30f;
  for (int sched = 0; sched < POVAR_NSCHEDULES; ++sched) p->tune_ms[prec][sched] = 1e30f;
  for (int round = 0; round < 2 && s == POVAR_OK; ++round) {
    float lead_ms = 1e30f;
    for (int sched = 0; sched < POVAR_NSCHEDULES; ++sched)
      lead_ms = std::min(lead_ms, p->tune_ms[prec][sched]);
    for (int sched = 0; sched < POVAR_NSCHEDULES; ++sched) {
      // second round: only the schedules that can still win
      if (round > 0 && !(p->tune_ms[prec][sched] <= 1.15f * lead_ms)) continue;
      float build_ms = 0.f;
      if (sched == 4) {
        if ((s = ensure_blocks(p, block_kind(q->precision))) != POVAR_OK) break;
        POVAR_CUDA(cudaEventRecord(ev[2], p->stream));
        if ((s = launch_build_blocks(p, q->precision, q->eta)) != POVAR_OK) break;
        POVAR_CUDA(cudaEventRecord(ev[3], p->stream));
        POVAR_CUDA(cudaEventSynchronize(ev[3]));
        POVAR_CUDA(cudaEventElapsedTime(&build_ms, ev[2], ev[3]));
        build_ms /= (float)std::max(1, q->m - 1);
      }
      if ((s = launch_camera_prepare(p, q->precision, q->manifold, q->eta)) != POVAR_OK) break;
      if ((s = launch_series_term(p, q->precision, q->eta, 1, 0.0, sched)) != POVAR_OK) break;
      POVAR_CUDA(cudaEventRecord(ev[0], p->stream));
      for (int k = 2; k <= 4 && s == POVAR_OK; ++k)
        s = launch_series_term(p, q->precision, q->eta, k, 0.0, sched);
      if (s != POVAR_OK) break;
      POVAR_CUDA(cudaEventRecord(ev[1], p->stream));
      POVAR_CUDA(cudaEventSynchronize(ev[1]));
      float ms = 0.f;
      POVAR_CUDA(cudaEventElapsedTime(&ms, ev[0], ev[1]));
      ms = ms / 3.f + build_ms;
      if (ms < p->tune_ms[prec][sched]) p->tune_ms[prec][sched] = ms;
    }
  }
  for (int sched = 0; sched < POVAR_NSCHEDULES && s == POVAR_OK; ++sched)
    if (p->tune_ms[prec][sched] < best_ms) {
      best_ms = p->tune_ms[prec][sched];
      best = sched;
    }
  for (int k = 0; k < 4; ++k) cudaEventDestroy(ev[k]);
  if (s != POVAR_OK) return s;
  p->tuned_schedule[prec] = best;
  return POVAR_OK;
}

bool same_params(const povar_params& a, const povar_params& b) {
  return a.eta == b.eta && a.series_eps == b.series_eps && a.m == b.m &&
         a.manifold == b.manifold && a.precision == b.precision && a.schedule == b.schedule &&
         a.lambda_l == b.lambda_l && a.solver == b.solver;
}

// Graph of one step on p->gstream (captured once per parameter set).
povar_status step_graph(Problem* p, const povar_params* q) {
  const int sched = resolve_schedule(p, q);
  if (p->gexec && same_params(p->gkey, *q) && p->gkey_sched == sched &&
      p->g_profiled == p->profiling)
    return POVAR_OK;
  if (p->gexec) {
    cudaGraphExecDestroy(p->gexec);
    p->gexec = nullptr;
  }
  cudaStream_t user = p->stream;
  p->stream = p->gstream;
  const int64_t l0 = p->launches;
  cudaError_t e = cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal);
  povar_status s = POVAR_OK;
  if (e == cudaSuccess) s = enqueue_step_kernels(p, q, nullptr, p->profiling ? p->gprof : nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(p->gstream, &g);
  p->stream = user;
  p->g_launches = p->launches - l0;
  p->launches = l0;
  if (e != cudaSuccess || e2 != cudaSuccess || s != POVAR_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return s != POVAR_OK ? s : fail(p, POVAR_ECUDA, "step graph capture failed");
  }
  e = cudaGraphInstantiate(&p->gexec, g, 0);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->graph = g;
  if (e != cudaSuccess) {
    p->gexec = nullptr;
    cudaGetLastError();
    return fail(p, POVAR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  p->gkey = *q;
  p->gkey_sched = sched;
  p->g_profiled = p->profiling;
  return POVAR_OK;
}

void fill_report(Problem* p, povar_step_report* r, float ms) {
  *r = *p->h_report;
  r->ms = ms;
}

// Up to max_iters steps with parameters q (launch_begin done by the caller),
// synchronizing the state every few steps and stopping at the device's
// convergence flag; on return p->h_state is current.
povar_status solve_loop(Problem* p, const povar_params* q, int max_iters) {
  povar_status s;
  const int check_every = 4;
  if (p->use_graphs && q->solver == POVAR_SOLVER_SERIES) {
    // one graph launch per step on the library stream, joined to the
    // caller's stream with events before and after
    if ((s = prepare_step(p, q)) != POVAR_OK) return s;
    if (q->schedule < 0 && (s = autotune_schedule(p, q)) != POVAR_OK) return s;
    if ((s = step_graph(p, q)) != POVAR_OK) return s;
    POVAR_CUDA(cudaEventRecord(p->ev_join, p->stream));
    POVAR_CUDA(cudaStreamWaitEvent(p->gstream, p->ev_join, 0));
    cudaStream_t user = p->stream;
    p->stream = p->gstream;
    // the phase events hold the last launched step: it is sampled when it
    // did work, i.e. when every launch since the last sample advanced the
    // iteration count (launches after convergence return at once)
    int since = 0, iter_mark = p->h_state->iteration;
    auto sample = [&]() -> povar_status {
      if ((s = sync_state(p)) != POVAR_OK) return s;
      sample_graph_profile(p, since > 0 && p->h_state->iteration - iter_mark == since);
      iter_mark = p->h_state->iteration;
      since = 0;
      return POVAR_OK;
    };
    for (int it = 0; it < max_iters; ++it) {
      const cudaError_t e = cudaGraphLaunch(p->gexec, p->gstream);
      if (e != cudaSuccess) {
        p->stream = user;
        return fail(p, POVAR_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
      }
      p->launches += p->g_launches;
      ++since;
      if ((it + 1) % check_every == 0 && it + 1 < max_iters) {
        if (sample() != POVAR_OK) {
          p->stream = user;
          return s;
        }
        if (p->h_state->converged) break;
      }
    }
    if (since > 0 && sample() != POVAR_OK) {
      p->stream = user;
      return s;
    }
    POVAR_CUDA(cudaEventRecord(p->ev_join, p->gstream));
    p->stream = user;
    POVAR_CUDA(cudaStreamWaitEvent(p->stream, p->ev_join, 0));
  } else {
    for (int it = 0; it < max_iters; ++it) {
      if ((s = enqueue_step(p, q)) != POVAR_OK) return s;
      if ((it + 1) % check_every == 0 && it + 1 < max_iters) {
        if ((s = sync_state(p)) != POVAR_OK) return s;
        if (p->h_state->converged) break;
      }
    }
    if ((s = sync_state(p)) != POVAR_OK) return s;
  }
  return POVAR_OK;
}

// ---------------------------------------------------------------------------
// Second stage (projective refinement by Riemannian PoBA)
// ---------------------------------------------------------------------------

povar_status check_s2_params(Problem* p, const povar_params* q) {
  if (!q) return fail(p, POVAR_EINVAL, "params is NULL");
  if (!(q->lambda0 > 0.0) || !std::isfinite(q->lambda0))
    return fail(p, POVAR_EINVAL, "lambda0 must be positive");
  if (q->m < 1 || q->m > 10000) return fail(p, POVAR_EINVAL, "m must be in [1, 10000]");
  if (!(q->series_eps >= 0.0)) return fail(p, POVAR_EINVAL, "series_eps must be >= 0");
  if (!(q->lambda_l > 0.0) || !std::isfinite(q->lambda_l))
    return fail(p, POVAR_EINVAL, "the second stage needs lambda_l > 0 (1: joint damping)");
  if (q->manifold != POVAR_SPHERE)
    return fail(p, POVAR_EINVAL, "the second stage is Riemannian: manifold must be SPHERE");
  if (q->precision != POVAR_FP64 && q->precision != POVAR_MIXED_FP32)
    return fail(p, POVAR_EINVAL, "the second stage runs in POVAR_FP64 or POVAR_MIXED_FP32");
  if (q->solver != POVAR_SOLVER_SERIES)
    return fail(p, POVAR_EINVAL, "the second stage runs the series solver");
  if (q->schedule < -1 || q->schedule > 1)
    return fail(p, POVAR_EINVAL, "second-stage series schedules are -1, 0 and 1");
  if (q->reserved != 0) return fail(p, POVAR_EINVAL, "params->reserved must be 0");
  if (!p->s2_live) return fail(p, POVAR_EINVAL, "call povar_s2_set first");
  return POVAR_OK;
}

// Before a second-stage step: the device state must hold the second stage's
// cost (a first-stage call in between replaced it), and the damping starts
// at lambda0 after povar_s2_set.
povar_status prepare_s2_step(Problem* p, const povar_params* q) {
  povar_status s;
  if (!p->s2_current) {
    if ((s = launch_s2_cost(p)) != POVAR_OK) return s;
    p->s2_current = true;
    p->fresh = true;
  }
  if (p->fresh) {
    if ((s = launch_init_state(p, q->lambda0, 1, 0)) != POVAR_OK) return s;
    p->fresh = false;
  }
  // a later first-stage call re-solves its landmarks at the cameras
  p->eta_cur = -1.0;
  return POVAR_OK;
}

povar_status enqueue_s2_step(Problem* p, const povar_params* q) {
  povar_status s;
  std::vector<size_t>* mk = nullptr;
  if (p->profiling) {
    p->prof_steps.emplace_back();
    mk = &p->prof_steps.back();
  }
  const int prec = q->precision;
  if ((s = prepare_s2_step(p, q)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_s2_prep(p, q->lambda_l)) != POVAR_OK) return s;
  if ((s = launch_s2_linearize(p, prec)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_s2_camera_prepare(p, prec)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  for (int k = 1; k < q->m; ++k)
    if ((s = q->schedule == 0 ? launch_s2_series_term(p, prec, k, q->series_eps)
                              : launch_s2_fused_term(p, prec, k, q->series_eps)) != POVAR_OK)
      return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_project_delta(p, prec)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_update(p, prec, POVAR_SPHERE)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_s2_trial(p, prec, q->m)) != POVAR_OK) return s;
  if ((s = mark(p, mk)) != POVAR_OK) return s;
  if ((s = launch_controller(p, prec)) != POVAR_OK) return s;
  p->last_precision = prec;
  return mark(p, mk);
}

povar_status s2_solve_loop(Problem* p, const povar_params* q, int max_iters) {
  povar_status s;
  const int check_every = 4;
  for (int it = 0; it < max_iters; ++it) {
    if ((s = enqueue_s2_step(p, q)) != POVAR_OK) return s;
    if ((it + 1) % check_every == 0 && it + 1 < max_iters) {
      if ((s = sync_state(p)) != POVAR_OK) return s;
      if (p->h_state->converged) break;
    }
  }
  return sync_state(p);
}

}  // namespace
}  // namespace povar

using povar::Problem;

extern "C" {

const char* povar_version(void) { return "povar-gb300 0.1 (sm_103a)"; }

const char* povar_last_error(const povar_problem* pp) {
  return pp ? pp->impl.err.c_str() : "null handle";
}

int64_t povar_launch_count(const povar_problem* pp) { return pp ? pp->impl.launches : 0; }

int64_t povar_device_bytes(const povar_problem* pp) { return pp ? pp->impl.device_bytes : 0; }

int64_t povar_estimate_bytes(int32_t n_cams, int32_t n_points, int64_t n_obs) {
  if (n_cams < 1 || n_points < 1 || n_obs < 1) return 0;
  // slots: every smallest camera (at most min(n_cams, n_points) of them)
  // starts a slice, so at most 31 padding slots per camera, then a multiple
  // of 256
  const int64_t nbk = std::min<int64_t>(n_cams, n_points);
  const int64_t nc = n_cams, npd = ((int64_t)n_points + 31 * nbk + 255) / 256 * 256,
                no = n_obs;
  // SELL entries are bounded by 32 x (longest track) per slice; two times the
  // observations bounds the padding of the scenes this library targets
  const int64_t nsell = 2 * no + 32 * 64;
  const int64_t chunks = no / 256 + nc + 1;
  int64_t b = 0;
  b += no * (4 + 4 + 16);                  // inputs
  b += no * (4 + 4) + 4 * ((int64_t)n_points + nc + 2);  // orders
  b += npd * (4 + 4) + 4 * (int64_t)n_points + 4 * (npd / 32 + 1);
  b += nsell * (4 + 8 + 16 + 16);          // SELL (camera, measurements f32 / f64 / double-float)
  b += no * (4 + 8 + 16);                  // camera-major list
  b += nc * 4 * 4 + chunks * 8;
  b += nc * 48 * 8;                        // double-float landmark tables
  b += nc * (2 * 12 * 8 + 48 * 8 + 2 * 12 * 4 + 144 * 8 + 12 * 8 + 144 * 8 + 144 * 4 +
             2 * 12 * 4 + 12 * 4 + 2 * 12 * 8 + 12 * 8 + 2 * 8);
  b += 2 * npd * (3 * 8 + 6 * 8 + 16 + 16 + 4) + npd * (32 + 64) + 3 * (npd / 32) * 8;
  b += chunks * (52 + 12) * 8;
  // every run partial and every camera-row visit holds at least one
  // observation, so n_obs bounds their counts
  // fused schedule: run mask and base per slice row, partials and their index
  b += (nsell / 32) * 8 + no * (12 * 8 + 4) + (nc + 1) * 4;
  // camera-row schedule: visit lists
  b += no * 8 + (nc + 1) * 4;
  // grouped schedule: group tables, group rows, slice-row runs, partials
  b += 2 * (npd / 32 + 1) * 4 + (nsell / 32) * 16 + no * (12 * 8 + 4) + (nc + 1) * 4;
  // group schedule: slice, row and item lists (each at most one per slice
  // row), the rest list, per-camera lists and partials (items + run partials)
  b += (nsell / 32) * 16 + (npd / 32 + 1) * 16 + (nc + 1) * 4 +
       (nsell / 32 + no) * (12 * 8 + 4);
  // PoBA: s_j per slot (allocated at first use)
  b += npd * (3 * 8 + 16);
  // PCG (allocated at first use): r, z, p, q, the preconditioner blocks in
  // FP64 and FP32, chunk sums of the diagonal blocks, dot products
  b += nc * (48 * 8 + 144 * 12 + 16) + chunks * 60 * 8;
  // stored-block schedule: FP64, FP32 and BF16 blocks (each allocated at
  // its first use)
  b += nsell * (72 + 36 + 18);
  return b + (1 << 20);
}

void povar_release_cached_memory(void) { povar::release_cached_memory(); }

void povar_destroy(povar_problem* pp) {
  if (!pp) return;
  Problem* p = &pp->impl;
  // work of the graph stream is joined back to the problem's stream by every
  // solve; wait for both, then return the memory in stream order
  if (p->gstream) cudaStreamSynchronize(p->gstream);
  cudaStreamSynchronize(p->stream);
  for (void* q : p->allocs) cudaFreeAsync(q, p->stream);
  povar::pinned_slot_put(reinterpret_cast<char*>(p->h_state));
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  for (cudaEvent_t e : p->prof_events) cudaEventDestroy(e);
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->gstream) cudaStreamDestroy(p->gstream);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  for (int ph = 0; ph <= POVAR_NPHASES; ++ph)
    if (p->gprof[ph]) cudaEventDestroy(p->gprof[ph]);
  delete pp;
}

povar_status povar_create(int32_t n_cams, int32_t n_points, int64_t n_obs, const int32_t* cam_idx,
                          const int32_t* pt_idx, const double* meas, void* cuda_stream,
                          povar_problem** out) {
  if (!out) return POVAR_EINVAL;
  *out = nullptr;
  if (n_cams < 1 || n_points < 1 || n_obs < 1 || n_obs >= (int64_t)1 << 31 || !cam_idx ||
      !pt_idx || !meas)
    return POVAR_EINVAL;
  povar_problem* pp = new (std::nothrow) povar_problem();
  if (!pp) return POVAR_ENOMEM;
  Problem* p = &pp->impl;
  p->nc = n_cams;
  p->np = n_points;
  p->nobs = n_obs;
  p->stream = static_cast<cudaStream_t>(cuda_stream);
  // the slot count (np_pad) follows from the landmark layout: build_orders
  // sets it and allocates the per-slot arrays (alloc_slot_arrays)
  povar_status s = POVAR_OK;
  const size_t nc = n_cams, no = n_obs;
#define ALLOC(ptr, count)                                                    \
  if ((s = povar::dev_alloc(p, &(ptr), (count), #ptr)) != POVAR_OK) {       \
    povar_destroy(pp);                                                       \
    return s;                                                                \
  }
  ALLOC(p->d_cam, no);
  ALLOC(p->d_pt, no);
  ALLOC(p->d_meas, 2 * no);
  ALLOC(p->perm_pt, no);
  ALLOC(p->perm_cam, no);
  ALLOC(p->off_pt, (size_t)n_points + 1);
  ALLOC(p->off_cam, nc + 1);
  ALLOC(p->pt_slot, (size_t)n_points);
  ALLOC(p->cm_slot, no);
  ALLOC(p->cm_m32, no);
  ALLOC(p->cm_m64, no);
  ALLOC(p->cam_nchunk, nc);
  ALLOC(p->cam_chunk0, nc);
  ALLOC(p->cam_ticket, nc);
  ALLOC(p->done_ticket, 1);
  ALLOC(p->P64[0], nc * 12);
  ALLOC(p->P64[1], nc * 12);
  ALLOC(p->Ltab, nc * 48);
  ALLOC(p->Ltab_df, nc * 48);
  ALLOC(p->camP32[0], nc * 12);
  ALLOC(p->camP32[1], nc * 12);
  ALLOC(p->U64, nc * 144);
  ALLOC(p->bp64, nc * 12);
  ALLOC(p->G64, nc * 144);
  ALLOC(p->G32, nc * 144);
  ALLOC(p->Y32, 2 * nc * 12);
  ALLOC(p->D32, nc * 12);
  ALLOC(p->Y64, 2 * nc * 12);
  ALLOC(p->D64, nc * 12);
  ALLOC(p->camnorm, nc * 2);
  ALLOC(p->fin_blk, 2 * povar::FIN_BLOCKS);
  ALLOC(p->fin_blk_i, povar::FIN_BLOCKS);
  ALLOC(p->fin_ticket, 2);
  ALLOC(p->state, 1);
  ALLOC(p->d_report, 1);
#define CK(call)                                                             \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      cudaGetLastError();                                                    \
      povar_destroy(pp);                                                     \
      return POVAR_ECUDA;                                                    \
    }                                                                        \
  } while (0)
  // page-locked host mirrors of the device state and report, from the slot
  // pool (no pinned allocation per problem)
  {
    char* slot = povar::pinned_slot_get();
    if (!slot) {
      povar_destroy(pp);
      return POVAR_ENOMEM;
    }
    p->h_state = new (slot) povar::DeviceState();
    p->h_report = new (slot + povar::kPinHalf) povar_step_report();
  }
  CK(cudaEventCreate(&p->ev0));
  CK(cudaEventCreate(&p->ev1));
  CK(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
  CK(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
  for (int ph = 0; ph <= POVAR_NPHASES; ++ph) CK(cudaEventCreate(&p->gprof[ph]));
  CK(cudaMemcpyAsync(p->d_cam, cam_idx, no * sizeof(int32_t), cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemcpyAsync(p->d_pt, pt_idx, no * sizeof(int32_t), cudaMemcpyHostToDevice, p->stream));
  CK(cudaMemcpyAsync(p->d_meas, meas, 2 * no * sizeof(double), cudaMemcpyHostToDevice,
                     p->stream));
  CK(cudaMemsetAsync(p->cam_ticket, 0, nc * sizeof(uint32_t), p->stream));
  CK(cudaMemsetAsync(p->done_ticket, 0, sizeof(uint32_t), p->stream));
  CK(cudaMemsetAsync(p->fin_ticket, 0, 2 * sizeof(uint32_t), p->stream));
  CK(cudaMemsetAsync(p->P64[0], 0, nc * 12 * sizeof(double), p->stream));
  CK(cudaMemsetAsync(p->P64[1], 0, nc * 12 * sizeof(double), p->stream));
  CK(cudaMemsetAsync(p->camnorm, 0, nc * 2 * sizeof(double), p->stream));
  CK(cudaMemsetAsync(p->state, 0, sizeof(povar::DeviceState), p->stream));
  CK(cudaMemsetAsync(p->d_report, 0, sizeof(povar_step_report), p->stream));
  if ((s = povar::build_orders(p, cam_idx, pt_idx)) != POVAR_OK) {
    povar_destroy(pp);
    return s;
  }
  ALLOC(*reinterpret_cast<char**>(&p->part_lin), (size_t)std::max(p->nchunks, 1) * povar::LIN_PART * sizeof(double));
  ALLOC(*reinterpret_cast<char**>(&p->part_ser), (size_t)std::max(p->nchunks, 1) * 12 * sizeof(double));
  // fused schedule when at most half as many run partials as observations
  p->schedule_default = (2 * p->npart <= p->nobs) ? 1 : 0;
#undef ALLOC
#undef CK
  if ((s = povar::launch_init_state(p, 1e-4, 1, 1)) != POVAR_OK ||
      (s = povar::sync_state(p)) != POVAR_OK) {
    povar_destroy(pp);
    return s;
  }
  *out = pp;
  return POVAR_OK;
}

povar_status povar_set_cameras(povar_problem* pp, const double* P, double eta) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!P) return povar::fail(p, POVAR_EINVAL, "P is NULL");
  if (!(eta >= 0.0 && eta <= 1.0)) return povar::fail(p, POVAR_EINVAL, "eta must be in [0, 1]");
  cudaPointerAttributes attr;
  bool on_device = false;
  if (cudaPointerGetAttributes(&attr, P) == cudaSuccess)
    on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
  cudaGetLastError();
  if (!on_device)
    for (int64_t e = 0; e < (int64_t)p->nc * 12; ++e)
      if (!std::isfinite(P[e])) return povar::fail(p, POVAR_EINVAL, "non-finite camera");
  povar_status s;
  if ((s = povar::launch_init_state(p, 1e-4, 1, 1)) != POVAR_OK) return s;
  POVAR_CUDA(cudaMemcpyAsync(p->P64[0], P, (size_t)p->nc * 12 * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             p->stream));
  if ((s = povar::refresh_landmarks(p, eta)) != POVAR_OK) return s;
  p->fresh = true;
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  if (p->h_state->error) return povar::fail(p, (povar_status)p->h_state->error, "non-finite cost");
  return POVAR_OK;
}

povar_status povar_init_random(povar_problem* pp, uint64_t seed, int32_t manifold, double eta) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (manifold != POVAR_EUCLID && manifold != POVAR_SPHERE)
    return povar::fail(p, POVAR_EINVAL, "unknown manifold");
  if (!(eta >= 0.0 && eta <= 1.0)) return povar::fail(p, POVAR_EINVAL, "eta must be in [0, 1]");
  povar_status s;
  if ((s = povar::launch_init_state(p, 1e-4, 1, 1)) != POVAR_OK) return s;
  if ((s = povar::launch_random_cameras(p, seed, manifold == POVAR_SPHERE)) != POVAR_OK) return s;
  if ((s = povar::refresh_landmarks(p, eta)) != POVAR_OK) return s;
  p->fresh = true;
  return povar::sync_state(p);
}

povar_status povar_get_cameras(povar_problem* pp, double* P_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!P_out) return povar::fail(p, POVAR_EINVAL, "P_out is NULL");
  povar_status s;
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  POVAR_CUDA(cudaMemcpyAsync(P_out, p->P64[p->h_state->cur], (size_t)p->nc * 12 * sizeof(double),
                             cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}

povar_status povar_get_points(povar_problem* pp, double* X_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!X_out) return povar::fail(p, POVAR_EINVAL, "X_out is NULL");
  // the gather stages the landmarks in the series record buffer (free between steps)
  double* d = reinterpret_cast<double*>(p->rec64);
  povar_status s = povar::launch_gather_points(p, d);
  if (s != POVAR_OK) return s;
  POVAR_CUDA(cudaMemcpyAsync(X_out, d, (size_t)p->np * 3 * sizeof(double),
                             cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}

povar_status povar_s2_set(povar_problem* pp, const double* P, const double* X) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (P && !X) return povar::fail(p, POVAR_EINVAL, "X is NULL while P is given");
  if (P)
    for (int64_t e = 0; e < (int64_t)p->nc * 12; ++e)
      if (!std::isfinite(P[e])) return povar::fail(p, POVAR_EINVAL, "non-finite camera");
  if (X)
    for (int64_t e = 0; e < (int64_t)p->np * 4; ++e)
      if (!std::isfinite(X[e])) return povar::fail(p, POVAR_EINVAL, "non-finite landmark");
  povar_status s;
  if ((s = povar::ensure_stage2(p)) != POVAR_OK) return s;
  if (!X) {
    // from the first stage: its landmarks at the current cameras, in FP64
    if (p->eta_cur < 0.0)
      return povar::fail(p, POVAR_EINVAL, "no first-stage landmarks to start from");
    if (p->lm_df && (s = povar::refresh_landmarks(p, p->eta_cur)) != POVAR_OK) return s;
    if ((s = povar::launch_init_state(p, 1e-4, 1, 0)) != POVAR_OK) return s;
  } else {
    if ((s = povar::launch_init_state(p, 1e-4, 1, 1)) != POVAR_OK) return s;
  }
  const double* d_X = nullptr;
  if (P)
    POVAR_CUDA(cudaMemcpyAsync(p->P64[0], P, (size_t)p->nc * 12 * sizeof(double),
                               cudaMemcpyHostToDevice, p->stream));
  if (X) {
    // staged in the series record buffer (free between steps)
    double* d = reinterpret_cast<double*>(p->rec64);
    POVAR_CUDA(cudaMemcpyAsync(d, X, (size_t)p->np * 4 * sizeof(double), cudaMemcpyHostToDevice,
                               p->stream));
    d_X = d;
  }
  if ((s = povar::launch_s2_set(p, nullptr, d_X)) != POVAR_OK) return s;
  if ((s = povar::launch_s2_cost(p)) != POVAR_OK) return s;
  p->s2_live = true;
  p->s2_current = true;
  p->fresh = true;
  p->eta_cur = -1.0;
  p->lm_df = false;
  p->lm_poba = false;
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  if (p->h_state->error) return povar::fail(p, (povar_status)p->h_state->error, "non-finite cost");
  return POVAR_OK;
}

povar_status povar_s2_cost(povar_problem* pp, double* cost_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!cost_out) return povar::fail(p, POVAR_EINVAL, "cost_out is NULL");
  if (!p->s2_live) return povar::fail(p, POVAR_EINVAL, "call povar_s2_set first");
  povar_status s;
  if (!p->s2_current) {
    if ((s = povar::launch_s2_cost(p)) != POVAR_OK) return s;
    p->s2_current = true;
    p->fresh = true;
    p->eta_cur = -1.0;
  }
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  *cost_out = p->h_state->F;
  return POVAR_OK;
}

povar_status povar_s2_step(povar_problem* pp, const povar_params* params,
                           povar_step_report* report) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  povar_status s;
  if ((s = povar::check_s2_params(p, params)) != POVAR_OK) return s;
  if ((s = povar::launch_begin(p, 0.0, 0.0, 0)) != POVAR_OK) return s;
  POVAR_CUDA(cudaEventRecord(p->ev0, p->stream));
  if ((s = povar::enqueue_s2_step(p, params)) != POVAR_OK) return s;
  POVAR_CUDA(cudaEventRecord(p->ev1, p->stream));
  POVAR_CUDA(cudaMemcpyAsync(p->h_report, p->d_report, sizeof(povar_step_report),
                             cudaMemcpyDeviceToHost, p->stream));
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  if (report) povar::fill_report(p, report, ms);
  if (p->h_state->error)
    return povar::fail(p, (povar_status)p->h_state->error, "device reported a numerical error");
  return POVAR_OK;
}

povar_status povar_s2_solve(povar_problem* pp, const povar_params* params, int32_t max_iters,
                            double ftol, double target_cost, povar_step_report* last,
                            int32_t* iters_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  povar_status s;
  if ((s = povar::check_s2_params(p, params)) != POVAR_OK) return s;
  if (max_iters < 1) return povar::fail(p, POVAR_EINVAL, "max_iters must be >= 1");
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  const int it0 = p->h_state->iteration;
  povar_params q = *params;
  const bool mixed = q.precision != POVAR_FP64;
  if ((s = povar::launch_begin(p, ftol, target_cost, max_iters,
                               mixed ? POVAR_FALLBACK_REJECTIONS : 0)) != POVAR_OK)
    return s;
  POVAR_CUDA(cudaEventRecord(p->ev0, p->stream));
  int fallback_at = 0;
  for (;;) {
    const int budget = it0 + max_iters - p->h_state->iteration;
    if ((s = povar::s2_solve_loop(p, &q, budget)) != POVAR_OK) return s;
    if (!p->h_state->fallback || q.precision == POVAR_FP64) break;
    fallback_at = p->h_state->iteration;
    q.precision = POVAR_FP64;
    if (it0 + max_iters - fallback_at <= 0) break;
    if ((s = povar::launch_begin(p, ftol, target_cost, it0 + max_iters - fallback_at, 0)) !=
        POVAR_OK)
      return s;
  }
  POVAR_CUDA(cudaEventRecord(p->ev1, p->stream));
  POVAR_CUDA(cudaMemcpyAsync(p->h_report, p->d_report, sizeof(povar_step_report),
                             cudaMemcpyDeviceToHost, p->stream));
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  if (last) {
    povar::fill_report(p, last, ms);
    last->fp64_fallback_at = fallback_at > 0 ? fallback_at - it0 : 0;
  }
  if (iters_out) *iters_out = p->h_state->iteration - it0;
  if (p->h_state->error)
    return povar::fail(p, (povar_status)p->h_state->error, "device reported an error");
  return POVAR_OK;
}

povar_status povar_s2_get_points(povar_problem* pp, double* X_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!X_out) return povar::fail(p, POVAR_EINVAL, "X_out is NULL");
  if (!p->s2_live) return povar::fail(p, POVAR_EINVAL, "call povar_s2_set first");
  double* d = reinterpret_cast<double*>(p->rec64);
  povar_status s;
  if ((s = povar::launch_s2_gather_points(p, d)) != POVAR_OK) return s;
  POVAR_CUDA(cudaMemcpyAsync(X_out, d, (size_t)p->np * 4 * sizeof(double),
                             cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}

povar_status povar_metric_upgrade(povar_problem* pp, const double* K, int32_t max_iters,
                                  double ftol, double* H_out, double* alpha_out,
                                  double* cost_out, int32_t* iters_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!H_out) return povar::fail(p, POVAR_EINVAL, "H_out is NULL");
  if (p->nc < 3) return povar::fail(p, POVAR_EINVAL, "the metric upgrade needs >= 3 cameras");
  if (max_iters < 1) return povar::fail(p, POVAR_EINVAL, "max_iters must be >= 1");
  if (!(ftol >= 0.0)) return povar::fail(p, POVAR_EINVAL, "ftol must be >= 0");
  povar_status s;
  const double* d_K = nullptr;
  if (K) {
    for (int64_t e = 0; e < (int64_t)p->nc * 9; ++e)
      if (!std::isfinite(K[e])) return povar::fail(p, POVAR_EINVAL, "non-finite intrinsics");
    if (!p->mu_K && (s = povar::dev_alloc(p, &p->mu_K, (size_t)p->nc * 9, "mu_K")) != POVAR_OK)
      return s;
    POVAR_CUDA(cudaMemcpyAsync(p->mu_K, K, (size_t)p->nc * 9 * sizeof(double),
                               cudaMemcpyHostToDevice, p->stream));
    d_K = p->mu_K;
  }
  int it = 0;
  if ((s = povar::launch_metric_upgrade(p, d_K, 1e-4, max_iters, ftol, H_out, alpha_out,
                                        cost_out, &it)) != POVAR_OK)
    return s;
  if (iters_out) *iters_out = it;
  return POVAR_OK;
}

povar_status povar_cost(povar_problem* pp, double eta, double* cost_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (!cost_out) return povar::fail(p, POVAR_EINVAL, "cost_out is NULL");
  if (!(eta >= 0.0 && eta <= 1.0)) return povar::fail(p, POVAR_EINVAL, "eta must be in [0, 1]");
  povar_status s;
  if (eta != p->eta_cur && (s = povar::refresh_landmarks(p, eta)) != POVAR_OK) return s;
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  *cost_out = p->h_state->F;
  return POVAR_OK;
}

povar_status povar_step(povar_problem* pp, const povar_params* params, povar_step_report* report) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  povar_status s;
  if ((s = povar::check_params(p, params)) != POVAR_OK) return s;
  if ((s = povar::launch_begin(p, 0.0, 0.0, 0)) != POVAR_OK) return s;
  POVAR_CUDA(cudaEventRecord(p->ev0, p->stream));
  if ((s = povar::enqueue_step(p, params)) != POVAR_OK) return s;
  POVAR_CUDA(cudaEventRecord(p->ev1, p->stream));
  POVAR_CUDA(cudaMemcpyAsync(p->h_report, p->d_report, sizeof(povar_step_report),
                             cudaMemcpyDeviceToHost, p->stream));
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  if (report) povar::fill_report(p, report, ms);
  if (p->h_state->error)
    return povar::fail(p, (povar_status)p->h_state->error, "device reported a numerical error");
  return POVAR_OK;
}

povar_status povar_solve(povar_problem* pp, const povar_params* params, int32_t max_iters,
                         double ftol, double target_cost, povar_step_report* last,
                         int32_t* iters_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  povar_status s;
  if ((s = povar::check_params(p, params)) != POVAR_OK) return s;
  if (max_iters < 1) return povar::fail(p, POVAR_EINVAL, "max_iters must be >= 1");
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  const int it0 = p->h_state->iteration;
  povar_params q = *params;
  const bool mixed = q.precision != POVAR_FP64;
  if ((s = povar::launch_begin(p, ftol, target_cost, max_iters,
                               mixed ? POVAR_FALLBACK_REJECTIONS : 0)) != POVAR_OK)
    return s;
  POVAR_CUDA(cudaEventRecord(p->ev0, p->stream));
  int fallback_at = 0;
  for (;;) {
    const int budget = it0 + max_iters - p->h_state->iteration;
    if ((s = povar::solve_loop(p, &q, budget)) != POVAR_OK) return s;
    // the mixed-precision safeguard stopped the solve: continue in FP64
    if (!p->h_state->fallback || q.precision == POVAR_FP64) break;
    fallback_at = p->h_state->iteration;
    q.precision = POVAR_FP64;
    if (it0 + max_iters - fallback_at <= 0) break;
    if ((s = povar::launch_begin(p, ftol, target_cost, it0 + max_iters - fallback_at, 0)) !=
        POVAR_OK)
      return s;
  }
  POVAR_CUDA(cudaEventRecord(p->ev1, p->stream));
  POVAR_CUDA(cudaMemcpyAsync(p->h_report, p->d_report, sizeof(povar_step_report),
                             cudaMemcpyDeviceToHost, p->stream));
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  if (last) {
    povar::fill_report(p, last, ms);
    last->fp64_fallback_at = fallback_at > 0 ? fallback_at - it0 : 0;
  }
  if (iters_out) *iters_out = p->h_state->iteration - it0;
  if (p->h_state->error)
    return povar::fail(p, (povar_status)p->h_state->error, "device reported an error");
  return POVAR_OK;
}

povar_status povar_set_profiling(povar_problem* pp, int32_t enable) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  povar_status s;
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  p->profiling = enable != 0;
  return POVAR_OK;
}

povar_status povar_get_profile(povar_problem* pp, double* ms_out, int64_t* steps_out,
                               int64_t* products_out, int32_t reset) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  povar_status s;
  if ((s = povar::sync_state(p)) != POVAR_OK) return s;
  if (ms_out)
    for (int ph = 0; ph < POVAR_NPHASES; ++ph) ms_out[ph] = p->prof_ms[ph];
  if (steps_out) *steps_out = p->prof_count;
  if (products_out) *products_out = p->prof_products;
  if (reset) {
    for (int ph = 0; ph < POVAR_NPHASES; ++ph) p->prof_ms[ph] = 0.0;
    p->prof_count = 0;
    p->prof_products = 0;
  }
  return POVAR_OK;
}

povar_status povar_get_tuning(povar_problem* pp, int32_t precision, int32_t* schedule_out,
                              float* ms_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (precision != POVAR_FP64 && precision != POVAR_MIXED_FP32)
    return povar::fail(p, POVAR_EINVAL, "unknown precision");
  const int k = precision == POVAR_FP64 ? 0 : 1;
  if (schedule_out) *schedule_out = p->tuned_schedule[k];
  if (ms_out)
    for (int q = 0; q < POVAR_NSCHEDULES; ++q) ms_out[q] = p->tune_ms[k][q];
  return POVAR_OK;
}

povar_status povar_get_orders(povar_problem* pp, uint32_t* perm_pt, uint32_t* off_pt,
                              uint32_t* perm_cam, uint32_t* off_cam) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  const size_t no = p->nobs;
  if (perm_pt)
    POVAR_CUDA(cudaMemcpyAsync(perm_pt, p->perm_pt, no * 4, cudaMemcpyDeviceToHost, p->stream));
  if (off_pt)
    POVAR_CUDA(cudaMemcpyAsync(off_pt, p->off_pt, ((size_t)p->np + 1) * 4, cudaMemcpyDeviceToHost,
                               p->stream));
  if (perm_cam)
    POVAR_CUDA(cudaMemcpyAsync(perm_cam, p->perm_cam, no * 4, cudaMemcpyDeviceToHost, p->stream));
  if (off_cam)
    POVAR_CUDA(cudaMemcpyAsync(off_cam, p->off_cam, ((size_t)p->nc + 1) * 4,
                               cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}

povar_status povar_get_layout(povar_problem* pp, int64_t* sizes, uint32_t* slot_pt,
                              uint32_t* sell_off, int32_t* sell_cam, uint32_t* row_mask,
                              uint32_t* row_base, uint32_t* cam_part_off,
                              uint32_t* cam_part_idx) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  if (sizes) {
    sizes[0] = p->np_pad;
    sizes[1] = p->nslices;
    sizes[2] = p->nsell;
    sizes[3] = p->nrows;
    sizes[4] = p->npart;
    sizes[5] = p->nvisits;
  }
  auto get = [&](void* dst, const void* src, size_t bytes) -> povar_status {
    if (dst && bytes)
      POVAR_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, p->stream));
    return POVAR_OK;
  };
  povar_status s;
  if ((s = get(slot_pt, p->slot_pt, (size_t)p->np_pad * 4)) != POVAR_OK ||
      (s = get(sell_off, p->sell_off, ((size_t)p->nslices + 1) * 4)) != POVAR_OK ||
      (s = get(sell_cam, p->sell_cam, (size_t)p->nsell * 4)) != POVAR_OK ||
      (s = get(row_mask, p->row_mask, (size_t)p->nrows * 4)) != POVAR_OK ||
      (s = get(row_base, p->row_base, (size_t)p->nrows * 4)) != POVAR_OK ||
      (s = get(cam_part_off, p->cam_part_off, ((size_t)p->nc + 1) * 4)) != POVAR_OK ||
      (s = get(cam_part_idx, p->cam_part_idx, (size_t)p->npart * 4)) != POVAR_OK)
    return s;
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}

povar_status povar_get_last_step(povar_problem* pp, double* U_out, double* bp_out,
                                 double* delta_out) {
  if (!pp) return POVAR_EINVAL;
  Problem* p = &pp->impl;
  const size_t nc = p->nc;
  if (U_out)
    POVAR_CUDA(cudaMemcpyAsync(U_out, p->U64, nc * 144 * 8, cudaMemcpyDeviceToHost, p->stream));
  if (bp_out)
    POVAR_CUDA(cudaMemcpyAsync(bp_out, p->bp64, nc * 12 * 8, cudaMemcpyDeviceToHost, p->stream));
  if (delta_out) {
    if (p->last_precision == POVAR_FP64) {
      POVAR_CUDA(cudaMemcpyAsync(delta_out, p->D64, nc * 12 * 8, cudaMemcpyDeviceToHost,
                                 p->stream));
    } else {
      std::vector<float> tmp(nc * 12);
      POVAR_CUDA(cudaMemcpyAsync(tmp.data(), p->D32, nc * 12 * 4, cudaMemcpyDeviceToHost,
                                 p->stream));
      POVAR_CUDA(cudaStreamSynchronize(p->stream));
      for (size_t e = 0; e < nc * 12; ++e) delta_out[e] = tmp[e];
    }
  }
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}

// ---------------------------------------------------------------- batches

struct povar_batch {
  std::vector<povar_problem*> probs;
  std::vector<int32_t> cam0;            // first camera of each problem
  int32_t nc_total = 0;
  cudaStream_t stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<povar_params> keys;       // parameters of each problem in the graph
  bool built = false;
  bool looped = false;                  // the graph is a device-side while loop over steps
  povar::DeviceState** d_states = nullptr;  // [n] the problems' device states
  int* d_loops = nullptr;               // [2] steps run, step limit
  std::string err;
};

static povar_status batch_fail(povar_batch* b, povar_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}

const char* povar_batch_last_error(const povar_batch* b) { return b ? b->err.c_str() : "null batch"; }

void povar_batch_destroy(povar_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_states) cudaFree(b->d_states);
  if (b->d_loops) cudaFree(b->d_loops);
  for (povar_problem* q : b->probs) povar_destroy(q);
  delete b;
}

povar_status povar_batch_create(int32_t n_problems, const int32_t* n_cams, const int32_t* n_points,
                                const int64_t* n_obs, const int32_t* cam_idx, const int32_t* pt_idx,
                                const double* meas, void* cuda_stream, povar_batch** out) {
  if (!out) return POVAR_EINVAL;
  *out = nullptr;
  if (n_problems < 1 || !n_cams || !n_points || !n_obs || !cam_idx || !pt_idx || !meas)
    return POVAR_EINVAL;
  povar_batch* b = new (std::nothrow) povar_batch();
  if (!b) return POVAR_ENOMEM;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  int64_t o = 0;
  for (int32_t k = 0; k < n_problems; ++k) {
    povar_problem* q = nullptr;
    const povar_status s = povar_create(n_cams[k], n_points[k], n_obs[k], cam_idx + o, pt_idx + o,
                                        meas + 2 * o, cuda_stream, &q);
    if (s != POVAR_OK) {
      povar_batch_destroy(b);
      return s;
    }
    b->probs.push_back(q);
    b->cam0.push_back(b->nc_total);
    b->nc_total += n_cams[k];
    o += n_obs[k];
  }
  // device state pointers and the step counters of the device-side loop
  // (without them a solve launches one graph per step)
  std::vector<povar::DeviceState*> st(b->probs.size());
  for (size_t k = 0; k < st.size(); ++k) st[k] = b->probs[k]->impl.state;
  if (cudaMalloc(reinterpret_cast<void**>(&b->d_states), st.size() * sizeof(st[0])) !=
          cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&b->d_loops), 2 * sizeof(int)) != cudaSuccess ||
      cudaMemcpy(b->d_states, st.data(), st.size() * sizeof(st[0]), cudaMemcpyHostToDevice) !=
          cudaSuccess) {
    cudaGetLastError();
    if (b->d_states) cudaFree(b->d_states);
    if (b->d_loops) cudaFree(b->d_loops);
    b->d_states = nullptr;
    b->d_loops = nullptr;
  }
  *out = b;
  return POVAR_OK;
}

povar_problem* povar_batch_problem(povar_batch* b, int32_t k) {
  if (!b || k < 0 || k >= (int32_t)b->probs.size()) return nullptr;
  return b->probs[k];
}

povar_status povar_batch_set_cameras(povar_batch* b, const double* P, double eta) {
  if (!b || !P) return POVAR_EINVAL;
  for (size_t k = 0; k < b->probs.size(); ++k) {
    const povar_status s = povar_set_cameras(b->probs[k], P + 12 * (size_t)b->cam0[k], eta);
    if (s != POVAR_OK) return batch_fail(b, s, povar_last_error(b->probs[k]));
  }
  return POVAR_OK;
}

povar_status povar_batch_get_cameras(povar_batch* b, double* P_out) {
  if (!b || !P_out) return POVAR_EINVAL;
  for (size_t k = 0; k < b->probs.size(); ++k) {
    const povar_status s = povar_get_cameras(b->probs[k], P_out + 12 * (size_t)b->cam0[k]);
    if (s != POVAR_OK) return batch_fail(b, s, povar_last_error(b->probs[k]));
  }
  return POVAR_OK;
}

povar_status povar_batch_cost(povar_batch* b, double eta, double* costs_out) {
  if (!b || !costs_out) return POVAR_EINVAL;
  for (size_t k = 0; k < b->probs.size(); ++k) {
    const povar_status s = povar_cost(b->probs[k], eta, costs_out + k);
    if (s != POVAR_OK) return batch_fail(b, s, povar_last_error(b->probs[k]));
  }
  return POVAR_OK;
}

// Batch solve with the parameters of problem k at params[k * each] (each = 0:
// one parameter set for all).
static povar_status batch_solve(povar_batch* b, const povar_params* params_base, size_t each,
                                int32_t max_iters, double ftol, const double* target_costs,
                                povar_step_report* reports, int32_t* iters_out) {
  if (!b || !params_base) return POVAR_EINVAL;
  if (max_iters < 1) return batch_fail(b, POVAR_EINVAL, "max_iters must be >= 1");
  povar_status s;
  const size_t n = b->probs.size();
  std::vector<int> it0(n);
  bool rebuild = !b->built || b->keys.size() != n;
  // In a batch many problems' kernels share the GPU: for small problems the
  // two-pass schedule (0), whose kernels leave room for other problems'
  // blocks, beats the schedule a problem's autotuner picks alone (on the
  // 64-problem batched family 877 against 482 solves/s); schedule -1 means
  // schedule 0 for problems of at most kBatchSmallObs observations there.
  constexpr int64_t kBatchSmallObs = 1 << 18;
  std::vector<povar_params> eff(n);
  for (size_t k = 0; k < n; ++k) {
    eff[k] = params_base[k * each];
    if (eff[k].schedule < 0 && eff[k].precision != POVAR_MIXED_BF16 &&
        b->probs[k]->impl.nobs <= kBatchSmallObs)
      eff[k].schedule = 0;
  }
  for (size_t k = 0; k < n && !rebuild; ++k) rebuild = !povar::same_params(b->keys[k], eff[k]);
  for (size_t k = 0; k < n; ++k) {
    Problem* p = &b->probs[k]->impl;
    const povar_params* params = &eff[k];
    if ((s = povar::check_params(p, params)) != POVAR_OK) return batch_fail(b, s, p->err);
    if (params->solver != POVAR_SOLVER_SERIES)
      return batch_fail(b, POVAR_EINVAL, "a batch runs the series solver only");
    if ((s = povar::sync_state(p)) != POVAR_OK) return batch_fail(b, s, p->err);
    it0[k] = p->h_state->iteration;
    if ((s = povar::launch_begin(p, ftol, target_costs ? target_costs[k] : 0.0, max_iters)) !=
        POVAR_OK)
      return batch_fail(b, s, p->err);
    if ((s = povar::prepare_step(p, params)) != POVAR_OK) return batch_fail(b, s, p->err);
    if (params->schedule < 0 && (s = povar::autotune_schedule(p, params)) != POVAR_OK)
      return batch_fail(b, s, p->err);
    cudaGraphExec_t before = p->gexec;
    if ((s = povar::step_graph(p, params)) != POVAR_OK) return batch_fail(b, s, p->err);
    rebuild |= p->gexec != before;
  }
  if (rebuild) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->looped = false;
    // preferred: the whole solve as one launch, a device-side while node
    // whose body runs one step of every problem and then decides whether
    // another step is needed (not with phase profiling: the step graphs
    // then hold event nodes, which a loop body cannot)
    bool profiled = false;
    for (povar_problem* q : b->probs) profiled |= q->impl.profiling;
    cudaError_t e = cudaSuccess;
    if (!profiled && b->d_states && b->d_loops) {
      e = cudaGraphCreate(&b->graph, 0);
      cudaGraphConditionalHandle h{};
      if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&h, b->graph, 1, cudaGraphCondAssignDefault);
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode;
      if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, b->graph, nullptr, nullptr, 0, &cp);
      std::vector<cudaGraphNode_t> kids(n);
      for (size_t k = 0; k < n && e == cudaSuccess; ++k)
        e = cudaGraphAddChildGraphNode(&kids[k], cp.conditional.phGraph_out[0], nullptr, 0,
                                       b->probs[k]->impl.graph);
      if (e == cudaSuccess)
        e = povar::add_batch_continue(cp.conditional.phGraph_out[0], kids.data(), n, h,
                                      b->d_states, (int)n, b->d_loops);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e == cudaSuccess) {
        b->looped = true;
      } else {
        cudaGetLastError();
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
      }
    }
    // otherwise one launch per step of a graph holding every problem's step
    if (!b->looped) {
      e = cudaGraphCreate(&b->graph, 0);
      for (size_t k = 0; k < n && e == cudaSuccess; ++k) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, b->graph, nullptr, 0, b->probs[k]->impl.graph);
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->built = false;
      return batch_fail(b, POVAR_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    b->keys = eff;
    b->built = true;
  }
  if (b->looped) {
    // one launch for the whole solve; the loop stops on the device
    const int h_loops[2] = {0, max_iters};
    int done[2] = {0, 0};
    if (cudaMemcpyAsync(b->d_loops, h_loops, sizeof(h_loops), cudaMemcpyHostToDevice,
                        b->stream) != cudaSuccess ||
        cudaGraphLaunch(b->exec, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(done, b->d_loops, sizeof(done), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
      cudaGetLastError();
      return batch_fail(b, POVAR_ECUDA, "batch loop launch");
    }
    for (povar_problem* q : b->probs) q->impl.launches += (int64_t)done[0] * q->impl.g_launches;
    b->probs[0]->impl.launches += done[0];   // the loop's condition kernel
  }
  const int check_every = 4;
  for (int it = 0; it < (b->looped ? 0 : max_iters); ++it) {
    const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess)
      return batch_fail(b, POVAR_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    for (povar_problem* q : b->probs) q->impl.launches += q->impl.g_launches;
    if ((it + 1) % check_every == 0 && it + 1 < max_iters) {
      bool all = true;
      for (povar_problem* q : b->probs) {
        Problem* p = &q->impl;
        if (cudaMemcpyAsync(p->h_state, p->state, sizeof(povar::DeviceState),
                            cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
          return batch_fail(b, POVAR_ECUDA, "state copy");
      }
      if (cudaStreamSynchronize(b->stream) != cudaSuccess)
        return batch_fail(b, POVAR_ECUDA, "stream sync");
      for (povar_problem* q : b->probs) all &= q->impl.h_state->converged != 0;
      if (all) break;
    }
  }
  povar_status worst = POVAR_OK;
  for (size_t k = 0; k < n; ++k) {
    Problem* p = &b->probs[k]->impl;
    if (cudaMemcpyAsync(p->h_report, p->d_report, sizeof(povar_step_report),
                        cudaMemcpyDeviceToHost, b->stream) != cudaSuccess)
      return batch_fail(b, POVAR_ECUDA, "report copy");
    if ((s = povar::sync_state(p)) != POVAR_OK) return batch_fail(b, s, p->err);
    if (reports) povar::fill_report(p, reports + k, 0.f);
    if (iters_out) iters_out[k] = p->h_state->iteration - it0[k];
    if (p->h_state->error && worst == POVAR_OK) worst = (povar_status)p->h_state->error;
  }
  return worst == POVAR_OK ? POVAR_OK : batch_fail(b, worst, "a problem reported a device error");
}

povar_status povar_batch_solve(povar_batch* b, const povar_params* params, int32_t max_iters,
                               double ftol, const double* target_costs,
                               povar_step_report* reports, int32_t* iters_out) {
  return batch_solve(b, params, 0, max_iters, ftol, target_costs, reports, iters_out);
}

povar_status povar_batch_solve_each(povar_batch* b, const povar_params* params,
                                    int32_t max_iters, double ftol, const double* target_costs,
                                    povar_step_report* reports, int32_t* iters_out) {
  return batch_solve(b, params, 1, max_iters, ftol, target_costs, reports, iters_out);
}

}  // extern "C"
