// a1: observation orders (built once per problem).
//
// The point-major and camera-major orders are stable sorts of the
// observation ids by landmark and by camera (ties keep the input order), so
// they equal a CPU stable sort bit for bit. The sort is an LSD radix sort
// with 8-bit digits; each pass ranks the keys of a 2048-key tile with warp
// match/ballot and a per-digit running count, which keeps it stable.
#include "povar_internal.cuh"


#include <algorithm>

namespace povar {
namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

__global__ void k_iota(uint32_t* v, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = (uint32_t)i;
}

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                             uint32_t* __restrict__ hist, int ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = 0; k < RS_ITEMS; ++k) {
    const int64_t i = base + (int64_t)k * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one tile: chunk c of the tile is items [c*256, c*256+256)
// in input order; warp w owns 32 consecutive items of the chunk.
__global__ void k_radix_scatter(const uint32_t* __restrict__ kin,
                                const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                int64_t n, int shift, const uint32_t* __restrict__ offs,
                                int ntiles) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t wcnt[RS_WARPS][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  run[threadIdx.x] = 0;
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int c = 0; c < RS_ITEMS; ++c) {
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) wcnt[q][threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = base + (int64_t)c * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    uint32_t key = 0, val = 0;
    unsigned d = 256u + (unsigned)lane;  // unique sentinel for invalid lanes
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = (key >> shift) & 255u;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt_mask);
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[w][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t acc = run[threadIdx.x];
#pragma unroll
      for (int q = 0; q < RS_WARPS; ++q) {
        const uint32_t t = wcnt[q][threadIdx.x];
        wcnt[q][threadIdx.x] = acc;
        acc += t;
      }
      run[threadIdx.x] = acc;
    }
    __syncthreads();
    if (valid) {
      const uint32_t pos = offs[(size_t)d * ntiles + blockIdx.x] + wcnt[w][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
  }
}

// Exclusive scan of 2048 elements per block (256 threads x 8 consecutive).
__global__ void k_scan_block(uint32_t* __restrict__ data, int64_t n,
                             uint32_t* __restrict__ block_sums) {
  __shared__ uint32_t warp_tot[RS_WARPS];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  uint32_t v[RS_ITEMS];
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    v[k] = (base + k < n) ? data[base + k] : 0u;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint32_t wbase = 0, tot = 0;
#pragma unroll
  for (int q = 0; q < RS_WARPS; ++q) {
    if (q < w) wbase += warp_tot[q];
    tot += warp_tot[q];
  }
  uint32_t run = wbase + incl - s;
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k) {
    if (base + k < n) data[base + k] = run;
    run += v[k];
  }
  if (block_sums != nullptr && threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(uint32_t* __restrict__ data, int64_t n,
                           const uint32_t* __restrict__ block_off) {
  const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)threadIdx.x * RS_ITEMS;
  const uint32_t a = block_off[blockIdx.x];
#pragma unroll
  for (int k = 0; k < RS_ITEMS; ++k)
    if (base + k < n) data[base + k] += a;
}

// off[k] = first position whose sorted key is >= k, for k in [0, nkeys].
__global__ void k_offsets(const uint32_t* __restrict__ skeys, int64_t n, int64_t nkeys,
                          uint32_t* __restrict__ off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = skeys[i];
  const int64_t prev = (i == 0) ? -1 : (int64_t)skeys[i - 1];
  for (int64_t q = prev + 1; q <= k; ++q) off[q] = (uint32_t)i;
  if (i == n - 1)
    for (int64_t q = k + 1; q <= nkeys; ++q) off[q] = (uint32_t)n;
}

// Per landmark: track length and smallest camera index.
__global__ void k_point_stats(const uint32_t* __restrict__ off_pt,
                              const uint32_t* __restrict__ perm_pt,
                              const int32_t* __restrict__ cam, int np,
                              uint32_t* __restrict__ len, uint32_t* __restrict__ mincam) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const uint32_t b = off_pt[j], e = off_pt[j + 1];
  uint32_t mc = 0xffffffffu;
  for (uint32_t r = b; r < e; ++r) mc = min(mc, (uint32_t)cam[perm_pt[r]]);
  len[j] = e - b;
  mincam[j] = mc;
}

// Slot key: smallest camera first, then track length descending. Landmarks
// whose tracks start at the same camera are adjacent, so when tracks are
// contiguous runs of cameras (video, trajectories) the lanes of a slice visit
// the same camera at the same track position; within one start camera the
// lengths descend, so a slice's lanes have nearly equal track lengths.
__global__ void k_slot_keys(const uint32_t* __restrict__ len,
                            const uint32_t* __restrict__ mincam, int np, uint32_t maxlen,
                            int len_bits, int use_cam, uint32_t* __restrict__ key) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  uint32_t k = maxlen - len[j];
  if (use_cam) k |= mincam[j] << len_bits;
  key[j] = k;
}

// Slice width = longest track among its 32 slots (times 32 entries per row).
// SELL measurements split into double-float pairs (u_hi, u_lo, v_hi, v_lo)
// for the double-float landmark kernel (padding entries are zero).
__global__ void k_split_meas(const double2* __restrict__ m, int64_t n, float4* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double2 x = m[i];
  const float uh = (float)x.x, vh = (float)x.y;
  out[i] = make_float4(uh, (float)(x.x - (double)uh), vh, (float)(x.y - (double)vh));
}

__global__ void k_slice_width(const uint32_t* __restrict__ slot_len, int nslices,
                              uint32_t* __restrict__ w32) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslices) return;
  uint32_t w = 0;
  for (int l = 0; l < SLICE; ++l) w = max(w, slot_len[s * SLICE + l]);
  w32[s] = w * SLICE;
}

__global__ void k_fill_sell(const uint32_t* __restrict__ slot_pt,
                            const uint32_t* __restrict__ slot_len,
                            const uint32_t* __restrict__ sell_off,
                            const uint32_t* __restrict__ off_pt,
                            const uint32_t* __restrict__ perm_pt,
                            const int32_t* __restrict__ cam, const double* __restrict__ meas,
                            int nslots, int32_t* __restrict__ sell_cam,
                            float2* __restrict__ m32, double2* __restrict__ m64) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nslots) return;
  const uint32_t j = slot_pt[s];
  if (j == 0xffffffffu) return;   // padding slot
  const uint32_t len = slot_len[s];
  const uint32_t b = off_pt[j];
  const uint32_t base = sell_off[s / SLICE] + (uint32_t)(s % SLICE);
  for (uint32_t t = 0; t < len; ++t) {
    const uint32_t o = perm_pt[b + t];
    const uint32_t pos = base + t * SLICE;
    const double u = meas[2 * (size_t)o], v = meas[2 * (size_t)o + 1];
    sell_cam[pos] = cam[o];
    m32[pos] = make_float2((float)u, (float)v);
    m64[pos] = make_double2(u, v);
  }
}

__global__ void k_fill_cm(const uint32_t* __restrict__ perm_cam,
                          const int32_t* __restrict__ pt, const uint32_t* __restrict__ pt_slot,
                          const double* __restrict__ meas, int64_t n,
                          uint32_t* __restrict__ cm_slot, float2* __restrict__ m32,
                          double2* __restrict__ m64) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t o = perm_cam[r];
  const double u = meas[2 * (size_t)o], v = meas[2 * (size_t)o + 1];
  cm_slot[r] = pt_slot[pt[o]];
  m32[r] = make_float2((float)u, (float)v);
  m64[r] = make_double2(u, v);
}

// keys[r] = pt[perm[r]], vals[r] = perm[r]
__global__ void k_keys_through(const int32_t* __restrict__ pt, const uint32_t* __restrict__ perm,
                               int64_t n, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint32_t o = perm[r];
  keys[r] = (uint32_t)pt[o];
  vals[r] = o;
}

__global__ void k_to_u32(const int32_t* __restrict__ src, uint32_t* __restrict__ dst, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (uint32_t)src[i];
}

// Input check before any index is used: every camera and landmark index in
// range and every measurement finite; flag bit 0 set otherwise.
__global__ void k_validate(const int32_t* __restrict__ cam, const int32_t* __restrict__ pt,
                           const double* __restrict__ meas, int64_t n, int nc, int np,
                           uint32_t* __restrict__ flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (i < n) {
    const int32_t c = cam[i], j = pt[i];
    bad = c < 0 || c >= nc || j < 0 || j >= np || !isfinite(meas[2 * i]) ||
          !isfinite(meas[2 * i + 1]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Longest track (stats[0]) and whether some landmark has no observation
// (stats[1] = 1).
__global__ void k_len_stats(const uint32_t* __restrict__ len, int np,
                            uint32_t* __restrict__ stats) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t l = j < np ? len[j] : 1u;
  const uint32_t mx = __reduce_max_sync(0xffffffffu, l);
  const bool empty = __any_sync(0xffffffffu, j < np && l == 0u);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(stats, mx);
    if (empty) atomicOr(stats + 1, 1u);
  }
}

// Bucket-aligned slot sequence. The landmarks sorted by (smallest camera,
// track length descending) form one bucket per smallest camera; every bucket
// starts a new slice (its last slice is padded to 32 slots), so that a slice
// never mixes landmarks whose tracks start at different cameras: for tracks
// over consecutive cameras every row of a slice then sees one camera.
//   k_bucket_flags: flag[i] = 1 where the sorted order starts a new bucket;
//   k_bucket_first: bfirst[b] = first sorted index of bucket b;
//   k_bucket_pad:   psize[b] = size of bucket b rounded up to 32 slots;
//   k_seq_fill:     seq[pstart[b] + (i - bfirst[b])] = order[i].
__global__ void k_bucket_flags(const uint32_t* __restrict__ order,
                               const uint32_t* __restrict__ mincam, int np,
                               uint32_t* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  // without mincam (the camera does not fit the sort key): a single bucket
  flag[i] = (i == 0 || (mincam && mincam[order[i]] != mincam[order[i - 1]])) ? 1u : 0u;
}

// excl = exclusive scan of the flags: the bucket of i is excl[i + 1] - 1
__global__ void k_bucket_first(const uint32_t* __restrict__ excl, int np,
                               uint32_t* __restrict__ bfirst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > np) return;
  if (i == np) {
    bfirst[excl[np]] = (uint32_t)np;
    return;
  }
  if (excl[i + 1] != excl[i]) bfirst[excl[i]] = (uint32_t)i;
}

__global__ void k_bucket_pad(const uint32_t* __restrict__ bfirst, int nb,
                             uint32_t* __restrict__ psize) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const uint32_t sz = bfirst[b + 1] - bfirst[b];
  psize[b] = (sz + SLICE - 1) / SLICE * SLICE;
}

__global__ void k_seq_fill(const uint32_t* __restrict__ order, const uint32_t* __restrict__ excl,
                           const uint32_t* __restrict__ bfirst,
                           const uint32_t* __restrict__ pstart, int np,
                           uint32_t* __restrict__ seq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const uint32_t b = excl[i + 1] - 1;
  seq[pstart[b] + ((uint32_t)i - bfirst[b])] = order[i];
}

// Slice order: slice sl of the aligned sequence gets the key maxlen - (its
// longest track), so a stable ascending sort puts the widest slices first and
// keeps the sequence order among equal widths.
__global__ void k_slice_keys(const uint32_t* __restrict__ seq, const uint32_t* __restrict__ len,
                             int nsl, uint32_t maxlen, uint32_t* __restrict__ wkey,
                             uint32_t* __restrict__ wval) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nsl) return;
  uint32_t w = 0;
  for (int l = 0; l < SLICE; ++l) {
    const uint32_t j = seq[(size_t)sl * SLICE + l];
    if (j != 0xffffffffu) w = max(w, len[j]);
  }
  wkey[sl] = maxlen - w;
  wval[sl] = (uint32_t)sl;
}

// Slot q: the slices of the aligned sequence in the width order sl_order,
// then padding up to np_pad.
__global__ void k_slot_fill(const uint32_t* __restrict__ seq,
                            const uint32_t* __restrict__ sl_order,
                            const uint32_t* __restrict__ len, int nsl, int np_pad,
                            uint32_t* __restrict__ slot_pt, uint32_t* __restrict__ slot_len,
                            uint32_t* __restrict__ pt_slot) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np_pad) return;
  uint32_t j = 0xffffffffu;
  const int sl = q / SLICE;
  if (sl < nsl) j = seq[(size_t)sl_order[sl] * SLICE + (q % SLICE)];
  slot_pt[q] = j;
  slot_len[q] = j == 0xffffffffu ? 0u : len[j];
  if (j != 0xffffffffu) pt_slot[j] = (uint32_t)q;
}

// Run table of the fused schedule, one warp per slice row (the row's 32
// camera indices, -1 for padding). A row whose valid lanes all see one
// camera is uniform: mask 0, its camera in rcam, one partial. Otherwise bit l
// of the mask marks a lane whose camera differs from lane l - 1's (bit 0
// always), rcam = -1, and every marked lane with a valid camera opens a
// partial. nvis counts the row's distinct valid cameras (its camera-row
// visits).
__global__ void k_row_runs(const int32_t* __restrict__ cam, int64_t nrows,
                           uint32_t* __restrict__ mask, int32_t* __restrict__ rcam,
                           uint32_t* __restrict__ npart, uint32_t* __restrict__ nvis) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;  // the whole warp
  const int32_t c = cam[row * SLICE + lane];
  const bool valid = c >= 0;
  const uint32_t vb = __ballot_sync(0xffffffffu, valid);
  const int32_t c0 = __shfl_sync(0xffffffffu, c, vb ? __ffs(vb) - 1 : 0);
  const bool uniform = vb != 0u && __ballot_sync(0xffffffffu, valid && c != c0) == 0u;
  const int32_t prev = __shfl_up_sync(0xffffffffu, c, 1);
  const uint32_t start = __ballot_sync(0xffffffffu, lane == 0 || c != prev);
  const uint32_t same = __match_any_sync(0xffffffffu, c);
  const uint32_t firsts = __ballot_sync(0xffffffffu, valid && __ffs(same) - 1 == lane);
  if (lane == 0) {
    mask[row] = uniform ? 0u : start;
    rcam[row] = uniform ? c0 : -1;
    npart[row] = uniform ? 1u : (uint32_t)__popc(start & vb);
    nvis[row] = (uint32_t)__popc(firsts);
  }
}

// Cameras of the partials (pcam, in partial order) and the camera-row visits
// (vcam, vrow: the row's distinct valid cameras in lane order), at the
// row offsets pbase and vbase.
__global__ void k_row_fill(const int32_t* __restrict__ cam, int64_t nrows,
                           const uint32_t* __restrict__ mask, const int32_t* __restrict__ rcam,
                           const uint32_t* __restrict__ pbase, const uint32_t* __restrict__ vbase,
                           uint32_t* __restrict__ pcam, uint32_t* __restrict__ vcam,
                           uint32_t* __restrict__ vrow) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;  // the whole warp
  const int32_t c = cam[row * SLICE + lane];
  const bool valid = c >= 0;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t vb = __ballot_sync(0xffffffffu, valid);
  const uint32_t m = mask[row];
  if (m == 0u) {
    if (lane == 0) pcam[pbase[row]] = (uint32_t)rcam[row];
  } else {
    const uint32_t sv = m & vb;
    if ((sv >> lane) & 1u) pcam[pbase[row] + __popc(sv & lt)] = (uint32_t)c;
  }
  const uint32_t same = __match_any_sync(0xffffffffu, c);
  const uint32_t firsts = __ballot_sync(0xffffffffu, valid && __ffs(same) - 1 == lane);
  if ((firsts >> lane) & 1u) {
    const uint32_t q = vbase[row] + __popc(firsts & lt);
    vcam[q] = (uint32_t)c;
    vrow[q] = (uint32_t)row;
  }
}

// Slice of every slice row.
__global__ void k_row_slice(const uint32_t* __restrict__ sell_off, int nslices,
                            uint32_t* __restrict__ row_slice) {
  const int sl = blockIdx.x * blockDim.x + threadIdx.x;
  if (sl >= nslices) return;
  for (uint32_t r = sell_off[sl] / SLICE; r < sell_off[sl + 1] / SLICE; ++r) row_slice[r] = sl;
}

// Camera-row lists: visit q of the camera-sorted order is the row vrow[v]
// (v = vidx[q]), given as the SELL position of the row and the slot of its
// lane 0.
__global__ void k_visit_fill(const uint32_t* __restrict__ vidx, const uint32_t* __restrict__ vrow,
                             const uint32_t* __restrict__ row_slice, int64_t nvis,
                             uint32_t* __restrict__ pos0, uint32_t* __restrict__ slot0) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nvis) return;
  const uint32_t row = vrow[vidx[q]];
  pos0[q] = row * SLICE;
  slot0[q] = row_slice[row] * SLICE;
}

// Tables of the grouped schedule with one slice per group: group g is slice
// g, its rows are the slice rows, and the partial space is the fused one.
__global__ void k_group_tables(int64_t nrows, const uint32_t* __restrict__ mask,
                               const int32_t* __restrict__ rcam,
                               const uint32_t* __restrict__ pbase,
                               int32_t* __restrict__ grow_cam, uint32_t* __restrict__ grow_base,
                               uint32_t* __restrict__ srow_mask,
                               uint32_t* __restrict__ srow_base) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const bool u = rcam[r] >= 0;
  grow_cam[r] = rcam[r];
  grow_base[r] = u ? pbase[r] : 0u;
  srow_mask[r] = u ? 0u : mask[r];
  srow_base[r] = u ? 0u : pbase[r];
}

__global__ void k_group_rows(const uint32_t* __restrict__ sell_off, int nslices,
                             uint32_t* __restrict__ grp_slice0, uint32_t* __restrict__ grp_row0) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g > nslices) return;
  grp_slice0[g] = (uint32_t)g;
  grp_row0[g] = sell_off[g] / SLICE;
}

int bits_for(uint64_t maxval) {
  int b = 0;
  while (b < 32 && (maxval >> b) != 0) ++b;
  return std::max(b, 1);
}

// Copies of the set-up tables between host vectors and the device run on the
// problem's stream and are waited for: a plain cudaMemcpy runs on the legacy
// default stream, which is not ordered with a caller's non-blocking stream,
// so it could read a table before the set-up kernels have written it, or a
// kernel could read a table before its upload has landed.
template <class T>
povar_status copy_sync(Problem* p, T* dst, const T* src, size_t count, cudaMemcpyKind kind) {
  POVAR_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(T), kind, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return POVAR_OK;
}
#define POVAR_COPY(dst, src, count, kind)                                    \
  do {                                                                       \
    const povar_status cs_ = copy_sync(p, dst, src, count, kind);            \
    if (cs_ != POVAR_OK) return cs_;                                         \
  } while (0)

// Scratch buffers of the set-up, from the stream-ordered allocator on the
// problem's stream and returned in stream order when the scope ends (after
// every kernel enqueued before that point).
struct Scratch {
  cudaStream_t stream;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : stream(s) {}
  ~Scratch() {
    for (void* q : ptrs) cudaFreeAsync(q, stream);
  }
  template <class T>
  T* get(size_t count) {
    void* q = nullptr;
    cudaMemPool_t pool;
    if (library_pool(&pool) != cudaSuccess ||
        cudaMallocFromPoolAsync(&q, std::max<size_t>(count, 1) * sizeof(T), pool, stream) !=
            cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    ptrs.push_back(q);
    return static_cast<T*>(q);
  }
};

povar_status scan_exclusive(Problem* p, Scratch& sc, uint32_t* data, int64_t n) {
  const int64_t nb = (n + RS_TILE - 1) / RS_TILE;
  if (nb <= 1) {
    k_scan_block<<<1, RS_THREADS, 0, p->stream>>>(data, n, nullptr);
    ++p->launches;
    return check_launch(p, "scan");
  }
  uint32_t* sums = sc.get<uint32_t>(nb);
  if (!sums) return fail(p, POVAR_ENOMEM, "scan scratch");
  k_scan_block<<<(unsigned)nb, RS_THREADS, 0, p->stream>>>(data, n, sums);
  ++p->launches;
  povar_status s = scan_exclusive(p, sc, sums, nb);
  if (s != POVAR_OK) return s;
  k_scan_add<<<(unsigned)nb, RS_THREADS, 0, p->stream>>>(data, n, sums);
  ++p->launches;
  return check_launch(p, "scan_add");
}

// Stable sort of (keys, vals) by keys < 2^key_bits. Results end in (*k, *v).
povar_status radix_sort(Problem* p, Scratch& sc, uint32_t** k, uint32_t** v, int64_t n,
                        int key_bits) {
  const int ntiles = (int)((n + RS_TILE - 1) / RS_TILE);
  uint32_t* k2 = sc.get<uint32_t>(n);
  uint32_t* v2 = sc.get<uint32_t>(n);
  uint32_t* hist = sc.get<uint32_t>((size_t)256 * ntiles);
  if (!k2 || !v2 || !hist) return fail(p, POVAR_ENOMEM, "radix scratch");
  uint32_t *ka = *k, *va = *v, *kb = k2, *vb = v2;
  for (int shift = 0; shift < key_bits; shift += 8) {
    k_radix_hist<<<ntiles, RS_THREADS, 0, p->stream>>>(ka, n, shift, hist, ntiles);
    ++p->launches;
    povar_status s = scan_exclusive(p, sc, hist, (int64_t)256 * ntiles);
    if (s != POVAR_OK) return s;
    k_radix_scatter<<<ntiles, RS_THREADS, 0, p->stream>>>(ka, va, kb, vb, n, shift, hist,
                                                         ntiles);
    ++p->launches;
    if ((s = check_launch(p, "radix_scatter")) != POVAR_OK) return s;
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  *k = ka;
  *v = va;
  return POVAR_OK;
}

}  // namespace

povar_status build_runs(Problem* p);
povar_status build_groups5(Problem* p, const int32_t* d_rcam);

povar_status build_orders(Problem* p, const int32_t* h_cam, const int32_t* h_pt) {
  (void)h_cam;
  (void)h_pt;
  Scratch sc(p->stream);
  const int64_t n = p->nobs;
  const unsigned gb = grid_for(n, 256);
  povar_status s;

  // ---- indices in range and measurements finite, before any index is used
  {
    uint32_t* flag = sc.get<uint32_t>(1);
    if (!flag) return fail(p, POVAR_ENOMEM, "validation scratch");
    POVAR_CUDA(cudaMemsetAsync(flag, 0, sizeof(uint32_t), p->stream));
    k_validate<<<gb, 256, 0, p->stream>>>(p->d_cam, p->d_pt, p->d_meas, n, p->nc, p->np, flag);
    ++p->launches;
    uint32_t h_flag = 0;
    POVAR_COPY(&h_flag, flag, 1, cudaMemcpyDeviceToHost);
    if (h_flag) return fail(p, POVAR_EINVAL, "index out of range or non-finite measurement");
  }

  // ---- point-major and camera-major stable orders
  for (int which = 0; which < 2; ++which) {
    uint32_t* keys = sc.get<uint32_t>(n);
    uint32_t* vals = sc.get<uint32_t>(n);
    if (!keys || !vals) return fail(p, POVAR_ENOMEM, "order scratch");
    k_to_u32<<<gb, 256, 0, p->stream>>>(which == 0 ? p->d_pt : p->d_cam, keys, n);
    k_iota<<<gb, 256, 0, p->stream>>>(vals, n);
    p->launches += 2;
    const int64_t nkeys = which == 0 ? p->np : p->nc;
    uint32_t *kk = keys, *vv = vals;
    if ((s = radix_sort(p, sc, &kk, &vv, n, bits_for((uint64_t)(nkeys - 1)))) != POVAR_OK)
      return s;
    uint32_t* perm = which == 0 ? p->perm_pt : p->perm_cam;
    uint32_t* off = which == 0 ? p->off_pt : p->off_cam;
    POVAR_CUDA(cudaMemcpyAsync(perm, vv, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                               p->stream));
    k_offsets<<<gb, 256, 0, p->stream>>>(kk, n, nkeys, off);
    ++p->launches;
    if ((s = check_launch(p, "offsets")) != POVAR_OK) return s;
  }

  // ---- observations of each landmark in camera order (stable sort of the
  //      camera-major order by landmark): the SELL rows follow this order
  uint32_t* perm_ptcam = nullptr;
  {
    uint32_t* keys = sc.get<uint32_t>(n);
    uint32_t* vals = sc.get<uint32_t>(n);
    if (!keys || !vals) return fail(p, POVAR_ENOMEM, "order scratch");
    k_keys_through<<<gb, 256, 0, p->stream>>>(p->d_pt, p->perm_cam, n, keys, vals);
    ++p->launches;
    uint32_t *kk = keys, *vv = vals;
    if ((s = radix_sort(p, sc, &kk, &vv, n, bits_for((uint64_t)(p->np - 1)))) != POVAR_OK)
      return s;
    perm_ptcam = vv;
  }

  // ---- landmark slots: smallest camera first, then track length (desc)
  uint32_t* len = sc.get<uint32_t>(p->np);
  uint32_t* mincam = sc.get<uint32_t>(p->np);
  uint32_t* skey = sc.get<uint32_t>(p->np);
  uint32_t* sval = sc.get<uint32_t>(p->np);
  if (!len || !mincam || !skey || !sval) return fail(p, POVAR_ENOMEM, "slot scratch");
  const unsigned gp = grid_for(p->np, 256);
  k_point_stats<<<gp, 256, 0, p->stream>>>(p->off_pt, p->perm_pt, p->d_cam, p->np, len,
                                           mincam);
  ++p->launches;
  // longest track, and every landmark must be observed
  uint32_t* stats = sc.get<uint32_t>(2);
  if (!stats) return fail(p, POVAR_ENOMEM, "slot scratch");
  POVAR_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(uint32_t), p->stream));
  k_len_stats<<<gp, 256, 0, p->stream>>>(len, p->np, stats);
  ++p->launches;
  uint32_t h_stats[2] = {0, 0};
  POVAR_COPY(h_stats, stats, 2, cudaMemcpyDeviceToHost);
  if (h_stats[1]) return fail(p, POVAR_EINVAL, "landmark without observations");
  const uint32_t maxlen = h_stats[0];
  const int len_bits = bits_for(maxlen);
  const int cam_bits = bits_for((uint64_t)(p->nc - 1));
  const int use_cam = (len_bits + cam_bits <= 32) ? 1 : 0;
  k_slot_keys<<<gp, 256, 0, p->stream>>>(len, mincam, p->np, maxlen, len_bits, use_cam, skey);
  k_iota<<<gp, 256, 0, p->stream>>>(sval, p->np);
  p->launches += 2;
  {
    uint32_t *kk = skey, *vv = sval;
    if ((s = radix_sort(p, sc, &kk, &vv, p->np, use_cam ? len_bits + cam_bits : len_bits)) !=
        POVAR_OK)
      return s;
    // Bucket-aligned sequence (every smallest camera starts a slice; when the
    // camera does not fit the sort key, one bucket), then all of its slices
    // ordered by width (longest track first, stable) so that the warps of a
    // block get similar work; padding up to a multiple of BLOCK slots at the
    // end. Every slice is its own group (GROUP = 1).
    static_assert(GROUP == 1, "the slot order and the run tables take one slice per group");
    uint32_t* flag = sc.get<uint32_t>((size_t)p->np + 1);
    uint32_t* bfirst = sc.get<uint32_t>((size_t)p->np + 1);
    uint32_t* pstart = sc.get<uint32_t>((size_t)p->np + 1);
    if (!flag || !bfirst || !pstart) return fail(p, POVAR_ENOMEM, "bucket scratch");
    POVAR_CUDA(cudaMemsetAsync(flag, 0, ((size_t)p->np + 1) * sizeof(uint32_t), p->stream));
    k_bucket_flags<<<gp, 256, 0, p->stream>>>(vv, use_cam ? mincam : nullptr, p->np, flag);
    if ((s = scan_exclusive(p, sc, flag, (int64_t)p->np + 1)) != POVAR_OK) return s;
    k_bucket_first<<<grid_for((int64_t)p->np + 1, 256), 256, 0, p->stream>>>(flag, p->np,
                                                                            bfirst);
    p->launches += 2;
    uint32_t nb = 0;
    POVAR_COPY(&nb, flag + p->np, 1, cudaMemcpyDeviceToHost);
    POVAR_CUDA(cudaMemsetAsync(pstart, 0, ((size_t)nb + 1) * sizeof(uint32_t), p->stream));
    k_bucket_pad<<<grid_for(nb, 256), 256, 0, p->stream>>>(bfirst, (int)nb, pstart);
    ++p->launches;
    if ((s = scan_exclusive(p, sc, pstart, (int64_t)nb + 1)) != POVAR_OK) return s;
    uint32_t total = 0;
    POVAR_COPY(&total, pstart + nb, 1, cudaMemcpyDeviceToHost);
    p->np_pad = (int32_t)(((int64_t)total + BLOCK - 1) / BLOCK * BLOCK);
    p->nslices = p->np_pad / SLICE;
    p->n_slot_blocks = p->np_pad / BLOCK;
    if ((s = alloc_slot_arrays(p)) != POVAR_OK) return s;
    uint32_t* seq = sc.get<uint32_t>(total);
    if (!seq) return fail(p, POVAR_ENOMEM, "bucket scratch");
    POVAR_CUDA(cudaMemsetAsync(seq, 0xff, (size_t)total * sizeof(uint32_t), p->stream));
    k_seq_fill<<<gp, 256, 0, p->stream>>>(vv, flag, bfirst, pstart, p->np, seq);
    ++p->launches;
    const int nsl = (int)(total / SLICE);
    uint32_t* wkey = sc.get<uint32_t>(nsl);
    uint32_t* wval = sc.get<uint32_t>(nsl);
    if (!wkey || !wval) return fail(p, POVAR_ENOMEM, "slice scratch");
    k_slice_keys<<<grid_for(nsl, 256), 256, 0, p->stream>>>(seq, len, nsl, maxlen, wkey, wval);
    ++p->launches;
    uint32_t *wk = wkey, *wv = wval;
    if ((s = radix_sort(p, sc, &wk, &wv, nsl, bits_for(maxlen))) != POVAR_OK) return s;
    k_slot_fill<<<grid_for(p->np_pad, 256), 256, 0, p->stream>>>(
        seq, wv, len, nsl, p->np_pad, p->slot_pt, p->slot_len, p->pt_slot);
    ++p->launches;
    if ((s = check_launch(p, "slot order")) != POVAR_OK) return s;
    p->ngroups = p->nslices;
  }
  // ---- SELL offsets
  uint32_t* w = sc.get<uint32_t>(p->nslices + 1);
  if (!w) return fail(p, POVAR_ENOMEM, "sell scratch");
  POVAR_CUDA(cudaMemsetAsync(w, 0, (p->nslices + 1) * sizeof(uint32_t), p->stream));
  k_slice_width<<<grid_for(p->nslices, 256), 256, 0, p->stream>>>(p->slot_len, p->nslices, w);
  ++p->launches;
  if ((s = scan_exclusive(p, sc, w, p->nslices + 1)) != POVAR_OK) return s;
  POVAR_CUDA(cudaMemcpyAsync(p->sell_off, w, (p->nslices + 1) * sizeof(uint32_t),
                             cudaMemcpyDeviceToDevice, p->stream));
  uint32_t nsell = 0;
  POVAR_CUDA(cudaMemcpyAsync(&nsell, w + p->nslices, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  p->nsell = nsell;
  if ((s = dev_alloc(p, &p->sell_cam, std::max<int64_t>(nsell, 1), "sell_cam")) ||
      (s = dev_alloc(p, &p->sell_m32, std::max<int64_t>(nsell, 1), "sell_m32")) ||
      (s = dev_alloc(p, &p->sell_m64, std::max<int64_t>(nsell, 1), "sell_m64")) ||
      (s = dev_alloc(p, &p->sell_mdf, std::max<int64_t>(nsell, 1), "sell_mdf")))
    return s;
  POVAR_CUDA(cudaMemsetAsync(p->sell_cam, 0xff, nsell * sizeof(int32_t), p->stream));
  POVAR_CUDA(cudaMemsetAsync(p->sell_m32, 0, nsell * sizeof(float2), p->stream));
  POVAR_CUDA(cudaMemsetAsync(p->sell_m64, 0, nsell * sizeof(double2), p->stream));
  k_fill_sell<<<grid_for(p->np_pad, 256), 256, 0, p->stream>>>(
      p->slot_pt, p->slot_len, p->sell_off, p->off_pt, perm_ptcam, p->d_cam, p->d_meas,
      p->np_pad, p->sell_cam, p->sell_m32, p->sell_m64);
  k_fill_cm<<<gb, 256, 0, p->stream>>>(p->perm_cam, p->d_pt, p->pt_slot, p->d_meas, n,
                                       p->cm_slot, p->cm_m32, p->cm_m64);
  k_split_meas<<<grid_for((int64_t)nsell, 256), 256, 0, p->stream>>>(p->sell_m64, nsell,
                                                                    p->sell_mdf);
  p->launches += 3;
  if ((s = check_launch(p, "fill layouts")) != POVAR_OK) return s;

  // ---- camera-major chunks (host: n_cams entries)
  std::vector<uint32_t> h_offc(p->nc + 1);
  POVAR_CUDA(cudaMemcpyAsync(h_offc.data(), p->off_cam, (p->nc + 1) * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  std::vector<uint32_t> cb;
  std::vector<int32_t> ccam, cn(p->nc), c0(p->nc);
  int active = 0;
  for (int c = 0; c < p->nc; ++c) {
    const uint32_t b = h_offc[c], e = h_offc[c + 1];
    c0[c] = (int32_t)ccam.size();
    cn[c] = (int32_t)((e - b + CHUNK - 1) / CHUNK);
    if (e > b) ++active;
    for (uint32_t q = b; q < e; q += CHUNK) {
      cb.push_back(q);
      ccam.push_back(c);
    }
  }
  cb.push_back((uint32_t)n);
  p->nchunks = (int32_t)ccam.size();
  p->nc_active = active;
  if ((s = dev_alloc(p, &p->chunk_beg, cb.size(), "chunk_beg")) ||
      (s = dev_alloc(p, &p->chunk_cam, std::max<size_t>(ccam.size(), 1), "chunk_cam")))
    return s;
  POVAR_COPY(p->chunk_beg, cb.data(), cb.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->chunk_cam, ccam.data(), ccam.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->cam_nchunk, cn.data(), p->nc, cudaMemcpyHostToDevice);
  POVAR_COPY(p->cam_chunk0, c0.data(), p->nc, cudaMemcpyHostToDevice);
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  return build_runs(p);
}

// Run structure of the fused series schedule. For each slice s and track
// position t (a "slice row", index sell_off[s] / 32 + t) the cameras of the
// 32 lanes are known at creation time. A row is "uniform" when every valid
// lane has the same camera (one partial sum, reduced over the whole warp);
// otherwise it is split into runs of consecutive lanes with equal camera
// (one partial per run with a valid camera). row_mask = 0 marks a uniform
// row; otherwise bit l is set when lane l starts a run (bit 0 always set).
// row_base is the index of the row's first partial. The partials of camera
// i are listed, in increasing index, at cam_part_idx[cam_part_off[i] ..).
// The same pass lists, per camera, the slice rows that contain it (camera-row
// schedule), and the grouped schedule's tables follow from the runs (one
// slice per group). Everything is built on the device: per-row counts (one
// warp per row), exclusive scans, per-row fills, and stable radix sorts by
// camera for the per-camera lists.
povar_status build_runs(Problem* p) {
  povar_status s;
  Scratch sc(p->stream);
  const int64_t nrows = p->nsell / SLICE;
  const unsigned gw = grid_for(nrows * SLICE, 256);   // one warp per row
  const unsigned gr = grid_for(nrows, 256);
  int32_t* rcam = sc.get<int32_t>(nrows);
  uint32_t* nvis = sc.get<uint32_t>(nrows + 1);
  uint32_t* row_slice = sc.get<uint32_t>(nrows);
  if (!rcam || !nvis || !row_slice) return fail(p, POVAR_ENOMEM, "run scratch");
  if ((s = dev_alloc(p, &p->row_mask, std::max<int64_t>(nrows, 1), "row_mask")) ||
      (s = dev_alloc(p, &p->row_base, nrows + 1, "row_base")))
    return s;
  POVAR_CUDA(cudaMemsetAsync(p->row_base, 0, (nrows + 1) * sizeof(uint32_t), p->stream));
  POVAR_CUDA(cudaMemsetAsync(nvis, 0, (nrows + 1) * sizeof(uint32_t), p->stream));
  k_row_runs<<<gw, 256, 0, p->stream>>>(p->sell_cam, nrows, p->row_mask, rcam, p->row_base,
                                        nvis);
  ++p->launches;
  if ((s = check_launch(p, "row runs")) != POVAR_OK) return s;
  // counts -> offsets; the last entries hold the totals
  if ((s = scan_exclusive(p, sc, p->row_base, nrows + 1)) != POVAR_OK) return s;
  if ((s = scan_exclusive(p, sc, nvis, nrows + 1)) != POVAR_OK) return s;
  uint32_t npart = 0, nvisit = 0;
  POVAR_COPY(&npart, p->row_base + nrows, 1, cudaMemcpyDeviceToHost);
  POVAR_COPY(&nvisit, nvis + nrows, 1, cudaMemcpyDeviceToHost);
  if (npart == 0 || nvisit == 0) return fail(p, POVAR_EINVAL, "no observation in the layout");
  uint32_t* pcam = sc.get<uint32_t>(npart);
  uint32_t* pval = sc.get<uint32_t>(npart);
  uint32_t* vcam = sc.get<uint32_t>(nvisit);
  uint32_t* vrow = sc.get<uint32_t>(nvisit);
  uint32_t* vval = sc.get<uint32_t>(nvisit);
  if (!pcam || !pval || !vcam || !vrow || !vval) return fail(p, POVAR_ENOMEM, "run scratch");
  k_row_fill<<<gw, 256, 0, p->stream>>>(p->sell_cam, nrows, p->row_mask, rcam, p->row_base, nvis,
                                        pcam, vcam, vrow);
  k_row_slice<<<grid_for(p->nslices, 256), 256, 0, p->stream>>>(p->sell_off, p->nslices,
                                                                row_slice);
  k_iota<<<grid_for(npart, 256), 256, 0, p->stream>>>(pval, npart);
  k_iota<<<grid_for(nvisit, 256), 256, 0, p->stream>>>(vval, nvisit);
  p->launches += 4;
  if ((s = check_launch(p, "row fill")) != POVAR_OK) return s;
  const int cbits = bits_for((uint64_t)(p->nc - 1));

  // partials of each camera in index order
  p->nrows = nrows;
  p->npart = npart;
  if ((s = dev_alloc(p, &p->cam_part_off, (size_t)p->nc + 1, "cam_part_off")) ||
      (s = dev_alloc(p, &p->cam_part_idx, npart, "cam_part_idx")) ||
      (s = dev_alloc_bytes(p, &p->part_run, (size_t)npart * 12 * sizeof(double), "part_run")))
    return s;
  {
    uint32_t *kk = pcam, *vv = pval;
    if ((s = radix_sort(p, sc, &kk, &vv, npart, cbits)) != POVAR_OK) return s;
    POVAR_CUDA(cudaMemcpyAsync(p->cam_part_idx, vv, (size_t)npart * sizeof(uint32_t),
                               cudaMemcpyDeviceToDevice, p->stream));
    k_offsets<<<grid_for(npart, 256), 256, 0, p->stream>>>(kk, npart, p->nc, p->cam_part_off);
    ++p->launches;
  }
  std::vector<uint32_t> poff((size_t)p->nc + 1);
  POVAR_COPY(poff.data(), p->cam_part_off, poff.size(), cudaMemcpyDeviceToHost);
  p->nc_parts = 0;
  for (int c = 0; c < p->nc; ++c) p->nc_parts += poff[c + 1] > poff[c] ? 1 : 0;

  // camera-row lists: every distinct valid camera of every slice row, per
  // camera in row order
  p->nvisits = nvisit;
  if ((s = dev_alloc(p, &p->cam_row_off, (size_t)p->nc + 1, "cam_row_off")) ||
      (s = dev_alloc(p, &p->cam_row_pos0, nvisit, "cam_row_pos0")) ||
      (s = dev_alloc(p, &p->cam_row_slot0, nvisit, "cam_row_slot0")))
    return s;
  {
    uint32_t *kk = vcam, *vv = vval;
    if ((s = radix_sort(p, sc, &kk, &vv, nvisit, cbits)) != POVAR_OK) return s;
    k_visit_fill<<<grid_for(nvisit, 256), 256, 0, p->stream>>>(vv, vrow, row_slice, nvisit,
                                                               p->cam_row_pos0,
                                                               p->cam_row_slot0);
    k_offsets<<<grid_for(nvisit, 256), 256, 0, p->stream>>>(kk, nvisit, p->nc, p->cam_row_off);
    p->launches += 2;
  }

  // grouped schedule (one slice per group): the fused runs in the group
  // layout; its partial lists are the fused ones
  p->ngrows = nrows;
  p->npart3 = npart;
  if ((s = dev_alloc(p, &p->grp_slice0, (size_t)p->ngroups + 1, "grp_slice0")) ||
      (s = dev_alloc(p, &p->grp_row0, (size_t)p->ngroups + 1, "grp_row0")) ||
      (s = dev_alloc(p, &p->grow_cam, std::max<int64_t>(nrows, 1), "grow_cam")) ||
      (s = dev_alloc(p, &p->grow_base, std::max<int64_t>(nrows, 1), "grow_base")) ||
      (s = dev_alloc(p, &p->srow_mask, std::max<int64_t>(nrows, 1), "srow_mask")) ||
      (s = dev_alloc(p, &p->srow_base, std::max<int64_t>(nrows, 1), "srow_base")))
    return s;
  k_group_tables<<<gr, 256, 0, p->stream>>>(nrows, p->row_mask, rcam, p->row_base, p->grow_cam,
                                            p->grow_base, p->srow_mask, p->srow_base);
  k_group_rows<<<grid_for((int64_t)p->ngroups + 1, 256), 256, 0, p->stream>>>(
      p->sell_off, p->ngroups, p->grp_slice0, p->grp_row0);
  p->launches += 2;
  p->cam_part3_off = p->cam_part_off;
  p->cam_part3_idx = p->cam_part_idx;
  p->part3 = p->part_run;   // schedules 1 and 3 never run at the same time
  if ((s = check_launch(p, "run tables")) != POVAR_OK) return s;
  return build_groups5(p, rcam);
}

// Tables of the group schedule (5), built on the host from the row tables
// (O(rows + partials) work). A slice joins a group when every row of it is
// warp-uniform and its row cameras agree with the group's at every row index
// both have; slices arrive widest first, so a group's first slice fixes its
// row count and the slices that reach row k are a prefix of the group.
povar_status build_groups5(Problem* p, const int32_t* d_rcam) {
  const int64_t nrows = p->nrows;
  const int nsl = p->nslices;
  std::vector<uint32_t> off((size_t)nsl + 1), rbase((size_t)nrows + 1), poff((size_t)p->nc + 1),
      pidx((size_t)p->npart);
  std::vector<int32_t> rcam((size_t)nrows);
  POVAR_COPY(off.data(), p->sell_off, off.size(), cudaMemcpyDeviceToHost);
  POVAR_COPY(rcam.data(), d_rcam, rcam.size(), cudaMemcpyDeviceToHost);
  POVAR_COPY(rbase.data(), p->row_base, rbase.size(), cudaMemcpyDeviceToHost);
  POVAR_COPY(poff.data(), p->cam_part_off, poff.size(), cudaMemcpyDeviceToHost);
  POVAR_COPY(pidx.data(), p->cam_part_idx, pidx.size(), cudaMemcpyDeviceToHost);
  // groups as fixed-capacity records (no allocation per group); open[c] is
  // the group last opened for first-row camera c
  struct Grp {
    uint32_t ns = 0, nr = 0, rows = 0;   // slices, rows, staged measurement rows
    uint32_t sl[G5_SLICES];
    int32_t cam[G5_ROWS];
  };
  std::vector<Grp> groups;
  groups.reserve((size_t)nsl / 4 + 16);
  std::vector<uint32_t> rest;
  std::vector<int> open((size_t)p->nc, -1);
  for (int sidx = 0; sidx < nsl; ++sidx) {
    const uint32_t r0 = off[sidx] / SLICE, w = (off[sidx + 1] - off[sidx]) / SLICE;
    bool uni = w > 0 && w <= (uint32_t)G5_ROWS && w <= (uint32_t)G5_MROWS;
    for (uint32_t k = 0; uni && k < w; ++k) uni = rcam[r0 + k] >= 0;
    if (!uni) {
      rest.push_back((uint32_t)sidx);
      continue;
    }
    const int32_t key = rcam[r0];
    int gi = open[(size_t)key];
    if (gi >= 0) {
      const Grp& g = groups[(size_t)gi];
      bool ok = g.ns < (uint32_t)G5_SLICES && g.rows + w <= (uint32_t)G5_MROWS;
      const uint32_t kk = std::min<uint32_t>(w, g.nr);
      for (uint32_t k = 0; ok && k < kk; ++k) ok = g.cam[k] == rcam[r0 + k];
      if (!ok) gi = -1;
    }
    if (gi < 0) {
      gi = (int)groups.size();
      groups.emplace_back();
      open[(size_t)key] = gi;
    }
    Grp& g = groups[(size_t)gi];
    g.sl[g.ns++] = (uint32_t)sidx;
    g.rows += w;
    for (uint32_t k = g.nr; k < w; ++k) g.cam[g.nr++] = rcam[r0 + k];
  }
  // flat tables; items: for row k the slices that reach it (a prefix of the
  // group, widest first) in ranges of at most G5_ITEM slices
  const size_t ngr = groups.size();
  size_t nrow_tot = 0, nitem_tot = 0;
  for (const Grp& g : groups) {
    nrow_tot += g.nr;
    nitem_tot += (size_t)g.nr * ((g.ns + G5_ITEM - 1) / G5_ITEM);
  }
  std::vector<uint32_t> goff, gsl, roff, ioff, items, sinfo;
  std::vector<int32_t> rowcam, ghdr, item_cam;
  goff.reserve(ngr + 1);
  roff.reserve(ngr + 1);
  ioff.reserve(ngr + 1);
  ghdr.reserve(2 * ngr);
  gsl.reserve((size_t)nsl);
  sinfo.reserve(4 * (size_t)G5_SLICES * ngr);
  rowcam.reserve(nrow_tot);
  items.reserve(nitem_tot);
  item_cam.reserve(nitem_tot);
  goff.push_back(0);
  roff.push_back(0);
  ioff.push_back(0);
  std::vector<char> grouped_part((size_t)p->npart, 0);
  int64_t g_obs_rows = 0;
  for (const Grp& g : groups) {
    uint32_t width[G5_SLICES];
    uint32_t mrow = 0;
    const size_t sbase = sinfo.size();
    for (uint32_t j = 0; j < g.ns; ++j) {
      const uint32_t sidx = g.sl[j];
      gsl.push_back(sidx);
      const uint32_t w = (off[sidx + 1] - off[sidx]) / SLICE;
      width[j] = w;
      sinfo.insert(sinfo.end(), {sidx, off[sidx], w, mrow});
      mrow += w;
      const uint32_t r0 = off[sidx] / SLICE;
      for (uint32_t k = 0; k < w; ++k) grouped_part[rbase[r0 + k]] = 1;   // uniform: one partial
      g_obs_rows += w;
    }
    sinfo.resize(sbase + 4 * (size_t)G5_SLICES, 0u);   // G5_SLICES entries per group
    goff.push_back((uint32_t)gsl.size());
    bool consecutive = g.nr > 0;
    for (uint32_t k = 1; consecutive && k < g.nr; ++k)
      consecutive = g.cam[k] == g.cam[0] + (int32_t)k;
    ghdr.push_back((int32_t)mrow);
    ghdr.push_back(consecutive ? g.cam[0] : -1);
    rowcam.insert(rowcam.end(), g.cam, g.cam + g.nr);
    roff.push_back((uint32_t)rowcam.size());
    // row k is reached by the slices of width > k: a prefix, as the widths
    // do not increase within a group
    uint32_t n = g.ns;
    for (uint32_t k = 0; k < g.nr; ++k) {
      while (n > 0 && width[n - 1] <= k) --n;
      for (uint32_t j0 = 0; j0 < n; j0 += G5_ITEM) {
        const uint32_t j1 = std::min<uint32_t>(n, j0 + G5_ITEM);
        items.push_back((k << 16) | (j0 << 8) | j1);
        item_cam.push_back(g.cam[k]);
      }
    }
    ioff.push_back((uint32_t)items.size());
  }
  const int64_t nitems = (int64_t)items.size();
  // per camera: its items in item order, then its remaining run partials
  // (a counting sort by camera). An item's partial is written at its list
  // position (idest), so a list entry of an item indexes itself; run
  // partials follow all lists.
  std::vector<uint32_t> c5off((size_t)p->nc + 1, 0), c5nd((size_t)p->nc, 0),
      idest((size_t)nitems);
  for (int64_t q = 0; q < nitems; ++q) ++c5nd[(size_t)item_cam[(size_t)q]];
  int64_t nlist = nitems;
  for (int c = 0; c < p->nc; ++c) {
    uint32_t nrun = 0;
    for (uint32_t e = poff[c]; e < poff[c + 1]; ++e) nrun += grouped_part[pidx[e]] ? 0 : 1;
    nlist += nrun;
    c5off[(size_t)c + 1] = c5off[(size_t)c] + c5nd[(size_t)c] + nrun;
  }
  if (nlist + p->npart >= ((int64_t)1 << 32))
    return fail(p, POVAR_EINVAL, "group schedule: partial list size");
  std::vector<uint32_t> c5idx((size_t)nlist), cursor(c5off.begin(), c5off.end() - 1);
  for (int64_t q = 0; q < nitems; ++q) {
    const uint32_t d = cursor[(size_t)item_cam[(size_t)q]]++;
    idest[(size_t)q] = d;
    c5idx[d] = d;
  }
  for (int c = 0; c < p->nc; ++c) {
    uint32_t d = cursor[(size_t)c];
    for (uint32_t e = poff[c]; e < poff[c + 1]; ++e)
      if (!grouped_part[pidx[e]]) c5idx[d++] = (uint32_t)nlist + pidx[e];
  }
  p->g5_ngroups = (int32_t)groups.size();
  p->g5_nrest = (int32_t)rest.size();
  p->g5_nitems = nitems;
  p->g5_nlist = nlist;
  p->g5_nslices = (int64_t)gsl.size();
  p->g5_obs = g_obs_rows;
  povar_status s;
  auto up32 = [&](uint32_t** dst, const std::vector<uint32_t>& v, const char* what) {
    povar_status r = dev_alloc(p, dst, std::max<size_t>(v.size(), 1), what);
    if (r != POVAR_OK || v.empty()) return r;
    return copy_sync(p, *dst, v.data(), v.size(), cudaMemcpyHostToDevice);
  };
  if ((s = up32(&p->g5_off, goff, "g5_off")) || (s = up32(&p->g5_slices, gsl, "g5_slices")) ||
      (s = up32(&p->g5_roff, roff, "g5_roff")) || (s = up32(&p->g5_ioff, ioff, "g5_ioff")) ||
      (s = up32(&p->g5_items, items, "g5_items")) || (s = up32(&p->g5_rest, rest, "g5_rest")) ||
      (s = up32(&p->cam5_off, c5off, "cam5_off")) || (s = up32(&p->cam5_idx, c5idx, "cam5_idx")) ||
      (s = up32(&p->g5_sinfo, sinfo, "g5_sinfo")) ||
      (s = up32(&p->g5_idest, idest, "g5_idest")) ||
      (s = up32(&p->cam5_ndirect, c5nd, "cam5_ndirect")))
    return s;
  if ((s = dev_alloc(p, &p->g5_ghdr, std::max<size_t>(ghdr.size(), 2), "g5_ghdr"))) return s;
  if (!ghdr.empty()) POVAR_COPY(p->g5_ghdr, ghdr.data(), ghdr.size(), cudaMemcpyHostToDevice);
  if ((s = dev_alloc(p, &p->g5_rowcam, std::max<size_t>(rowcam.size(), 1), "g5_rowcam")))
    return s;
  if (!rowcam.empty())
    POVAR_COPY(p->g5_rowcam, rowcam.data(), rowcam.size(), cudaMemcpyHostToDevice);
  if ((s = dev_alloc_bytes(p, &p->part5,
                           (size_t)(nlist + (int64_t)p->npart) * 12 * sizeof(double), "part5")))
    return s;
  return setup_group_kernels(p);
}

}  // namespace povar
