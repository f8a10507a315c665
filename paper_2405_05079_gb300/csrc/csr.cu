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
                            int np, int32_t* __restrict__ sell_cam,
                            float2* __restrict__ m32, double2* __restrict__ m64) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= np) return;
  const uint32_t j = slot_pt[s];
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

// Scratch buffer list freed at the end of build_orders.
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* q : ptrs) cudaFree(q);
  }
  template <class T>
  T* get(size_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
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

povar_status build_orders(Problem* p, const int32_t* h_cam, const int32_t* h_pt) {
  (void)h_pt;
  Scratch sc;
  const int64_t n = p->nobs;
  const unsigned gb = grid_for(n, 256);
  povar_status s;

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
  std::vector<uint32_t> h_off(p->np + 1);
  POVAR_CUDA(cudaMemcpyAsync(h_off.data(), p->off_pt, (p->np + 1) * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, p->stream));
  POVAR_CUDA(cudaStreamSynchronize(p->stream));
  uint32_t maxlen = 0;
  for (int j = 0; j < p->np; ++j) {
    const uint32_t l = h_off[j + 1] - h_off[j];
    if (l == 0) return fail(p, POVAR_EINVAL, "landmark without observations");
    maxlen = std::max(maxlen, l);
  }
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
    // Full slices of the sorted order are grouped: up to GROUP consecutive
    // slices whose first landmarks share the smallest camera (their rows
    // then tend to see the same camera, row by row). Groups are ordered by
    // width (longest track first, stable) so that the warps of a block get
    // similar work; the last partial slice and the pads stay at the end,
    // one group each.
    std::vector<uint32_t> order(p->np), h_len(p->np), h_min(p->np);
    POVAR_COPY(order.data(), vv, p->np, cudaMemcpyDeviceToHost);
    POVAR_COPY(h_len.data(), len, p->np, cudaMemcpyDeviceToHost);
    POVAR_COPY(h_min.data(), mincam, p->np, cudaMemcpyDeviceToHost);
    const int nfull = p->np / SLICE;
    std::vector<uint32_t> width(nfull, 0);
    for (int sl = 0; sl < nfull; ++sl)
      for (int l = 0; l < SLICE; ++l) width[sl] = std::max(width[sl], h_len[order[sl * SLICE + l]]);
    std::vector<std::pair<int, int>> groups;  // [first, last) sorted slices
    for (int sl = 0; sl < nfull;) {
      int e = sl + 1;
      while (e < nfull && e - sl < GROUP && h_min[order[e * SLICE]] == h_min[order[sl * SLICE]]) ++e;
      groups.emplace_back(sl, e);
      sl = e;
    }
    std::vector<uint32_t> gwidth(groups.size(), 0);
    for (size_t g = 0; g < groups.size(); ++g)
      for (int sl = groups[g].first; sl < groups[g].second; ++sl)
        gwidth[g] = std::max(gwidth[g], width[sl]);
    std::vector<int> g_order(groups.size());
    for (size_t g = 0; g < groups.size(); ++g) g_order[g] = (int)g;
    std::stable_sort(g_order.begin(), g_order.end(),
                     [&](int x, int y) { return gwidth[x] > gwidth[y]; });
    std::vector<int> sl_order;
    sl_order.reserve(nfull);
    p->h_grp_slice0.assign(1, 0u);
    for (int g : g_order) {
      for (int sl = groups[g].first; sl < groups[g].second; ++sl) sl_order.push_back(sl);
      p->h_grp_slice0.push_back((uint32_t)sl_order.size());
    }
    for (int sl = nfull; sl < p->nslices; ++sl) p->h_grp_slice0.push_back((uint32_t)sl + 1);
    p->ngroups = (int32_t)p->h_grp_slice0.size() - 1;
    std::vector<uint32_t> slot_pt(p->np_pad, 0xffffffffu), slot_len(p->np_pad, 0),
        pt_slot(p->np);
    for (int sl = 0; sl < nfull; ++sl)
      for (int l = 0; l < SLICE; ++l) slot_pt[sl * SLICE + l] = order[sl_order[sl] * SLICE + l];
    for (int q = nfull * SLICE; q < p->np; ++q) slot_pt[q] = order[q];
    for (int q = 0; q < p->np; ++q) {
      slot_len[q] = h_len[slot_pt[q]];
      pt_slot[slot_pt[q]] = (uint32_t)q;
    }
    POVAR_COPY(p->slot_pt, slot_pt.data(), p->np_pad, cudaMemcpyHostToDevice);
    POVAR_COPY(p->slot_len, slot_len.data(), p->np_pad, cudaMemcpyHostToDevice);
    POVAR_COPY(p->pt_slot, pt_slot.data(), (size_t)p->np, cudaMemcpyHostToDevice);
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
  k_fill_sell<<<gp, 256, 0, p->stream>>>(p->slot_pt, p->slot_len, p->sell_off, p->off_pt,
                                         perm_ptcam, p->d_cam, p->d_meas, p->np, p->sell_cam,
                                         p->sell_m32, p->sell_m64);
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
povar_status build_group_runs(Problem* p, const std::vector<int32_t>& cam,
                              const std::vector<uint32_t>& off);

povar_status build_runs(Problem* p) {
  povar_status s;
  const int64_t nrows = p->nsell / SLICE;
  std::vector<int32_t> cam(p->nsell);
  std::vector<uint32_t> off(p->nslices + 1);
  POVAR_COPY(cam.data(), p->sell_cam, p->nsell, cudaMemcpyDeviceToHost);
  POVAR_COPY(off.data(), p->sell_off, (p->nslices + 1), cudaMemcpyDeviceToHost);
  std::vector<uint32_t> mask(std::max<int64_t>(nrows, 1)), base(std::max<int64_t>(nrows, 1));
  std::vector<int32_t> pcam;
  pcam.reserve(nrows + nrows / 4);
  for (int64_t row = 0; row < nrows; ++row) {
    const int32_t* c = cam.data() + row * SLICE;
    int32_t c0 = -1;
    bool uniform = true;
    for (int l = 0; l < SLICE; ++l) {
      if (c[l] < 0) continue;
      if (c0 < 0) c0 = c[l];
      else if (c[l] != c0) uniform = false;
    }
    base[row] = (uint32_t)pcam.size();
    if (uniform && c0 >= 0) {
      mask[row] = 0;
      pcam.push_back(c0);
      continue;
    }
    uint32_t m = 0;
    for (int l = 0; l < SLICE; ++l) {
      if (l == 0 || c[l] != c[l - 1]) {
        m |= 1u << l;
        if (c[l] >= 0) pcam.push_back(c[l]);
      }
    }
    mask[row] = m;
  }
  // camera-row lists: every distinct valid camera of every slice row
  std::vector<uint32_t> voff(p->nc + 1, 0);
  std::vector<std::pair<uint32_t, uint32_t>> vis;  // (camera, row) in row order
  {
    std::vector<uint32_t> row_slice(std::max<int64_t>(nrows, 1), 0);
    for (int sl = 0; sl < p->nslices; ++sl)
      for (uint32_t r = off[sl] / SLICE; r < off[sl + 1] / SLICE; ++r) row_slice[r] = sl;
    vis.reserve(nrows + nrows / 4);
    int32_t seen[SLICE];
    for (int64_t row = 0; row < nrows; ++row) {
      const int32_t* c = cam.data() + row * SLICE;
      int nseen = 0;
      for (int l = 0; l < SLICE; ++l) {
        if (c[l] < 0) continue;
        bool dup = false;
        for (int q = 0; q < nseen; ++q) dup |= seen[q] == c[l];
        if (!dup) {
          seen[nseen++] = c[l];
          vis.emplace_back((uint32_t)c[l], (uint32_t)row);
        }
      }
    }
    for (const auto& v : vis) ++voff[v.first + 1];
    for (int c = 0; c < p->nc; ++c) voff[c + 1] += voff[c];
    std::vector<uint32_t> cursor(voff.begin(), voff.end() - 1);
    std::vector<uint32_t> pos0(std::max<size_t>(vis.size(), 1)), slot0(std::max<size_t>(vis.size(), 1));
    for (const auto& v : vis) {
      const uint32_t q = cursor[v.first]++;
      pos0[q] = v.second * SLICE;
      slot0[q] = row_slice[v.second] * SLICE;
    }
    p->nvisits = (int64_t)vis.size();
    if ((s = dev_alloc(p, &p->cam_row_off, voff.size(), "cam_row_off")) ||
        (s = dev_alloc(p, &p->cam_row_pos0, pos0.size(), "cam_row_pos0")) ||
        (s = dev_alloc(p, &p->cam_row_slot0, slot0.size(), "cam_row_slot0")))
      return s;
    POVAR_COPY(p->cam_row_off, voff.data(), voff.size(), cudaMemcpyHostToDevice);
    POVAR_COPY(p->cam_row_pos0, pos0.data(), pos0.size(), cudaMemcpyHostToDevice);
    POVAR_COPY(p->cam_row_slot0, slot0.data(), slot0.size(), cudaMemcpyHostToDevice);
  }
  const int64_t npart = (int64_t)pcam.size();
  std::vector<uint32_t> poff(p->nc + 1, 0), pidx(std::max<int64_t>(npart, 1));
  for (int32_t c : pcam) ++poff[c + 1];
  for (int c = 0; c < p->nc; ++c) poff[c + 1] += poff[c];
  {
    std::vector<uint32_t> cursor(poff.begin(), poff.end() - 1);
    for (int64_t q = 0; q < npart; ++q) pidx[cursor[pcam[q]]++] = (uint32_t)q;
  }
  p->nrows = nrows;
  p->npart = npart;
  p->nc_parts = 0;
  for (int c = 0; c < p->nc; ++c) p->nc_parts += poff[c + 1] > poff[c] ? 1 : 0;
  if ((s = dev_alloc(p, &p->row_mask, mask.size(), "row_mask")) ||
      (s = dev_alloc(p, &p->row_base, base.size(), "row_base")) ||
      (s = dev_alloc(p, &p->cam_part_off, poff.size(), "cam_part_off")) ||
      (s = dev_alloc(p, &p->cam_part_idx, pidx.size(), "cam_part_idx")) ||
      (s = dev_alloc_bytes(p, &p->part_run, std::max<int64_t>(npart, 1) * 12 * sizeof(double),
                           "part_run")))
    return s;
  POVAR_COPY(p->row_mask, mask.data(), mask.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->row_base, base.data(), base.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->cam_part_off, poff.data(), poff.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->cam_part_idx, pidx.data(), pidx.size(), cudaMemcpyHostToDevice);
  return build_group_runs(p, cam, off);
}

// Run structure of the grouped schedule. Group g holds the slices
// h_grp_slice0[g] .. h_grp_slice0[g+1]-1; its rows t = 0 .. (widest slice)-1
// are numbered from grp_row0[g]. A group row whose valid lanes (over all of
// the group's slices that reach row t) all see one camera is "uniform": one
// partial, at grow_base, camera in grow_cam. For any other group row,
// grow_cam = -1 and every slice row in it gets the run description of the
// fused schedule (srow_mask, srow_base) in the grouped partial space. The
// partials of camera i are listed at cam_part3_idx[cam_part3_off[i] ..).
povar_status build_group_runs(Problem* p, const std::vector<int32_t>& cam,
                              const std::vector<uint32_t>& off) {
  povar_status s;
  const int ng = p->ngroups;
  const int64_t nrows = p->nsell / SLICE;
  std::vector<uint32_t> grow0(ng + 1, 0), gbase, smask(std::max<int64_t>(nrows, 1), 0),
      sbase(std::max<int64_t>(nrows, 1), 0);
  std::vector<int32_t> gcam, pcam;
  for (int g = 0; g < ng; ++g) {
    const uint32_t s0 = p->h_grp_slice0[g], s1 = p->h_grp_slice0[g + 1];
    uint32_t W = 0;
    for (uint32_t sl = s0; sl < s1; ++sl) W = std::max(W, (off[sl + 1] - off[sl]) / SLICE);
    grow0[g] = (uint32_t)gcam.size();
    for (uint32_t t = 0; t < W; ++t) {
      int32_t c0 = -1;
      bool uniform = true;
      for (uint32_t sl = s0; sl < s1; ++sl) {
        if (t >= (off[sl + 1] - off[sl]) / SLICE) continue;
        const int32_t* c = cam.data() + (size_t)off[sl] + (size_t)t * SLICE;
        for (int l = 0; l < SLICE; ++l) {
          if (c[l] < 0) continue;
          if (c0 < 0) c0 = c[l];
          else if (c[l] != c0) uniform = false;
        }
      }
      if (uniform && c0 >= 0) {
        gcam.push_back(c0);
        gbase.push_back((uint32_t)pcam.size());
        pcam.push_back(c0);
        continue;
      }
      gcam.push_back(-1);
      gbase.push_back(0);
      for (uint32_t sl = s0; sl < s1; ++sl) {
        if (t >= (off[sl + 1] - off[sl]) / SLICE) continue;
        const int64_t row = off[sl] / SLICE + t;
        const int32_t* c = cam.data() + row * SLICE;
        int32_t r0 = -1;
        bool ru = true;
        for (int l = 0; l < SLICE; ++l) {
          if (c[l] < 0) continue;
          if (r0 < 0) r0 = c[l];
          else if (c[l] != r0) ru = false;
        }
        sbase[row] = (uint32_t)pcam.size();
        if (ru && r0 >= 0) {
          smask[row] = 0;
          pcam.push_back(r0);
          continue;
        }
        uint32_t m = 0;
        for (int l = 0; l < SLICE; ++l) {
          if (l == 0 || c[l] != c[l - 1]) {
            m |= 1u << l;
            if (c[l] >= 0) pcam.push_back(c[l]);
          }
        }
        smask[row] = m;
      }
    }
  }
  grow0[ng] = (uint32_t)gcam.size();
  const int64_t npart = (int64_t)pcam.size();
  std::vector<uint32_t> poff(p->nc + 1, 0), pidx(std::max<int64_t>(npart, 1));
  for (int32_t c : pcam) ++poff[c + 1];
  for (int c = 0; c < p->nc; ++c) poff[c + 1] += poff[c];
  {
    std::vector<uint32_t> cursor(poff.begin(), poff.end() - 1);
    for (int64_t q = 0; q < npart; ++q) pidx[cursor[pcam[q]]++] = (uint32_t)q;
  }
  p->ngrows = (int64_t)gcam.size();
  p->npart3 = npart;
  if (gcam.empty()) {
    gcam.push_back(-1);
    gbase.push_back(0);
  }
  if ((s = dev_alloc(p, &p->grp_slice0, p->h_grp_slice0.size(), "grp_slice0")) ||
      (s = dev_alloc(p, &p->grp_row0, grow0.size(), "grp_row0")) ||
      (s = dev_alloc(p, &p->grow_cam, gcam.size(), "grow_cam")) ||
      (s = dev_alloc(p, &p->grow_base, gbase.size(), "grow_base")) ||
      (s = dev_alloc(p, &p->srow_mask, smask.size(), "srow_mask")) ||
      (s = dev_alloc(p, &p->srow_base, sbase.size(), "srow_base")) ||
      (s = dev_alloc(p, &p->cam_part3_off, poff.size(), "cam_part3_off")) ||
      (s = dev_alloc(p, &p->cam_part3_idx, pidx.size(), "cam_part3_idx")) ||
      (s = dev_alloc_bytes(p, &p->part3, std::max<int64_t>(npart, 1) * 12 * sizeof(double),
                           "part3")))
    return s;
  POVAR_COPY(p->grp_slice0, p->h_grp_slice0.data(), p->h_grp_slice0.size(),
             cudaMemcpyHostToDevice);
  POVAR_COPY(p->grp_row0, grow0.data(), grow0.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->grow_cam, gcam.data(), gcam.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->grow_base, gbase.data(), gbase.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->srow_mask, smask.data(), smask.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->srow_base, sbase.data(), sbase.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->cam_part3_off, poff.data(), poff.size(), cudaMemcpyHostToDevice);
  POVAR_COPY(p->cam_part3_idx, pidx.data(), pidx.size(), cudaMemcpyHostToDevice);
  return POVAR_OK;
}

}  // namespace povar
