// After the stack kernel: exact counts of the emitted cells, deterministic
// ordering, and the contributing detection ids (Sec. 2.1 step 3; Sec. 3.3).
#include "sas_count.cuh"

namespace sas {

namespace {

constexpr int kWarpsPerBlock = 8;

__device__ __forceinline__ bool key_less(const Key& p, const Key& q) {
  if (p.a != q.a) return p.a < q.a;
  if (p.b != q.b) return p.b < q.b;
  return p.c < q.c;
}

__device__ __forceinline__ Key max_key() {
  Key k;
  k.a = ~0ull;
  k.b = ~0ull;
  k.c = ~0u;
  k.pad = 0;
  return k;
}

// The detections of epoch e that fall in bin (bx, by) at lattice point (kx, ky):
// the bin's source window at epoch e is exactly one bin shifted by s[k][e], and
// the buckets covering that window are scanned with the exact membership test.
struct BinWindow {
  int32_t ox, oy;       // window origin (mpx)
  int cxa, cxb, cya, cyb;
};

__device__ __forceinline__ bool bin_window(const SearchGeom& g, const CoarseGeom& cg, uint32_t e,
                                           uint32_t kx, uint32_t ky, uint32_t bx, uint32_t by,
                                           const int32_t* sxt, const int32_t* syt, BinWindow& w) {
  w.ox = g.x_min + (int32_t)bx * g.bin + sxt[(size_t)kx * g.E + e];
  w.oy = g.y_min + (int32_t)by * g.bin + syt[(size_t)ky * g.E + e];
  w.cxa = max(floor_div32(w.ox - cg.gx0, cg.cell), 0);
  w.cxb = min(floor_div32(w.ox + g.bin - 1 - cg.gx0, cg.cell), cg.ncx - 1);
  w.cya = max(floor_div32(w.oy - cg.gy0, cg.cell), 0);
  w.cyb = min(floor_div32(w.oy + g.bin - 1 - cg.gy0, cg.cell), cg.ncy - 1);
  return w.cxa <= w.cxb && w.cya <= w.cyb;
}

// One warp per emitted super-bin (count_superbin); every bin that reaches
// the super-bin's threshold (n_low for a tile-local peak, else n_min) appends
// its key.
constexpr int kMaxS = 4;

template <bool W>
__global__ void k_cell_count(const Emit* __restrict__ emits, uint32_t n_emit, int sb, SearchGeom g,
                             CoarseGeom cg, uint64_t cell_m, uint64_t bin_m, const Det* __restrict__ dets,
                             const uint32_t* __restrict__ boff, const uint32_t* __restrict__ ecount,
                             const int32_t* __restrict__ sxt, const int32_t* __restrict__ syt,
                             uint32_t n_min, uint32_t n_low, Key* __restrict__ keys,
                             uint32_t* __restrict__ n_valid, unsigned long long* __restrict__ raw_total,
                             const uint8_t* __restrict__ wts) {
  const uint32_t w = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (w >= n_emit) return;  // whole warps leave together
  const Emit em = emits[w];
  const uint32_t thr = (em.flags & kEmitLowPeak) ? n_low : n_min;
  count_superbin<W>(em, sb, g, cg, cell_m, bin_m, dets, boff, ecount, sxt, syt, thr, lane,
                 [&](int, uint32_t bx, uint32_t by, uint32_t distinct, uint32_t raw) {
                   Key k;
                   k.a = ((uint64_t)(~distinct) << 32) | (uint64_t)(~raw);
                   k.b = ((uint64_t)em.v_idx << 32) | (uint64_t)by;
                   k.c = bx;
                   k.pad = 0;
                   keys[atomicAdd(n_valid, 1u)] = k;  // compacted; the sort fixes the order
                   atomicAdd(raw_total, (unsigned long long)raw);
                 },
                 wts);
}

__global__ void k_fill_max(Key* keys, uint32_t from, uint32_t to) {
  const uint32_t i = from + blockIdx.x * blockDim.x + threadIdx.x;
  if (i < to) keys[i] = max_key();
}

// ---- bitonic sort of keys (total order; ascending) --------------------------

constexpr int kSortChunk = 2048;
constexpr int kSortThreads = 1024;

__device__ __forceinline__ void cmp_swap(Key& p, Key& q, bool asc) {
  if (key_less(q, p) == asc) {
    const Key t = p;
    p = q;
    q = t;
  }
}

// The bitonic network sorts every aligned segment of `seg` keys ascending: the
// direction of stage k is the usual ((i & k) == 0) below k = seg, and ascending
// at k = seg (one segment = the whole array for a single sort).

// Stages k = 2..len inside each chunk of `len` keys (len <= kSortChunk).
__global__ void k_bitonic_local_sort(Key* keys, uint32_t len, uint32_t seg) {
  __shared__ Key s[kSortChunk];
  const uint32_t base = blockIdx.x * len;
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) s[i] = keys[base + i];
  __syncthreads();
  for (uint32_t k = 2; k <= len; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) cmp_swap(s[i], s[ixj], ((base + i) & k) == 0 || k >= seg);
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) keys[base + i] = s[i];
}

// Steps j < kSortChunk of stage k, one chunk per block.
__global__ void k_bitonic_local_merge(Key* keys, uint32_t k, uint32_t seg) {
  __shared__ Key s[kSortChunk];
  const uint32_t base = blockIdx.x * kSortChunk;
  for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) s[i] = keys[base + i];
  __syncthreads();
  for (uint32_t j = kSortChunk >> 1; j > 0; j >>= 1) {
    for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
      const uint32_t ixj = i ^ j;
      if (ixj > i) cmp_swap(s[i], s[ixj], ((base + i) & k) == 0 || k >= seg);
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < kSortChunk; i += blockDim.x) keys[base + i] = s[i];
}

// One step (k, j >= kSortChunk) over global memory.
__global__ void k_bitonic_global(Key* keys, uint32_t n_pad, uint32_t k, uint32_t j, uint32_t seg) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  const uint32_t ixj = i ^ j;
  if (ixj > i) {
    Key p = keys[i], q = keys[ixj];
    const bool asc = (i & k) == 0 || k >= seg;
    if (key_less(q, p) == asc) {
      keys[i] = q;
      keys[ixj] = p;
    }
  }
}

__global__ void k_key_raw(const Key* __restrict__ keys, uint32_t n, uint32_t* __restrict__ raw) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) raw[i] = ~(uint32_t)keys[i].a;
}

// One warp per candidate: collect the ids of every detection in the cell
// (unordered, through a per-warp cursor), then order them ascending by rank
// (ids are distinct, so the ranks are a permutation).
__global__ void k_gather_ids(const Key* __restrict__ keys, uint32_t n,
                             const unsigned long long* __restrict__ id_off, SearchGeom g,
                             CoarseGeom cg, const Det* __restrict__ dets,
                             const uint32_t* __restrict__ boff, const uint32_t* __restrict__ ecount,
                             const int32_t* __restrict__ sxt, const int32_t* __restrict__ syt,
                             uint32_t* __restrict__ ids_tmp, uint32_t* __restrict__ ids,
                             uint32_t* __restrict__ flags) {
  __shared__ uint32_t s_cursor[kWarpsPerBlock];
  const int wl = threadIdx.x >> 5;
  const uint32_t w = blockIdx.x * kWarpsPerBlock + wl;
  const int lane = threadIdx.x & 31;
  if (w >= n) return;
  const Key key = keys[w];
  const uint32_t v_idx = (uint32_t)(key.b >> 32), by = (uint32_t)key.b, bx = key.c;
  const uint32_t raw = ~(uint32_t)key.a;
  const uint32_t kx = v_idx % (uint32_t)g.nvx, ky = v_idx / (uint32_t)g.nvx;
  const unsigned long long off = id_off[w];
  if (lane == 0) s_cursor[wl] = 0;
  __syncwarp();
  for (uint32_t eb = 0; eb < g.E; eb += 32) {
    const uint32_t e = eb + lane;
    BinWindow bw;
    if (e < g.E && ecount[e] > 0 && bin_window(g, cg, e, kx, ky, bx, by, sxt, syt, bw)) {
      for (int cy = bw.cya; cy <= bw.cyb; ++cy) {
        const size_t b0 = ((size_t)e * cg.ncy + cy) * cg.ncx;
        const uint32_t k1 = boff[b0 + bw.cxb + 1];
        for (uint32_t k = boff[b0 + bw.cxa]; k < k1; ++k) {
          const Det d = dets[k];
          if (((uint32_t)(d.x - bw.ox) < (uint32_t)g.bin) &&
              ((uint32_t)(d.y - bw.oy) < (uint32_t)g.bin)) {
            const uint32_t p = atomicAdd(&s_cursor[wl], 1u);
            if (p < raw) ids_tmp[off + p] = d.id;
          }
        }
      }
    }
  }
  __syncwarp();
  const uint32_t got = s_cursor[wl];
  if (got != raw) {
    if (lane == 0) atomicOr(flags, kFlagInternal);
    return;
  }
  for (uint32_t i = lane; i < raw; i += 32) {
    const uint32_t v = ids_tmp[off + i];
    uint32_t r = 0;
    for (uint32_t j = 0; j < raw; ++j) r += ids_tmp[off + j] < v;
    ids[off + r] = v;
  }
}

__global__ void k_write_candidates(const Key* __restrict__ keys, uint32_t n,
                                   const unsigned long long* __restrict__ id_off,
                                   sas_candidate* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Key k = keys[i];
  sas_candidate c;
  c.v_idx = (uint32_t)(k.b >> 32);
  c.by = (uint32_t)k.b;
  c.bx = k.c;
  c.count = ~(uint32_t)(k.a >> 32);
  c.raw = ~(uint32_t)k.a;
  c.id_len = c.raw;
  c.id_off = id_off[i];
  out[i] = c;
}

unsigned blocks_for(uint64_t n, unsigned per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

cudaError_t launch_cell_count(const Emit* emits, uint32_t n_emit, int s_bins, const SearchGeom& g,
                              const CoarseGeom& cg, const Det* dets, const uint32_t* boff,
                              const uint32_t* ecount, const int32_t* sxt, const int32_t* syt,
                              uint32_t n_min, uint32_t n_low, Key* keys, uint32_t* n_valid,
                              unsigned long long* raw_total, const uint8_t* wts, cudaStream_t s) {
  if (n_emit == 0) return cudaSuccess;
  if (s_bins < 1 || s_bins > kMaxS) return cudaErrorInvalidValue;
  auto kern = wts ? k_cell_count<true> : k_cell_count<false>;
  kern<<<blocks_for(n_emit, kWarpsPerBlock), kWarpsPerBlock * 32, 0, s>>>(
      emits, n_emit, s_bins, g, cg, div_magic((uint32_t)cg.cell), div_magic((uint32_t)g.bin), dets, boff,
      ecount, sxt, syt, n_min, n_low, keys, n_valid, raw_total, wts);
  note_launch();
  return cudaGetLastError();
}

// Sorts keys[0..n_pad) ascending; keys[n..n_pad) are set to the maximum key first.
cudaError_t launch_sort_keys(Key* keys, uint32_t n, uint32_t n_pad, cudaStream_t s) {
  if (n_pad <= 1) return cudaSuccess;
  if (n_pad > n) {
    k_fill_max<<<blocks_for(n_pad - n, 256), 256, 0, s>>>(keys, n, n_pad);
    note_launch();
  }
  return launch_sort_segments(keys, n_pad, n_pad, s);
}

cudaError_t launch_sort_segments(Key* keys, uint32_t n_total, uint32_t seg, cudaStream_t s) {
  if (seg <= 1 || n_total == 0) return cudaSuccess;
  if (seg <= (uint32_t)kSortChunk) {
    k_bitonic_local_sort<<<n_total / seg, kSortThreads, 0, s>>>(keys, seg, seg);
    note_launch();
    return cudaGetLastError();
  }
  k_bitonic_local_sort<<<n_total / kSortChunk, kSortThreads, 0, s>>>(keys, kSortChunk, seg);
  note_launch();
  for (uint32_t k = 2 * kSortChunk; k <= seg; k <<= 1) {
    for (uint32_t j = k >> 1; j >= (uint32_t)kSortChunk; j >>= 1) {
      k_bitonic_global<<<blocks_for(n_total, 256), 256, 0, s>>>(keys, n_total, k, j, seg);
      note_launch();
    }
    k_bitonic_local_merge<<<n_total / kSortChunk, kSortThreads, 0, s>>>(keys, k, seg);
    note_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_key_raw(const Key* keys, uint32_t n, uint32_t* raw, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_key_raw<<<blocks_for(n, 256), 256, 0, s>>>(keys, n, raw);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_ids(const Key* keys, uint32_t n, const unsigned long long* id_off,
                              const SearchGeom& g, const CoarseGeom& cg, const Det* dets,
                              const uint32_t* boff, const uint32_t* ecount, const int32_t* sxt,
                              const int32_t* syt, uint32_t* ids_tmp, uint32_t* ids,
                              uint32_t* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_gather_ids<<<blocks_for(n, kWarpsPerBlock), kWarpsPerBlock * 32, 0, s>>>(
      keys, n, id_off, g, cg, dets, boff, ecount, sxt, syt, ids_tmp, ids, flags);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_write_candidates(const Key* keys, uint32_t n, const unsigned long long* id_off,
                                    sas_candidate* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_write_candidates<<<blocks_for(n, 256), 256, 0, s>>>(keys, n, id_off, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace sas
