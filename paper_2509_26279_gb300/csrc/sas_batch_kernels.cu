// Device side of the batched search: many fields in one pass of each kernel.
//
// Every kernel here covers all fields of a batch in one launch; a thread, warp
// or block finds its field from prefix offsets (binary search over n_fields + 1
// entries).  The arithmetic per field is the same as in sas_prep.cu,
// sas_stack.cu and sas_post.cu.
#include <climits>

#include "sas_batch.cuh"
#include "sas_count.cuh"

namespace sas {

namespace {

__device__ __forceinline__ int find_field(const unsigned long long* off, int n_fields,
                                          unsigned long long i) {
  int lo = 0, hi = n_fields;  // largest f with off[f] <= i
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ Key max_key_b() {
  Key k;
  k.a = ~0ull;
  k.b = ~0ull;
  k.c = ~0u;
  k.pad = 0;
  return k;
}

__device__ __forceinline__ bool key_less_b(const Key& p, const Key& q) {
  if (p.a != q.a) return p.a < q.a;
  if (p.b != q.b) return p.b < q.b;
  return p.c < q.c;
}

// Validation, per-epoch counts and per-bucket counts of every detection.
__global__ void k_batch_ingest(const BatchField* __restrict__ F, int n_fields,
                               const unsigned long long* __restrict__ det_off,
                               uint32_t* __restrict__ bucket_count, uint32_t* __restrict__ bucket_of) {
  const unsigned long long total = det_off[n_fields];
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int f = find_field(det_off, n_fields, i);
    const BatchField& bf = F[f];
    const unsigned long long k = i - det_off[f];
    const uint32_t e = bf.epoch[k];
    const int32_t xi = bf.x[k], yi = bf.y[k];
    uint32_t b = kInvalidBucket;
    if (e >= bf.E) {
      atomicOr(bf.counters + kCtrFlags, kFlagEpoch);
    } else {
      atomicAdd(&bf.ecount[e], 1u);
      if (xi <= -kLimPos || xi >= kLimPos || yi <= -kLimPos || yi >= kLimPos) {
        atomicOr(bf.counters + kCtrFlags, kFlagPos);
      } else {
        const CoarseGeom& cg = bf.args.cg;
        const int64_t cx = floor_div64((int64_t)xi - cg.gx0, cg.cell);
        const int64_t cy = floor_div64((int64_t)yi - cg.gy0, cg.cell);
        if (cx >= 0 && cx < cg.ncx && cy >= 0 && cy < cg.ncy) {
          b = (uint32_t)(bf.bucket_base +
                         ((uint64_t)e * cg.ncy + (uint64_t)cy) * cg.ncx + (uint64_t)cx);
          atomicAdd(&bucket_count[b], 1u);
        }
      }
    }
    bucket_of[i] = b;
  }
}

__global__ void k_batch_scatter(const BatchField* __restrict__ F, int n_fields,
                                const unsigned long long* __restrict__ det_off,
                                const uint32_t* __restrict__ bucket_of, uint32_t* __restrict__ cursor,
                                Det* __restrict__ dets) {
  const unsigned long long total = det_off[n_fields];
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t b = bucket_of[i];
    if (b == kInvalidBucket) continue;
    const int f = find_field(det_off, n_fields, i);
    const BatchField& bf = F[f];
    const unsigned long long k = i - det_off[f];
    Det d;
    d.x = bf.x[k];
    d.y = bf.y[k];
    d.e = bf.epoch[k];
    d.id = (uint32_t)k;
    dets[atomicAdd(&cursor[b], 1u)] = d;
  }
}

// Sec. 2.1 step 1 per field: t0 = earliest time with a detection, dt = t - t0.
__global__ void k_batch_epoch_setup(const BatchField* __restrict__ F) {
  const BatchField& bf = F[blockIdx.x];
  __shared__ long long s_min[32];
  long long m = LLONG_MAX;
  for (uint32_t e = threadIdx.x; e < bf.E; e += blockDim.x)
    if (bf.ecount[e] > 0 && bf.t[e] < m) m = bf.t[e];
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(0xffffffffu, m, o);
    m = other < m ? other : m;
  }
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t0 = s_min[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t0 = s_min[w] < t0 ? s_min[w] : t0;
    s_min[0] = t0;
    bf.t0[0] = t0;
  }
  __syncthreads();
  const long long t0 = s_min[0];
  for (uint32_t e = threadIdx.x; e < bf.E; e += blockDim.x)
    bf.dt[e] = bf.ecount[e] > 0 ? (int64_t)(bf.t[e] - t0) : 0;
}

// Sec. 2 Eq. 1-2 per field: x and y shift tables, one thread per entry.
__global__ void k_batch_shift(const BatchField* __restrict__ F, int n_fields,
                              const unsigned long long* __restrict__ tab_off) {
  const unsigned long long total = tab_off[n_fields];
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int f = find_field(tab_off, n_fields, i);
    const BatchField& bf = F[f];
    const SearchGeom& g = bf.args.g;
    unsigned long long k = i - tab_off[f];
    const unsigned long long nx = (unsigned long long)g.nvx * g.E;
    const bool is_x = k < nx;
    if (!is_x) k -= nx;
    const uint32_t c = (uint32_t)(k / g.E), e = (uint32_t)(k % g.E);
    const int64_t v = is_x ? (int64_t)g.vx0 + (int64_t)c * g.dvx : (int64_t)g.vy0 + (int64_t)c * g.dvy;
    const int64_t s = floor_div64(v * bf.dt[e], g.tph);
    int32_t sv = 0;
    if (s <= -kLimDomain || s >= kLimDomain) {
      if (bf.ecount[e] > 0) atomicOr(bf.counters + kCtrFlags, kFlagShift);
    } else {
      sv = (int32_t)s;
    }
    (is_x ? bf.sxt : bf.syt)[k] = sv;
  }
}

constexpr int kWarps = 8;

// Exact counts of every bin of every emitted super-bin of every field; one warp
// per emission slot (slots beyond a field's emission count exit).
// Grid: x blocks per field, y = field; each warp walks the field's emissions.
__global__ void k_batch_cell_count(const BatchField* __restrict__ F, const Det* __restrict__ dets,
                                   const uint32_t* __restrict__ boff) {
  const int lane = threadIdx.x & 31;
  const BatchField& bf = F[blockIdx.y];
  const uint32_t n_emit = min(bf.counters[kCtrEmit], bf.emit_cap);
  const SearchGeom& g = bf.args.g;
  const CoarseGeom& cg = bf.args.cg;
  const uint64_t cell_m = div_magic((uint32_t)cg.cell), bin_m = div_magic((uint32_t)g.bin);
  for (uint32_t j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < n_emit; j += gridDim.x * kWarps) {
    const Emit em = bf.args.emits[j];
    count_superbin(em, bf.args.tc.s, g, cg, cell_m, bin_m, dets, boff + bf.bucket_base, bf.ecount, bf.sxt,
                   bf.syt, (em.flags & kEmitLowPeak) ? bf.args.n_low : bf.args.n_min, lane,
                   [&](int, uint32_t bx, uint32_t by, uint32_t distinct, uint32_t raw) {
                     Key k;
                     k.a = ((uint64_t)(~distinct) << 32) | (uint64_t)(~raw);
                     k.b = ((uint64_t)em.v_idx << 32) | (uint64_t)by;
                     k.c = bx;
                     k.pad = 0;
                     const uint32_t p = atomicAdd(bf.counters + kCtrValid, 1u);
                     if (p < bf.key_cap) bf.keys[p] = k; else atomicOr(bf.counters + kCtrFlags, kFlagEmitCap);
                   });
  }
}

// Keys slots beyond a field's valid keys get the maximum key, so the segmented
// sort leaves the valid keys first; a field with more valid keys than slots
// gets its capacity flag (and is recomputed on the single-field path).
__global__ void k_batch_pad(const BatchField* __restrict__ F, Key* __restrict__ keys_all, uint64_t total,
                            uint32_t key_seg) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const BatchField& bf = F[i / key_seg];
  const uint32_t local = (uint32_t)(i % key_seg);
  const uint32_t n_valid = bf.counters[kCtrValid];
  if (local >= n_valid) keys_all[i] = max_key_b();
  if (local == 0 && n_valid > key_seg) atomicOr(bf.counters + kCtrFlags, kFlagEmitCap);
}

// One block per field, after the sort: the exclusive scan of the raw counts of
// the first n_out keys gives the id offsets.
__global__ void __launch_bounds__(1024) k_batch_offsets(const BatchField* __restrict__ F) {
  __shared__ unsigned long long s_warp[33];
  const BatchField& bf = F[blockIdx.x];
  const uint32_t n_valid = min(bf.counters[kCtrValid], bf.key_cap);
  const uint32_t n_out = min(n_valid, bf.max_out);
  unsigned long long carry = 0;
  for (uint32_t base = 0; base < n_out; base += blockDim.x) {
    const uint32_t i = base + threadIdx.x;
    const unsigned long long r = i < n_out ? (unsigned long long)(~(uint32_t)bf.keys[i].a) : 0ull;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = r;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long n = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += n;
    }
    if (lane == 31) s_warp[w] = inc;
    __syncthreads();
    if (w == 0) {
      const int nw = blockDim.x >> 5;
      const unsigned long long x = lane < nw ? s_warp[lane] : 0ull;
      unsigned long long sc = x;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(0xffffffffu, sc, o);
        if (lane >= o) sc += n;
      }
      if (lane < nw) s_warp[lane] = sc - x;
      if (lane == nw - 1) s_warp[32] = sc;
    }
    __syncthreads();
    if (i < n_out) bf.id_off[i] = carry + s_warp[w] + inc - r;
    carry += s_warp[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bf.counters[kCtrOut] = n_out;
    bf.id_off[n_out] = carry;
    bf.counters[kCtrIdsLo] = (uint32_t)carry;
    bf.counters[kCtrIdsHi] = (uint32_t)(carry >> 32);
    if (carry > bf.ids_cap) atomicOr(bf.counters + kCtrFlags, kFlagEmitCap);
  }
}

// Contributing ids (ascending) and the candidate records of every field; one
// warp per candidate slot.
// Grid: x blocks per field, y = field; each warp walks the field's candidates.
__global__ void k_batch_ids(const BatchField* __restrict__ F, const Det* __restrict__ dets,
                            const uint32_t* __restrict__ boff) {
  __shared__ uint32_t s_cursor[kWarps];
  const int wl = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const BatchField& bf = F[blockIdx.y];
  const uint32_t n_out = (bf.counters[kCtrFlags] & kFlagEmitCap) ? 0u : bf.counters[kCtrOut];
  for (uint32_t c = blockIdx.x * kWarps + wl; c < n_out; c += gridDim.x * kWarps) {
  const SearchGeom& g = bf.args.g;
  const CoarseGeom& cg = bf.args.cg;
  const Key key = bf.keys[c];
  const uint32_t v_idx = (uint32_t)(key.b >> 32), by = (uint32_t)key.b, bx = key.c;
  const uint32_t raw = ~(uint32_t)key.a;
  const uint32_t kx = v_idx % (uint32_t)g.nvx, ky = v_idx / (uint32_t)g.nvx;
  const unsigned long long off = bf.id_off[c];
  if (lane == 0) {
    sas_candidate rec;
    rec.v_idx = v_idx;
    rec.bx = bx;
    rec.by = by;
    rec.count = ~(uint32_t)(key.a >> 32);
    rec.raw = raw;
    rec.id_len = raw;
    rec.id_off = off;
    bf.cands[c] = rec;
    s_cursor[wl] = 0;
  }
  __syncwarp();
  for (uint32_t eb = 0; eb < g.E; eb += 32) {
    const uint32_t e = eb + lane;
    if (e >= g.E || bf.ecount[e] == 0) continue;
    const int32_t ox = g.x_min + (int32_t)bx * g.bin + bf.sxt[(size_t)kx * g.E + e];
    const int32_t oy = g.y_min + (int32_t)by * g.bin + bf.syt[(size_t)ky * g.E + e];
    const int cxa = max(floor_div32(ox - cg.gx0, cg.cell), 0);
    const int cxb = min(floor_div32(ox + g.bin - 1 - cg.gx0, cg.cell), cg.ncx - 1);
    const int cya = max(floor_div32(oy - cg.gy0, cg.cell), 0);
    const int cyb = min(floor_div32(oy + g.bin - 1 - cg.gy0, cg.cell), cg.ncy - 1);
    for (int cy = cya; cy <= cyb && cxa <= cxb; ++cy) {
      const size_t b0 = bf.bucket_base + ((size_t)e * cg.ncy + cy) * cg.ncx;
      const uint32_t k1 = boff[b0 + cxb + 1];
      for (uint32_t k = boff[b0 + cxa]; k < k1; ++k) {
        const Det d = dets[k];
        if (((uint32_t)(d.x - ox) < (uint32_t)g.bin) && ((uint32_t)(d.y - oy) < (uint32_t)g.bin)) {
          const uint32_t p = atomicAdd(&s_cursor[wl], 1u);
          if (p < raw) bf.ids_tmp[off + p] = d.id;
        }
      }
    }
  }
  __syncwarp();
  if (s_cursor[wl] != raw) {
    if (lane == 0) atomicOr(bf.counters + kCtrFlags, kFlagInternal);
  } else {
    for (uint32_t i = lane; i < raw; i += 32) {
      const uint32_t v = bf.ids_tmp[off + i];
      uint32_t r = 0;
      for (uint32_t j = 0; j < raw; ++j) r += bf.ids_tmp[off + j] < v;
      bf.ids[off + r] = v;
    }
  }
  __syncwarp();  // the cursor is reset for the next candidate only after every lane read it
  }
}

// Ownership over a batch: grid x blocks per field, y = field; warp per candidate.
__global__ void k_batch_owner(const BatchField* __restrict__ F, const unsigned long long* __restrict__ det_off,
                              const uint8_t* __restrict__ active, uint32_t* __restrict__ owner) {
  const int f = blockIdx.y;
  if (!active[f]) return;
  const BatchField& bf = F[f];
  const uint32_t n_out = bf.counters[kCtrOut];
  const uint32_t lane = threadIdx.x & 31;
  uint32_t* own = owner + det_off[f];
  for (uint32_t c = blockIdx.x * kWarps + (threadIdx.x >> 5); c < n_out; c += gridDim.x * kWarps) {
    const sas_candidate cd = bf.cands[c];
    for (uint32_t j = lane; j < cd.id_len; j += 32) atomicMin(&own[bf.ids[cd.id_off + j]], c);
  }
}

__global__ void k_batch_owned_flag(const BatchField* __restrict__ F, const unsigned long long* __restrict__ det_off,
                                   const unsigned long long* __restrict__ cand_off, const uint8_t* __restrict__ active,
                                   const uint32_t* __restrict__ owner, uint32_t* __restrict__ flag) {
  const int f = blockIdx.y;
  if (!active[f]) return;
  const BatchField& bf = F[f];
  const uint32_t n_out = bf.counters[kCtrOut];
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t* own = owner + det_off[f];
  for (uint32_t c = blockIdx.x * kWarps + (threadIdx.x >> 5); c < n_out; c += gridDim.x * kWarps) {
    const sas_candidate cd = bf.cands[c];
    uint32_t mine = 0;
    for (uint32_t j = lane; j < cd.id_len; j += 32) mine += own[bf.ids[cd.id_off + j]] == c;
    mine = __reduce_add_sync(0xffffffffu, mine);
    if (lane == 0) flag[cand_off[f] + c] = 2ull * mine >= cd.id_len || mine >= bf.args.n_low;
  }
}

__global__ void k_batch_compact(const unsigned long long* __restrict__ cand_off, int n_fields, uint64_t total,
                                const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off,
                                uint32_t* __restrict__ field_out, uint32_t* __restrict__ cand_out) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= total || !flag[i]) return;
  const int f = find_field(cand_off, n_fields, i);
  field_out[off[i]] = (uint32_t)f;
  cand_out[off[i]] = (uint32_t)(i - cand_off[f]);
}

unsigned grid_for(unsigned long long n, int threads) {
  unsigned long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152ull * 64) b = 152ull * 64;
  return (unsigned)b;
}

}  // namespace

cudaError_t batch_launch_prep(const BatchDev& B, cudaStream_t s) {
  k_batch_ingest<<<grid_for(B.total_dets, 256), 256, 0, s>>>(B.fields, B.n_fields, B.det_off,
                                                              B.bucket_count, B.bucket_of);
  note_launch();
  cudaError_t e = launch_scan_u32(B.bucket_count, B.boff, B.total_buckets, B.scan_scratch, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(B.cursor, B.boff, B.total_buckets * sizeof(uint32_t),
                      cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  k_batch_scatter<<<grid_for(B.total_dets, 256), 256, 0, s>>>(B.fields, B.n_fields, B.det_off,
                                                               B.bucket_of, B.cursor, B.dets);
  k_batch_epoch_setup<<<B.n_fields, 1024, 0, s>>>(B.fields);
  k_batch_shift<<<grid_for(B.total_tab, 256), 256, 0, s>>>(B.fields, B.n_fields, B.tab_off);
  note_launch(3);
  return cudaGetLastError();
}

cudaError_t batch_launch_post(const BatchDev& B, cudaStream_t s) {
  k_batch_cell_count<<<dim3(64, B.n_fields), kWarps * 32, 0, s>>>(B.fields, B.dets, B.boff);
  k_batch_pad<<<(unsigned)((B.total_cand + 255) / 256), 256, 0, s>>>(B.fields, B.keys_all, B.total_cand, B.key_seg);
  note_launch(2);
  cudaError_t e = launch_sort_segments(B.keys_all, (uint32_t)B.total_cand, B.key_seg, s);
  if (e != cudaSuccess) return e;
  k_batch_offsets<<<B.n_fields, 1024, 0, s>>>(B.fields);
  k_batch_ids<<<dim3(32, B.n_fields), kWarps * 32, 0, s>>>(B.fields, B.dets, B.boff);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t batch_set_attrs() { return cudaSuccess; }

cudaError_t batch_launch_owned(const BatchDev& B, const uint8_t* active, uint32_t* owner, uint32_t* flag,
                               cudaStream_t s) {
  k_batch_owner<<<dim3(32, B.n_fields), kWarps * 32, 0, s>>>(B.fields, B.det_off, active, owner);
  k_batch_owned_flag<<<dim3(32, B.n_fields), kWarps * 32, 0, s>>>(B.fields, B.det_off, B.cand_off, active, owner,
                                                                    flag);
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t batch_launch_compact(const BatchDev& B, const uint32_t* flag, const uint32_t* off,
                                 uint32_t* field_out, uint32_t* cand_out, cudaStream_t s) {
  k_batch_compact<<<(unsigned)((B.total_cand + 255) / 256), 256, 0, s>>>(B.cand_off, B.n_fields, B.total_cand,
                                                                       flag, off, field_out, cand_out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace sas
