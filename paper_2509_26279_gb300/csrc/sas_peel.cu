// Cluster finding (Sec. 2.1 step 3) over a finished search's candidates.
//
// The paper loops: take the histogram's maximum cell; stop when it is below
// N_min; otherwise the detections that contributed to it form a cluster and are
// removed from the histogram.  Removing detections only lowers counts, so every
// later maximum is already among the search's candidates (every cell >= N_min):
// the loop runs over that list.  Maximum = the search's total order on the
// current counts (distinct desc, raw desc, v_idx, by, bx).
//
// Two implementations of the same loop:
//
// * Rounds of local maxima (default).  The keys the loop picks strictly
//   decrease, and a live candidate whose current key beats every live candidate
//   it shares a remaining detection with is picked by the loop, sooner or later,
//   with exactly its current detections: no candidate that could take one of
//   them can be picked before it.  Picking all such candidates at once and
//   removing their detections leaves a state from which the loop picks the
//   same remaining clusters, so each round picks every local maximum (at least
//   the global one) in parallel; the picks, sorted by the key they were picked
//   with, are the loop's output in order.  A round: recount every live
//   candidate and publish its key on each remaining detection (64-bit
//   atomicMax), test which candidates hold the maximum on all of theirs, copy
//   their detections out, mark them removed.  The loop's cut (the first
//   max_clusters clusters) is final once that many picks beat every live key.
//
// * One persistent 1024-thread block running the loop as stated, one cluster
//   per iteration: a block-wide argmax, the winner's remaining ids appended in
//   ascending order, removal, and a warp per affected candidate (found through
//   an inverted detection -> candidates index) recounting its remaining ids.
#include <algorithm>
#include <vector>

#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr int kPeelThreads = 1024;
constexpr uint32_t kNone = 0xFFFFFFFFu;

__global__ void k_epoch_of(const Det* __restrict__ dets, const uint32_t* __restrict__ n_ptr,
                           uint16_t* __restrict__ epoch_of) {
  const uint32_t n = *n_ptr;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    epoch_of[dets[i].id] = (uint16_t)dets[i].e;
}

// Inverted index detection -> candidates: counts, then (after a scan) fill.
__global__ void k_inv_count(const sas_candidate* __restrict__ c, uint32_t n, const uint32_t* __restrict__ ids,
                            uint32_t* __restrict__ cnt) {
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const sas_candidate ci = c[w];
  for (uint32_t j = threadIdx.x & 31; j < ci.id_len; j += 32) atomicAdd(&cnt[ids[ci.id_off + j]], 1u);
}

__global__ void k_inv_fill(const sas_candidate* __restrict__ c, uint32_t n, const uint32_t* __restrict__ ids,
                           const uint32_t* __restrict__ off, uint32_t* __restrict__ cursor,
                           uint32_t* __restrict__ inv) {
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  if (w >= n) return;
  const sas_candidate ci = c[w];
  for (uint32_t j = threadIdx.x & 31; j < ci.id_len; j += 32) {
    const uint32_t d = ids[ci.id_off + j];
    inv[off[d] + atomicAdd(&cursor[d], 1u)] = (uint32_t)w;
  }
}

struct Best {
  uint32_t d, r, v, by, bx, i;
};

// a precedes b in the total order on (d desc, r desc, v, by, bx); kNone last
__device__ __forceinline__ bool precedes(const Best& a, const Best& b) {
  if (a.i == kNone) return false;
  if (b.i == kNone) return true;
  if (a.d != b.d) return a.d > b.d;
  if (a.r != b.r) return a.r > b.r;
  if (a.v != b.v) return a.v < b.v;
  if (a.by != b.by) return a.by < b.by;
  return a.bx < b.bx;
}

__device__ __forceinline__ Best shfl_best(const Best& b, int o) {
  Best x;
  x.d = __shfl_xor_sync(0xffffffffu, b.d, o);
  x.r = __shfl_xor_sync(0xffffffffu, b.r, o);
  x.v = __shfl_xor_sync(0xffffffffu, b.v, o);
  x.by = __shfl_xor_sync(0xffffffffu, b.by, o);
  x.bx = __shfl_xor_sync(0xffffffffu, b.bx, o);
  x.i = __shfl_xor_sync(0xffffffffu, b.i, o);
  return x;
}

__global__ void __launch_bounds__(kPeelThreads) k_peel(
    const sas_candidate* __restrict__ c, uint32_t n_cand, const uint32_t* __restrict__ ids,
    const uint16_t* __restrict__ epoch_of, const uint32_t* __restrict__ inv_off, const uint32_t* __restrict__ inv,
    uint32_t* __restrict__ cur_d, uint32_t* __restrict__ cur_r, uint8_t* __restrict__ removed,
    uint32_t* __restrict__ aff_flag, uint32_t* __restrict__ aff, uint32_t n_min, uint32_t max_clusters,
    uint32_t* __restrict__ picks, uint32_t* __restrict__ out_ids, uint32_t* __restrict__ totals) {
  __shared__ Best s_warp[32];
  __shared__ Best s_best;
  __shared__ uint32_t s_naff, s_nids;
  __shared__ uint32_t s_mask[32][32];  // per warp: epochs 0..1023
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (uint32_t i = tid; i < n_cand; i += kPeelThreads) {
    cur_d[i] = c[i].count;
    cur_r[i] = c[i].raw;
  }
  if (tid == 0) {
    s_naff = 0;
    s_nids = 0;
  }
  __syncthreads();
  uint32_t npick = 0;
  for (; npick < max_clusters; ++npick) {
    // argmax under the total order
    Best b{0, 0, 0, 0, 0, kNone};
    for (uint32_t i = tid; i < n_cand; i += kPeelThreads) {
      const uint32_t d = cur_d[i];
      if (d < n_min) continue;
      const Best x{d, cur_r[i], c[i].v_idx, c[i].by, c[i].bx, i};
      if (precedes(x, b)) b = x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      const Best x = shfl_best(b, o);
      if (precedes(x, b)) b = x;
    }
    if (lane == 0) s_warp[warp] = b;
    __syncthreads();
    if (warp == 0) {
      b = s_warp[lane];
      for (int o = 16; o > 0; o >>= 1) {
        const Best x = shfl_best(b, o);
        if (precedes(x, b)) b = x;
      }
      if (lane == 0) s_best = b;
    }
    __syncthreads();
    const Best w = s_best;
    if (w.i == kNone) break;
    // the cluster: the winner's remaining ids, ascending (its list is ascending)
    const sas_candidate cw = c[w.i];
    if (warp == 0) {
      uint32_t base = s_nids;
      for (uint32_t j0 = 0; j0 < cw.id_len; j0 += 32) {
        const uint32_t j = j0 + lane;
        const uint32_t d = j < cw.id_len ? ids[cw.id_off + j] : 0u;
        const bool keep = j < cw.id_len && !removed[d];
        const uint32_t m = __ballot_sync(0xffffffffu, keep);
        if (keep) out_ids[base + __popc(m & ((1u << lane) - 1u))] = d;
        base += __popc(m);
      }
      if (lane == 0) {
        picks[4 * npick] = w.i;
        picks[4 * npick + 1] = w.d;
        picks[4 * npick + 2] = w.r;
        picks[4 * npick + 3] = s_nids;  // offset of the cluster's ids
        s_nids = base;
      }
    }
    __syncthreads();
    // remove them; every candidate holding one of them is recounted
    for (uint32_t j = tid; j < cw.id_len; j += kPeelThreads) {
      const uint32_t d = ids[cw.id_off + j];
      if (removed[d]) continue;
      removed[d] = 1;
      for (uint32_t k = inv_off[d]; k < inv_off[d + 1]; ++k) {
        const uint32_t cand = inv[k];
        if (atomicCAS(&aff_flag[cand], 0u, 1u) == 0u) aff[atomicAdd(&s_naff, 1u)] = cand;
      }
    }
    __syncthreads();
    const uint32_t naff = s_naff;
    for (uint32_t a = warp; a < naff; a += kPeelThreads / 32) {
      const uint32_t k = aff[a];
      const sas_candidate ck = c[k];
      s_mask[warp][lane] = 0;
      __syncwarp();
      uint32_t r = 0;
      for (uint32_t j = lane; j < ck.id_len; j += 32) {
        const uint32_t d = ids[ck.id_off + j];
        if (!removed[d]) {
          const uint32_t e = epoch_of[d];
          atomicOr(&s_mask[warp][e >> 5], 1u << (e & 31));
          ++r;
        }
      }
      __syncwarp();
      const uint32_t dist = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(s_mask[warp][lane]));
      r = __reduce_add_sync(0xffffffffu, r);
      if (lane == 0) {
        cur_d[k] = dist;
        cur_r[k] = r;
        aff_flag[k] = 0u;
      }
      __syncwarp();
    }
    __syncthreads();
    if (tid == 0) s_naff = 0;
    __syncthreads();
  }
  if (tid == 0) {
    totals[0] = npick;
    totals[1] = s_nids;
  }
}

// picks[4 i ..] = (candidate, distinct, raw, id offset) -> candidate records.
__global__ void k_peel_write(const sas_candidate* __restrict__ c, const uint32_t* __restrict__ picks,
                             uint32_t n, sas_candidate* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const sas_candidate ci = c[picks[4 * i]];
  sas_candidate o;
  o.v_idx = ci.v_idx;
  o.bx = ci.bx;
  o.by = ci.by;
  o.count = picks[4 * i + 1];
  o.raw = picks[4 * i + 2];
  o.id_len = picks[4 * i + 2];
  o.id_off = picks[4 * i + 3];
  out[i] = o;
}


// ---- rounds of local maxima ---------------------------------------------------

constexpr int kRoundThreads = 256;
constexpr int kRoundWarps = kRoundThreads / 32;

// Packed key of a live candidate, larger = earlier in the total order:
// distinct (11 bits, E <= 1024) | raw (rb bits) | (2^tb - 1 - t), t = the
// candidate's rank in (v_idx, by, bx) order.
struct Pack {
  uint32_t rb, tb;
  __device__ __forceinline__ uint64_t key(uint32_t d, uint32_t r, uint32_t t) const {
    return ((uint64_t)d << (rb + tb)) | ((uint64_t)r << tb) | (((1ull << tb) - 1ull) - t);
  }
  __device__ __forceinline__ uint32_t distinct(uint64_t k) const { return (uint32_t)(k >> (rb + tb)); }
  __device__ __forceinline__ uint32_t raw(uint64_t k) const {
    return (uint32_t)((k >> tb) & ((1ull << rb) - 1ull));
  }
};

// Control words of the round loop.
struct RoundCtl {
  uint32_t n_live[2];   // entries of the two live lists
  uint32_t n_pick;      // picks so far
  uint32_t id_cursor;   // ids copied out so far
  uint32_t pick_first;  // first pick of the current round
  uint32_t n_final;     // picks that beat every live key (cut test)
  unsigned long long max_key;  // largest live key of the current round
};

__global__ void k_tie_keys(const sas_candidate* __restrict__ c, uint32_t n, Key* __restrict__ keys) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Key k;
  k.a = 0;
  k.b = ((uint64_t)c[i].v_idx << 32) | c[i].by;
  k.c = c[i].bx;
  k.pad = i;
  keys[i] = k;
}

// rank[cand] = position in (v_idx, by, bx) order; live list 0 = every candidate
__global__ void k_tie_rank(const Key* __restrict__ keys, uint32_t n, uint32_t* __restrict__ rank,
                           uint32_t* __restrict__ live0) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  rank[keys[j].pad] = j;
  live0[j] = j;
}

// Recount every live candidate from its remaining ids; the ones still >= n_min
// go to the next live list and publish their key on each remaining detection.
__global__ void __launch_bounds__(kRoundThreads) k_round_recount(
    const sas_candidate* __restrict__ c, const uint32_t* __restrict__ ids, const uint16_t* __restrict__ epoch_of,
    const uint8_t* __restrict__ removed, const uint32_t* __restrict__ rank, Pack pk, uint32_t n_min,
    const uint32_t* __restrict__ live_in, uint32_t* __restrict__ live_out, RoundCtl* __restrict__ ctl, int in_buf,
    unsigned long long* __restrict__ key_of, unsigned long long* __restrict__ best) {
  __shared__ uint32_t s_mask[kRoundWarps][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) ctl->pick_first = ctl->n_pick;
  const uint32_t n_in = ctl->n_live[in_buf];
  const uint32_t stride = gridDim.x * kRoundWarps;
  for (uint32_t w = blockIdx.x * kRoundWarps + wib; w < n_in; w += stride) {
    const uint32_t k = live_in[w];
    const sas_candidate ck = c[k];
    s_mask[wib][lane] = 0;
    __syncwarp();
    uint32_t r = 0;
    for (uint32_t j = lane; j < ck.id_len; j += 32) {
      const uint32_t d = ids[ck.id_off + j];
      if (!removed[d]) {
        const uint32_t e = epoch_of[d];
        atomicOr(&s_mask[wib][e >> 5], 1u << (e & 31));
        ++r;
      }
    }
    __syncwarp();
    const uint32_t dist = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(s_mask[wib][lane]));
    r = __reduce_add_sync(0xffffffffu, r);
    __syncwarp();
    if (dist < n_min) continue;
    const unsigned long long key = pk.key(dist, r, rank[k]);
    if (lane == 0) {
      key_of[k] = key;
      live_out[atomicAdd(&ctl->n_live[in_buf ^ 1], 1u)] = k;
      atomicMax(&ctl->max_key, key);
    }
    for (uint32_t j = lane; j < ck.id_len; j += 32) {
      const uint32_t d = ids[ck.id_off + j];
      if (!removed[d]) atomicMax(&best[d], key);
    }
  }
}

// A live candidate holding the maximum key on every remaining detection is a
// pick: its remaining ids (ascending) are copied out.  Nothing is removed here,
// so every test of the round sees the same remaining detections.
__global__ void __launch_bounds__(kRoundThreads) k_round_pick(
    const sas_candidate* __restrict__ c, const uint32_t* __restrict__ ids, const uint8_t* __restrict__ removed,
    Pack pk, const uint32_t* __restrict__ live, RoundCtl* __restrict__ ctl, int buf,
    const unsigned long long* __restrict__ key_of, const unsigned long long* __restrict__ best,
    unsigned long long* __restrict__ pick_key, uint32_t* __restrict__ pick_cand, uint32_t* __restrict__ pick_off,
    uint32_t* __restrict__ tmp_ids) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const uint32_t n = ctl->n_live[buf];
  const uint32_t stride = gridDim.x * kRoundWarps;
  for (uint32_t w = blockIdx.x * kRoundWarps + wib; w < n; w += stride) {
    const uint32_t k = live[w];
    const unsigned long long key = key_of[k];
    const sas_candidate ck = c[k];
    bool ok = true;
    for (uint32_t j = lane; j < ck.id_len; j += 32) {
      const uint32_t d = ids[ck.id_off + j];
      if (!removed[d] && best[d] != key) ok = false;
    }
    if (!__all_sync(0xffffffffu, ok)) continue;
    uint32_t slot = 0, base = 0;
    if (lane == 0) {
      slot = atomicAdd(&ctl->n_pick, 1u);
      base = atomicAdd(&ctl->id_cursor, pk.raw(key));
      pick_key[slot] = key;
      pick_cand[slot] = k;
      pick_off[slot] = base;
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    for (uint32_t j0 = 0; j0 < ck.id_len; j0 += 32) {
      const uint32_t j = j0 + lane;
      const uint32_t d = j < ck.id_len ? ids[ck.id_off + j] : 0u;
      const bool keep = j < ck.id_len && !removed[d];
      const uint32_t m = __ballot_sync(0xffffffffu, keep);
      if (keep) tmp_ids[base + __popc(m & ((1u << lane) - 1u))] = d;
      base += __popc(m);
    }
  }
}

// Removes the detections of the round's picks.
__global__ void k_round_remove(Pack pk, const RoundCtl* __restrict__ ctl,
                               const unsigned long long* __restrict__ pick_key,
                               const uint32_t* __restrict__ pick_off, const uint32_t* __restrict__ tmp_ids,
                               uint8_t* __restrict__ removed) {
  const int lane = threadIdx.x & 31;
  const uint32_t first = ctl->pick_first, n = ctl->n_pick;
  const uint32_t stride = gridDim.x * (blockDim.x >> 5);
  for (uint32_t p = first + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n; p += stride) {
    const uint32_t off = pick_off[p], r = pk.raw(pick_key[p]);
    for (uint32_t j = lane; j < r; j += 32) removed[tmp_ids[off + j]] = 1;
  }
}

// Cut test: how many picks beat every key still live.
__global__ void k_round_final(const RoundCtl* __restrict__ ctl_in, const unsigned long long* __restrict__ pick_key,
                              RoundCtl* __restrict__ ctl) {
  const uint32_t n = ctl_in->n_pick;
  const unsigned long long m = ctl_in->max_key;
  uint32_t cnt = 0;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    cnt += pick_key[p] > m;
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctl->n_final, cnt);
}

// Sort keys of the picks: descending packed key = ascending complement.
__global__ void k_pick_keys(const unsigned long long* __restrict__ pick_key, uint32_t n, Key* __restrict__ keys) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Key k;
  k.a = ~pick_key[i];
  k.b = 0;
  k.c = 0;
  k.pad = i;
  keys[i] = k;
}

__global__ void k_pick_len(const Key* __restrict__ keys, uint32_t n, Pack pk,
                           const unsigned long long* __restrict__ pick_key, uint32_t* __restrict__ len) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) len[j] = pk.raw(pick_key[keys[j].pad]);
}

// Cluster j (in order) -> its record and ids.
__global__ void k_pick_write(const sas_candidate* __restrict__ c, const Key* __restrict__ keys, uint32_t n, Pack pk,
                             const unsigned long long* __restrict__ pick_key, const uint32_t* __restrict__ pick_cand,
                             const uint32_t* __restrict__ pick_off, const uint32_t* __restrict__ tmp_ids,
                             const uint32_t* __restrict__ out_off, sas_candidate* __restrict__ out,
                             uint32_t* __restrict__ out_ids) {
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * (blockDim.x >> 5);
  for (uint32_t j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n; j += stride) {
    const uint32_t p = keys[j].pad;
    const unsigned long long key = pick_key[p];
    const uint32_t r = pk.raw(key), src = pick_off[p], dst = out_off[j];
    for (uint32_t i = lane; i < r; i += 32) out_ids[dst + i] = tmp_ids[src + i];
    if (lane == 0) {
      const sas_candidate ci = c[pick_cand[p]];
      sas_candidate o;
      o.v_idx = ci.v_idx;
      o.bx = ci.bx;
      o.by = ci.by;
      o.count = pk.distinct(key);
      o.raw = r;
      o.id_len = r;
      o.id_off = dst;
      out[j] = o;
    }
  }
}

}  // namespace

namespace {

uint32_t ceil_log2(uint64_t n) {
  uint32_t b = 0;
  while ((1ull << b) < n) ++b;
  return b;
}

uint32_t pow2_at_least(uint32_t n) {
  uint32_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

unsigned blocks_of(uint64_t n, unsigned per) { return (unsigned)std::max<uint64_t>(1, (n + per - 1) / per); }

// Stream-ordered scratch, freed (stream-ordered) when the scope ends.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  cudaError_t get(T** p, uint64_t count) {
    cudaError_t e = cudaMallocAsync((void**)p, std::max<uint64_t>(count * sizeof(T), 16), s);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

cudaError_t peel_sequential(const CandView& v, uint32_t n_min, uint32_t max_clusters, uint64_t n_ids,
                            const uint16_t* epoch_of, uint8_t* removed, Scratch& sc, cudaStream_t s,
                            uint32_t* picks4, uint32_t* ids_tmp, uint32_t* totals) {
  const uint64_t nd = v.n_det, nc = v.n;
  uint32_t *cnt, *off, *scr, *cursor, *inv, *cur_d, *cur_r, *aff_flag, *aff;
  cudaError_t e = sc.get(&cnt, nd);
  if (e == cudaSuccess) e = sc.get(&off, nd + 1);
  if (e == cudaSuccess) e = sc.get(&scr, scan_scratch_elems(nd));
  if (e == cudaSuccess) e = sc.get(&cursor, nd);
  if (e == cudaSuccess) e = sc.get(&inv, n_ids);
  if (e == cudaSuccess) e = sc.get(&cur_d, nc);
  if (e == cudaSuccess) e = sc.get(&cur_r, nc);
  if (e == cudaSuccess) e = sc.get(&aff_flag, nc);
  if (e == cudaSuccess) e = sc.get(&aff, nc);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, nd * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, nd * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(aff_flag, 0, nc * 4, s);
  if (e != cudaSuccess) return e;
  k_inv_count<<<blocks_of(nc * 32, 256), 256, 0, s>>>(v.cands, (uint32_t)nc, v.ids, cnt);
  note_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_scan_u32(cnt, off, nd, scr, s)) != cudaSuccess) return e;
  k_inv_fill<<<blocks_of(nc * 32, 256), 256, 0, s>>>(v.cands, (uint32_t)nc, v.ids, off, cursor, inv);
  k_peel<<<1, kPeelThreads, 0, s>>>(v.cands, (uint32_t)nc, v.ids, epoch_of, off, inv, cur_d, cur_r,
                                    removed, aff_flag, aff, n_min, max_clusters, picks4,
                                    ids_tmp, totals);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace

int peel_clusters(const CandView& v, uint32_t n_min, uint32_t max_clusters, bool sequential, cudaStream_t s,
                  PeelOut* out) {
  *out = PeelOut{};
  if (v.n == 0 || max_clusters == 0) return SAS_OK;
  if (v.n >= (1ull << 31) || v.n_det >= (1ull << 31))
    return set_error(SAS_ERR_RANGE, "too many candidates or detections for cluster finding");
  const uint64_t nd = v.n_det, nc = v.n;
  uint64_t n_ids = 0;
  {
    sas_candidate last;
    cudaError_t e = cudaMemcpyAsync(&last, v.cands + nc - 1, sizeof(last), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_errorf(SAS_ERR_CUDA, "cluster finding: %s", cudaGetErrorString(e));
    n_ids = last.id_off + last.id_len;
  }
  // The packed key holds distinct (11 bits), raw (< 2^31: at most n_det) and
  // the (v_idx, by, bx) rank; when they do not fit, the single-block loop runs.
  Pack pk;
  pk.tb = std::max<uint32_t>(1, ceil_log2(nc));
  pk.rb = 64 - 11 - pk.tb;
  if (pk.rb < 32 && (nd >> pk.rb) != 0) sequential = true;

  uint32_t n_out = 0, n_out_ids = 0;
  cudaError_t e = cudaSuccess;
  {
    Scratch sc(s);
    uint16_t* epoch_of;
    uint8_t* removed;
    uint32_t* tmp_ids;
    e = sc.get(&epoch_of, nd);
    if (e == cudaSuccess) e = sc.get(&removed, nd);
    if (e == cudaSuccess) e = sc.get(&tmp_ids, std::max<uint64_t>(nd, n_ids));
    if (e == cudaSuccess) e = cudaMemsetAsync(removed, 0, nd, s);
    const uint64_t nb = (uint64_t)v.g.E * v.cg.ncy * v.cg.ncx;
    if (e == cudaSuccess) {
      k_epoch_of<<<152 * 8, 256, 0, s>>>(v.dets, v.boff + nb, epoch_of);
      note_launch();
      e = cudaGetLastError();
    }
    if (sequential) {
      uint32_t *picks4 = nullptr, *totals = nullptr;
      const uint32_t cap = (uint32_t)std::min<uint64_t>(max_clusters, nc);
      if (e == cudaSuccess) e = sc.get(&picks4, (uint64_t)cap * 4);
      if (e == cudaSuccess) e = sc.get(&totals, 2);
      if (e == cudaSuccess) e = cudaMemsetAsync(totals, 0, 8, s);
      if (e == cudaSuccess)
        e = peel_sequential(v, n_min, cap, n_ids, epoch_of, removed, sc, s, picks4, tmp_ids, totals);
      uint32_t h_tot[2] = {0, 0};
      if (e == cudaSuccess) e = cudaMemcpyAsync(h_tot, totals, 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&out->cands, std::max<size_t>(h_tot[0], 1) * sizeof(sas_candidate), s);
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&out->ids, std::max<size_t>(h_tot[1], 1) * 4, s);
      if (e == cudaSuccess && h_tot[0]) {
        k_peel_write<<<blocks_of(h_tot[0], 256), 256, 0, s>>>(v.cands, picks4, h_tot[0], out->cands);
        note_launch();
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && h_tot[1])
        e = cudaMemcpyAsync(out->ids, tmp_ids, (size_t)h_tot[1] * 4, cudaMemcpyDeviceToDevice, s);
      n_out = h_tot[0];
      n_out_ids = h_tot[1];
    } else {
      const uint32_t n_pad = pow2_at_least((uint32_t)nc);
      Key* keys;
      uint32_t *rank, *live[2], *pick_cand, *pick_off, *len, *ooff, *scr;
      unsigned long long *key_of, *best, *pick_key;
      RoundCtl* ctl;
      if (e == cudaSuccess) e = sc.get(&keys, n_pad);
      if (e == cudaSuccess) e = sc.get(&rank, nc);
      if (e == cudaSuccess) e = sc.get(&live[0], nc);
      if (e == cudaSuccess) e = sc.get(&live[1], nc);
      if (e == cudaSuccess) e = sc.get(&key_of, nc);
      if (e == cudaSuccess) e = sc.get(&best, nd);
      if (e == cudaSuccess) e = sc.get(&pick_key, nc);
      if (e == cudaSuccess) e = sc.get(&pick_cand, nc);
      if (e == cudaSuccess) e = sc.get(&pick_off, nc);
      if (e == cudaSuccess) e = sc.get(&ctl, 2);
      // ranks in (v_idx, by, bx) order, live list 0 = all candidates
      if (e == cudaSuccess) {
        k_tie_keys<<<blocks_of(nc, 256), 256, 0, s>>>(v.cands, (uint32_t)nc, keys);
        note_launch();
        e = launch_sort_keys(keys, (uint32_t)nc, n_pad, s);
      }
      if (e == cudaSuccess) {
        k_tie_rank<<<blocks_of(nc, 256), 256, 0, s>>>(keys, (uint32_t)nc, rank, live[0]);
        note_launch();
        e = cudaGetLastError();
      }
      RoundCtl init{};
      init.n_live[0] = (uint32_t)nc;
      if (e == cudaSuccess) e = cudaMemcpyAsync(ctl, &init, sizeof(init), cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // init is a stack object
      const unsigned grid = (unsigned)std::min<uint64_t>(blocks_of(nc, kRoundWarps), 152u * 8u);
      int buf = 0;
      uint32_t n_pick = 0;
      for (uint32_t round = 0; e == cudaSuccess && round <= nc; ++round) {
        // reset: the output list, the round's max key, the per-detection maxima
        e = cudaMemsetAsync(&ctl->n_live[buf ^ 1], 0, 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(&ctl->max_key, 0, 8, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(best, 0, nd * 8, s);
        if (e != cudaSuccess) break;
        k_round_recount<<<grid, kRoundThreads, 0, s>>>(v.cands, v.ids, epoch_of, removed, rank, pk, n_min, live[buf],
                                                       live[buf ^ 1], ctl, buf, key_of, best);
        note_launch();
        if (n_pick >= max_clusters) {
          // ctl[1] collects the cut count of this round
          e = cudaMemsetAsync(&ctl[1].n_final, 0, 4, s);
          if (e != cudaSuccess) break;
          k_round_final<<<blocks_of(n_pick, 256), 256, 0, s>>>(ctl, pick_key, ctl + 1);
          note_launch();
        }
        buf ^= 1;
        k_round_pick<<<grid, kRoundThreads, 0, s>>>(v.cands, v.ids, removed, pk, live[buf], ctl, buf, key_of, best,
                                                    pick_key, pick_cand, pick_off, tmp_ids);
        k_round_remove<<<grid, kRoundThreads, 0, s>>>(pk, ctl, pick_key, pick_off, tmp_ids, removed);
        note_launch(2);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        RoundCtl hc[2];
        if ((e = cudaMemcpyAsync(hc, ctl, sizeof(hc), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        const bool cut = n_pick >= max_clusters && hc[1].n_final >= max_clusters;
        n_pick = hc[0].n_pick;
        if (cut || hc[0].n_live[buf] == 0) break;
      }
      // the picks in the loop's order, cut to max_clusters
      n_out = std::min<uint32_t>(n_pick, max_clusters);
      const uint32_t p_pad = pow2_at_least(std::max<uint32_t>(n_pick, 1));
      Key* pkeys = nullptr;
      if (e == cudaSuccess) e = sc.get(&pkeys, p_pad);
      if (e == cudaSuccess) e = sc.get(&len, (uint64_t)n_out + 1);
      if (e == cudaSuccess) e = sc.get(&ooff, (uint64_t)n_out + 1);
      if (e == cudaSuccess) e = sc.get(&scr, scan_scratch_elems(n_out + 1));
      if (e == cudaSuccess && n_pick) {
        k_pick_keys<<<blocks_of(n_pick, 256), 256, 0, s>>>(pick_key, n_pick, pkeys);
        note_launch();
        e = launch_sort_keys(pkeys, n_pick, p_pad, s);
      }
      if (e == cudaSuccess && n_out) {
        k_pick_len<<<blocks_of(n_out, 256), 256, 0, s>>>(pkeys, n_out, pk, pick_key, len);
        note_launch();
        e = launch_scan_u32(len, ooff, n_out, scr, s);
      }
      if (e == cudaSuccess && n_out) e = cudaMemcpyAsync(&n_out_ids, ooff + n_out, 4, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&out->cands, std::max<size_t>(n_out, 1) * sizeof(sas_candidate), s);
      if (e == cudaSuccess) e = cudaMallocAsync((void**)&out->ids, std::max<size_t>(n_out_ids, 1) * 4, s);
      if (e == cudaSuccess && n_out) {
        k_pick_write<<<blocks_of(n_out, kRoundWarps), kRoundThreads, 0, s>>>(
            v.cands, pkeys, n_out, pk, pick_key, pick_cand, pick_off, tmp_ids, ooff, out->cands, out->ids);
        note_launch();
        e = cudaGetLastError();
      }
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (out->cands) cudaFree(out->cands);
    if (out->ids) cudaFree(out->ids);
    *out = PeelOut{};
    return set_errorf(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, "cluster finding: %s",
                      cudaGetErrorString(e));
  }
  out->n = n_out;
  out->n_ids = n_out_ids;
  return SAS_OK;
}

}  // namespace sas
