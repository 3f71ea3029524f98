// Cluster finding (Sec. 2.1 step 3) over a finished search's candidates.
//
// The paper loops: take the histogram's maximum cell; stop when it is below
// N_min; otherwise the detections that contributed to it form a cluster and are
// removed from the histogram.  Removing detections only lowers counts, so every
// later maximum is already among the search's candidates (every cell >= N_min):
// the loop runs over that list, recounting only the candidates that shared a
// removed detection.  Maximum = the search's total order on the current counts
// (distinct desc, raw desc, v_idx, by, bx).
//
// One persistent block of 1024 threads runs the whole loop (one round per
// cluster, at most max_clusters rounds): a block-wide argmax, the winner's
// remaining ids appended in ascending order, removal, and a warp per affected
// candidate recounting its remaining ids (epoch bitmask in shared memory).
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

}  // namespace

int peel_clusters(const CandView& v, uint32_t n_min, uint32_t max_clusters, cudaStream_t s, PeelOut* out) {
  *out = PeelOut{};
  if (v.n == 0) return SAS_OK;
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
  std::vector<void*> ptrs;
  auto alloc = [&](void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, std::max<size_t>(bytes, 16), s);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  };
  uint16_t* epoch_of = nullptr;
  uint32_t *cnt = nullptr, *off = nullptr, *scr = nullptr, *cursor = nullptr, *inv = nullptr, *cur_d = nullptr,
           *cur_r = nullptr, *aff_flag = nullptr, *aff = nullptr, *picks = nullptr, *ids_tmp = nullptr,
           *totals = nullptr;
  uint8_t* removed = nullptr;
  cudaError_t e = alloc((void**)&epoch_of, nd * 2);
  if (e == cudaSuccess) e = alloc((void**)&cnt, nd * 4);
  if (e == cudaSuccess) e = alloc((void**)&off, (nd + 1) * 4);
  if (e == cudaSuccess) e = alloc((void**)&scr, scan_scratch_elems(nd) * 4);
  if (e == cudaSuccess) e = alloc((void**)&cursor, nd * 4);
  if (e == cudaSuccess) e = alloc((void**)&inv, n_ids * 4);
  if (e == cudaSuccess) e = alloc((void**)&cur_d, nc * 4);
  if (e == cudaSuccess) e = alloc((void**)&cur_r, nc * 4);
  if (e == cudaSuccess) e = alloc((void**)&aff_flag, nc * 4);
  if (e == cudaSuccess) e = alloc((void**)&aff, nc * 4);
  if (e == cudaSuccess) e = alloc((void**)&picks, (size_t)max_clusters * 16);
  if (e == cudaSuccess) e = alloc((void**)&ids_tmp, n_ids * 4);
  if (e == cudaSuccess) e = alloc((void**)&totals, 8);
  if (e == cudaSuccess) e = alloc((void**)&removed, nd);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, nd * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, nd * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(removed, 0, nd, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(aff_flag, 0, nc * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(totals, 0, 8, s);
  const uint64_t nb = (uint64_t)v.g.E * v.cg.ncy * v.cg.ncx;
  if (e == cudaSuccess) {
    k_epoch_of<<<152 * 8, 256, 0, s>>>(v.dets, v.boff + nb, epoch_of);
    k_inv_count<<<(unsigned)((nc * 32 + 255) / 256), 256, 0, s>>>(v.cands, (uint32_t)nc, v.ids, cnt);
    note_launch(2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_scan_u32(cnt, off, nd, scr, s);
  if (e == cudaSuccess) {
    k_inv_fill<<<(unsigned)((nc * 32 + 255) / 256), 256, 0, s>>>(v.cands, (uint32_t)nc, v.ids, off, cursor, inv);
    k_peel<<<1, kPeelThreads, 0, s>>>(v.cands, (uint32_t)nc, v.ids, epoch_of, off, inv, cur_d, cur_r, removed,
                                      aff_flag, aff, n_min, max_clusters, picks, ids_tmp, totals);
    note_launch(2);
    e = cudaGetLastError();
  }
  uint32_t h_tot[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_tot, totals, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&out->cands, std::max<size_t>(h_tot[0], 1) * sizeof(sas_candidate), s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&out->ids, std::max<size_t>(h_tot[1], 1) * 4, s);
  if (e == cudaSuccess && h_tot[0]) {
    k_peel_write<<<(h_tot[0] + 255) / 256, 256, 0, s>>>(v.cands, picks, h_tot[0], out->cands);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && h_tot[1]) e = cudaMemcpyAsync(out->ids, ids_tmp, (size_t)h_tot[1] * 4, cudaMemcpyDeviceToDevice, s);
  for (void* p : ptrs) cudaFreeAsync(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (out->cands) cudaFree(out->cands);
    if (out->ids) cudaFree(out->ids);
    *out = PeelOut{};
    return set_errorf(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, "cluster finding: %s",
                      cudaGetErrorString(e));
  }
  out->n = h_tot[0];
  out->n_ids = h_tot[1];
  return SAS_OK;
}

}  // namespace sas
