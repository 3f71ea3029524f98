// Local peaks of a candidate list: the candidates that no neighbour within one
// lattice step (kx, ky) and one bin (bx, by) precedes in the output order.
//
// A mover makes a cluster of threshold crossings around its best cell (nearby
// velocities and bins also collect its detections; Sec. 2.2's velocity
// tolerance spans several lattice steps).  The paper removes such duplicates by
// peeling the best cluster (Sec. 2.1 step 3); keeping local peaks is the cheap,
// order-defined stand-in that the vetter runs on.
//
// Cells go into an open-addressing hash table (cell -> candidate index); each
// candidate then looks up its 80 neighbours.  Flags are compacted in order by
// an exclusive scan, so the peak list is ascending like the candidate list.
#include <algorithm>

#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t cell_hash(uint32_t v, uint32_t bx, uint32_t by) {
  uint64_t h = (uint64_t)v * 0x9E3779B97F4A7C15ull;
  h ^= (uint64_t)bx * 0xC2B2AE3D27D4EB4Full;
  h ^= (uint64_t)by * 0x165667B19E3779F9ull;
  h ^= h >> 29;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 32;
  return (uint32_t)h;
}

__global__ void k_peak_insert(const sas_candidate* __restrict__ c, uint64_t n, uint32_t* table,
                              uint32_t mask) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t h = cell_hash(c[i].v_idx, c[i].bx, c[i].by) & mask;
  // the table has more slots than keys, so an empty slot is always found
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    if (atomicCAS(&table[h], kEmpty, (uint32_t)i) == kEmpty) return;
    h = (h + 1) & mask;
  }
}

__global__ void k_peak_flags(const sas_candidate* __restrict__ c, uint64_t n, int32_t nvx, int32_t nvy,
                             const uint32_t* __restrict__ table, uint32_t mask, uint32_t* __restrict__ flag) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const sas_candidate ci = c[i];
  const int kx = (int)(ci.v_idx % (uint32_t)nvx), ky = (int)(ci.v_idx / (uint32_t)nvx);
  uint32_t peak = 1;
  for (int dky = -1; dky <= 1 && peak; ++dky) {
    const int ky2 = ky + dky;
    if (ky2 < 0 || ky2 >= nvy) continue;
    for (int dkx = -1; dkx <= 1 && peak; ++dkx) {
      const int kx2 = kx + dkx;
      if (kx2 < 0 || kx2 >= nvx) continue;
      const uint32_t v2 = (uint32_t)ky2 * (uint32_t)nvx + (uint32_t)kx2;
      for (int dby = -1; dby <= 1 && peak; ++dby) {
        const int64_t by2 = (int64_t)ci.by + dby;
        if (by2 < 0) continue;
        for (int dbx = -1; dbx <= 1 && peak; ++dbx) {
          const int64_t bx2 = (int64_t)ci.bx + dbx;
          if (bx2 < 0 || (dkx == 0 && dky == 0 && dbx == 0 && dby == 0)) continue;
          uint32_t h = cell_hash(v2, (uint32_t)bx2, (uint32_t)by2) & mask;
          for (uint32_t probe = 0; probe <= mask; ++probe) {
            const uint32_t j = table[h];
            if (j == kEmpty) break;
            const sas_candidate cj = c[j];
            if (cj.v_idx == v2 && cj.bx == (uint32_t)bx2 && cj.by == (uint32_t)by2) {
              if (j < i) peak = 0;
              break;
            }
            h = (h + 1) & mask;
          }
        }
      }
    }
  }
  flag[i] = peak;
}

__global__ void k_compact(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ off, uint64_t n,
                          uint32_t* __restrict__ idx) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n && flag[i]) idx[off[i]] = (uint32_t)i;
}

// Ownership: warp per candidate.  owner[d] = min index of a candidate whose ids
// contain detection d.
__global__ void k_owner_min(const sas_candidate* __restrict__ c, uint64_t n, const uint32_t* __restrict__ ids,
                            uint32_t* __restrict__ owner) {
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (w >= n) return;  // whole warps leave together
  const sas_candidate ci = c[w];
  for (uint32_t j = lane; j < ci.id_len; j += 32) atomicMin(&owner[ids[ci.id_off + j]], (uint32_t)w);
}

__global__ void k_owned_flag(const sas_candidate* __restrict__ c, uint64_t n, const uint32_t* __restrict__ ids,
                             const uint32_t* __restrict__ owner, uint32_t n_keep, uint32_t* __restrict__ flag) {
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint32_t lane = threadIdx.x & 31;
  if (w >= n) return;
  const sas_candidate ci = c[w];
  uint32_t mine = 0;
  for (uint32_t j = lane; j < ci.id_len; j += 32) mine += owner[ids[ci.id_off + j]] == (uint32_t)w;
  mine = __reduce_add_sync(0xffffffffu, mine);
  if (lane == 0) flag[w] = 2ull * mine >= ci.id_len || (n_keep > 0 && mine >= n_keep);
}

unsigned blocks_for(uint64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Scratch of a selection: flags, their exclusive scan and the scan's scratch.
struct Select {
  cudaStream_t s;
  uint32_t *flag = nullptr, *off = nullptr, *scratch = nullptr, *aux = nullptr;
  explicit Select(cudaStream_t st) : s(st) {}
  ~Select() {
    for (void* p : {(void*)flag, (void*)off, (void*)scratch, (void*)aux})
      if (p) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(uint64_t n, uint64_t aux_words) {
    cudaError_t e = cudaMallocAsync(&flag, n * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&off, (n + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&scratch, scan_scratch_elems(n) * 4, s);
    if (e == cudaSuccess && aux_words) e = cudaMallocAsync(&aux, aux_words * 4, s);
    if (e == cudaSuccess && aux_words) e = cudaMemsetAsync(aux, 0xFF, aux_words * 4, s);
    return e;
  }
  // In-order compaction of the flagged indices into idx; *n_out on the host.
  int finish(cudaError_t e, uint64_t n, uint32_t* idx, uint64_t* n_out, const char* what) {
    if (e == cudaSuccess) e = launch_scan_u32(flag, off, n, scratch, s);
    if (e == cudaSuccess) {
      k_compact<<<blocks_for(n, 256), 256, 0, s>>>(flag, off, n, idx);
      note_launch();
      e = cudaGetLastError();
    }
    uint32_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, off + n, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
      return set_errorf(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, "%s: %s", what,
                        cudaGetErrorString(e));
    *n_out = total;
    return SAS_OK;
  }
};

}  // namespace

int select_peaks(const CandView& v, uint32_t* idx, uint64_t* n_peaks, cudaStream_t s) {
  *n_peaks = 0;
  if (v.n == 0) return SAS_OK;
  if (v.n >= (1ull << 31)) return set_error(SAS_ERR_RANGE, "too many candidates for peak selection");
  uint64_t slots = 1;
  while (slots < 2 * v.n) slots <<= 1;
  Select sel(s);
  cudaError_t e = sel.alloc(v.n, slots);  // aux = hash table, all slots empty
  if (e == cudaSuccess) {
    k_peak_insert<<<blocks_for(v.n, 256), 256, 0, s>>>(v.cands, v.n, sel.aux, (uint32_t)(slots - 1));
    k_peak_flags<<<blocks_for(v.n, 256), 256, 0, s>>>(v.cands, v.n, v.g.nvx, v.g.nvy, sel.aux,
                                                      (uint32_t)(slots - 1), sel.flag);
    note_launch(2);
    e = cudaGetLastError();
  }
  return sel.finish(e, v.n, idx, n_peaks, "peak selection");
}

int select_owned(const CandView& v, uint32_t n_keep, uint32_t* idx, uint64_t* n_kept, cudaStream_t s) {
  *n_kept = 0;
  if (v.n == 0) return SAS_OK;
  if (v.n >= (1ull << 31)) return set_error(SAS_ERR_RANGE, "too many candidates for ownership selection");
  Select sel(s);
  cudaError_t e = sel.alloc(v.n, std::max<uint64_t>(v.n_det, 1));  // aux = owner per detection, all empty
  if (e == cudaSuccess) {
    const unsigned blocks = blocks_for(v.n * 32, 256);
    k_owner_min<<<blocks, 256, 0, s>>>(v.cands, v.n, v.ids, sel.aux);
    k_owned_flag<<<blocks, 256, 0, s>>>(v.cands, v.n, v.ids, sel.aux, n_keep, sel.flag);
    note_launch(2);
    e = cudaGetLastError();
  }
  return sel.finish(e, v.n, idx, n_kept, "ownership selection");
}

}  // namespace sas
