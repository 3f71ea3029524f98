// Count stamps of candidates: the input of the candidate vetter.
//
// Stamp of candidate (v_idx, bx, by): 9 x 15 x 15 distinct-epoch counts.  Plane
// q = (dy + 1) * 3 + (dx + 1) is the histogram (Sec. 2.1 step 2) of lattice
// point (kx + dx, ky + dy); element (i, j) is its bin (bx - 7 + j, by - 7 + i).
// Points off the lattice and bins off the domain count 0.
#include "sas_batch.cuh"

namespace sas {

namespace {

constexpr int kStampThreads = 256;
constexpr int kSide = 15;
constexpr int kCells = kSide * kSide;

// One candidate's stamp, by one block.  For each of the 9 velocities the block
// marks, in a shared epoch bitmask per stamp cell, the epochs of the
// detections that fall in the 15 x 15-bin window (one bucket scan per epoch),
// then writes the popcounts.  s_mask holds kCells * ceil(E / 32) words.
__device__ void stamp_one(const sas_candidate& cd, const SearchGeom& g, const CoarseGeom& cg,
                          const Det* __restrict__ dets, const uint32_t* __restrict__ boff,
                          const uint32_t* __restrict__ ecount, const int32_t* __restrict__ sxt,
                          const int32_t* __restrict__ syt, uint16_t* __restrict__ out, uint32_t* s_mask) {
  const uint32_t W = (g.E + 31) / 32;
  const int kx = (int)(cd.v_idx % (uint32_t)g.nvx), ky = (int)(cd.v_idx / (uint32_t)g.nvx);
  for (int q = 0; q < 9; ++q) {
    const int kx2 = kx + q % 3 - 1, ky2 = ky + q / 3 - 1;
    uint16_t* o = out + q * kCells;
    if (kx2 < 0 || kx2 >= g.nvx || ky2 < 0 || ky2 >= g.nvy) {
      for (int i = threadIdx.x; i < kCells; i += blockDim.x) o[i] = 0;
      continue;
    }
    for (uint32_t i = threadIdx.x; i < kCells * W; i += blockDim.x) s_mask[i] = 0;
    __syncthreads();
    for (uint32_t e = threadIdx.x; e < g.E; e += blockDim.x) {
      if (ecount[e] == 0) continue;
      // window origin: bin (bx - 7, by - 7) shifted back to epoch e
      const int32_t ox = g.x_min + ((int32_t)cd.bx - 7) * g.bin + sxt[(size_t)kx2 * g.E + e];
      const int32_t oy = g.y_min + ((int32_t)cd.by - 7) * g.bin + syt[(size_t)ky2 * g.E + e];
      const int32_t span = kSide * g.bin;
      const int cxa = max(floor_div32(ox - cg.gx0, cg.cell), 0);
      const int cxb = min(floor_div32(ox + span - 1 - cg.gx0, cg.cell), cg.ncx - 1);
      const int cya = max(floor_div32(oy - cg.gy0, cg.cell), 0);
      const int cyb = min(floor_div32(oy + span - 1 - cg.gy0, cg.cell), cg.ncy - 1);
      for (int cy = cya; cy <= cyb && cxa <= cxb; ++cy) {
        const size_t b0 = ((size_t)e * cg.ncy + cy) * cg.ncx;
        const uint32_t k1 = boff[b0 + cxb + 1];
        for (uint32_t k = boff[b0 + cxa]; k < k1; ++k) {
          const Det d = dets[k];
          const uint32_t X = (uint32_t)(d.x - ox), Y = (uint32_t)(d.y - oy);
          if (X >= (uint32_t)span || Y >= (uint32_t)span) continue;
          const int j = (int)(X / (uint32_t)g.bin), i = (int)(Y / (uint32_t)g.bin);
          const int bxx = (int)cd.bx - 7 + j, byy = (int)cd.by - 7 + i;
          if (bxx < 0 || bxx >= g.nbx || byy < 0 || byy >= g.nby) continue;
          atomicOr(&s_mask[(i * kSide + j) * W + (e >> 5)], 1u << (e & 31));
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kCells; i += blockDim.x) {
      uint32_t d = 0;
      for (uint32_t w = 0; w < W; ++w) d += __popc(s_mask[i * W + w]);
      o[i] = (uint16_t)min(d, 65535u);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kStampThreads) k_stamps(
    const sas_candidate* __restrict__ cands, const uint32_t* __restrict__ idx, uint64_t first,
    uint64_t n, SearchGeom g, CoarseGeom cg, const Det* __restrict__ dets,
    const uint32_t* __restrict__ boff, const uint32_t* __restrict__ ecount,
    const int32_t* __restrict__ sxt, const int32_t* __restrict__ syt, uint16_t* __restrict__ out) {
  extern __shared__ uint32_t s_mask[];
  for (uint64_t c = blockIdx.x; c < n; c += gridDim.x) {
    const sas_candidate cd = cands[idx ? (uint64_t)idx[c] : first + c];
    stamp_one(cd, g, cg, dets, boff, ecount, sxt, syt, out + c * 9 * kCells, s_mask);
  }
}

// Stamps of (field[i], cand[i]) items of a batch; the field's own geometry,
// buckets and shift tables.
__global__ void __launch_bounds__(kStampThreads) k_batch_stamps(
    const BatchField* __restrict__ F, const uint32_t* __restrict__ field, const uint32_t* __restrict__ cand,
    uint64_t n, uint16_t* __restrict__ out) {
  extern __shared__ uint32_t s_mask[];
  for (uint64_t c = blockIdx.x; c < n; c += gridDim.x) {
    const BatchField& bf = F[field[c]];
    const sas_candidate cd = bf.cands[cand[c]];
    stamp_one(cd, bf.args.g, bf.args.cg, bf.args.dets, bf.args.boff, bf.ecount, bf.sxt, bf.syt,
              out + c * 9 * kCells, s_mask);
  }
}

}  // namespace

cudaError_t launch_batch_stamps(const BatchField* F, uint32_t max_e, const uint32_t* field, const uint32_t* cand,
                                uint64_t n, uint16_t* out, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t smem = (size_t)kCells * ((max_e + 31) / 32) * 4;
  cudaError_t e = cudaFuncSetAttribute(k_batch_stamps, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(n < 152ull * 16 ? n : 152ull * 16);
  k_batch_stamps<<<blocks, kStampThreads, smem, s>>>(F, field, cand, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_stamps(const CandView& v, const uint32_t* idx, uint64_t first, uint64_t count,
                          uint16_t* out, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const size_t smem = (size_t)kCells * ((v.g.E + 31) / 32) * 4;
  cudaError_t e = cudaFuncSetAttribute(k_stamps, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(count < 152ull * 16 ? count : 152ull * 16);
  k_stamps<<<blocks, kStampThreads, smem, s>>>(v.cands, idx, first, count, v.g, v.cg, v.dets, v.boff,
                                                v.ecount, v.sxt, v.syt, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace sas
