// Exact distinct-epoch counts of the bins of one emitted super-bin (Sec. 2.1
// step 2 for the cells the stack kernel flagged), shared by the single-field
// and the batched count kernels.
#pragma once

#include "sas_internal.cuh"

namespace sas {

// Division by a constant d >= 1 through a 64-bit reciprocal:
// umulhi64(x, ceil(2^64 / d)) == x / d for every 32-bit x (the rounding error
// of the reciprocal times x stays below 2^-32 < 1/d).  d == 1 is stored as 0.
__host__ __device__ inline uint64_t div_magic(uint32_t d) { return d <= 1 ? 0ull : (~0ull) / d + 1; }
__device__ __forceinline__ uint32_t div_by(uint32_t x, uint64_t m) {
  return m ? (uint32_t)__umul64hi((uint64_t)x, m) : x;
}

// Buckets [ca, cb] covering [o, o + span) along one axis (empty when ca > cb);
// o is relative to the bucket grid origin.
__device__ __forceinline__ void bucket_range(int32_t o, int32_t span, uint64_t cell_m, int n, int& ca, int& cb) {
  const int32_t hi = o + span - 1;
  ca = o < 0 ? 0 : (int)div_by((uint32_t)o, cell_m);
  cb = hi < 0 ? -1 : min((int)div_by((uint32_t)hi, cell_m), n - 1);
}

// One warp per emitted super-bin of sb x sb bins: lane l handles epochs l,
// l + 32, ...  For every bin q the epochs with at least one detection in it
// form one bitmask per 32-epoch block (ballot) whose popcounts add up to the
// exact distinct-epoch count.  Weighted (W): each lane keeps, per bin, the
// largest weight among its epoch's detections there, and the warp sums of
// those maxima add up to the bin's score instead.  Raw detection counts are
// taken afterwards, only for the bins in the domain that reach n_min; lane 0
// then calls out(q, bx, by, distinct or score, raw) for each of them.
template <bool W = false, typename Out>
__device__ __forceinline__ void count_superbin(const Emit& em, int sb, const SearchGeom& g, const CoarseGeom& cg,
                                               uint64_t cell_m, uint64_t bin_m, const Det* __restrict__ dets,
                                               const uint32_t* __restrict__ boff,
                                               const uint32_t* __restrict__ ecount,
                                               const int32_t* __restrict__ sxt, const int32_t* __restrict__ syt,
                                               uint32_t n_min, int lane, Out out,
                                               const uint8_t* __restrict__ wts = nullptr) {
  constexpr int kMaxQ = 16;  // super-bins up to 4 x 4 bins
  const uint32_t kx = em.v_idx % (uint32_t)g.nvx, ky = em.v_idx / (uint32_t)g.nvx;
  const int nq = sb * sb;
  const int32_t span = sb * g.bin;
  uint32_t distinct[kMaxQ];
#pragma unroll
  for (int q = 0; q < kMaxQ; ++q) distinct[q] = 0;
  for (uint32_t eb = 0; eb < g.E; eb += 32) {
    const uint32_t e = eb + lane;
    uint32_t hit = 0;
    uint32_t wmax[W ? kMaxQ : 1];
#pragma unroll
    for (int q = 0; q < (W ? kMaxQ : 1); ++q) wmax[q] = 0;
    if (e < g.E && ecount[e] > 0) {
      const int32_t ox = g.x_min + (int32_t)em.bx * g.bin + sxt[(size_t)kx * g.E + e];
      const int32_t oy = g.y_min + (int32_t)em.by * g.bin + syt[(size_t)ky * g.E + e];
      int cxa, cxb, cya, cyb;
      bucket_range(ox - cg.gx0, span, cell_m, cg.ncx, cxa, cxb);
      bucket_range(oy - cg.gy0, span, cell_m, cg.ncy, cya, cyb);
      for (int cy = cya; cy <= cyb && cxa <= cxb; ++cy) {
        const size_t b0 = ((size_t)e * cg.ncy + cy) * cg.ncx;
        const uint32_t k1 = boff[b0 + cxb + 1];
        for (uint32_t k = boff[b0 + cxa]; k < k1; ++k) {
          const Det d = dets[k];
          const uint32_t X = (uint32_t)(d.x - ox), Y = (uint32_t)(d.y - oy);
          if (X < (uint32_t)span && Y < (uint32_t)span) {
            const int qd = (int)div_by(Y, bin_m) * sb + (int)div_by(X, bin_m);
            hit |= 1u << qd;
            if constexpr (W) {
              const uint32_t wd = wts[d.id];
#pragma unroll
              for (int q = 0; q < kMaxQ; ++q)
                if (q == qd) wmax[q] = max(wmax[q], wd);
            }
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kMaxQ; ++q) {
      if (q >= nq) continue;
      if constexpr (W)
        distinct[q] += __reduce_add_sync(0xffffffffu, wmax[q]);
      else
        distinct[q] += __popc(__ballot_sync(0xffffffffu, (hit >> q) & 1u));
    }
  }
  // bins that become candidates (warp-uniform: the counts are)
  uint32_t need = 0;
#pragma unroll
  for (int q = 0; q < kMaxQ; ++q) {
    const uint32_t bx = em.bx + (uint32_t)(q % sb), by = em.by + (uint32_t)(q / sb);
    if (q < nq && distinct[q] >= n_min && bx < (uint32_t)g.nbx && by < (uint32_t)g.nby) need |= 1u << q;
  }
  while (need) {
    const int q = __ffs(need) - 1;
    need &= need - 1;
    const uint32_t bx = em.bx + (uint32_t)(q % sb), by = em.by + (uint32_t)(q / sb);
    uint32_t raw = 0;
    for (uint32_t eb = 0; eb < g.E; eb += 32) {
      const uint32_t e = eb + lane;
      if (e >= g.E || ecount[e] == 0) continue;
      const int32_t ox = g.x_min + (int32_t)bx * g.bin + sxt[(size_t)kx * g.E + e];
      const int32_t oy = g.y_min + (int32_t)by * g.bin + syt[(size_t)ky * g.E + e];
      int cxa, cxb, cya, cyb;
      bucket_range(ox - cg.gx0, g.bin, cell_m, cg.ncx, cxa, cxb);
      bucket_range(oy - cg.gy0, g.bin, cell_m, cg.ncy, cya, cyb);
      for (int cy = cya; cy <= cyb && cxa <= cxb; ++cy) {
        const size_t b0 = ((size_t)e * cg.ncy + cy) * cg.ncx;
        const uint32_t k1 = boff[b0 + cxb + 1];
        for (uint32_t k = boff[b0 + cxa]; k < k1; ++k) {
          const Det d = dets[k];
          raw += ((uint32_t)(d.x - ox) < (uint32_t)g.bin) & ((uint32_t)(d.y - oy) < (uint32_t)g.bin);
        }
      }
    }
    raw = __reduce_add_sync(0xffffffffu, raw);
    uint32_t dq = 0;  // distinct[q] without a dynamic register index
#pragma unroll
    for (int qq = 0; qq < kMaxQ; ++qq) dq = qq == q ? distinct[qq] : dq;
    if (lane == 0) out(q, bx, by, dq, raw);
  }
}

}  // namespace sas
