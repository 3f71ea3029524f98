// The stack kernel: Sec. 2.1 steps 1-3 for one block of the 3-D histogram at a time.
//
// Work unit = (spatial tile) x (velocity block).  A velocity block is BVX x BVY
// velocity tiles of KX x KY lattice points.  For a unit, the detections whose
// projection can land in the tile at any velocity of the block are found through
// the (epoch, coarse cell) buckets, filtered to the exact union window of each
// epoch and staged ONCE in shared memory as 8-byte records.  Then every velocity
// tile of the block runs against shared memory only: per record, KX + KY
// projections (the shift is separable: sx depends on kx, sy on ky) and one
// shared-memory atomicAdd per (detection, velocity) pair that lands in the tile.
//
// Counters: one narrow counter (CB = 8/16/32 bits, packed along kx so lane and
// increment are compile-time constants) per S x S block of bins ("super-bin")
// per velocity, counting raw detections.  Distinct epochs <= raw detections of a
// bin <= raw detections of its super-bin, so the super-bins whose count reaches
// N_min contain every bin that can reach N_min distinct epochs; the exact
// per-bin distinct-epoch counts (epoch bitmasks + popcount) are taken afterwards
// in sas_post.cu, which also discards the rest.
//
// Weighted stacking: every detection carries an integer weight w (1 without
// weights) and adds w instead of 1, so a super-bin's counter holds the sum of
// its weights, which bounds every bin's score (sum over epochs of the largest
// weight) from above; N_min is then the score threshold.
//
// A counter starts at 2^(CB-1) - N_min, so its top bit is set exactly when its
// count reaches N_min.  The hot loop therefore only adds (the atomics' old
// values are never read).  The pass that resets a tile's counters after its
// velocity tile is done reads them first: every counter with the top bit set is
// emitted once, and the counters' excess over their start value is summed.  A
// counter that wrapped (more than 2^(CB-1) - 1 + N_min detections) makes that sum
// fall short of the number of pairs added, by 255 or 256 per wrap; the kernel
// accumulates (sum - pairs) into a global balance and the host reruns with wider
// counters when it is not zero, so the result is exact for any input.
//
// Two thresholds (n_low < N_min): the counters start at 2^(CB-1) - n_low and a
// counter with the top bit set is emitted when its count reaches N_min (its
// bins are counted against N_min, as above) or when no counter of the tile
// adjacent to it -- lattice points and super-bins differing by at most one in
// each of kx, ky, super-bin column and row -- holds a larger count (a
// tile-local peak: its bins are counted against n_low).  A linear mover
// raises a whole neighbourhood of velocities and super-bins, and a noise
// alignment the velocities next to it; the peak test keeps the best of each
// such group before any bin is counted.  With the peaks alone (kSelectPeaks)
// the counters at or over N_min that are not peaks are dropped as well.  Only
// a counter with the top bit set can be larger than a tested one, so a word
// holding one is reset after every test of the tile (a second pass) and every
// other word as soon as it is read.  The kernel is instantiated with and
// without the peak tests (PEAKS), in two translation units.
#pragma once

#include <type_traits>

#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr int kNT = 1024;
constexpr int32_t kOutside = -(1 << 30);  // table entry of a lattice column that does not exist

struct SmemLayout {
  size_t cells, staged, ox, oy, win, seg_pos, seg_src, emit, peaks, misc, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// Shift-table rows per epoch in shared memory, padded by 4 words so that the
// rows of consecutive epochs start in different banks (a warp's records span
// one to three epochs; unpadded, their 16-byte loads hit the same banks).
__host__ __device__ inline int ox_stride(const TileCfg& tc) { return tc.bvx * tc.kx + 4; }
__host__ __device__ inline int oy_stride(const TileCfg& tc) { return tc.bvy * tc.ky + 4; }

__host__ __device__ inline SmemLayout layout(const TileCfg& tc) {
  SmemLayout L;
  const int per_word = 32 / tc.cb;
  size_t off = 0;
  L.cells = off;
  off += align16((size_t)tc.ky * (tc.kx / per_word) * tc.tx * tc.ty * 4);
  L.staged = off;
  off += align16((size_t)tc.scap * 8);
  L.ox = off;
  off += align16((size_t)tc.ec * ox_stride(tc) * 4);
  L.oy = off;
  off += align16((size_t)tc.ec * oy_stride(tc) * 4);
  L.win = off;
  off += align16((size_t)tc.ec * 4 * 4);
  L.seg_pos = off;
  off += align16((size_t)(tc.seg_cap + 1) * 4);
  L.seg_src = off;
  off += align16((size_t)tc.seg_cap * 4);
  L.emit = off;
  off += align16((size_t)tc.emit_cap * sizeof(Emit));
  L.peaks = off;
  off += align16((size_t)tc.peak_cap * 4);
  L.misc = off;
  off += 512;
  L.total = off;
  return L;
}

// Block-wide exclusive scan of one value per thread (kNT threads).
__device__ inline uint32_t block_scan(uint32_t v, uint32_t* s_tmp, uint32_t& total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  if (lane == 31) s_tmp[w] = inc;
  __syncthreads();
  if (w == 0) {
    constexpr int nw = kNT / 32;
    const uint32_t x = lane < nw ? s_tmp[lane] : 0u;
    uint32_t s = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t n = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += n;
    }
    if (lane < nw) s_tmp[lane] = s - x;
    if (lane == nw - 1) s_tmp[32] = s;
  }
  __syncthreads();
  const uint32_t r = s_tmp[w] + inc - v;
  total = s_tmp[32];
  __syncthreads();
  return r;
}

// Bit set of the lattice points of a velocity tile (bit ky * KX + kx).
template <int KX, int KY>
using Mask = typename std::conditional<(KX * KY > 32), uint64_t, uint32_t>::type;

template <int CB>
struct Counter {
  static constexpr int P = 32 / CB;  // counters per word
  static constexpr uint32_t CMASK = CB == 32 ? 0xffffffffu : ((1u << CB) - 1u);
};

// Unconditional shared-memory reduction.  On the merged paths (the usual
// ones) lanes with nothing to add give a zero increment at a harmless address
// instead of a predicate: predicated reductions measured one divergent branch
// each per warp.
__device__ __forceinline__ void red_shared(uint32_t addr, uint32_t inc) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
}

// Predicated shared-memory reduction: adds inc to the word at shared address
// addr when pred is nonzero (the per-lattice-point path, taken only when the
// planner cannot prove the merged reductions' two-run property; the zero-add
// form spills registers there).
__device__ __forceinline__ void red_shared_if(uint32_t pred, uint32_t addr, uint32_t inc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %0, 0;\n\t@p red.shared.add.u32 [%1], %2;\n\t}" ::"r"(pred),
      "r"(addr), "r"(inc));
}

// Counter increments of a mask of lattice columns within one word: bit q
// becomes 1 at the lowest bit of counter q.
template <int CB>
__device__ __forceinline__ uint32_t spread_bits(uint32_t b) {
  if constexpr (CB == 8) return (b * 0x00204081u) & 0x01010101u;  // bit q -> bit 8q (q < 4)
  else if constexpr (CB == 16) return (b * 0x00008001u) & 0x00010001u;  // bit q -> bit 16q (q < 2)
  else return b;
}

// One staged detection against every velocity of the tile (Sec. 2.1 steps 1-2).
// ox/oy hold the tile origin plus the shift of each lattice column/row, relative
// to the same window origin as the staged coordinates, so X = xr - ox[k] is the
// projected position relative to the tile origin.  Returns the number of
// (detection, velocity) pairs that landed in the tile.
template <int KX, int KY, int CB, bool MASKED, bool MERGE, bool WT>
__device__ __forceinline__ uint32_t process_rec(uint32_t xr, uint32_t yr,
                                                const int32_t* __restrict__ ox,
                                                const int32_t* __restrict__ oy,
                                                uint32_t cells_s, uint32_t tw_x,
                                                uint32_t tw_y, uint32_t magic, bool one, int tx,
                                                int txty, Mask<KX, KY> act, uint32_t w_in) {
  using C = Counter<CB>;
  const uint32_t w = WT ? w_in : 1u;  // unweighted: a compile-time 1
  // where a lane adds zero: one counter word per lane, in distinct banks (the
  // tile holds at least 32 words); adding zero changes no counter
  const uint32_t safe = cells_s + 4u * (threadIdx.x & 31u);
  int32_t oxv[KX], oyv[KY];
  if constexpr (KX % 4 == 0) {
#pragma unroll
    for (int k = 0; k < KX; k += 4) {
      const int4 q = *reinterpret_cast<const int4*>(ox + k);
      oxv[k] = q.x; oxv[k + 1] = q.y; oxv[k + 2] = q.z; oxv[k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < KX; ++k) oxv[k] = ox[k];
  }
  if constexpr (KY % 4 == 0) {
#pragma unroll
    for (int k = 0; k < KY; k += 4) {
      const int4 q = *reinterpret_cast<const int4*>(oy + k);
      oyv[k] = q.x; oyv[k + 1] = q.y; oyv[k + 2] = q.z; oyv[k + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < KY; ++k) oyv[k] = oy[k];
  }
  uint32_t col4[KX], okxb = 0;  // byte offset of the counter word in its row
#pragma unroll
  for (int k = 0; k < KX; ++k) {
    const uint32_t X = xr - (uint32_t)oxv[k];
    okxb |= (uint32_t)(X < tw_x) << k;
    col4[k] = (one ? X : __umulhi(X, magic)) * 4u;
  }
  uint32_t rbase4[KY], okyb = 0;  // shared address of the counter row
#pragma unroll
  for (int k = 0; k < KY; ++k) {
    const uint32_t Y = yr - (uint32_t)oyv[k];
    okyb |= (uint32_t)(Y < tw_y) << k;
    rbase4[k] = cells_s + (one ? Y : __umulhi(Y, magic)) * (uint32_t)(4 * tx);
  }
  if constexpr (MERGE && C::P >= 2 && !MASKED) {
    // Every lattice point of the tile is searched: a record's pairs are the
    // valid columns times the valid rows, so each word group's two increments
    // (runs of equal columns, see below) are formed once and reused per row.
    constexpr uint32_t gmask = (1u << C::P) - 1u;
    uint32_t lo[KX / C::P], hi[KX / C::P];
#pragma unroll
    for (int g = 0; g < KX / C::P; ++g) {
      uint32_t e = 0;
#pragma unroll
      for (int q = 0; q < C::P; ++q) e |= (uint32_t)(col4[g * C::P + q] == col4[g * C::P]) << q;
      const uint32_t xb = (okxb >> (g * C::P)) & gmask;
      lo[g] = spread_bits<CB>(xb & e) * w;
      hi[g] = spread_bits<CB>(xb & ~e) * w;
    }
#pragma unroll
    for (int ky = 0; ky < KY; ++ky) {
      const bool row = (okyb >> ky) & 1u;
#pragma unroll
      for (int g = 0; g < KX / C::P; ++g) {
        const uint32_t plane = rbase4[ky] + (uint32_t)((ky * (KX / C::P) + g) * txty * 4);
        const uint32_t a = row ? lo[g] : 0u, b = row ? hi[g] : 0u;
        red_shared(a ? plane + col4[g * C::P] : safe, a);
        red_shared(b ? plane + col4[g * C::P + C::P - 1] : safe, b);
      }
    }
    return (uint32_t)(__popc(okxb) * __popc(okyb));
  }
  using M = Mask<KX, KY>;
  M m = 0;
#pragma unroll
  for (int ky = 0; ky < KY; ++ky)
    if ((okyb >> ky) & 1u) m |= (M)okxb << (ky * KX);
  if (MASKED) m &= act;
  if constexpr (MERGE && C::P >= 2) {
    // The columns of one counter word project into at most two adjacent
    // super-bins (the planner proved it), and the projection is monotone in kx:
    // the columns equal to the word's first column form one run, the rest
    // equal its last column.  One reduction per run carries every column's
    // increment.
    constexpr uint32_t gmask = (1u << C::P) - 1u;
    uint32_t eqm[KX / C::P];
#pragma unroll
    for (int g = 0; g < KX / C::P; ++g) {
      uint32_t e = 0;
#pragma unroll
      for (int q = 0; q < C::P; ++q) e |= (uint32_t)(col4[g * C::P + q] == col4[g * C::P]) << q;
      eqm[g] = e;
    }
#pragma unroll
    for (int ky = 0; ky < KY; ++ky) {
#pragma unroll
      for (int g = 0; g < KX / C::P; ++g) {
        const uint32_t rb = (uint32_t)(m >> (ky * KX + g * C::P)) & gmask;
        const uint32_t lo = spread_bits<CB>(rb & eqm[g]) * w, hi = spread_bits<CB>(rb & ~eqm[g]) * w;
        const uint32_t plane = rbase4[ky] + (uint32_t)((ky * (KX / C::P) + g) * txty * 4);
        red_shared(lo ? plane + col4[g * C::P] : safe, lo);
        red_shared(hi ? plane + col4[g * C::P + C::P - 1] : safe, hi);
      }
    }
  } else {
#pragma unroll
    for (int ky = 0; ky < KY; ++ky) {
#pragma unroll
      for (int kx = 0; kx < KX; ++kx) {
        const uint32_t addr = rbase4[ky] + col4[kx] + (uint32_t)((ky * (KX / C::P) + kx / C::P) * txty * 4);
        red_shared_if((uint32_t)(m >> (ky * KX + kx)) & 1u, addr, w << (CB * (kx % C::P)));
      }
    }
  }
  if constexpr (sizeof(M) == 8) return (uint32_t)__popcll(m);
  else return (uint32_t)__popc(m);
}

// Sum of the counters packed in one word.
template <int CB>
__device__ __forceinline__ uint32_t word_sum(uint32_t w) {
  if constexpr (CB == 8) return __dp4a(w, 0x01010101u, 0u);
  else if constexpr (CB == 16) return (w & 0xffffu) + (w >> 16);
  else return w;
}

// Everything one work unit needs lives in shared memory: the counter tile, the
// staged records, the shift tables, the windows and the bucket segments.
template <int KX, int KY, int CB, bool PEAKS>
__device__ __forceinline__ void run_unit(const StackArgs& a, uint64_t unit, unsigned char* smem,
                                         bool init_cells, int64_t& balance, uint64_t& pairs64,
                                         uint32_t& my_flags) {
  using C = Counter<CB>;
  const TileCfg& tc = a.tc;
  const SmemLayout L = layout(tc);
  uint32_t* cells = reinterpret_cast<uint32_t*>(smem + L.cells);
  const uint32_t cells_s = (uint32_t)__cvta_generic_to_shared(cells);
  uint2* staged = reinterpret_cast<uint2*>(smem + L.staged);
  int32_t* s_ox = reinterpret_cast<int32_t*>(smem + L.ox);
  int32_t* s_oy = reinterpret_cast<int32_t*>(smem + L.oy);
  int32_t* s_win = reinterpret_cast<int32_t*>(smem + L.win);  // [ec][4]: xlo, xw, ylo, yw
  uint32_t* s_seg_pos = reinterpret_cast<uint32_t*>(smem + L.seg_pos);
  uint32_t* s_seg_src = reinterpret_cast<uint32_t*>(smem + L.seg_src);
  Emit* s_emit = reinterpret_cast<Emit*>(smem + L.emit);
  uint32_t* s_peaks = reinterpret_cast<uint32_t*>(smem + L.peaks);
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + L.misc);
  // s_misc: [0..33) scan scratch, [42] active mask (points 0-31), [45] (points 32-63),
  //         [43] emission count,
  //         [44] flush base, [46] peak-test list fill
  const int tid = threadIdx.x;
  constexpr int P = C::P;
  const uint32_t n_words = (uint32_t)KY * (KX / P) * tc.tx * tc.ty;
  const int txty = tc.tx * tc.ty;
  const SearchGeom& g = a.g;
  const CoarseGeom& cg = a.cg;
  const uint32_t E = g.E;
  const int n_st = a.nst_x * a.nst_y;
  const int bxk = tc.bvx * KX, byk = tc.bvy * KY;  // lattice columns / rows of a block
  const int oxs = ox_stride(tc), oys = oy_stride(tc);  // their shift-table rows per epoch
  const int sbins = tc.s;                          // bins per super-bin side
  const int rows_per_epoch = tc.rows;
  const bool single_chunk = E <= (uint32_t)tc.ec;
  // counter start value: the top bit turns on when the count reaches n_low
  // (n_min with one threshold)
  const uint32_t start = (1u << (CB - 1)) - a.n_low;
  uint32_t start_word = 0;
#pragma unroll
  for (int q = 0; q < P; ++q) start_word |= start << (CB * q);
  uint32_t tmask = 0;  // the top bit of every counter in a word
#pragma unroll
  for (int q = 0; q < P; ++q) tmask |= (1u << (CB - 1)) << (CB * q);
  const uint4 start4 = make_uint4(start_word, start_word, start_word, start_word);
  if (init_cells) {  // first unit of this block, or of another field
    for (uint32_t i = tid; i < n_words / 4; i += kNT) reinterpret_cast<uint4*>(cells)[i] = start4;
    if (tid == 0) s_misc[43] = 0;
    __syncthreads();
  }

    const int vb = (int)(unit / n_st), st = (int)(unit % n_st);
    const int kxa = a.kx_lo + (vb % a.nvt_x) * bxk;   // nvt_x/nvt_y count velocity BLOCKS
    const int kya = a.ky_lo + (vb / a.nvt_x) * byk;
    const int kxb = min(kxa + bxk, g.nvx) - 1;
    const int kyb = min(kya + byk, g.nvy) - 1;
    const int bx0 = (st % a.nst_x) * tc.tx * sbins;
    const int by0 = (st / a.nst_x) * tc.ty * sbins;
    const uint32_t tw_x = (uint32_t)min(tc.tx * sbins, g.nbx - bx0) * (uint32_t)g.bin;
    const uint32_t tw_y = (uint32_t)min(tc.ty * sbins, g.nby - by0) * (uint32_t)g.bin;
    const int32_t X0 = g.x_min + bx0 * g.bin, Y0 = g.y_min + by0 * g.bin;

    // --- prepare one epoch chunk: windows, shift tables, bucket segments -----
    auto prepare_chunk = [&](uint32_t e_base) -> uint32_t {
      const int ne = (int)min((uint32_t)tc.ec, E - e_base);
      if (tid < ne) {
        const uint32_t e = e_base + tid;
        int32_t xlo = 0, xw = 0, ylo = 0, yw = 0;
        if (a.ecount[e] > 0) {
          const int32_t s0 = a.sxt[(size_t)kxa * E + e], s1 = a.sxt[(size_t)kxb * E + e];
          const int32_t t0 = a.syt[(size_t)kya * E + e], t1 = a.syt[(size_t)kyb * E + e];
          xlo = X0 + min(s0, s1);
          xw = max(s0, s1) - min(s0, s1) + (int32_t)tw_x;
          ylo = Y0 + min(t0, t1);
          yw = max(t0, t1) - min(t0, t1) + (int32_t)tw_y;
          // staged x fits 24 bits (the chunk epoch rides above it), and so does a weighted search's y
          if (xw >= (1 << 24) || (a.w && yw >= (1 << 24))) my_flags |= kFlagInternal;
        }
        s_win[tid * 4 + 0] = xlo;
        s_win[tid * 4 + 1] = xw;
        s_win[tid * 4 + 2] = ylo;
        s_win[tid * 4 + 3] = yw;
      }
      __syncthreads();
      for (int i = tid; i < ne * (bxk + byk); i += kNT) {
        if (i < ne * bxk) {
          // Columns past the lattice edge take the last column's origin: their
          // pairs are masked out (active_mask), and a counter word that straddles
          // the edge keeps projections that differ by less than a super-bin,
          // which the merged reductions rely on.
          const int el = i / bxk, k = i % bxk, kx = min(kxa + k, g.nvx - 1);
          s_ox[el * oxs + k] = s_win[el * 4 + 1] > 0
                                   ? X0 + a.sxt[(size_t)kx * E + e_base + el] - s_win[el * 4]
                                   : kOutside;
        } else {
          const int j = i - ne * bxk;
          const int el = j / byk, k = j % byk, ky = kya + k;
          s_oy[el * oys + k] = (ky < g.nvy && s_win[el * 4 + 3] > 0)
                                   ? Y0 + a.syt[(size_t)ky * E + e_base + el] - s_win[el * 4 + 2]
                                   : kOutside;
        }
      }
      // One segment per (epoch, bucket row): thread t owns item t.
      uint32_t len = 0, src = 0;
      {
        const int el = tid / rows_per_epoch, r = tid % rows_per_epoch;
        if (el < ne && s_win[el * 4 + 1] > 0) {
          const int32_t xlo = s_win[el * 4], ylo = s_win[el * 4 + 2];
          const int cxa = max(floor_div32(xlo - cg.gx0, cg.cell), 0);
          const int cxb = min(floor_div32(xlo + s_win[el * 4 + 1] - 1 - cg.gx0, cg.cell), cg.ncx - 1);
          const int cya = max(floor_div32(ylo - cg.gy0, cg.cell), 0);
          const int cyb = min(floor_div32(ylo + s_win[el * 4 + 3] - 1 - cg.gy0, cg.cell), cg.ncy - 1);
          const int cy = cya + r;
          if (cxa <= cxb && cy <= cyb) {
            const size_t b0 = ((size_t)(e_base + el) * cg.ncy + cy) * cg.ncx;
            src = a.boff[b0 + cxa];
            len = a.boff[b0 + cxb + 1] - src;
          }
          if (r == rows_per_epoch - 1 && cyb - cya + 1 > rows_per_epoch) my_flags |= kFlagInternal;
        }
      }
      uint32_t total;
      const uint32_t pos = block_scan(len, s_misc, total);
      s_seg_pos[tid] = pos;
      s_seg_src[tid] = src;
      __syncthreads();
      return total;
    };

    // --- stage detections [p0, p1) of the chunk that lie in the window, in
    //     bucket order (records of one epoch stay together, so the shift-table
    //     loads of a warp are broadcasts) ----------------------------------------
    auto stage = [&](uint32_t e_base, uint32_t p0, uint32_t p1) -> uint32_t {
      uint32_t n_kept = 0;
      for (uint32_t j0 = p0; j0 < p1; j0 += kNT) {
        const uint32_t j = j0 + tid;
        uint32_t keep = 0;
        uint2 rec = make_uint2(0, 0);
        if (j < p1) {
          uint32_t lo = 0, hi = kNT;
          while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_seg_pos[mid] <= j) lo = mid; else hi = mid;
          }
          const Det d = a.dets[s_seg_src[lo] + (j - s_seg_pos[lo])];
          const int el = (int)(d.e - e_base);
          const uint32_t xr = (uint32_t)(d.x - s_win[el * 4]);
          const uint32_t yr = (uint32_t)(d.y - s_win[el * 4 + 2]);
          keep = xr < (uint32_t)s_win[el * 4 + 1] && yr < (uint32_t)s_win[el * 4 + 3];
          // weighted: the detection's weight rides in the top byte of y
          rec = make_uint2(xr | ((uint32_t)el << 24), a.w ? (yr | ((uint32_t)a.w[d.id] << 24)) : yr);
        }
        uint32_t total;
        const uint32_t pos = block_scan(keep, s_misc, total);
        if (keep) staged[n_kept + pos] = rec;
        n_kept += total;
      }
      __syncthreads();
      return n_kept;
    };

    // --- which lattice points of a velocity tile are searched ----------------
    auto active_mask = [&](int kx0, int ky0) -> Mask<KX, KY> {
      constexpr int kWarpsM = (KX * KY + 31) / 32;
      if (tid < 32 * kWarpsM) {
        bool act = false;
        if (tid < KX * KY) {
          const int kx = kx0 + tid % KX, ky = ky0 + tid / KX;
          if (kx < g.nvx && ky <= kyb) {
            const uint64_t v = (uint64_t)ky * g.nvx + kx;
            act = v >= g.v_begin && v < g.v_end;
            if (act && (g.smin != 0 || g.smax != 0)) {
              const int64_t vx = (int64_t)g.vx0 + (int64_t)kx * g.dvx;
              const int64_t vy = (int64_t)g.vy0 + (int64_t)ky * g.dvy;
              const int64_t s2 = vx * vx + vy * vy;
              act = s2 >= (int64_t)g.smin * g.smin && s2 <= (int64_t)g.smax * g.smax;
            }
          }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, act);
        if ((tid & 31) == 0) s_misc[(tid >> 5) ? 45 : 42] = m;  // lattice points 0-31, 32-63
      }
      __syncthreads();
      Mask<KX, KY> act = s_misc[42];
      if constexpr (KX * KY > 32) act |= (Mask<KX, KY>)s_misc[45] << 32;
      __syncthreads();
      return act;
    };

    // --- run one velocity tile of the block against the staged records -------
    auto compute = [&](int vtx, int vty, Mask<KX, KY> act, uint32_t n_staged) {
      using M = Mask<KX, KY>;
      const M full = (KX * KY == 8 * (int)sizeof(M)) ? ~(M)0 : (((M)1 << (KX * KY)) - 1);
      const int oxo = vtx * KX, oyo = vty * KY;
      uint32_t pairs = 0, added = 0;  // pairs, and the weight they added
      auto run = [&](auto masked, auto merge, auto weighted) {
        constexpr bool WT = decltype(weighted)::value;
        for (uint32_t j = tid; j < n_staged; j += kNT) {
          const uint2 r = staged[j];
          const int el = (int)(r.x >> 24);
          const uint32_t w = WT ? r.y >> 24 : 1u;
          const uint32_t p = process_rec<KX, KY, CB, decltype(masked)::value, decltype(merge)::value, WT>(
              r.x & 0xffffffu, WT ? r.y & 0xffffffu : r.y, s_ox + el * oxs + oxo, s_oy + el * oys + oyo, cells_s,
              tw_x, tw_y, a.magic, a.bin_is_one, tc.tx, txty, act, w);
          pairs += p;
          added += WT ? p * w : p;
        }
      };
      using T = std::true_type;
      using F = std::false_type;
      auto run_w = [&](auto weighted) {
        if (act == full) {
          if (a.merge) run(F{}, T{}, weighted); else run(F{}, F{}, weighted);
        } else {
          if (a.merge) run(T{}, T{}, weighted); else run(T{}, F{}, weighted);
        }
      };
      if (a.w) run_w(T{}); else run_w(F{});
      pairs64 += pairs;
      balance -= added;
      __syncthreads();  // the reductions above are asm: order them before any reader
    };

    // --- read every counter of the tile: emit those at or over n_min (and,
    //     with peak selection, the tile-local peaks at or over n_low), add up
    //     the counts, and reset them to the start value -----------------------
    // One threshold: each counter at or over n_min is emitted by the thread
    // that reads it, and every word is reset as soon as it is read.
    auto finish_plain = [&](int kx0, int ky0) {
      __syncthreads();
      // counter sums of this thread's words: 32 bits suffice below 32-bit counters
      // (the tile has at most 232448 / 16 uint4, so at most 15 per thread x 16 counters x 65535)
      using Acc = typename std::conditional<CB <= 16, uint32_t, uint64_t>::type;
      Acc acc = 0;
      uint32_t n_vec = 0;
      for (uint32_t i = tid; i < n_words / 4; i += kNT) {
        const uint4 v = reinterpret_cast<const uint4*>(cells)[i];
        acc += (Acc)word_sum<CB>(v.x) + (Acc)word_sum<CB>(v.y) + (Acc)word_sum<CB>(v.z) + (Acc)word_sum<CB>(v.w);
        ++n_vec;
        if ((v.x | v.y | v.z | v.w) & tmask) {
          const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
          for (int q = 0; q < 4; ++q) {
            for (int lane = 0; lane < P; ++lane) {
              if (!((wv[q] >> (CB * lane + CB - 1)) & 1u)) continue;
              const uint32_t widx = 4 * i + q;
              const uint32_t r = widx / (uint32_t)txty, rem = widx % (uint32_t)txty;
              const uint32_t row = rem / (uint32_t)tc.tx, col = rem % (uint32_t)tc.tx;
              const uint32_t ky = r / (KX / P), kx = (r % (KX / P)) * P + lane;
              Emit em;
              em.v_idx = (uint32_t)(ky0 + ky) * (uint32_t)g.nvx + (uint32_t)(kx0 + kx);
              em.bx = (uint32_t)bx0 + col * sbins;
              em.by = (uint32_t)by0 + row * sbins;
              em.flags = kEmitPlain;
              const uint32_t p = atomicAdd(&s_misc[43], 1u);
              if (p < (uint32_t)tc.emit_cap) {
                s_emit[p] = em;
              } else {
                const uint32_t gp = atomicAdd(a.n_emit, 1u);
                if (gp < a.emit_cap) a.emits[gp] = em; else my_flags |= kFlagEmitCap;
              }
            }
          }
        }
        reinterpret_cast<uint4*>(cells)[i] = start4;
      }
      balance += (int64_t)acc - (int64_t)n_vec * 4 * P * start;
      __syncthreads();
      const uint32_t ne_tile = min(s_misc[43], (uint32_t)tc.emit_cap);
      if (ne_tile) {
        if (tid == 0) s_misc[44] = atomicAdd(a.n_emit, ne_tile);
        __syncthreads();
        const uint32_t base = s_misc[44];
        for (uint32_t i = tid; i < ne_tile; i += kNT) {
          if (base + i < a.emit_cap) a.emits[base + i] = s_emit[i]; else my_flags |= kFlagEmitCap;
        }
        __syncthreads();
      }
      if (tid == 0) s_misc[43] = 0;
    };

    // Peak selection.  A first pass reads every word like the one-threshold
    // pass (and resets the words with no counter at or over n_low: only such
    // a counter can be larger than one that is); a second pass takes, warp by
    // warp, only the rounds in which some lane holds one, and the words it
    // read are reset after a barrier.
    auto finish_peaks = [&](int kx0, int ky0) {
      __syncthreads();
      using Acc = typename std::conditional<CB <= 16, uint32_t, uint64_t>::type;
      Acc acc = 0;
      uint32_t n_vec = 0;
      const int wl = tid & 31;
      const uint32_t lt_mask = (1u << wl) - 1u;
      const uint32_t nv4 = n_words / 4;
      uint32_t hit = 0;   // bit k: this thread's word of round k holds a counter with the top bit set
      uint32_t ntop = 0;  // how many such counters this thread's words hold
      {
        uint32_t k = 0;
        for (uint32_t i = tid; i < nv4; i += kNT, ++k) {
          const uint4 v = reinterpret_cast<const uint4*>(cells)[i];
          acc += (Acc)word_sum<CB>(v.x) + (Acc)word_sum<CB>(v.y) + (Acc)word_sum<CB>(v.z) + (Acc)word_sum<CB>(v.w);
          ++n_vec;
          if ((v.x | v.y | v.z | v.w) & tmask) {
            hit |= 1u << k;
            ntop += __popc(v.x & tmask) + __popc(v.y & tmask) + __popc(v.z & tmask) + __popc(v.w & tmask);
          } else {
            reinterpret_cast<uint4*>(cells)[i] = start4;
          }
        }
      }
      balance += (int64_t)acc - (int64_t)n_vec * 4 * P * start;
      // Second pass: the counters with the top bit set are listed in s_peaks
      // (as counter index widx * P + lane; slots from a block-wide scan of the
      // per-thread counts, in batches of tc.peak_cap) and tested by groups of
      // G threads each (G = 32 for a short list, down to 1 for a long one),
      // whichever warps hold them; a group's threads split the 27 (ky, row,
      // col) neighbour positions between them.
      const uint32_t cap = (uint32_t)tc.peak_cap;
      if (cap == 0) my_flags |= kFlagInternal;  // the plan reserves the list with peak selection
      uint32_t n_top = 0, off = 0;
      if (__syncthreads_or(cap != 0 && ntop != 0))  // one barrier for a tile with no candidate
        off = block_scan(cap ? ntop : 0u, s_misc, n_top);
      for (uint32_t b0 = 0; b0 < n_top; b0 += cap) {
        const uint32_t n_list = min(n_top - b0, cap);
        if (ntop && off < b0 + n_list && off + ntop > b0) {
          uint32_t idx = off, rr = hit;
          while (rr && idx < b0 + n_list) {
            const uint32_t k = (uint32_t)(__ffs(rr) - 1);
            rr &= rr - 1;
            const uint4 v = reinterpret_cast<const uint4*>(cells)[k * kNT + tid];
            uint32_t todo = 0;
#pragma unroll
            for (int l = 0; l < P; ++l) {
              const int sh = CB * l + CB - 1;
              todo |= ((v.x >> sh) & 1u) << l;
              todo |= ((v.y >> sh) & 1u) << (P + l);
              todo |= ((v.z >> sh) & 1u) << (2 * P + l);
              todo |= ((v.w >> sh) & 1u) << (3 * P + l);
            }
            while (todo && idx < b0 + n_list) {
              const int bb = __ffs(todo) - 1;
              todo &= todo - 1;
              if (idx >= b0) s_peaks[idx - b0] = (4u * (k * kNT + tid) + (uint32_t)(bb / P)) * P + (uint32_t)(bb % P);
              ++idx;
            }
          }
        }
        __syncthreads();
        const int G = n_list <= kNT / 32 ? 32 : n_list <= kNT / 8 ? 8 : n_list <= kNT / 4 ? 4 : 1;
        const uint32_t gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (wl & ~(G - 1));
        const int j = tid % G;
        for (uint32_t e0 = 0; e0 < n_list; e0 += (uint32_t)(kNT / G)) {
          const uint32_t e = e0 + (uint32_t)(tid / G);
          uint32_t why = 0;
          Emit em;
          bool bigger = false;
          int kx = 0, ky = 0, row = 0, col = 0;
          uint32_t c = 0;
          if (e < n_list) {
            const uint32_t ci = s_peaks[e];
            const uint32_t widx = ci / P;
            const int q = (int)(widx & 3u), l = (int)(ci % P);
            const uint4 v = reinterpret_cast<const uint4*>(cells)[widx >> 2];
            const uint32_t wq = q == 0 ? v.x : q == 1 ? v.y : q == 2 ? v.z : v.w;
            c = (wq >> (CB * l)) & C::CMASK;
            const uint32_t r = widx / (uint32_t)txty, rem_w = widx % (uint32_t)txty;
            row = (int)(rem_w / (uint32_t)tc.tx);
            col = (int)(rem_w % (uint32_t)tc.tx);
            ky = (int)(r / (KX / P));
            kx = (int)(r % (KX / P)) * P + l;
            // neighbours already in registers: kx -/+ 1 in this word, and in
            // the words of col -/+ 1 of the same row held by this uint4
#pragma unroll
            for (int dq = -1; dq <= 1; ++dq) {
              const int q2 = q + dq;
              if (q2 < 0 || q2 > 3 || col + dq < 0 || col + dq >= tc.tx) continue;
              const uint32_t w2 = q2 == 0 ? v.x : q2 == 1 ? v.y : q2 == 2 ? v.z : v.w;
#pragma unroll
              for (int dl = -1; dl <= 1; ++dl) {
                const int l2 = l + dl;
                if (l2 < 0 || l2 >= P) continue;
                bigger |= ((w2 >> (CB * l2)) & C::CMASK) > c;
              }
            }
            if (!bigger) {
              // this thread's share of the 27 positions (ky + t/9 - 1, row +
              // (t/3)%3 - 1, col + t%3 - 1), every kx - 1 .. kx + 1 (the
              // counter itself is not larger than itself)
              const int xa = max(kx - 1, 0), xb = min(kx + 1, KX - 1);
              for (int t = j; t < 27; t += G) {
                const int ky2 = ky + t / 9 - 1, r2 = row + (t / 3) % 3 - 1, c2 = col + t % 3 - 1;
                if (ky2 < 0 || ky2 >= KY || r2 < 0 || r2 >= tc.ty || c2 < 0 || c2 >= tc.tx) continue;
                const uint32_t* wb = cells + (uint32_t)(r2 * tc.tx + c2) + (uint32_t)(ky2 * (KX / P)) * (uint32_t)txty;
                for (int g2 = xa / P; g2 <= xb / P; ++g2) {
                  const uint32_t w = wb[(uint32_t)g2 * (uint32_t)txty];
#pragma unroll
                  for (int l2 = 0; l2 < P; ++l2) {
                    const int kx2 = g2 * P + l2;
                    if (kx2 >= xa && kx2 <= xb) bigger |= ((w >> (CB * l2)) & C::CMASK) > c;
                  }
                }
              }
            }
          }
          const bool any_bigger = (__ballot_sync(0xffffffffu, bigger) & gmask) != 0u;
          if (e < n_list && j == 0) {
            why = (a.select == kSelectPlainAndPeaks && c - start >= a.n_min) ? kEmitPlain : 0u;
            if (!any_bigger) why |= kEmitLowPeak;
            em.v_idx = (uint32_t)(ky0 + ky) * (uint32_t)g.nvx + (uint32_t)(kx0 + kx);
            em.bx = (uint32_t)bx0 + (uint32_t)col * sbins;
            em.by = (uint32_t)by0 + (uint32_t)row * sbins;
            em.flags = why;
          }
          const uint32_t m = __ballot_sync(0xffffffffu, why != 0);
          if (!m) continue;
          const int lead = __ffs(m) - 1;
          uint32_t base = 0;
          if (wl == lead) base = atomicAdd(&s_misc[43], (uint32_t)__popc(m));
          base = __shfl_sync(0xffffffffu, base, lead);
          const uint32_t p = base + (uint32_t)__popc(m & lt_mask);
          const bool over = why != 0 && p >= (uint32_t)tc.emit_cap;
          if (why != 0 && !over) s_emit[p] = em;
          const uint32_t mo = __ballot_sync(0xffffffffu, over);
          if (mo) {
            const int lo = __ffs(mo) - 1;
            uint32_t gb = 0;
            if (wl == lo) gb = atomicAdd(a.n_emit, (uint32_t)__popc(mo));
            gb = __shfl_sync(0xffffffffu, gb, lo);
            if (over) {
              const uint32_t gp = gb + (uint32_t)__popc(mo & lt_mask);
              if (gp < a.emit_cap) a.emits[gp] = em; else my_flags |= kFlagEmitCap;
            }
          }
        }
        __syncthreads();  // the list's reads before its next batch
      }
      __syncthreads();
      while (hit) {  // every peak test has read its neighbours
        const uint32_t k = (uint32_t)(__ffs(hit) - 1);
        hit &= hit - 1;
        reinterpret_cast<uint4*>(cells)[k * kNT + tid] = start4;
      }
      const uint32_t ne_tile = min(s_misc[43], (uint32_t)tc.emit_cap);
      if (ne_tile) {
        if (tid == 0) s_misc[44] = atomicAdd(a.n_emit, ne_tile);
        __syncthreads();
        const uint32_t base = s_misc[44];
        for (uint32_t i = tid; i < ne_tile; i += kNT) {
          if (base + i < a.emit_cap) a.emits[base + i] = s_emit[i]; else my_flags |= kFlagEmitCap;
        }
        __syncthreads();
      }
      if (tid == 0) s_misc[43] = 0;
    };

    auto finish = [&](int kx0, int ky0) {
      if constexpr (PEAKS) finish_peaks(kx0, ky0); else finish_plain(kx0, ky0);
    };

    const int nvt_bx = min(tc.bvx, (kxb - kxa) / KX + 1);
    const int nvt_by = min(tc.bvy, (kyb - kya) / KY + 1);
    if (single_chunk) {
      const uint32_t D = prepare_chunk(0);
      const bool once = D <= (uint32_t)tc.scap;
      const uint32_t ns_once = once ? stage(0, 0, D) : 0u;  // staged once for the whole block
      for (int vty = 0; vty < nvt_by; ++vty)
        for (int vtx = 0; vtx < nvt_bx; ++vtx) {
          const int kx0 = kxa + vtx * KX, ky0 = kya + vty * KY;
          const auto act = active_mask(kx0, ky0);
          if (act == 0) continue;
          if (once) {
            compute(vtx, vty, act, ns_once);
          } else {
            for (uint32_t p0 = 0; p0 < D; p0 += tc.scap) {
              const uint32_t ns = stage(0, p0, min(D, p0 + (uint32_t)tc.scap));
              compute(vtx, vty, act, ns);
              __syncthreads();
            }
          }
          finish(kx0, ky0);
        }
    } else {
      for (int vty = 0; vty < nvt_by; ++vty)
        for (int vtx = 0; vtx < nvt_bx; ++vtx) {
          const int kx0 = kxa + vtx * KX, ky0 = kya + vty * KY;
          const auto act = active_mask(kx0, ky0);
          if (act == 0) continue;
          for (uint32_t e_base = 0; e_base < E; e_base += tc.ec) {
            const uint32_t D = prepare_chunk(e_base);
            for (uint32_t p0 = 0; p0 < D; p0 += tc.scap) {
              const uint32_t ns = stage(e_base, p0, min(D, p0 + (uint32_t)tc.scap));
              compute(vtx, vty, act, ns);
              __syncthreads();
            }
          }
          finish(kx0, ky0);
        }
    }
}

// Single field: StackArgs as the kernel parameter.  Several fields (one
// persistent launch over all their units): fargs[f] for field f, whose units
// are [unit_base[f], unit_base[f + 1]) of one global work counter.
struct MultiArgs {
  const StackArgs* fargs;
  const unsigned long long* unit_base;  // [n_fields + 1]
  int n_fields;
  unsigned long long* counter;
};

template <int KX, int KY, int CB, bool MULTI, bool PEAKS>
__global__ void __launch_bounds__(kNT, 1) k_stack(StackArgs a0, MultiArgs m) {
  static_assert(KX % (32 / CB) == 0, "kx must be a multiple of the counters per word");
  static_assert(KX * KY <= 64, "at most 64 velocities per tile");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ StackArgs s_args;
  __shared__ unsigned long long s_unit, s_local;
  __shared__ int s_field;
  const int tid = threadIdx.x;
  int cur_field = -1;
  while (true) {
    if (tid == 0) {
      const unsigned long long t = atomicAdd(MULTI ? m.counter : a0.tile_counter, 1ull);
      s_unit = t;
      if (MULTI) {
        const unsigned long long total = m.unit_base[m.n_fields];
        int f = 0;
        if (t < total) {
          int lo = 0, hi = m.n_fields;  // largest f with unit_base[f] <= t
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (m.unit_base[mid] <= t) lo = mid; else hi = mid;
          }
          f = lo;
        }
        s_field = f;
        s_local = t < total ? t - m.unit_base[f] : ~0ull;
      } else {
        s_field = 0;
        s_local = t < a0.n_tiles ? t : ~0ull;
      }
    }
    __syncthreads();
    const unsigned long long local = s_local;
    const int field = s_field;
    if (local == ~0ull) break;
    if (MULTI && field != cur_field) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&m.fargs[field]);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&s_args);
      for (int i = tid; i < (int)(sizeof(StackArgs) / 4); i += kNT) dst[i] = src[i];
      __syncthreads();
    }
    const StackArgs& a = MULTI ? s_args : a0;
    int64_t balance = 0;  // (counted excess over the start values) - (pairs added)
    uint64_t pairs64 = 0;
    uint32_t my_flags = 0;
    run_unit<KX, KY, CB, PEAKS>(a, local, smem, field != cur_field, balance, pairs64, my_flags);
    cur_field = field;
    // Per-unit statistics of this field: one global atomic each per warp.
    for (int o = 16; o > 0; o >>= 1) {
      pairs64 += __shfl_xor_sync(0xffffffffu, pairs64, o);
      balance += __shfl_xor_sync(0xffffffffu, balance, o);
      my_flags |= __shfl_xor_sync(0xffffffffu, my_flags, o);
    }
    if ((tid & 31) == 0) {
      if (pairs64) atomicAdd(a.n_pairs, (unsigned long long)pairs64);
      if (balance) atomicAdd(a.balance, (unsigned long long)balance);
      if (my_flags) atomicOr(a.flags, my_flags);
    }
    __syncthreads();
  }
}

template <int KX, int KY, int CB, bool PEAKS>
cudaError_t launch_t(const StackArgs& a, int grid, cudaStream_t s) {
  MultiArgs m{};
  k_stack<KX, KY, CB, false, PEAKS><<<grid, kNT, a.tc.smem, s>>>(a, m);
  note_launch();
  return cudaGetLastError();
}

template <int KX, int KY, int CB, bool PEAKS>
cudaError_t launch_multi_t(const StackArgs& proto, const StackArgs* fargs,
                           const unsigned long long* unit_base, int n_fields,
                           unsigned long long* counter, size_t smem, int grid, cudaStream_t s) {
  MultiArgs m{fargs, unit_base, n_fields, counter};
  k_stack<KX, KY, CB, true, PEAKS><<<grid, kNT, smem, s>>>(proto, m);
  note_launch();
  return cudaGetLastError();
}

// Lets kernel f take `smem` bytes of dynamic shared memory.  The limit is only
// ever raised, and then to the device's whole opt-in size: launches of one
// kernel with different tile sizes (several batches, or a batch and single
// searches) never lower it under one another.
inline cudaError_t raise_smem_limit(const void* f, size_t smem) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  if ((size_t)fa.maxDynamicSharedSizeBytes >= smem) return cudaSuccess;
  int dev = 0, optin = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  const int64_t lim = (int64_t)optin - (int64_t)fa.sharedSizeBytes;
  if ((int64_t)smem > lim) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
}

template <int KX, int KY, int CB, bool PEAKS>
cudaError_t attr_t(size_t smem) {
  cudaError_t e = raise_smem_limit((const void*)k_stack<KX, KY, CB, false, PEAKS>, smem);
  if (e != cudaSuccess) return e;
  return raise_smem_limit((const void*)k_stack<KX, KY, CB, true, PEAKS>, smem);
}

// Supported (KX, KY, CB) instantiations.
#define SAS_STACK_CONFIGS(X) \
  X(4, 1, 8) X(4, 2, 8) X(4, 4, 8) X(8, 2, 8) X(8, 4, 8) X(8, 8, 8) \
  X(4, 1, 16) X(4, 2, 16) X(4, 4, 16) X(8, 2, 16) X(8, 4, 16) X(8, 8, 16) \
  X(4, 1, 32) X(4, 2, 32) X(4, 4, 32) X(8, 2, 32) X(8, 4, 32) X(8, 8, 32)

}  // namespace

}  // namespace sas
