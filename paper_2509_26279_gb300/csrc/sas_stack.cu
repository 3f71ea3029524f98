// The stack kernel: Sec. 2.1 steps 1-3 for one tile of the 3-D histogram at a time.
//
// A CTA owns a tile of KX x KY lattice velocities x TX x TY spatial bins and keeps
// one narrow counter per cell in shared memory.  For every detection whose
// projection can land in the tile (found through the (epoch, coarse cell)
// buckets), it computes the projected bin at each of the tile's velocities --
// the shift is separable, sx depends on kx only and sy on ky only, so a
// detection costs KX + KY divisions -- and does one shared-memory atomicAdd per
// (detection, velocity) pair that lands in the tile.  The counter counts
// detections; a cell whose counter goes from N_min - 1 to N_min is emitted
// exactly once (the crossing is a unique event).  Since distinct epochs <= raw
// detections, the emitted set contains every cell with >= N_min distinct epochs;
// the exact distinct-epoch count (bitmask + popcount) of each emitted cell is
// taken afterwards (sas_post.cu), which also discards the rest.
//
// Counters are packed CB bits wide, 32/CB per 32-bit word, and the packing runs
// along kx so the byte lane and increment of every pair are compile-time
// constants.  A counter that would wrap sets kFlagCounter and the host reruns
// with wider counters, so results stay exact for any input.
#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr int kNT = 512;
constexpr int32_t kOutside = -(1 << 30);  // table entry of a lattice column that does not exist

struct SmemLayout {
  size_t cells, ox, oy, seg_pos, seg_src, emit, misc, total;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__host__ __device__ inline SmemLayout layout(int kx, int ky, int tx, int ty, int cb, int ec,
                                             int seg_cap, int emit_cap) {
  SmemLayout L;
  const int per_word = 32 / cb;
  size_t off = 0;
  L.cells = off;
  off += align16((size_t)ky * (kx / per_word) * tx * ty * 4);
  L.ox = off;
  off += align16((size_t)ec * kx * 4);
  L.oy = off;
  off += align16((size_t)ec * ky * 4);
  L.seg_pos = off;
  off += align16((size_t)(seg_cap + 1) * 4);
  L.seg_src = off;
  off += align16((size_t)seg_cap * 4);
  L.emit = off;
  off += align16((size_t)emit_cap * sizeof(Emit));
  L.misc = off;
  off += 512;
  L.total = off;
  return L;
}

// Block-wide exclusive scan of two values at once (kNT threads).
__device__ inline void scan2(uint32_t a, uint32_t b, uint32_t* s_tmp, uint32_t& ea, uint32_t& eb,
                             uint32_t& ta, uint32_t& tb) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t ia = a, ib = b;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t na = __shfl_up_sync(0xffffffffu, ia, o);
    const uint32_t nb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) { ia += na; ib += nb; }
  }
  if (lane == 31) { s_tmp[w] = ia; s_tmp[32 + w] = ib; }
  __syncthreads();
  if (w == 0) {
    constexpr int nw = kNT / 32;
    const uint32_t va = lane < nw ? s_tmp[lane] : 0u;
    const uint32_t vb = lane < nw ? s_tmp[32 + lane] : 0u;
    uint32_t sa = va, sb = vb;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t na = __shfl_up_sync(0xffffffffu, sa, o);
      const uint32_t nb = __shfl_up_sync(0xffffffffu, sb, o);
      if (lane >= o) { sa += na; sb += nb; }
    }
    if (lane < nw) { s_tmp[lane] = sa - va; s_tmp[32 + lane] = sb - vb; }
    if (lane == nw - 1) { s_tmp[64] = sa; s_tmp[65] = sb; }
  }
  __syncthreads();
  ea = s_tmp[w] + ia - a;
  eb = s_tmp[32 + w] + ib - b;
  ta = s_tmp[64];
  tb = s_tmp[65];
  __syncthreads();
}

template <int KX, int KY, int CB>
struct Tile {
  static constexpr int P = 32 / CB;            // counters per word
  static constexpr uint32_t CMASK = CB == 32 ? 0xffffffffu : ((1u << CB) - 1u);
};

// Where a threshold crossing is recorded: the CTA's buffer, else the global list.
struct EmitCtx {
  Emit* s_emit;
  uint32_t* s_count;
  uint32_t s_cap;
  Emit* g_emit;
  uint32_t* g_count;
  uint32_t g_cap;
  uint32_t v_base;  // v_idx of the tile's (kx0, ky0)
  uint32_t nvx;
  uint32_t bx0, by0;
  uint32_t flags;
};

__device__ __noinline__ void emit_cell(EmitCtx& ec, uint32_t dv, uint32_t bxl, uint32_t byl) {
  Emit em;
  em.v_idx = ec.v_base + dv;
  em.bx = ec.bx0 + bxl;
  em.by = ec.by0 + byl;
  em.pad = 0;
  const uint32_t p = atomicAdd(ec.s_count, 1u);
  if (p < ec.s_cap) {
    ec.s_emit[p] = em;
  } else {
    const uint32_t gp = atomicAdd(ec.g_count, 1u);
    if (gp < ec.g_cap) ec.g_emit[gp] = em; else ec.flags |= kFlagEmitCap;
  }
}

// One detection against every velocity of the tile (Sec. 2.1 steps 1-2).
template <int KX, int KY, int CB, bool MASKED>
__device__ __forceinline__ void process_det(const Det& d, int el, const int32_t* __restrict__ s_ox,
                                            const int32_t* __restrict__ s_oy,
                                            uint32_t* __restrict__ cells, uint32_t tw_x,
                                            uint32_t tw_y, uint32_t magic, bool bin_one, int tx,
                                            int txty, uint32_t act, uint32_t nmin1,
                                            uint64_t& pairs, EmitCtx& ec) {
  using T = Tile<KX, KY, CB>;
  uint32_t col[KX];
  bool okx[KX];
#pragma unroll
  for (int k = 0; k < KX; ++k) {
    const uint32_t X = (uint32_t)(d.x - s_ox[el * KX + k]);
    okx[k] = X < tw_x;
    col[k] = bin_one ? X : __umulhi(X, magic);
  }
  uint32_t row[KY];
  bool oky[KY];
#pragma unroll
  for (int k = 0; k < KY; ++k) {
    const uint32_t Y = (uint32_t)(d.y - s_oy[el * KY + k]);
    oky[k] = Y < tw_y;
    row[k] = bin_one ? Y : __umulhi(Y, magic);
  }
#pragma unroll
  for (int ky = 0; ky < KY; ++ky) {
    const uint32_t rbase = row[ky] * (uint32_t)tx;
#pragma unroll
    for (int kx = 0; kx < KX; ++kx) {
      bool ok = okx[kx] && oky[ky];
      if (MASKED) ok = ok && ((act >> (ky * KX + kx)) & 1u);
      if (ok) {
        const uint32_t widx = (uint32_t)((ky * (KX / T::P) + kx / T::P) * txty) + rbase + col[kx];
        const int sh = CB * (kx % T::P);  // folds to a constant once unrolled
        const uint32_t old = atomicAdd(&cells[widx], 1u << sh);
        const uint32_t c = (old >> sh) & T::CMASK;
        ++pairs;
        if (c >= nmin1) {
          if (c == nmin1) emit_cell(ec, (uint32_t)ky * ec.nvx + kx, col[kx], row[ky]);
          if (c == T::CMASK) ec.flags |= kFlagCounter;  // counter wrapped: rerun wider
        }
      }
    }
  }
}

template <int KX, int KY, int CB>
__global__ void __launch_bounds__(kNT, 2) k_stack(StackArgs a) {
  static_assert(KX % (32 / CB) == 0, "kx must be a multiple of the counters per word");
  static_assert(KX * KY <= 31, "at most 31 velocities per tile");
  extern __shared__ __align__(16) unsigned char smem[];
  const TileCfg& tc = a.tc;
  const SmemLayout L = layout(KX, KY, tc.tx, tc.ty, CB, tc.ec, tc.seg_cap, tc.emit_cap);
  uint32_t* cells = reinterpret_cast<uint32_t*>(smem + L.cells);
  int32_t* s_ox = reinterpret_cast<int32_t*>(smem + L.ox);
  int32_t* s_oy = reinterpret_cast<int32_t*>(smem + L.oy);
  uint32_t* s_seg_pos = reinterpret_cast<uint32_t*>(smem + L.seg_pos);
  uint32_t* s_seg_src = reinterpret_cast<uint32_t*>(smem + L.seg_src);
  Emit* s_emit = reinterpret_cast<Emit*>(smem + L.emit);
  uint32_t* s_misc = reinterpret_cast<uint32_t*>(smem + L.misc);
  // s_misc: [0..66) scan scratch, [70] tile lo, [71] tile hi, [72] active mask,
  //         [73] emission count, [74] flags
  const int tid = threadIdx.x;
  const int P = 32 / CB;
  const uint32_t n_words = (uint32_t)KY * (KX / P) * tc.tx * tc.ty;
  const int txty = tc.tx * tc.ty;
  const SearchGeom& g = a.g;
  const CoarseGeom& cg = a.cg;
  const uint32_t E = g.E;
  const uint32_t nmin1 = a.n_min - 1u;
  const int n_st = a.nst_x * a.nst_y;

  for (uint32_t i = tid; i < n_words / 4; i += kNT)
    reinterpret_cast<uint4*>(cells)[i] = make_uint4(0, 0, 0, 0);
  uint64_t pairs = 0;
  uint32_t my_flags = 0;

  while (true) {
    if (tid == 0) {
      const unsigned long long t = atomicAdd(a.tile_counter, 1ull);
      s_misc[70] = (uint32_t)t;
      s_misc[71] = (uint32_t)(t >> 32);
      s_misc[73] = 0;
    }
    __syncthreads();
    const uint64_t tile = (uint64_t)s_misc[70] | ((uint64_t)s_misc[71] << 32);
    if (tile >= a.n_tiles) break;
    const int vt = (int)(tile / n_st), st = (int)(tile % n_st);
    const int kx0 = a.kx_lo + (vt % a.nvt_x) * KX;
    const int ky0 = a.ky_lo + (vt / a.nvt_x) * KY;
    const int bx0 = (st % a.nst_x) * tc.tx;
    const int by0 = (st / a.nst_x) * tc.ty;
    const int txe = min(tc.tx, g.nbx - bx0), tye = min(tc.ty, g.nby - by0);
    const uint32_t tw_x = (uint32_t)txe * (uint32_t)g.bin, tw_y = (uint32_t)tye * (uint32_t)g.bin;
    const int32_t X0 = g.x_min + bx0 * g.bin, Y0 = g.y_min + by0 * g.bin;

    // Which (kx, ky) of the tile are searched: inside the lattice, inside the
    // requested index range and inside the speed annulus.
    if (tid < 32) {
      bool act = false;
      if (tid < KX * KY) {
        const int kx = kx0 + tid % KX, ky = ky0 + tid / KX;
        if (kx < g.nvx && ky < g.nvy) {
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
      if (tid == 0) s_misc[72] = m;
    }
    __syncthreads();
    const uint32_t act = s_misc[72];
    if (act == 0) continue;  // nothing searched here; every thread sees the same value
    const uint32_t full = (KX * KY == 32) ? 0xffffffffu : ((1u << (KX * KY)) - 1u);
    const bool masked = act != full;
    const int kxl = min(kx0 + KX, g.nvx) - 1;  // last lattice column of the tile
    const int kyl = min(ky0 + KY, g.nvy) - 1;

    for (uint32_t e_base = 0; e_base < E; e_base += tc.ec) {
      const int ne = (int)min((uint32_t)tc.ec, E - e_base);
      // Shift table of this chunk, offset by the tile origin.
      for (int i = tid; i < ne * (KX + KY); i += kNT) {
        if (i < ne * KX) {
          const int el = i / KX, k = i % KX;
          const int kx = kx0 + k;
          s_ox[el * KX + k] = kx < g.nvx ? X0 + a.sxt[(size_t)kx * E + e_base + el] : kOutside;
        } else {
          const int j = i - ne * KX;
          const int el = j / KY, k = j % KY;
          const int ky = ky0 + k;
          s_oy[el * KY + k] = ky < g.nvy ? Y0 + a.syt[(size_t)ky * E + e_base + el] : kOutside;
        }
      }
      // Source window of the tile at this epoch -> bucket rows.
      uint32_t nrows = 0, ndet = 0;
      int cxa = 0, cxb = -1, cya = 0, cyb = -1;
      const uint32_t e = e_base + tid;
      if (tid < ne && a.ecount[e] > 0) {
        const int32_t s0 = a.sxt[(size_t)kx0 * E + e], s1 = a.sxt[(size_t)kxl * E + e];
        const int32_t t0 = a.syt[(size_t)ky0 * E + e], t1 = a.syt[(size_t)kyl * E + e];
        const int32_t xa = X0 + min(s0, s1), xb = X0 + max(s0, s1) + (int32_t)tw_x;  // [xa, xb)
        const int32_t ya = Y0 + min(t0, t1), yb = Y0 + max(t0, t1) + (int32_t)tw_y;
        cxa = max(floor_div32(xa - cg.gx0, cg.cell), 0);
        cxb = min(floor_div32(xb - 1 - cg.gx0, cg.cell), cg.ncx - 1);
        cya = max(floor_div32(ya - cg.gy0, cg.cell), 0);
        cyb = min(floor_div32(yb - 1 - cg.gy0, cg.cell), cg.ncy - 1);
        if (cxa <= cxb && cya <= cyb) {
          for (int cy = cya; cy <= cyb; ++cy) {  // rows holding at least one detection
            const size_t b0 = ((size_t)e * cg.ncy + cy) * cg.ncx;
            const uint32_t len = a.boff[b0 + cxb + 1] - a.boff[b0 + cxa];
            if (len) { ++nrows; ndet += len; }
          }
        }
      }
      uint32_t seg_off, det_off, nseg, D;
      scan2(nrows, ndet, s_misc, seg_off, det_off, nseg, D);
      if (nseg > (uint32_t)tc.seg_cap) {  // cannot happen with host-chosen sizes
        my_flags |= kFlagInternal;
        nseg = 0;
        D = 0;
      } else if (nrows) {
        uint32_t si = seg_off, pos = det_off;
        for (int cy = cya; cy <= cyb; ++cy) {
          const size_t b0 = ((size_t)e * cg.ncy + cy) * cg.ncx;
          const uint32_t st0 = a.boff[b0 + cxa];
          const uint32_t len = a.boff[b0 + cxb + 1] - st0;
          if (!len) continue;
          s_seg_pos[si] = pos;
          s_seg_src[si] = st0;
          ++si;
          pos += len;
        }
      }
      __syncthreads();

      EmitCtx ecx;
      ecx.s_emit = s_emit;
      ecx.s_count = &s_misc[73];
      ecx.s_cap = (uint32_t)tc.emit_cap;
      ecx.g_emit = a.emits;
      ecx.g_count = a.n_emit;
      ecx.g_cap = a.emit_cap;
      ecx.v_base = (uint32_t)ky0 * (uint32_t)g.nvx + (uint32_t)kx0;
      ecx.nvx = (uint32_t)g.nvx;
      ecx.bx0 = (uint32_t)bx0;
      ecx.by0 = (uint32_t)by0;
      ecx.flags = 0;
      for (uint32_t j = tid; j < D; j += kNT) {
        uint32_t lo = 0, hi = nseg;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (s_seg_pos[mid] <= j) lo = mid; else hi = mid;
        }
        const Det d = a.dets[s_seg_src[lo] + (j - s_seg_pos[lo])];
        const int el = (int)(d.e - e_base);
        if (masked)
          process_det<KX, KY, CB, true>(d, el, s_ox, s_oy, cells, tw_x, tw_y, a.magic,
                                        a.bin_is_one, tc.tx, txty, act, nmin1, pairs, ecx);
        else
          process_det<KX, KY, CB, false>(d, el, s_ox, s_oy, cells, tw_x, tw_y, a.magic,
                                         a.bin_is_one, tc.tx, txty, act, nmin1, pairs, ecx);
      }
      my_flags |= ecx.flags;
      __syncthreads();
    }

    // Flush this tile's emissions with one global atomic, then clear the tile.
    const uint32_t ne_tile = min(s_misc[73], (uint32_t)tc.emit_cap);
    if (ne_tile) {
      if (tid == 0) s_misc[74] = atomicAdd(a.n_emit, ne_tile);
      __syncthreads();
      const uint32_t base = s_misc[74];
      for (uint32_t i = tid; i < ne_tile; i += kNT) {
        if (base + i < a.emit_cap) a.emits[base + i] = s_emit[i]; else my_flags |= kFlagEmitCap;
      }
    }
    for (uint32_t i = tid; i < n_words / 4; i += kNT)
      reinterpret_cast<uint4*>(cells)[i] = make_uint4(0, 0, 0, 0);
    __syncthreads();
  }

  // Pair count and flags: one global atomic per warp.
  for (int o = 16; o > 0; o >>= 1) {
    pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    my_flags |= __shfl_xor_sync(0xffffffffu, my_flags, o);
  }
  if ((tid & 31) == 0) {
    if (pairs) atomicAdd(a.n_pairs, (unsigned long long)pairs);
    if (my_flags) atomicOr(a.flags, my_flags);
  }
}

template <int KX, int KY, int CB>
cudaError_t launch_t(const StackArgs& a, int grid, cudaStream_t s) {
  k_stack<KX, KY, CB><<<grid, kNT, a.tc.smem, s>>>(a);
  note_launch();
  return cudaGetLastError();
}

template <int KX, int KY, int CB>
cudaError_t attr_t(size_t smem) {
  return cudaFuncSetAttribute(k_stack<KX, KY, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

// Supported (KX, KY, CB) instantiations.
#define SAS_STACK_CONFIGS(X) \
  X(4, 1, 8) X(4, 2, 8) X(4, 4, 8) X(8, 2, 8) X(8, 3, 8) \
  X(4, 1, 16) X(4, 2, 16) X(4, 4, 16) X(8, 2, 16) X(8, 3, 16) \
  X(4, 1, 32) X(4, 2, 32) X(4, 4, 32) X(8, 2, 32) X(8, 3, 32)

}  // namespace

bool stack_config_supported(int kx, int ky, int cb) {
#define SAS_CHECK(KX, KY, CB) if (kx == KX && ky == KY && cb == CB) return true;
  SAS_STACK_CONFIGS(SAS_CHECK)
#undef SAS_CHECK
  return false;
}

size_t stack_smem_bytes(const TileCfg& tc) {
  return layout(tc.kx, tc.ky, tc.tx, tc.ty, tc.cb, tc.ec, tc.seg_cap, tc.emit_cap).total;
}

int stack_threads() { return kNT; }

cudaError_t launch_stack(const StackArgs& a, int grid, cudaStream_t s) {
#define SAS_LAUNCH(KX, KY, CB) \
  if (a.tc.kx == KX && a.tc.ky == KY && a.tc.cb == CB) return launch_t<KX, KY, CB>(a, grid, s);
  SAS_STACK_CONFIGS(SAS_LAUNCH)
#undef SAS_LAUNCH
  return cudaErrorInvalidValue;
}

cudaError_t stack_set_smem_attr(int kx, int ky, int cb, size_t smem) {
#define SAS_ATTR(KX, KY, CB) if (kx == KX && ky == KY && cb == CB) return attr_t<KX, KY, CB>(smem);
  SAS_STACK_CONFIGS(SAS_ATTR)
#undef SAS_ATTR
  return cudaErrorInvalidValue;
}

}  // namespace sas
