// Planning of one field's search: counter width, super-bin size, tile sizes,
// velocity blocks, staging capacity and bucket geometry.  Host code only.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "sas_internal.cuh"

namespace sas {

std::mutex g_dev_mu;
DevInfo g_dev[64];

int device_info(int dev, DevInfo* out) {
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (dev < 0 || dev >= 64) return set_error(SAS_ERR_ARG, "device ordinal out of range");
  DevInfo& d = g_dev[dev];
  if (!d.ready) {
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // Keep freed stream-ordered allocations cached in the pool between calls.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_errorf(SAS_ERR_CUDA, "device query: %s", cudaGetErrorString(e));
    d.ready = true;
  }
  *out = d;
  return SAS_OK;
}

uint32_t magic_for(int32_t bin) {  // ceil(2^32 / bin) for bin >= 2
  return (uint32_t)(((uint64_t)1 << 32) / (uint64_t)bin + 1);
}

// (X_max) * (magic * bin - 2^32) < 2^32 makes umulhi(X, magic) == X / bin for X <= X_max.
bool magic_exact(int32_t bin, int64_t x_max) {
  if (bin == 1) return true;
  const uint64_t m = magic_for(bin);
  const uint64_t err = m * (uint64_t)bin - ((uint64_t)1 << 32);
  return (unsigned __int128)x_max * err < ((unsigned __int128)1 << 32);
}

constexpr int kStackThreads = 1024;
constexpr int kSegCap = kStackThreads;  // one (epoch, bucket row) segment per thread
constexpr int kEmitCap = 256;
constexpr int kPeakCap = 1024;  // one counter per thread and batch
constexpr int kMaxEpochChunk = 256;     // staged records carry the epoch in 8 bits

struct Plan {
  TileCfg tc;
  CoarseGeom cg;
  int ky_lo, ky_hi;
};

// Upper bound of |floor(v*dt/TPH) - floor(v'*dt/TPH)| over dt in [0, dT] for
// |v - v'| <= dv_span.
int64_t spread_bound(int64_t dv_span, int64_t dT, int64_t tph) {
  const long double s = (long double)dv_span * (long double)dT / (long double)tph + 2.0L;
  return s > (long double)kLimDomain ? kLimDomain : (int64_t)s;
}

// log P(Poisson(lam) >= k), summed in log space.
double log_poisson_tail(double lam, int k) {
  if (k <= 0) return 0.0;
  if (lam <= 0) return -1e300;
  double lt = -lam + k * std::log(lam) - std::lgamma(k + 1.0), acc = lt, term = lt;
  for (int i = k + 1; i < k + 200; ++i) {
    term += std::log(lam) - std::log((double)i);
    acc = std::max(acc, term) + std::log1p(std::exp(-std::fabs(acc - term)));
    if (term < acc - 40) break;
  }
  return acc;
}

// Super-bin size: the largest s in 1..3 for which uniform noise of the
// catalog's mean density is expected to push few super-bins over n_min across
// the searched lattice -- at most max(4000, pairs / 1e5), each emission costing
// one exact recount.  Larger super-bins mean fewer counters to reset per
// detection-shift but more cells near true movers reach the threshold; measured
// on the DECam-like fields, s = 3 balances the two and s = 4 does not pay.
int choose_superbin(const sas_grid_desc& d, uint64_t n, uint32_t n_min, uint64_t nv) {
  if (n_min < 2) return 1;
  const double bins = (double)d.nbx * d.nby;
  const double lam_bin = (double)n / bins;  // detections per bin over all epochs
  const double pairs = (double)n * (double)nv;  // upper bound of detection-shifts
  const double budget = std::max(4000.0, pairs / 1e5);
  int best = 1;
  for (int s = 2; s <= 3; ++s) {
    if ((int64_t)s * d.bin >= kLimDomain / 4) break;
    const double cells = (double)nv * bins / (s * s);
    const double lt = log_poisson_tail(lam_bin * s * s, (int)n_min);
    if (std::log(cells) + lt < std::log(budget)) best = s;
  }
  return best;
}

int choose_tiles(const sas_grid_desc& d, uint32_t E, uint64_t n, int64_t dT, int64_t tph, int kx,
                 int ky, int cb, int sb, const sas_opts& o, const DevInfo& di, int n_rows,
                 const CoarseGeom* fixed_cg, Plan* p) {
  if (!stack_config_supported(kx, ky, cb))
    return set_errorf(SAS_ERR_ARG, "unsupported tile (kx=%d, ky=%d, counter_bits=%d)", kx, ky, cb);
  TileCfg tc{};
  tc.kx = kx;
  tc.ky = ky;
  tc.cb = cb;
  tc.s = sb;
  tc.nt = kStackThreads;
  tc.seg_cap = kSegCap;
  tc.emit_cap = kEmitCap;
  tc.peak_cap = (o.n_low || o.peaks_only) ? kPeakCap : 0;
  const int64_t budget = (int64_t)di.smem_optin - 1024;  // room for static shared memory
  const int64_t sbin = (int64_t)sb * d.bin;
  // velocity block: keep the union window within ~15% of the tile per axis
  const int64_t step_x = spread_bound(std::llabs((int64_t)d.dvx), dT, tph) - 1;
  const int64_t step_y = spread_bound(std::llabs((int64_t)d.dvy), dT, tph) - 1;
  const double lam1 = (double)n / ((double)E * d.nbx * d.nby);  // per bin per epoch
  // The shifts of one velocity tile may spread by at most 2^23 mpx over the
  // time span, so that staged coordinates fit their 24-bit field.
  if (spread_bound((int64_t)(kx - 1) * std::llabs((int64_t)d.dvx), dT, tph) >= (1 << 23) ||
      spread_bound((int64_t)(ky - 1) * std::llabs((int64_t)d.dvy), dT, tph) >= (1 << 23))
    return set_error(SAS_ERR_RANGE, "lattice step x time span too large (shift spread >= 2^23 mpx)");
  double cells_frac = 0.62;
  // 8 x 8 velocity tiles share each record's column projections over 8 rows;
  // with them, blocks of up to 4 x 4 tiles whose union window stays within
  // ~20 % of the tile per axis measured best (decam_tno and fast_movers).
  const bool tall = kx * ky > 32;
  int bv_cap = tall ? 4 : 8;
  const int64_t win_pct = tall ? 20 : 15;
  for (int iter = 0; iter < 200; ++iter) {
    const int64_t cells_bytes = (int64_t)(budget * cells_frac);
    int side = (int)std::sqrt((double)cells_bytes * 8.0 / ((double)kx * ky * cb));
    side = std::max(4, side & ~3);
    const int dom_x = (int)(((int64_t)d.nbx + sb - 1) / sb + 3) & ~3;
    const int dom_y = (int)(((int64_t)d.nby + sb - 1) / sb + 3) & ~3;
    tc.tx = o.tile_bx ? (int)o.tile_bx : std::min(side, dom_x);
    tc.ty = o.tile_by ? (int)o.tile_by : std::min(side, dom_y);
    if (!o.tile_bx && tc.ty < side)
      tc.tx = std::min((int)(cells_bytes * 8 / ((int64_t)kx * ky * cb * tc.ty)) & ~3, dom_x);
    if (!o.tile_by && tc.tx < side && tc.ty == side)
      tc.ty = std::min((int)(cells_bytes * 8 / ((int64_t)kx * ky * cb * tc.tx)) & ~3, dom_y);
    tc.tx = std::max(tc.tx, 4);
    tc.ty = std::max(tc.ty, 4);
    if (tc.tx >= 4096 || tc.ty >= 4096)  // the kernel packs tile positions in 12 bits
      return set_error(SAS_ERR_ARG, "tile_bx and tile_by must be below 4096");
    if (((int64_t)tc.tx * tc.ty) % 4 != 0)
      return set_error(SAS_ERR_ARG, "tile_bx * tile_by must be a multiple of 4");
    const int64_t tw = (int64_t)tc.tx * sbin, th = (int64_t)tc.ty * sbin;
    int bvx = (int)std::max<int64_t>(1, std::min<int64_t>(bv_cap, (tw * win_pct / 100) / std::max<int64_t>(1, step_x * kx)));
    int bvy = (int)std::max<int64_t>(1, std::min<int64_t>(bv_cap, (th * win_pct / 100) / std::max<int64_t>(1, step_y * ky)));
    if (o.velocity_block) bvx = bvy = (int)std::min<uint32_t>(o.velocity_block, 8);
    // enough work units to fill the GPU: shrink the velocity block, then the tile
    const uint64_t units = (uint64_t)div_ceil_u32(d.nvx, kx * bvx) * div_ceil_u32(n_rows, ky * bvy) *
                           div_ceil_u32(d.nbx, tc.tx * sb) * div_ceil_u32(d.nby, tc.ty * sb);
    if (units < 2ull * di.sms && !o.velocity_block && std::max(bvx, bvy) > 1) {
      bv_cap = std::max(bvx, bvy) / 2;
      continue;
    }
    if (units < 2ull * di.sms && !(o.tile_bx || o.tile_by) && std::min(tc.tx, tc.ty) > 16) {
      cells_frac *= 0.7;
      continue;
    }
    tc.bvx = bvx;
    tc.bvy = bvy;
    const int64_t spread_x = spread_bound((int64_t)(bvx * kx - 1) * std::llabs((int64_t)d.dvx), dT, tph);
    const int64_t spread_y = spread_bound((int64_t)(bvy * ky - 1) * std::llabs((int64_t)d.dvy), dT, tph);
    if (tw + spread_x >= (1 << 24) || th + spread_y >= ((int64_t)1 << 30)) {
      if (o.tile_bx || o.tile_by) return set_error(SAS_ERR_ARG, "tile too wide for staged records");
      cells_frac *= 0.8;
      continue;
    }
    if (!magic_exact((int32_t)std::min<int64_t>(sbin, INT32_MAX), std::max(tw, th) - 1)) {
      if (o.tile_bx || o.tile_by) return set_error(SAS_ERR_RANGE, "tile too large for exact division");
      cells_frac *= 0.8;
      continue;
    }
    // coarse bucket cell and rows per epoch window
    CoarseGeom cg{};
    if (fixed_cg) {
      cg = *fixed_cg;
    } else {
      int64_t cell = o.coarse_bins > 0 ? (int64_t)o.coarse_bins * d.bin : (th + spread_y + 5) / 6;
      cg.cell = (int32_t)std::max<int64_t>(1, std::min<int64_t>(cell, kLimDomain));
    }
    const int64_t rows = (th + spread_y) / cg.cell + 2;
    if (rows > kSegCap) {
      if (fixed_cg) return set_error(SAS_ERR_INTERNAL, "segment rows exceed capacity");
      return set_errorf(SAS_ERR_ARG, "coarse_bins too small for this tile (%lld rows)", (long long)rows);
    }
    tc.rows = (int)rows;
    tc.ec = (int)std::min<int64_t>(std::min<int64_t>(E, kMaxEpochChunk), kSegCap / rows);
    if (tc.ec < 1) tc.ec = 1;
    // staged records: what the union window holds on average, with headroom
    const double win = (double)(tw + spread_x) / d.bin * (double)(th + spread_y) / d.bin;
    const double est = lam1 * std::min<uint32_t>(E, tc.ec) * win;
    tc.scap = 0;
    const int64_t rest = budget - (int64_t)stack_smem_bytes(tc);
    const int64_t want = (int64_t)(1.5 * est) + 1024;
    if (rest < 8 * 256) {
      if (o.tile_bx || o.tile_by) return set_error(SAS_ERR_ARG, "tile does not fit in shared memory");
      cells_frac *= 0.9;
      continue;
    }
    if (rest / 8 < want && cells_frac > 0.15 && !(o.tile_bx || o.tile_by)) {
      cells_frac *= 0.93;  // give the staging area more room
      continue;
    }
    tc.scap = (int)std::min<int64_t>(rest / 8, std::max<int64_t>(want, 4096));
    tc.smem = stack_smem_bytes(tc);
    if ((int64_t)tc.smem > budget) {
      cells_frac *= 0.95;
      continue;
    }
    p->tc = tc;
    p->cg = cg;
    return SAS_OK;
  }
  return set_error(SAS_ERR_INTERNAL, "could not size the stack tile");
}



int64_t ceil_div64(int64_t a, int64_t b) { return -floor_div64(-a, b); }

int plan_field(const sas_grid_desc& d, uint64_t n, uint32_t E, const int64_t* t, int64_t tph,
               uint32_t n_min, uint64_t v_begin, uint64_t v_end, const sas_opts& o,
               const DevInfo& di, FieldPlan* fp) {
  int64_t tmin = t[0], tmax = t[0];
  for (uint32_t e = 1; e < E; ++e) {
    tmin = std::min(tmin, t[e]);
    tmax = std::max(tmax, t[e]);
  }
  const int64_t dT = tmax - tmin;
  // A CB-bit counter holds thresholds up to 2^(CB-1) (it starts at 2^(CB-1) - n_min).
  int cb = (int)o.counter_bits;
  if (cb == 0) cb = n_min <= 128 ? 8 : (n_min <= 32768 ? 16 : 32);
  if (cb != 8 && cb != 16 && cb != 32) return set_error(SAS_ERR_ARG, "counter_bits must be 8, 16 or 32");
  if (cb == 8 && n_min > 128) cb = 16;
  if (cb == 16 && n_min > 32768) cb = 32;
  const int kx = o.tile_kx ? (int)o.tile_kx : 8;
  // 8 x 8 tiles for 8-bit counters; wider counters leave 8 x 8 tiles too little area
  int ky = o.tile_ky ? (int)o.tile_ky : (cb == 8 ? 8 : 4);
  if (o.superbin > 4) return set_error(SAS_ERR_ARG, "superbin must be 0..4");
  const int sb = o.superbin ? (int)o.superbin : choose_superbin(d, n, n_min, v_end - v_begin);
  const int n_rows = (int)((v_end - 1) / d.nvx - v_begin / d.nvx + 1);
  Plan plan;
  if (int rc = choose_tiles(d, E, n, dT, tph, kx, ky, cb, sb, o, di, n_rows, nullptr, &plan)) {
    // the default 8 x 8 tile can exceed the staged coordinates' shift spread
    // where 8 x 4 does not: fall back to it unless the caller chose the tile
    if (o.tile_ky || ky != 8) return rc;
    ky = 4;
    if (int rc2 = choose_tiles(d, E, n, dT, tph, kx, ky, cb, sb, o, di, n_rows, nullptr, &plan)) return rc2;
  }
  // Bucket grid: every detection that can project into the domain for some
  // lattice velocity and some dt in [0, dT] lies inside it.
  const int64_t vxa = d.vx0, vxb = (int64_t)d.vx0 + (int64_t)(d.nvx - 1) * d.dvx;
  const int64_t vya = d.vy0, vyb = (int64_t)d.vy0 + (int64_t)(d.nvy - 1) * d.dvy;
  auto clampd = [](int64_t v) { return std::max(-kLimDomain, std::min(kLimDomain, v)); };
  const int64_t sx_lo = clampd(floor_div64(std::min<int64_t>(std::min(vxa, vxb), 0) * dT, tph));
  const int64_t sx_hi = clampd(ceil_div64(std::max<int64_t>(std::max(vxa, vxb), 0) * dT, tph));
  const int64_t sy_lo = clampd(floor_div64(std::min<int64_t>(std::min(vya, vyb), 0) * dT, tph));
  const int64_t sy_hi = clampd(ceil_div64(std::max<int64_t>(std::max(vya, vyb), 0) * dT, tph));
  CoarseGeom cg = plan.cg;
  for (;;) {
    cg.gx0 = (int32_t)(d.x_min + sx_lo);
    cg.gy0 = (int32_t)(d.y_min + sy_lo);
    cg.ncx = (int32_t)ceil_div64((int64_t)d.nbx * d.bin + (sx_hi - sx_lo) + 1, cg.cell);
    cg.ncy = (int32_t)ceil_div64((int64_t)d.nby * d.bin + (sy_hi - sy_lo) + 1, cg.cell);
    if ((uint64_t)E * cg.ncx * cg.ncy <= ((uint64_t)1 << 27)) break;
    if (cg.cell >= kLimDomain / 2) break;
    cg.cell *= 2;  // fewer, larger buckets
  }
  {  // the bucket cell may have grown: recompute the per-chunk epoch count
    Plan p2;
    if (int rc = choose_tiles(d, E, n, dT, tph, kx, ky, cb, sb, o, di, n_rows, &cg, &p2)) return rc;
    plan.tc = p2.tc;
  }
  fp->tc = plan.tc;
  fp->cg = cg;
  fp->kx = kx;
  fp->ky = ky;
  fp->cb = cb;
  fp->sb = sb;
  fp->dT = dT;
  fp->n_rows = n_rows;
  fp->ky_lo = (int)(v_begin / d.nvx);
  fp->ky_hi = (int)((v_end - 1) / d.nvx);
  fp->nb = (uint64_t)E * cg.ncx * cg.ncy;
  SearchGeom& g = fp->g;
  g = SearchGeom{};
  g.vx0 = d.vx0; g.vy0 = d.vy0; g.dvx = d.dvx; g.dvy = d.dvy;
  g.nvx = (int32_t)d.nvx; g.nvy = (int32_t)d.nvy;
  g.smin = d.speed_min; g.smax = d.speed_max;
  g.x_min = d.x_min; g.y_min = d.y_min;
  g.nbx = (int32_t)d.nbx; g.nby = (int32_t)d.nby; g.bin = d.bin;
  g.E = E; g.tph = tph;
  g.v_begin = v_begin; g.v_end = v_end;
  return SAS_OK;
}

int replan_wider(const sas_grid_desc& d, uint64_t n, uint32_t n_min, const sas_opts& o,
                 const DevInfo& di, FieldPlan* fp) {
  (void)n_min;
  if (fp->cb == 32) return set_error(SAS_ERR_INTERNAL, "32-bit counter wrapped");
  const int wider = fp->cb * 2;
  Plan p2;
  if (int rc = choose_tiles(d, fp->g.E, n, fp->dT, fp->g.tph, fp->kx, fp->ky, wider, fp->sb, o, di,
                            fp->n_rows, &fp->cg, &p2))
    return rc;
  fp->tc = p2.tc;
  fp->cb = wider;
  return SAS_OK;
}

void fill_stack_args(const FieldPlan& fp, uint32_t n_min, uint32_t n_low, uint32_t peaks_only, StackArgs* sa) {
  const TileCfg& tc = fp.tc;
  sa->g = fp.g;
  sa->cg = fp.cg;
  sa->tc = tc;
  const int64_t sbin = (int64_t)tc.s * fp.g.bin;
  sa->magic = sbin >= 2 ? magic_for((int32_t)sbin) : 0u;
  sa->bin_is_one = sbin == 1;
  // The projections of the P lattice columns that share a counter word differ
  // by at most spread_bound((P-1)|dvx|); below one super-bin they fall into at
  // most two adjacent super-bins, so the stack kernel needs two reductions per
  // word (one per run of equal columns) instead of P.
  const int per_word = 32 / tc.cb;
  sa->merge = per_word >= 2 &&
              spread_bound((int64_t)(per_word - 1) * std::llabs((int64_t)fp.g.dvx), fp.dT, fp.g.tph) < sbin;
  sa->n_min = n_min;
  sa->n_low = n_low && n_low < n_min ? n_low : n_min;
  sa->select = peaks_only ? kSelectPeaks : (sa->n_low < n_min ? kSelectPlainAndPeaks : kSelectAll);
  sa->kx_lo = 0;
  sa->ky_lo = fp.ky_lo;
  sa->nvt_x = (int)div_ceil_u32((uint32_t)fp.g.nvx, tc.kx * tc.bvx);
  sa->nvt_y = (int)div_ceil_u32((uint32_t)(fp.ky_hi - fp.ky_lo + 1), tc.ky * tc.bvy);
  sa->nst_x = (int)div_ceil_u32((uint32_t)fp.g.nbx, tc.tx * tc.s);
  sa->nst_y = (int)div_ceil_u32((uint32_t)fp.g.nby, tc.ty * tc.s);
  sa->n_tiles = (uint64_t)sa->nvt_x * sa->nvt_y * sa->nst_x * sa->nst_y;
}

}  // namespace sas
