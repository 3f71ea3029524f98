// C ABI of the shift-and-stack library: validation, planning and the launch
// sequence of one search (Sec. 2.1 steps 1-3).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sas_internal.cuh"

using namespace sas;

struct sas_grid {
  sas_grid_desc d;
  // emission count of the previous search on this grid: sizes the next
  // emission list so that repeated searches do not need an exact rerun
  std::atomic<uint32_t> emit_hint{0};
};

struct sas_result {
  int device;
  sas_candidate* d_cands;
  uint32_t* d_ids;
  sas_result_info info;
  // The search's bucketed catalog, per-epoch counts and shift tables, kept so
  // that stamps can be cut from the same search (sas_stamps).
  Det* d_dets;
  uint32_t* d_boff;
  uint32_t* d_ecount;
  int32_t* d_sxt;
  int32_t* d_syt;
  int64_t* d_dt;      // per-epoch time minus t0, ticks
  SearchGeom g;
  CoarseGeom cg;
  uint64_t n_det;     // catalog size (detection ids are < n_det)
  uint32_t n_min;     // the search's threshold (the score threshold when weighted)
  int complete;       // every cell >= n_min is in the list (no top-K cut)
  int weighted;       // counts are weighted scores
};

namespace {
thread_local std::string g_err;
}  // namespace

namespace sas {
std::atomic<unsigned long long> g_launches{0};
void note_launch(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int set_errorf(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
}  // namespace sas

namespace {

template <typename... Args>
int fail(int code, const char* fmt, Args... args) {
  return set_errorf(code, fmt, args...);
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

// Stream-ordered scratch, released when the search returns.
struct Scratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), s);
    if (e != cudaSuccess) return e;
    ptrs.push_back(q);
    *p = static_cast<T*>(q);
    return cudaSuccess;
  }
};

bool fits_i32(int64_t v) { return v >= INT32_MIN && v <= INT32_MAX; }

// Opt-in host-side tracing (environment variable SAS_TRACE=1): microseconds
// since the start of the call at each phase boundary, on stderr.
struct Tracer {
  bool on;
  std::chrono::steady_clock::time_point t0;
  Tracer() : on(std::getenv("SAS_TRACE") != nullptr), t0(std::chrono::steady_clock::now()) {}
  void mark(const char* what) const {
    if (!on) return;
    const double us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    std::fprintf(stderr, "[sas] %9.1f us  %s\n", us, what);
  }
};

}  // namespace

namespace sas {
CandView result_view(const sas_result* r) {
  CandView v;
  v.cands = r->d_cands;
  v.n = r->info.n_candidates;
  v.g = r->g;
  v.cg = r->cg;
  v.dets = r->d_dets;
  v.boff = r->d_boff;
  v.ecount = r->d_ecount;
  v.sxt = r->d_sxt;
  v.syt = r->d_syt;
  v.ids = r->d_ids;
  v.n_det = r->n_det;
  return v;
}
}  // namespace sas

extern "C" {

const char* sas_version(void) { return "sas-gb300 0.1 (sm_103a)"; }
int sas_abi_version(void) { return SAS_ABI_VERSION; }
uint64_t sas_kernel_launches(void) { return sas::g_launches.load(); }
const char* sas_last_error(void) { return g_err.c_str(); }

int sas_create_grid(const sas_grid_desc* desc, sas_grid** out) {
  if (!desc || !out) return fail(SAS_ERR_ARG, "null argument");
  const sas_grid_desc& d = *desc;
  if (d.nvx < 1 || d.nvy < 1 || d.nbx < 1 || d.nby < 1 || d.bin < 1)
    return fail(SAS_ERR_ARG, "lattice and domain sizes and the bin must be >= 1");
  if (d.speed_min < 0 || d.speed_max < d.speed_min)
    return fail(SAS_ERR_ARG, "need 0 <= speed_min <= speed_max");
  if ((uint64_t)d.nvx * d.nvy >= ((uint64_t)1 << 31))
    return fail(SAS_ERR_RANGE, "nvx*nvy must be < 2^31");
  if (std::llabs((int64_t)d.x_min) >= kLimDomain || std::llabs((int64_t)d.y_min) >= kLimDomain)
    return fail(SAS_ERR_RANGE, "|x_min|, |y_min| must be < 2^28");
  if ((int64_t)d.nbx * d.bin >= kLimDomain || (int64_t)d.nby * d.bin >= kLimDomain)
    return fail(SAS_ERR_RANGE, "nbx*bin and nby*bin must be < 2^28");
  if (!fits_i32((int64_t)d.vx0 + (int64_t)(d.nvx - 1) * d.dvx) ||
      !fits_i32((int64_t)d.vy0 + (int64_t)(d.nvy - 1) * d.dvy))
    return fail(SAS_ERR_RANGE, "lattice velocities must fit in int32");
  sas_grid* g = new (std::nothrow) sas_grid;
  if (!g) return fail(SAS_ERR_OOM, "host allocation");
  g->d = d;
  g->emit_hint.store(0);
  *out = g;
  return SAS_OK;
}

void sas_destroy_grid(sas_grid* grid) { delete grid; }

int sas_grid_get_desc(const sas_grid* grid, sas_grid_desc* desc) {
  if (!grid || !desc) return fail(SAS_ERR_ARG, "null argument");
  *desc = grid->d;
  return SAS_OK;
}

namespace {

// The search (Sec. 2.1 steps 1-3); with weights (one uint8 per detection, in
// host or device memory like the catalog) cells are scored by the sum over
// epochs of their largest weight and n_min is the score threshold.
int stack_impl(const sas_grid* grid, const sas_catalog* cat, const uint8_t* weights, uint32_t n_min,
               const sas_opts* opts, void* stream, sas_result** out) {
  if (!grid || !cat || !out) return fail(SAS_ERR_ARG, "null argument");
  const Tracer tr;
  const sas_grid_desc& d = grid->d;
  const uint32_t E = cat->n_epochs;
  const uint64_t n = cat->n;
  if (n_min < 1) return fail(SAS_ERR_ARG, "n_min must be >= 1");
  if (E < 1 || E > SAS_MAX_EPOCHS) return fail(SAS_ERR_RANGE, "n_epochs must be in [1, %d]", SAS_MAX_EPOCHS);
  if (!cat->t) return fail(SAS_ERR_ARG, "null epoch time table");
  if (cat->ticks_per_hour <= 0) return fail(SAS_ERR_ARG, "ticks_per_hour must be > 0");
  if (n >= ((uint64_t)1 << 31)) return fail(SAS_ERR_RANGE, "n must be < 2^31");
  if (n > 0 && (!cat->x || !cat->y || !cat->epoch)) return fail(SAS_ERR_ARG, "null catalog array");
  sas_opts o{};
  if (opts) o = *opts;
  const uint64_t nv = (uint64_t)d.nvx * d.nvy;
  uint64_t v_begin = o.v_begin, v_end = o.v_end;
  if (v_begin == 0 && v_end == 0) v_end = nv;
  if (v_begin > v_end || v_end > nv) return fail(SAS_ERR_ARG, "bad lattice index range");
  int64_t tmin = cat->t[0], tmax = cat->t[0];
  for (uint32_t e = 1; e < E; ++e) {
    tmin = std::min(tmin, cat->t[e]);
    tmax = std::max(tmax, cat->t[e]);
  }
  if ((__int128)tmax - tmin >= ((__int128)1 << 32)) return fail(SAS_ERR_RANGE, "time span must be < 2^32 ticks");
  const int64_t tph = cat->ticks_per_hour;

  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
  DevInfo di;
  if (int rc = device_info(dev, &di)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_min > (1u << 31)) return fail(SAS_ERR_ARG, "n_min must be <= 2^31");
  if (o.n_low > n_min) return fail(SAS_ERR_ARG, "n_low %u is above n_min %u", o.n_low, n_min);
  if ((o.n_low || o.peaks_only) && weights)
    return fail(SAS_ERR_ARG, "n_low and peaks_only are not supported by the weighted search");
  if (o.peaks_only > 1) return fail(SAS_ERR_ARG, "peaks_only must be 0 or 1");
  const uint32_t n_low = o.n_low ? o.n_low : n_min;

  sas_result* res = new (std::nothrow) sas_result;
  if (!res) return fail(SAS_ERR_OOM, "host allocation");
  memset(res, 0, sizeof(*res));
  res->device = dev;
  res->n_det = n;
  res->n_min = n_min;
  res->info.n_low = n_low;
  res->info.peaks_only = o.peaks_only;

  if (n == 0 || v_begin == v_end) {
    res->info.t0 = 0;
    res->complete = 1;
    *out = res;
    return SAS_OK;
  }

  res->weighted = weights != nullptr;
  if (weights && o.superbin == 0) {
    // the super-bin heuristic models unit increments: give it the distinct-epoch
    // count that a score of n_min needs at the largest weight
    uint32_t wmax = 0;
    if (cat->on_device) {
      std::vector<uint8_t> hw(n);
      ce = cudaMemcpy(hw.data(), weights, n, cudaMemcpyDeviceToHost);
      if (ce != cudaSuccess) {
        delete res;
        return cuda_fail(ce, "copy weights");
      }
      for (uint8_t v : hw) wmax = std::max<uint32_t>(wmax, v);
    } else {
      for (uint64_t i = 0; i < n; ++i) wmax = std::max<uint32_t>(wmax, weights[i]);
    }
    o.superbin = (uint32_t)choose_superbin(d, n, (n_min + std::max(wmax, 1u) - 1) / std::max(wmax, 1u), v_end - v_begin);
  }

  FieldPlan plan;
  if (int rc = plan_field(d, n, E, cat->t, tph, n_min, v_begin, v_end, o, di, &plan)) {
    delete res;
    return rc;
  }
  const CoarseGeom& cg = plan.cg;
  const uint64_t nb = plan.nb;
  const SearchGeom& g = plan.g;
  tr.mark("planned");

  cudaEvent_t ev0, ev1, evs0, evs1, evc0, evc1;
  cudaEventCreate(&ev0); cudaEventCreate(&ev1); cudaEventCreate(&evs0); cudaEventCreate(&evs1);
  cudaEventCreate(&evc0); cudaEventCreate(&evc1);
  struct EvGuard {
    cudaEvent_t e[6];
    ~EvGuard() { for (cudaEvent_t x : e) cudaEventDestroy(x); }
  } evg{{ev0, ev1, evs0, evs1, evc0, evc1}};
  cudaEventRecord(ev0, s);

  int rc = SAS_OK;
  {
    Scratch sc(s);
#define CK(expr, where)                          \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) {                     \
      rc = cuda_fail(e_, where);                 \
      goto done;                                 \
    }                                            \
  } while (0)
    const int32_t* dx = cat->x;
    const int32_t* dy = cat->y;
    const uint16_t* dep = cat->epoch;
    int32_t *hx = nullptr, *hy = nullptr;
    uint16_t* hep = nullptr;
    int64_t *d_t = nullptr, *d_dt = nullptr, *d_t0 = nullptr;  // d_dt is kept by the result
    const uint8_t* d_w = nullptr;
    uint8_t* hw_dev = nullptr;
    uint32_t *d_ecount = nullptr, *d_bcount = nullptr, *d_boff = nullptr, *d_cursor = nullptr,
             *d_bof = nullptr, *d_scan = nullptr;
    Det* d_dets = nullptr;
    int32_t *d_sxt = nullptr, *d_syt = nullptr;
    uint32_t* d_small = nullptr;  // [0] flags [1] n_emit [2] n_valid
    unsigned long long* d_small64 = nullptr;  // [0] pairs [1] tile counter [2] raw total
    Emit* d_emits = nullptr;
    Key* d_keys = nullptr;
    uint32_t* d_raw = nullptr;
    unsigned long long *d_idoff = nullptr, *d_scan64 = nullptr;
    uint32_t* d_ids_tmp = nullptr;
    const uint32_t hint = grid->emit_hint.load(std::memory_order_relaxed);
    uint32_t emit_cap = (uint32_t)std::min<uint64_t>(
        std::max<uint64_t>({(uint64_t)1 << 16, 2 * n, (uint64_t)hint + hint / 4 + 1024}), (uint64_t)1 << 26);
    uint32_t h_small[3] = {0, 0, 0};
    unsigned long long h_small64[4] = {0, 0, 0, 0};
    int64_t h_t0 = 0;
    uint32_t n_out = 0;
    unsigned long long n_ids = 0;
    StackArgs sa{};

    if (!cat->on_device) {
      CK(sc.alloc(&hx, n), "alloc x");
      CK(sc.alloc(&hy, n), "alloc y");
      CK(sc.alloc(&hep, n), "alloc epoch");
      CK(cudaMemcpyAsync(hx, cat->x, n * 4, cudaMemcpyHostToDevice, s), "copy x");
      CK(cudaMemcpyAsync(hy, cat->y, n * 4, cudaMemcpyHostToDevice, s), "copy y");
      CK(cudaMemcpyAsync(hep, cat->epoch, n * 2, cudaMemcpyHostToDevice, s), "copy epoch");
      dx = hx; dy = hy; dep = hep;
    }
    if (weights) {
      if (cat->on_device) {
        d_w = weights;
      } else {
        CK(sc.alloc(&hw_dev, n), "alloc weights");
        CK(cudaMemcpyAsync(hw_dev, weights, n, cudaMemcpyHostToDevice, s), "copy weights");
        d_w = hw_dev;
      }
    }
    CK(sc.alloc(&d_t, E), "alloc t");
    CK(cudaMallocAsync((void**)&d_dt, (size_t)E * 8, s), "alloc dt");
    res->d_dt = d_dt;
    CK(sc.alloc(&d_t0, 1), "alloc t0");
    CK(cudaMemcpyAsync(d_t, cat->t, E * 8, cudaMemcpyHostToDevice, s), "copy t");
    CK(cudaMallocAsync((void**)&d_ecount, (size_t)E * 4, s), "alloc ecount");
    res->d_ecount = d_ecount;
    // nb grid buckets plus one overflow bucket (detections outside the grid)
    CK(sc.alloc(&d_bcount, nb + 1), "alloc bucket counts");
    CK(cudaMallocAsync((void**)&d_boff, (nb + 2) * 4, s), "alloc bucket offsets");
    res->d_boff = d_boff;
    CK(sc.alloc(&d_cursor, nb + 1), "alloc cursor");
    CK(sc.alloc(&d_scan, scan_scratch_elems(nb + 1)), "alloc scan scratch");
    CK(sc.alloc(&d_bof, n), "alloc bucket_of");
    CK(cudaMallocAsync((void**)&d_dets, n * sizeof(Det), s), "alloc dets");
    res->d_dets = d_dets;
    CK(cudaMallocAsync((void**)&d_sxt, (size_t)d.nvx * E * 4, s), "alloc sx table");
    res->d_sxt = d_sxt;
    CK(cudaMallocAsync((void**)&d_syt, (size_t)d.nvy * E * 4, s), "alloc sy table");
    res->d_syt = d_syt;
    res->g = g;
    res->cg = cg;
    CK(sc.alloc(&d_small, 4), "alloc counters");
    CK(sc.alloc(&d_small64, 4), "alloc counters64");
    CK(cudaMemsetAsync(d_ecount, 0, E * 4, s), "memset");
    CK(cudaMemsetAsync(d_bcount, 0, (nb + 1) * 4, s), "memset");
    CK(cudaMemsetAsync(d_small, 0, 16, s), "memset");
    CK(cudaMemsetAsync(d_small64, 0, 32, s), "memset");
    tr.mark("allocated");

    // a1-a3: ingest and validate, bucket, reference epoch, shift tables
    CK(launch_ingest(dx, dy, dep, n, E, cg, d_bcount, d_ecount, d_bof, &d_small[0], s), "ingest");
    CK(launch_scan_u32(d_bcount, d_boff, nb + 1, d_scan, s), "bucket scan");
    CK(cudaMemcpyAsync(d_cursor, d_boff, (nb + 1) * 4, cudaMemcpyDeviceToDevice, s), "cursor");
    CK(launch_scatter(dx, dy, dep, n, d_bof, d_cursor, d_dets, s), "scatter");
    CK(launch_epoch_setup(E, d_t, d_ecount, d_dt, d_t0, s), "epoch setup");
    CK(launch_shift_tables(g, d_dt, d_ecount, d_sxt, d_syt, &d_small[0], s), "shift tables");
    tr.mark("prep launched");

    // a4-a6: the stack kernel; reruns (exact) with wider counters if one wrapped
    // or with a longer emission list if it overflowed.
    for (int attempt = 0;; ++attempt) {
      const TileCfg& tc = plan.tc;
      CK(sc.alloc(&d_emits, emit_cap), "alloc emissions");
      CK(stack_set_smem_attr(tc.kx, tc.ky, tc.cb, tc.smem), "smem attribute");
      fill_stack_args(plan, n_min, n_low, o.peaks_only, &sa);
      sa.w = d_w;
      sa.dets = d_dets;
      sa.boff = d_boff;
      sa.ecount = d_ecount;
      sa.sxt = d_sxt;
      sa.syt = d_syt;
      sa.emits = d_emits;
      sa.emit_cap = emit_cap;
      sa.n_emit = &d_small[1];
      sa.n_pairs = &d_small64[0];
      sa.balance = &d_small64[3];
      sa.flags = &d_small[0];
      sa.tile_counter = &d_small64[1];
      CK(cudaMemsetAsync(&d_small[1], 0, 4, s), "memset");
      CK(cudaMemsetAsync(d_small64, 0, 16, s), "memset");
      CK(cudaMemsetAsync(&d_small64[3], 0, 8, s), "memset");
      const int grid_sz = (int)std::min<uint64_t>((uint64_t)di.sms, std::max<uint64_t>(sa.n_tiles, 1));
      cudaEventRecord(evs0, s);
      tr.mark("stack configured");
      CK(launch_stack(sa, grid_sz, s), "stack kernel");
      cudaEventRecord(evs1, s);
      tr.mark("stack launched");
      CK(cudaMemcpyAsync(h_small, d_small, 12, cudaMemcpyDeviceToHost, s), "read counters");
      CK(cudaMemcpyAsync(h_small64, d_small64, 32, cudaMemcpyDeviceToHost, s), "read counters");
      CK(cudaMemcpyAsync(&h_t0, d_t0, 8, cudaMemcpyDeviceToHost, s), "read t0");
      CK(cudaStreamSynchronize(s), "stack sync");
      tr.mark("stack done");
      if (h_small[0] & kFlagEpoch) { rc = fail(SAS_ERR_RANGE, "an epoch index is >= n_epochs"); goto done; }
      if (h_small[0] & kFlagPos) { rc = fail(SAS_ERR_RANGE, "a detection has |x| or |y| >= 2^29"); goto done; }
      if (h_small[0] & kFlagShift) { rc = fail(SAS_ERR_RANGE, "a shift |v*(t-t0)/TPH| >= 2^28"); goto done; }
      if (h_small[0] & kFlagInternal) { rc = fail(SAS_ERR_INTERNAL, "stack kernel invariant"); goto done; }
      if (attempt >= 4) { rc = fail(SAS_ERR_INTERNAL, "stack kernel did not converge"); goto done; }
      if ((h_small[0] & kFlagCounter) || h_small64[3] != 0) {  // a counter wrapped
        CK(cudaMemsetAsync(&d_small[0], 0, 4, s), "memset");
        if (int r2 = replan_wider(d, n, n_min, o, di, &plan)) { rc = r2; goto done; }
        continue;
      }
      if (h_small[1] > emit_cap || (h_small[0] & kFlagEmitCap)) {
        if (h_small[1] >= (1u << 28)) {
          rc = fail(SAS_ERR_OOM, "more than 2^28 cells reach the threshold; raise n_min");
          goto done;
        }
        CK(cudaMemsetAsync(&d_small[0], 0, 4, s), "memset");
        emit_cap = h_small[1] + h_small[1] / 4 + 1024;
        continue;
      }
      break;
    }
    {
      const uint32_t n_emit = h_small[1];
      const_cast<sas_grid*>(grid)->emit_hint.store(n_emit, std::memory_order_relaxed);
      const uint64_t n_keys = (uint64_t)n_emit * plan.tc.s * plan.tc.s;
      if (n_keys >= (1ull << 31)) { rc = fail(SAS_ERR_OOM, "too many candidate bins; raise n_min"); goto done; }
      CK(sc.alloc(&d_keys, n_keys), "alloc keys");
      // a5/a7: exact distinct and raw counts of every bin of the emitted super-bins
      cudaEventRecord(evc0, s);
      CK(launch_cell_count(d_emits, n_emit, plan.tc.s, g, cg, d_dets, d_boff, d_ecount, d_sxt,
                           d_syt, n_min, sa.n_low, d_keys, &d_small[2], &d_small64[2], d_w, s), "cell count");
      CK(cudaMemcpyAsync(&h_small[2], &d_small[2], 4, cudaMemcpyDeviceToHost, s), "read n_valid");
      CK(cudaMemcpyAsync(&h_small64[2], &d_small64[2], 8, cudaMemcpyDeviceToHost, s), "read raw");
      CK(cudaStreamSynchronize(s), "count sync");
      tr.mark("counts done");
      {  // a8: total order of the valid keys
        const uint32_t n_valid = h_small[2];
        uint32_t n_pad = 1;
        while (n_pad < n_valid) n_pad <<= 1;
        Key* sort_buf = d_keys;
        if (n_pad > n_keys) {
          CK(sc.alloc(&sort_buf, n_pad), "alloc sort buffer");
          CK(cudaMemcpyAsync(sort_buf, d_keys, (size_t)n_valid * sizeof(Key), cudaMemcpyDeviceToDevice, s), "copy keys");
        }
        CK(launch_sort_keys(sort_buf, n_valid, n_pad, s), "sort");
        d_keys = sort_buf;
      }
      cudaEventRecord(evc1, s);
      n_out = h_small[2];
      if (o.max_candidates > 0 && n_out > o.max_candidates) n_out = (uint32_t)o.max_candidates;
      const uint64_t id_cap = std::max<uint64_t>(h_small64[2], 1);
      CK(sc.alloc(&d_raw, n_out), "alloc raw");
      CK(sc.alloc(&d_idoff, (size_t)n_out + 1), "alloc id offsets");
      CK(sc.alloc(&d_scan64, scan_scratch_elems(n_out)), "alloc scan scratch");
      CK(sc.alloc(&d_ids_tmp, id_cap), "alloc ids");
      CK(cudaMallocAsync((void**)&res->d_ids, id_cap * 4, s), "alloc result ids");
      CK(cudaMallocAsync((void**)&res->d_cands, std::max<size_t>(n_out, 1) * sizeof(sas_candidate), s),
         "alloc result candidates");
      // a7: contributing ids, ascending per candidate
      CK(launch_key_raw(d_keys, n_out, d_raw, s), "raw");
      CK(launch_scan_u32_to_u64(d_raw, d_idoff, n_out, d_scan64, s), "id offsets");
      CK(launch_gather_ids(d_keys, n_out, d_idoff, g, cg, d_dets, d_boff, d_ecount, d_sxt, d_syt,
                           d_ids_tmp, res->d_ids, &d_small[0], s), "gather ids");
      CK(launch_write_candidates(d_keys, n_out, d_idoff, res->d_cands, s), "write candidates");
      CK(cudaMemcpyAsync(&n_ids, &d_idoff[n_out], 8, cudaMemcpyDeviceToHost, s), "read n_ids");
      CK(cudaMemcpyAsync(&h_small[0], &d_small[0], 4, cudaMemcpyDeviceToHost, s), "read flags");
      cudaEventRecord(ev1, s);
      CK(cudaStreamSynchronize(s), "final sync");
      tr.mark("ids done");
      if (h_small[0] & kFlagInternal) { rc = fail(SAS_ERR_INTERNAL, "id gather invariant"); goto done; }
      res->info.n_candidates = n_out;
      res->complete = n_out == h_small[2];
      res->info.n_ids = n_ids;
      res->info.n_pairs = h_small64[0];
      res->info.n_emitted = n_emit;
      res->info.t0 = h_t0;
      res->info.counter_bits = (uint32_t)plan.tc.cb;
      res->info.tile_kx = (uint32_t)plan.tc.kx;
      res->info.tile_ky = (uint32_t)plan.tc.ky;
      res->info.tile_bx = (uint32_t)plan.tc.tx;
      res->info.tile_by = (uint32_t)plan.tc.ty;
      res->info.superbin = (uint32_t)plan.tc.s;
      res->info.vblock_x = (uint32_t)plan.tc.bvx;
      res->info.vblock_y = (uint32_t)plan.tc.bvy;
      res->info.staged_cap = (uint32_t)plan.tc.scap;
      cudaEventElapsedTime(&res->info.ms_stack, evs0, evs1);
      cudaEventElapsedTime(&res->info.ms_total, ev0, ev1);
      cudaEventElapsedTime(&res->info.ms_count, evc0, evc1);
      cudaEventElapsedTime(&res->info.ms_ids, evc1, ev1);
      cudaEventElapsedTime(&res->info.ms_prep, ev0, evs0);
    }
  done:;
#undef CK
  }
  if (rc != SAS_OK) {
    if (res->d_ids) cudaFreeAsync(res->d_ids, s);
    if (res->d_cands) cudaFreeAsync(res->d_cands, s);
    for (void* p : {(void*)res->d_dets, (void*)res->d_boff, (void*)res->d_ecount, (void*)res->d_sxt,
                    (void*)res->d_syt, (void*)res->d_dt})
      if (p) cudaFreeAsync(p, s);
    cudaStreamSynchronize(s);
    delete res;
    return rc;
  }
  *out = res;
  return SAS_OK;
}

}  // namespace

int sas_stack(const sas_grid* grid, const sas_catalog* cat, uint32_t n_min, const sas_opts* opts,
              void* stream, sas_result** out) {
  return stack_impl(grid, cat, nullptr, n_min, opts, stream, out);
}

int sas_stack_weighted(const sas_grid* grid, const sas_catalog* cat, const uint8_t* weights, uint32_t s_min,
                       const sas_opts* opts, void* stream, sas_result** out) {
  if (!weights && cat && cat->n) return fail(SAS_ERR_ARG, "null weights");
  return stack_impl(grid, cat, weights ? weights : (const uint8_t*)"", s_min, opts, stream, out);
}

int sas_result_get_info(const sas_result* r, sas_result_info* info) {
  if (!r || !info) return fail(SAS_ERR_ARG, "null argument");
  *info = r->info;
  return SAS_OK;
}

int sas_candidates(const sas_result* r, sas_candidate* out, uint64_t cap, uint64_t* n_total,
                   uint32_t* ids, uint64_t ids_cap, uint64_t* n_ids_total, int on_device) {
  if (!r) return fail(SAS_ERR_ARG, "null result");
  const uint64_t nc = r->info.n_candidates, ni = r->info.n_ids;
  if (n_total) *n_total = nc;
  if (n_ids_total) *n_ids_total = ni;
  const uint64_t c1 = std::min(cap, nc), i1 = std::min(ids_cap, ni);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (c1 && !out) return fail(SAS_ERR_ARG, "null candidate buffer");
  if (i1 && !ids) return fail(SAS_ERR_ARG, "null id buffer");
  // both copies on the legacy default stream (the search completed before it
  // returned), then one wait
  if (c1) {
    cudaError_t e = cudaMemcpyAsync(out, r->d_cands, c1 * sizeof(sas_candidate), kind, 0);
    if (e != cudaSuccess) return cuda_fail(e, "copy candidates");
  }
  if (i1) {
    cudaError_t e = cudaMemcpyAsync(ids, r->d_ids, i1 * sizeof(uint32_t), kind, 0);
    if (e != cudaSuccess) return cuda_fail(e, "copy ids");
  }
  if (c1 || i1) {
    cudaError_t e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) return cuda_fail(e, "copy candidates");
  }
  if (cap < nc || ids_cap < ni)
    return fail(SAS_ERR_OVERFLOW, "buffers too small: need %llu candidates and %llu ids",
                (unsigned long long)nc, (unsigned long long)ni);
  return SAS_OK;
}

int sas_stamps(const sas_result* r, uint64_t first, uint64_t count, uint16_t* out, void* stream) {
  if (!r) return fail(SAS_ERR_ARG, "null result");
  if (!r->d_dets && count) return fail(SAS_ERR_ARG, "this result keeps no catalog (a cluster list)");
  const uint64_t nc = r->info.n_candidates;
  if (first > nc || count > nc - first)
    return fail(SAS_ERR_ARG, "candidates [%llu, %llu) outside the result's %llu", (unsigned long long)first,
                (unsigned long long)(first + count), (unsigned long long)nc);
  if (count == 0) return SAS_OK;
  if (!out) return fail(SAS_ERR_ARG, "null stamp buffer");
  cudaError_t e = launch_stamps(result_view(r), nullptr, first, count, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stamps");
  return SAS_OK;
}

int sas_stamps_indexed(const sas_result* r, const uint32_t* idx, uint64_t count, uint16_t* out,
                       void* stream) {
  if (!r) return fail(SAS_ERR_ARG, "null result");
  if (!r->d_dets && count) return fail(SAS_ERR_ARG, "this result keeps no catalog (a cluster list)");
  if (count == 0) return SAS_OK;
  if (!idx || !out) return fail(SAS_ERR_ARG, "null index or stamp buffer");
  cudaError_t e = launch_stamps(result_view(r), idx, 0, count, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stamps");
  return SAS_OK;
}

int sas_peel(const sas_result* r, uint32_t n_min, uint32_t max_clusters, uint32_t flags, void* stream,
             sas_result** out) {
  if (!r || !out) return fail(SAS_ERR_ARG, "null argument");
  if (!r->d_dets && r->info.n_candidates)
    return fail(SAS_ERR_ARG, "cluster finding needs a search result (this one is a cluster list)");
  if (n_min < r->n_min || n_min == 0)
    return fail(SAS_ERR_ARG, "n_min %u is below the search's threshold %u (cells under it are not in the list)",
                n_min, r->n_min);
  if (!r->complete) return fail(SAS_ERR_ARG, "the search kept only its top candidates (max_candidates)");
  if (r->info.peaks_only)
    return fail(SAS_ERR_ARG, "the search kept only tile-local peaks (peaks_only): its list is not complete at n_min");
  if (r->weighted) return fail(SAS_ERR_ARG, "cluster finding counts distinct epochs; this search is weighted");
  if (flags & ~SAS_PEEL_SEQUENTIAL) return fail(SAS_ERR_ARG, "unknown flags 0x%x", flags);
  if (max_clusters == 0) max_clusters = 1000;
  cudaStream_t s = (cudaStream_t)stream;
  PeelOut po;
  if (int rc = peel_clusters(result_view(r), n_min, max_clusters, (flags & SAS_PEEL_SEQUENTIAL) != 0, s, &po))
    return rc;
  sas_result* res = new sas_result();
  std::memset(res, 0, sizeof(*res));
  res->device = r->device;
  res->d_cands = po.cands;
  res->d_ids = po.ids;
  res->info = r->info;
  res->info.n_candidates = po.n;
  res->info.n_ids = po.n_ids;
  res->g = r->g;
  res->cg = r->cg;
  res->n_det = r->n_det;
  res->n_min = n_min;
  res->complete = 0;
  *out = res;
  return SAS_OK;
}

struct sas_tracks {
  int device;
  sas_track* d_tracks;
  uint32_t* d_ids;
  uint64_t n, n_ids;
};

int sas_refine(const sas_result* search, const sas_result* clusters, const sas_refine_opts* opts, void* stream,
               sas_tracks** out) {
  if (!search || !clusters || !out) return fail(SAS_ERR_ARG, "null argument");
  const bool empty = clusters->info.n_candidates == 0;
  if ((!search->d_dets || !search->d_dt) && !(empty && search->complete))
    return fail(SAS_ERR_ARG, "`search` must be a search result");
  if (clusters->n_det != search->n_det)
    return fail(SAS_ERR_ARG, "clusters come from a catalog of %llu detections, the search has %llu",
                (unsigned long long)clusters->n_det, (unsigned long long)search->n_det);
  sas_refine_opts o = opts ? *opts : sas_refine_opts{};
  if (o.n_starts == 0) o.n_starts = 500;
  if (o.n_best == 0) o.n_best = 10;
  if (o.max_csteps == 0) o.max_csteps = 100;
  if (o.max_iter == 0) o.max_iter = 10;
  if (o.radius == 0) o.radius = search->g.bin;
  if (o.n_starts > 4096) return fail(SAS_ERR_ARG, "n_starts %u above 4096", o.n_starts);
  if (o.radius < 0 || o.radius > (1 << 26)) return fail(SAS_ERR_ARG, "radius %d outside [0, 2^26]", o.radius);
  o.n_best = std::min(o.n_best, o.n_starts);
  RefineIn in;
  in.search.dets = search->d_dets;
  in.search.boff = search->d_boff;
  in.search.dt = search->d_dt;
  in.search.g = search->g;
  in.search.cg = search->cg;
  in.search.n_det = search->n_det;
  in.clusters.cands = clusters->d_cands;
  in.clusters.n = clusters->info.n_candidates;
  in.clusters.ids = clusters->d_ids;
  RefineOut ro;
  if (!empty)
    if (int rc = refine_tracks(in, o, (cudaStream_t)stream, &ro)) return rc;
  sas_tracks* t = new sas_tracks();
  t->device = search->device;
  t->d_tracks = ro.tracks;
  t->d_ids = ro.ids;
  t->n = ro.n;
  t->n_ids = ro.n_ids;
  *out = t;
  return SAS_OK;
}

int sas_tracks_get(const sas_tracks* t, sas_track* out, uint64_t cap, uint64_t* n_total, uint32_t* ids,
                   uint64_t ids_cap, uint64_t* n_ids_total, int on_device) {
  if (!t) return fail(SAS_ERR_ARG, "null tracks");
  if (n_total) *n_total = t->n;
  if (n_ids_total) *n_ids_total = t->n_ids;
  const uint64_t c1 = std::min(cap, t->n), i1 = std::min(ids_cap, t->n_ids);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (c1) {
    if (!out) return fail(SAS_ERR_ARG, "null track buffer");
    cudaError_t e = cudaMemcpy(out, t->d_tracks, c1 * sizeof(sas_track), kind);
    if (e != cudaSuccess) return cuda_fail(e, "copy tracks");
  }
  if (i1) {
    if (!ids) return fail(SAS_ERR_ARG, "null id buffer");
    cudaError_t e = cudaMemcpy(ids, t->d_ids, i1 * sizeof(uint32_t), kind);
    if (e != cudaSuccess) return cuda_fail(e, "copy ids");
  }
  if (cap < t->n || ids_cap < t->n_ids)
    return fail(SAS_ERR_OVERFLOW, "buffers too small: need %llu tracks and %llu ids", (unsigned long long)t->n,
                (unsigned long long)t->n_ids);
  return SAS_OK;
}

void sas_tracks_free(sas_tracks* t) {
  if (!t) return;
  if (t->d_tracks) cudaFree(t->d_tracks);
  if (t->d_ids) cudaFree(t->d_ids);
  delete t;
}

int sas_owned(const sas_result* r, uint32_t n_keep, uint32_t* idx, uint64_t* n_kept, void* stream) {
  if (!r || !n_kept) return fail(SAS_ERR_ARG, "null argument");
  if (r->info.n_candidates && !idx) return fail(SAS_ERR_ARG, "null index buffer");
  return select_owned(result_view(r), n_keep, idx, n_kept, (cudaStream_t)stream);
}

int sas_peaks(const sas_result* r, uint32_t* idx, uint64_t* n_peaks, void* stream) {
  if (!r || !n_peaks) return fail(SAS_ERR_ARG, "null argument");
  if (r->info.n_candidates && !idx) return fail(SAS_ERR_ARG, "null index buffer");
  return select_peaks(result_view(r), idx, n_peaks, (cudaStream_t)stream);
}

void sas_result_free(sas_result* r) {
  if (!r) return;
  for (void* p : {(void*)r->d_cands, (void*)r->d_ids, (void*)r->d_dets, (void*)r->d_boff,
                  (void*)r->d_ecount, (void*)r->d_sxt, (void*)r->d_syt, (void*)r->d_dt})
    if (p) cudaFree(p);
  delete r;
}

int sas_cell_counts_noalloc(const sas_grid* grid, const sas_catalog* cat, const uint32_t* cells,
                            uint64_t n_cells, uint32_t* distinct, uint32_t* raw, void* stream) {
  if (!grid || !cat) return fail(SAS_ERR_ARG, "null argument");
  std::string err;
  const int rc = noalloc_cell_counts(grid->d, cat, cells, n_cells, distinct, raw, stream, &err);
  if (rc != SAS_OK) return fail(rc, "%s", err.c_str());
  return SAS_OK;
}

int sas_probe_shared_atomic_peak(uint32_t iters, void* stream, double* ops_per_s, double* sm_mhz) {
  if (!ops_per_s || !sm_mhz || iters == 0) return fail(SAS_ERR_ARG, "bad argument");
  cudaError_t e = run_atomic_probe(iters, (cudaStream_t)stream, ops_per_s, sm_mhz);
  if (e != cudaSuccess) return cuda_fail(e, "atomic probe");
  return SAS_OK;
}

int sas_probe_shared_or64_peak(uint32_t iters, void* stream, double* ops_per_s, double* sm_mhz) {
  if (!ops_per_s || !sm_mhz || iters == 0) return fail(SAS_ERR_ARG, "bad argument");
  cudaError_t e = run_or64_probe(iters, (cudaStream_t)stream, ops_per_s, sm_mhz);
  if (e != cudaSuccess) return cuda_fail(e, "64-bit atomicOr probe");
  return SAS_OK;
}

int sas_probe_shared_reduction_peak(uint32_t iters, void* stream, double* ops_per_s, double* sm_mhz) {
  if (!ops_per_s || !sm_mhz || iters == 0) return fail(SAS_ERR_ARG, "bad argument");
  cudaError_t e = run_red_probe(iters, (cudaStream_t)stream, ops_per_s, sm_mhz);
  if (e != cudaSuccess) return cuda_fail(e, "reduction probe");
  return SAS_OK;
}

}  // extern "C"
