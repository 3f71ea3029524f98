// Batched search: many fields (CCDs) with uneven detection and epoch counts in
// one pass of every kernel -- one persistent stack launch over the work units of
// all fields -- recorded once as a CUDA graph and replayed.
//
// sas_batch_create plans every field (tile shape from its own opts, e.g. the
// autotuner's pick for its size class), lays out one device arena for all of
// them with fixed capacities, and captures the whole device pipeline into a
// graph.  sas_batch_run replays the graph; when a field needed more candidate,
// emission or id slots than the arena has, the run grows them to what the
// field reported, rebuilds the arena and the graph, and replays; a field whose
// counters wrapped (or whose grown capacities would not fit) is recomputed
// exactly on the single-field path, so the results always equal sas_stack's.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sas_batch.cuh"

using namespace sas;

struct sas_batch {
  int device = 0;
  uint32_t n_fields = 0;
  std::vector<sas_grid*> grids;            // private copies (own descriptors)
  std::vector<sas_catalog> cats;
  std::vector<std::vector<int64_t>> times;
  std::vector<uint32_t> n_min;
  std::vector<sas_opts> opts;
  std::vector<FieldPlan> plans;
  std::vector<BatchField> hf;              // host copy of the field descriptors
  // Capacities of the arena: candidate-key slots per field (one power of two for
  // all fields: the segment of the segmented sort), emission slots and id slots
  // per field.  A replay that finds a field over one of them rebuilds the arena
  // and the graph at the sizes it reported, and replays.
  uint32_t key_seg = kBatchKeyCap;
  std::vector<uint32_t> emit_cap;
  std::vector<uint64_t> ids_cap;
  uint64_t rebuilds = 0;
  BatchDev dev{};
  void* arena = nullptr;
  uint32_t* h_ctr = nullptr;               // pinned [n_fields][kCtrN]
  unsigned long long* h_c64 = nullptr;     // pinned [n_fields][kC64N]
  uint32_t* d_ctr = nullptr;
  unsigned long long* d_c64 = nullptr;
  uint32_t* d_ecount_all = nullptr;
  size_t ecount_words = 0;
  // Fields grouped by stack kernel configuration (velocity tile, counter width,
  // peak selection): one persistent stack launch per group, each over its own
  // work counter and its fields' units.
  struct Group {
    int kx = 0, ky = 0, cb = 0;
    bool peaks = false;
    std::vector<uint32_t> fields;
    size_t smem = 0;
    int grid = 0;
    StackArgs* d_args = nullptr;
    unsigned long long* d_unit_base = nullptr;
    unsigned long long* d_work = nullptr;
  };
  std::vector<Group> groups;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<sas_result*> fallback;       // per field, after a run that needed it
  float ms_last = 0.f;
  uint64_t fallback_count = 0;
};

namespace {

int cuda_err(cudaError_t e, const char* where) {
  return set_errorf(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, "%s: %s", where,
                    cudaGetErrorString(e));
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Records the device work of one batch pass on stream s (used under capture).
cudaError_t record_pass(sas_batch* b, cudaStream_t s) {
  cudaError_t e;
  if ((e = cudaMemsetAsync(b->d_ctr, 0, (size_t)b->n_fields * kCtrN * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b->d_c64, 0, (size_t)b->n_fields * kC64N * 8, s)) != cudaSuccess) return e;
  for (const sas_batch::Group& g : b->groups)
    if ((e = cudaMemsetAsync(g.d_work, 0, 8, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b->d_ecount_all, 0, b->ecount_words * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(b->dev.bucket_count, 0, b->dev.total_buckets * 4, s)) != cudaSuccess) return e;
  if ((e = batch_launch_prep(b->dev, s)) != cudaSuccess) return e;
  for (const sas_batch::Group& g : b->groups)
    if ((e = launch_stack_multi(g.kx, g.ky, g.cb, g.peaks, g.d_args, g.d_unit_base, (int)g.fields.size(),
                                g.d_work, g.smem, g.grid, s)) != cudaSuccess)
      return e;
  if ((e = batch_launch_post(b->dev, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(b->h_ctr, b->d_ctr, (size_t)b->n_fields * kCtrN * 4,
                           cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  return cudaMemcpyAsync(b->h_c64, b->d_c64, (size_t)b->n_fields * kC64N * 8,
                         cudaMemcpyDeviceToHost, s);
}

// Releases the device arena and the recorded pass (capacities and plans stay).
void free_pass(sas_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->arena) cudaFree(b->arena);
  if (b->h_ctr) cudaFreeHost(b->h_ctr);
  if (b->h_c64) cudaFreeHost(b->h_c64);
  b->exec = nullptr;
  b->graph = nullptr;
  b->arena = nullptr;
  b->h_ctr = nullptr;
  b->h_c64 = nullptr;
}

void free_batch(sas_batch* b) {
  if (!b) return;
  free_pass(b);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  for (sas_result* r : b->fallback) sas_result_free(r);
  for (sas_grid* g : b->grids) sas_destroy_grid(g);
  delete b;
}

}  // namespace

namespace {

// Lays out the device arena for the current capacities, writes the field
// descriptors and records one pass of the whole pipeline as a graph.
int build_pass(sas_batch* b, const DevInfo& di, cudaStream_t s) {
  const uint32_t n_fields = b->n_fields;
  int rc = SAS_OK;
  cudaError_t ce = cudaSuccess;
  // --- sizes and arena layout --------------------------------------------------
  std::vector<unsigned long long> det_off(n_fields + 1, 0), tab_off(n_fields + 1, 0),
      emit_off(n_fields + 1, 0), cand_off(n_fields + 1, 0), unit_base(n_fields + 1, 0);
  std::vector<uint64_t> bucket_base(n_fields + 1, 0), ecount_base(n_fields + 1, 0);
  std::vector<StackArgs> hargs(n_fields);
  for (uint32_t f = 0; f < n_fields; ++f) {
    const FieldPlan& fp = b->plans[f];
    const sas_catalog& c = b->cats[f];
    det_off[f + 1] = det_off[f] + c.n;
    tab_off[f + 1] = tab_off[f] + (unsigned long long)(fp.g.nvx + fp.g.nvy) * fp.g.E;
    emit_off[f + 1] = emit_off[f] + b->emit_cap[f];
    cand_off[f + 1] = cand_off[f] + b->key_seg;
    bucket_base[f + 1] = bucket_base[f] + fp.nb;
    ecount_base[f + 1] = ecount_base[f] + fp.g.E;
    fill_stack_args(fp, b->n_min[f], b->opts[f].n_low, b->opts[f].peaks_only, &hargs[f]);
    unit_base[f + 1] = unit_base[f] + hargs[f].n_tiles;
  }
  BatchDev& B = b->dev;
  B.n_fields = (int)n_fields;
  B.total_dets = det_off[n_fields];
  B.total_buckets = bucket_base[n_fields];
  B.total_tab = tab_off[n_fields];
  B.total_emit = emit_off[n_fields];
  B.total_cand = cand_off[n_fields];
  B.key_seg = b->key_seg;
  b->ecount_words = ecount_base[n_fields];
  // one arena: [region sizes computed here]
  struct Reg { void** p; size_t bytes; };
  std::vector<Reg> regs;
  std::vector<Emit*> f_emits(n_fields);
  std::vector<Key*> f_keys(n_fields);
  std::vector<unsigned long long*> f_idoff(n_fields);
  std::vector<uint32_t*> f_ids(n_fields), f_idt(n_fields);
  std::vector<sas_candidate*> f_cands(n_fields);
  std::vector<int32_t*> f_sxt(n_fields), f_syt(n_fields);
  std::vector<int64_t*> f_t(n_fields), f_dt(n_fields);
  regs.push_back({(void**)&B.fields, n_fields * sizeof(BatchField)});
  for (sas_batch::Group& g : b->groups) {
    regs.push_back({(void**)&g.d_args, g.fields.size() * sizeof(StackArgs)});
    regs.push_back({(void**)&g.d_unit_base, (g.fields.size() + 1) * 8});
    regs.push_back({(void**)&g.d_work, 8});
  }
  regs.push_back({(void**)&B.det_off, (n_fields + 1) * 8});
  regs.push_back({(void**)&B.tab_off, (n_fields + 1) * 8});
  regs.push_back({(void**)&B.emit_off, (n_fields + 1) * 8});
  regs.push_back({(void**)&B.cand_off, (n_fields + 1) * 8});
  regs.push_back({(void**)&b->d_ctr, (size_t)n_fields * kCtrN * 4});
  regs.push_back({(void**)&b->d_c64, (size_t)n_fields * kC64N * 8});
  regs.push_back({(void**)&b->d_ecount_all, b->ecount_words * 4});
  regs.push_back({(void**)&B.bucket_count, B.total_buckets * 4});
  regs.push_back({(void**)&B.boff, (B.total_buckets + 1) * 4});
  regs.push_back({(void**)&B.cursor, B.total_buckets * 4});
  regs.push_back({(void**)&B.scan_scratch, scan_scratch_elems(B.total_buckets) * 4});
  regs.push_back({(void**)&B.bucket_of, B.total_dets * 4});
  regs.push_back({(void**)&B.dets, B.total_dets * sizeof(Det)});
  regs.push_back({(void**)&B.keys_all, B.total_cand * sizeof(Key)});
  for (uint32_t f = 0; f < n_fields; ++f) {
    const FieldPlan& fp = b->plans[f];
    regs.push_back({(void**)&f_t[f], fp.g.E * 8});
    regs.push_back({(void**)&f_dt[f], fp.g.E * 8});
    regs.push_back({(void**)&f_sxt[f], (size_t)fp.g.nvx * fp.g.E * 4});
    regs.push_back({(void**)&f_syt[f], (size_t)fp.g.nvy * fp.g.E * 4});
    regs.push_back({(void**)&f_emits[f], (emit_off[f + 1] - emit_off[f]) * sizeof(Emit)});
    regs.push_back({(void**)&f_idoff[f], ((size_t)b->key_seg + 1) * 8});
    regs.push_back({(void**)&f_ids[f], b->ids_cap[f] * 4});
    regs.push_back({(void**)&f_idt[f], b->ids_cap[f] * 4});
    regs.push_back({(void**)&f_cands[f], (size_t)b->key_seg * sizeof(sas_candidate)});
  }
  size_t total = 0;
  for (const Reg& r : regs) total += align256(std::max<size_t>(r.bytes, 1));
  if ((ce = cudaMalloc(&b->arena, total)) != cudaSuccess) { rc = cuda_err(ce, "batch arena"); return rc; }
  {
    size_t off = 0;
    for (const Reg& r : regs) {
      *r.p = static_cast<char*>(b->arena) + off;
      off += align256(std::max<size_t>(r.bytes, 1));
    }
  }
  for (uint32_t f = 0; f < n_fields; ++f) f_keys[f] = B.keys_all + cand_off[f];
  if ((ce = cudaMallocHost((void**)&b->h_ctr, (size_t)n_fields * kCtrN * 4)) != cudaSuccess ||
      (ce = cudaMallocHost((void**)&b->h_c64, (size_t)n_fields * kC64N * 8)) != cudaSuccess) {
    return cuda_err(ce, "pinned counters");
  }
  // --- field descriptors ---------------------------------------------------------
  b->hf.resize(n_fields);
  for (uint32_t f = 0; f < n_fields; ++f) {
    const FieldPlan& fp = b->plans[f];
    const sas_catalog& c = b->cats[f];
    StackArgs& sa = hargs[f];
    uint32_t* ctr = b->d_ctr + (size_t)f * kCtrN;
    unsigned long long* c64 = b->d_c64 + (size_t)f * kC64N;
    sa.dets = B.dets;
    sa.boff = B.boff + bucket_base[f];
    sa.ecount = b->d_ecount_all + ecount_base[f];
    sa.sxt = f_sxt[f];
    sa.syt = f_syt[f];
    sa.emits = f_emits[f];
    sa.emit_cap = (uint32_t)(emit_off[f + 1] - emit_off[f]);
    sa.n_emit = ctr + kCtrEmit;
    sa.n_pairs = c64 + kC64Pairs;
    sa.balance = c64 + kC64Balance;
    sa.flags = ctr + kCtrFlags;
    sa.tile_counter = nullptr;  // the group's work counter drives the multi-field launch
    BatchField& bf = b->hf[f];
    memset(&bf, 0, sizeof(bf));
    bf.args = sa;
    bf.x = c.x;
    bf.y = c.y;
    bf.epoch = c.epoch;
    bf.t = f_t[f];
    bf.E = fp.g.E;
    bf.emit_cap = sa.emit_cap;
    bf.ecount = const_cast<uint32_t*>(sa.ecount);
    bf.dt = f_dt[f];
    bf.t0 = reinterpret_cast<long long*>(c64 + kC64T0);
    bf.sxt = f_sxt[f];
    bf.syt = f_syt[f];
    bf.bucket_base = bucket_base[f];
    bf.counters = ctr;
    bf.keys = f_keys[f];
    bf.key_cap = b->key_seg;
    bf.max_out = b->opts[f].max_candidates ? (uint32_t)std::min<uint64_t>(b->opts[f].max_candidates, b->key_seg) : b->key_seg;
    bf.id_off = f_idoff[f];
    bf.ids = f_ids[f];
    bf.ids_tmp = f_idt[f];
    bf.ids_cap = b->ids_cap[f];
    bf.cands = f_cands[f];
    if ((ce = cudaMemcpyAsync(f_t[f], c.t, fp.g.E * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(B.fields, b->hf.data(), n_fields * sizeof(BatchField), cudaMemcpyHostToDevice, s);
  // per group: its fields' stack arguments and a unit base over its own units
  std::vector<std::vector<StackArgs>> gargs(b->groups.size());
  std::vector<std::vector<unsigned long long>> gbase(b->groups.size());
  for (size_t k = 0; k < b->groups.size(); ++k) {
    sas_batch::Group& g = b->groups[k];
    gbase[k].assign(1, 0ull);
    for (uint32_t f : g.fields) {
      gargs[k].push_back(hargs[f]);
      gbase[k].push_back(gbase[k].back() + hargs[f].n_tiles);
    }
    g.grid = (int)std::min<unsigned long long>((unsigned long long)di.sms, std::max<unsigned long long>(gbase[k].back(), 1));
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(g.d_args, gargs[k].data(), g.fields.size() * sizeof(StackArgs), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(g.d_unit_base, gbase[k].data(), (g.fields.size() + 1) * 8, cudaMemcpyHostToDevice, s);
  }
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(B.det_off, det_off.data(), (n_fields + 1) * 8, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(B.tab_off, tab_off.data(), (n_fields + 1) * 8, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(B.emit_off, emit_off.data(), (n_fields + 1) * 8, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(B.cand_off, cand_off.data(), (n_fields + 1) * 8, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  for (const sas_batch::Group& g : b->groups)
    if (ce == cudaSuccess) ce = stack_set_smem_attr(g.kx, g.ky, g.cb, g.smem);
  if (ce == cudaSuccess) ce = batch_set_attrs();
  // One launch of each group's stack kernel before the capture, with its work
  // counter far past the end (0x7F7F...: every CTA leaves at once, and the
  // counter cannot wrap): the kernel is loaded and its resources reserved
  // outside the capture.
  if (ce != cudaSuccess) { rc = cuda_err(ce, "batch setup"); return rc; }
  for (const sas_batch::Group& g : b->groups) {
    ce = cudaMemsetAsync(g.d_work, 0x7F, 8, s);
    if (ce == cudaSuccess)
      ce = launch_stack_multi(g.kx, g.ky, g.cb, g.peaks, g.d_args, g.d_unit_base, (int)g.fields.size(), g.d_work,
                              g.smem, g.grid, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess)
      return set_errorf(SAS_ERR_CUDA, "batch setup: stack kernel (kx %d, ky %d, %d-bit counters%s, %zu B shared, "
                                      "%d CTAs): %s", g.kx, g.ky, g.cb, g.peaks ? ", peaks" : "", g.smem, g.grid,
                        cudaGetErrorString(ce));
  }
  // --- record the pass as a graph ---------------------------------------------
  cudaStream_t cs;
  if ((ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) { rc = cuda_err(ce, "stream"); return rc; }
  ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cudaError_t ce2 = ce == cudaSuccess ? record_pass(b, cs) : ce;
  cudaGraph_t g = nullptr;
  if (ce == cudaSuccess) ce = cudaStreamEndCapture(cs, &g);
  if (ce2 != cudaSuccess) ce = ce2;  // the first failure inside the capture, not its consequence
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&b->exec, g, 0);
  b->graph = g;
  cudaStreamDestroy(cs);
  if (ce != cudaSuccess) { rc = cuda_err(ce, "graph capture"); return rc; }
  return SAS_OK;
}

}  // namespace

extern "C" {

int sas_batch_create(const sas_grid* const* grids, const sas_catalog* cats, const uint32_t* n_min,
                     uint32_t n_fields, const sas_opts* opts, void* stream, sas_batch** out) {
  if (!grids || !cats || !n_min || !out || n_fields == 0) return set_error(SAS_ERR_ARG, "null argument or no fields");
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return cuda_err(ce, "cudaGetDevice");
  DevInfo di;
  if (int rc = device_info(dev, &di)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  sas_batch* b = new (std::nothrow) sas_batch;
  if (!b) return set_error(SAS_ERR_OOM, "host allocation");
  b->device = dev;
  b->n_fields = n_fields;
  int rc = SAS_OK;
  // --- plan every field --------------------------------------------------------
  for (uint32_t f = 0; f < n_fields && rc == SAS_OK; ++f) {
    const sas_catalog& c = cats[f];
    if (!grids[f]) { rc = set_error(SAS_ERR_ARG, "null grid"); break; }
    if (!c.on_device) { rc = set_error(SAS_ERR_ARG, "batch catalogs must be in device memory"); break; }
    if (c.n_epochs < 1 || c.n_epochs > SAS_MAX_EPOCHS) { rc = set_error(SAS_ERR_RANGE, "n_epochs out of range"); break; }
    if (!c.t || c.ticks_per_hour <= 0) { rc = set_error(SAS_ERR_ARG, "bad epoch times"); break; }
    if (c.n == 0 || c.n >= ((uint64_t)1 << 31)) { rc = set_error(SAS_ERR_RANGE, "each field needs 1 <= n < 2^31 detections"); break; }
    if (!c.x || !c.y || !c.epoch) { rc = set_error(SAS_ERR_ARG, "null catalog array"); break; }
    if (n_min[f] < 1 || n_min[f] > 128) { rc = set_error(SAS_ERR_ARG, "batch fields need 1 <= n_min <= 128"); break; }
    int64_t tmin = c.t[0], tmax = c.t[0];
    for (uint32_t e = 1; e < c.n_epochs; ++e) { tmin = std::min(tmin, c.t[e]); tmax = std::max(tmax, c.t[e]); }
    if ((__int128)tmax - tmin >= ((__int128)1 << 32)) { rc = set_error(SAS_ERR_RANGE, "time span must be < 2^32 ticks"); break; }
    sas_grid* gcopy = nullptr;
    sas_grid_desc desc;
    // copy the grid through its public descriptor
    rc = sas_grid_get_desc(grids[f], &desc);
    if (rc == SAS_OK) rc = sas_create_grid(&desc, &gcopy);
    if (rc != SAS_OK) break;
    b->grids.push_back(gcopy);
    b->times.emplace_back(c.t, c.t + c.n_epochs);
    sas_catalog cc = c;
    cc.t = b->times.back().data();
    b->cats.push_back(cc);
    b->n_min.push_back(n_min[f]);
    sas_opts o{};
    if (opts) o = opts[f];
    if (o.n_low > n_min[f]) { rc = set_errorf(SAS_ERR_ARG, "field %u: n_low is above n_min", f); break; }
    if (o.n_low == 0) o.n_low = n_min[f];
    if (o.peaks_only > 1) { rc = set_errorf(SAS_ERR_ARG, "field %u: peaks_only must be 0 or 1", f); break; }
    // 8-bit counters (start 128 - n_low) wrap past 128 + n_low detections in
    // one super-bin: a field whose brightest mover (one detection per epoch)
    // plus a generous noise allowance could get there counts in 16 bits.  A
    // wrap is still detected and recomputed exactly; this keeps it rare.
    if (o.counter_bits == 0) {
      const double lam = (double)c.n * 9.0 / ((double)desc.nbx * desc.nby);  // per 3 x 3-bin super-bin
      const double reach = (double)c.n_epochs + lam + 6.0 * std::sqrt(lam) + 2.0;
      o.counter_bits = reach >= 128.0 + o.n_low ? 16 : 8;
    }
    o.v_begin = o.v_end = 0;
    b->opts.push_back(o);
    FieldPlan fp;
    rc = plan_field(desc, c.n, c.n_epochs, c.t, c.ticks_per_hour, n_min[f], 0,
                    (uint64_t)desc.nvx * desc.nvy, o, di, &fp);
    if (rc != SAS_OK && (o.tile_bx || o.tile_by) && (!opts || opts[f].counter_bits != o.counter_bits)) {
      // a spatial tile chosen for other counters (e.g. tuned with 8-bit ones)
      // may not fit the wider counters picked here: the planner sizes it
      o.tile_bx = o.tile_by = 0;
      rc = plan_field(desc, c.n, c.n_epochs, c.t, c.ticks_per_hour, n_min[f], 0,
                      (uint64_t)desc.nvx * desc.nvy, o, di, &fp);
    }
    if (rc != SAS_OK) break;
    b->plans.push_back(fp);
  }
  if (rc != SAS_OK) { free_batch(b); return rc; }
  // group the fields by stack kernel configuration
  for (uint32_t f = 0; f < n_fields; ++f) {
    const TileCfg& tc = b->plans[f].tc;
    sas_batch::Group* g = nullptr;
    const bool peaks = b->opts[f].peaks_only || b->opts[f].n_low < b->n_min[f];
    for (sas_batch::Group& h : b->groups)
      if (h.kx == tc.kx && h.ky == tc.ky && h.cb == tc.cb && h.peaks == peaks) g = &h;
    if (!g) {
      b->groups.emplace_back();
      g = &b->groups.back();
      g->kx = tc.kx;
      g->ky = tc.ky;
      g->cb = tc.cb;
      g->peaks = peaks;
    }
    g->fields.push_back(f);
    g->smem = std::max(g->smem, tc.smem);
  }
  b->emit_cap.resize(n_fields);
  b->ids_cap.resize(n_fields);
  for (uint32_t f = 0; f < n_fields; ++f) {
    b->emit_cap[f] = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(2 * b->cats[f].n, 1u << 18), 1u << 24);
    b->ids_cap[f] = (uint64_t)b->key_seg * (b->plans[f].g.E / 2 + 8);
  }
  if ((rc = build_pass(b, di, s)) != SAS_OK) { free_batch(b); return rc; }
  cudaEventCreate(&b->ev0);
  cudaEventCreate(&b->ev1);
  b->fallback.assign(n_fields, nullptr);
  *out = b;
  return SAS_OK;
}

int sas_batch_run(sas_batch* b, void* stream) {
  if (!b) return set_error(SAS_ERR_ARG, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  for (sas_result*& r : b->fallback) {
    if (r) sas_result_free(r);
    r = nullptr;
  }
  cudaEventRecord(b->ev0, s);
  cudaError_t ce = cudaGraphLaunch(b->exec, s);
  cudaEventRecord(b->ev1, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) return cuda_err(ce, "batch graph");
  cudaEventElapsedTime(&b->ms_last, b->ev0, b->ev1);
  // A field over a capacity (keys, emissions, ids) reports what it needed: grow
  // those capacities, rebuild the arena and the graph, and replay (a few times
  // at most: a field cut short at one stage can need more at the next).
  for (int round = 0; round < 4; ++round) {
    bool grow = false;
    uint32_t key_seg = b->key_seg;
    std::vector<uint32_t> emit_cap = b->emit_cap;
    std::vector<uint64_t> ids_cap = b->ids_cap;
    for (uint32_t f = 0; f < b->n_fields; ++f) {
      const uint32_t* ctr = b->h_ctr + (size_t)f * kCtrN;
      const uint32_t fl = ctr[kCtrFlags];
      if (fl & (kFlagEpoch | kFlagPos | kFlagShift | kFlagCounter | kFlagInternal)) continue;
      if (!(fl & kFlagEmitCap) && ctr[kCtrEmit] <= b->emit_cap[f]) continue;
      const uint64_t need_emit = ctr[kCtrEmit], need_keys = ctr[kCtrValid];
      const uint64_t need_ids = (uint64_t)ctr[kCtrIdsLo] | ((uint64_t)ctr[kCtrIdsHi] << 32);
      if (need_emit > emit_cap[f]) emit_cap[f] = (uint32_t)std::min<uint64_t>(need_emit + need_emit / 4 + 1024, 1u << 30);
      while (need_keys > key_seg && key_seg < kBatchKeyCapMax) key_seg *= 2;
      if (need_ids > ids_cap[f]) ids_cap[f] = need_ids + need_ids / 4 + 1024;
      grow = true;
    }
    if (!grow) break;
    // the new arena must fit in what the device has free now (plus the old arena)
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    uint64_t want = 0;
    for (uint32_t f = 0; f < b->n_fields; ++f)
      want += (uint64_t)key_seg * (sizeof(Key) + 8 + sizeof(sas_candidate)) + (uint64_t)emit_cap[f] * sizeof(Emit) +
              ids_cap[f] * 8;
    if (want > free_b / 2) break;  // leave it to the exact single-field fallback below
    b->key_seg = key_seg;
    b->emit_cap = emit_cap;
    b->ids_cap = ids_cap;
    free_pass(b);
    DevInfo di;
    int rc = device_info(b->device, &di);
    if (rc == SAS_OK) rc = build_pass(b, di, s);
    if (rc != SAS_OK) return rc;
    ++b->rebuilds;
    cudaEventRecord(b->ev0, s);
    ce = cudaGraphLaunch(b->exec, s);
    cudaEventRecord(b->ev1, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return cuda_err(ce, "batch graph");
    cudaEventElapsedTime(&b->ms_last, b->ev0, b->ev1);
  }
  // exact fallback for fields that still do not fit, or whose counters wrapped
  for (uint32_t f = 0; f < b->n_fields; ++f) {
    const uint32_t* ctr = b->h_ctr + (size_t)f * kCtrN;
    const unsigned long long* c64 = b->h_c64 + (size_t)f * kC64N;
    const uint32_t fl = ctr[kCtrFlags];
    if (fl & kFlagEpoch) return set_errorf(SAS_ERR_RANGE, "field %u: an epoch index is >= n_epochs", f);
    if (fl & kFlagPos) return set_errorf(SAS_ERR_RANGE, "field %u: a detection has |x| or |y| >= 2^29", f);
    if (fl & kFlagShift) return set_errorf(SAS_ERR_RANGE, "field %u: a shift |v*(t-t0)/TPH| >= 2^28", f);
    const bool redo = (fl & (kFlagEmitCap | kFlagCounter | kFlagInternal)) || c64[kC64Balance] != 0 ||
                      ctr[kCtrEmit] > b->hf[f].emit_cap;
    if (!redo) continue;
    sas_opts o = b->opts[f];
    o.counter_bits = 0;
    const int rc = sas_stack(b->grids[f], &b->cats[f], b->n_min[f], &o, stream, &b->fallback[f]);
    if (rc != SAS_OK) return rc;
    ++b->fallback_count;
  }
  return SAS_OK;
}

int sas_batch_field_info(const sas_batch* b, uint32_t field, sas_result_info* info) {
  if (!b || !info || field >= b->n_fields) return set_error(SAS_ERR_ARG, "bad argument");
  if (b->fallback[field]) return sas_result_get_info(b->fallback[field], info);
  const uint32_t* ctr = b->h_ctr + (size_t)field * kCtrN;
  const unsigned long long* c64 = b->h_c64 + (size_t)field * kC64N;
  memset(info, 0, sizeof(*info));
  info->n_candidates = ctr[kCtrOut];
  info->n_ids = (uint64_t)ctr[kCtrIdsLo] | ((uint64_t)ctr[kCtrIdsHi] << 32);
  info->n_pairs = c64[kC64Pairs];
  info->n_emitted = ctr[kCtrEmit];
  info->t0 = (int64_t)c64[kC64T0];
  const TileCfg& tc = b->plans[field].tc;
  info->counter_bits = (uint32_t)tc.cb;
  info->tile_kx = (uint32_t)tc.kx;
  info->tile_ky = (uint32_t)tc.ky;
  info->tile_bx = (uint32_t)tc.tx;
  info->tile_by = (uint32_t)tc.ty;
  info->superbin = (uint32_t)tc.s;
  info->vblock_x = (uint32_t)tc.bvx;
  info->vblock_y = (uint32_t)tc.bvy;
  info->staged_cap = (uint32_t)tc.scap;
  info->n_low = b->opts[field].n_low;
  info->peaks_only = b->opts[field].peaks_only;
  info->ms_total = b->ms_last;
  return SAS_OK;
}

int sas_batch_candidates(const sas_batch* b, uint32_t field, sas_candidate* out, uint64_t cap,
                         uint64_t* n_total, uint32_t* ids, uint64_t ids_cap, uint64_t* n_ids_total,
                         int on_device) {
  if (!b || field >= b->n_fields) return set_error(SAS_ERR_ARG, "bad argument");
  if (b->fallback[field])
    return sas_candidates(b->fallback[field], out, cap, n_total, ids, ids_cap, n_ids_total, on_device);
  sas_result_info info;
  sas_batch_field_info(b, field, &info);
  const uint64_t nc = info.n_candidates, ni = info.n_ids;
  if (n_total) *n_total = nc;
  if (n_ids_total) *n_ids_total = ni;
  const uint64_t c1 = std::min(cap, nc), i1 = std::min(ids_cap, ni);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (c1) {
    if (!out) return set_error(SAS_ERR_ARG, "null candidate buffer");
    cudaError_t e = cudaMemcpy(out, b->hf[field].cands, c1 * sizeof(sas_candidate), kind);
    if (e != cudaSuccess) return cuda_err(e, "copy candidates");
  }
  if (i1) {
    if (!ids) return set_error(SAS_ERR_ARG, "null id buffer");
    cudaError_t e = cudaMemcpy(ids, b->hf[field].ids, i1 * sizeof(uint32_t), kind);
    if (e != cudaSuccess) return cuda_err(e, "copy ids");
  }
  if (cap < nc || ids_cap < ni)
    return set_errorf(SAS_ERR_OVERFLOW, "buffers too small: need %llu candidates and %llu ids",
                      (unsigned long long)nc, (unsigned long long)ni);
  return SAS_OK;
}

namespace {

CandView batch_view(const sas_batch* b, uint32_t field) {
  if (b->fallback[field]) return result_view(b->fallback[field]);
  sas_result_info info;
  sas_batch_field_info(b, field, &info);
  const BatchField& f = b->hf[field];
  CandView v;
  v.cands = f.cands;
  v.n = info.n_candidates;
  v.g = f.args.g;
  v.cg = f.args.cg;
  v.dets = f.args.dets;
  v.boff = f.args.boff;
  v.ecount = f.ecount;
  v.sxt = f.sxt;
  v.syt = f.syt;
  v.ids = f.ids;
  v.n_det = b->cats[field].n;
  return v;
}

}  // namespace

int sas_batch_peaks(const sas_batch* b, uint32_t field, uint32_t* idx, uint64_t* n_peaks, void* stream) {
  if (!b || field >= b->n_fields || !n_peaks) return set_error(SAS_ERR_ARG, "bad argument");
  const CandView v = batch_view(b, field);
  if (v.n && !idx) return set_error(SAS_ERR_ARG, "null index buffer");
  return select_peaks(v, idx, n_peaks, (cudaStream_t)stream);
}

int sas_batch_owned(const sas_batch* b, uint32_t field, uint32_t n_keep, uint32_t* idx, uint64_t* n_kept,
                    void* stream) {
  if (!b || field >= b->n_fields || !n_kept) return set_error(SAS_ERR_ARG, "bad argument");
  const CandView v = batch_view(b, field);
  if (v.n && !idx) return set_error(SAS_ERR_ARG, "null index buffer");
  return select_owned(v, n_keep, idx, n_kept, (cudaStream_t)stream);
}

int sas_batch_stamps(const sas_batch* b, uint32_t field, const uint32_t* idx, uint64_t count, uint16_t* out,
                     void* stream) {
  if (!b || field >= b->n_fields) return set_error(SAS_ERR_ARG, "bad argument");
  const CandView v = batch_view(b, field);
  if (!idx && count > v.n)
    return set_errorf(SAS_ERR_ARG, "%llu stamps asked of a field with %llu candidates",
                      (unsigned long long)count, (unsigned long long)v.n);
  if (count == 0) return SAS_OK;
  if (!out) return set_error(SAS_ERR_ARG, "null stamp buffer");
  cudaError_t e = launch_stamps(v, idx, 0, count, out, (cudaStream_t)stream);
  return e == cudaSuccess ? SAS_OK : cuda_err(e, "batch stamps");
}

}  // extern "C"

namespace {

__global__ void k_fill_u32(uint32_t* p, uint64_t n, uint32_t v) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Device scratch of one sas_batch_vet call, released in stream order.
struct VetScratch {
  cudaStream_t s;
  std::vector<void*> ptrs;
  explicit VetScratch(cudaStream_t st) : s(st) {}
  ~VetScratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMallocAsync(&q, std::max<size_t>(count, 1) * sizeof(T), s);
    if (e == cudaSuccess) {
      ptrs.push_back(q);
      *p = static_cast<T*>(q);
    }
    return e;
  }
};

}  // namespace

extern "C" {

int sas_batch_vet(const sas_batch* b, sas_vet* vt, uint32_t* field_out, uint32_t* cand_out, float* logit_out,
                  uint64_t cap, uint64_t* n_out, void* stream) {
  if (!b || !vt || !n_out) return set_error(SAS_ERR_ARG, "null argument");
  *n_out = 0;
  if (vet_device(vt) != b->device) return set_error(SAS_ERR_ARG, "vetter and batch live on different devices");
  cudaStream_t s = (cudaStream_t)stream;
  const BatchDev& B = b->dev;
  VetScratch sc(s);
  uint8_t* d_active = nullptr;
  uint32_t *owner = nullptr, *flag = nullptr, *off = nullptr, *scratch = nullptr;
  std::vector<uint8_t> active(b->n_fields);
  uint32_t max_e = 1;
  for (uint32_t f = 0; f < b->n_fields; ++f) {
    active[f] = b->fallback[f] ? 0 : 1;
    max_e = std::max(max_e, b->hf[f].E);
  }
  cudaError_t e = sc.alloc(&d_active, b->n_fields);
  if (e == cudaSuccess) e = sc.alloc(&owner, B.total_dets);
  if (e == cudaSuccess) e = sc.alloc(&flag, B.total_cand);
  if (e == cudaSuccess) e = sc.alloc(&off, B.total_cand + 1);
  if (e == cudaSuccess) e = sc.alloc(&scratch, scan_scratch_elems(B.total_cand));
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_active, active.data(), b->n_fields, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(owner, 0xFF, std::max<uint64_t>(B.total_dets, 1) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, std::max<uint64_t>(B.total_cand, 1) * 4, s);
  if (e == cudaSuccess) e = batch_launch_owned(B, d_active, owner, flag, s);
  if (e == cudaSuccess) e = launch_scan_u32(flag, off, B.total_cand, scratch, s);
  uint32_t n_batched = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n_batched, off + B.total_cand, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "batch vetting");
  if (n_batched > cap) return set_errorf(SAS_ERR_OVERFLOW, "room for %llu items, %u needed", (unsigned long long)cap, n_batched);
  if (n_batched && (!field_out || !cand_out || !logit_out)) return set_error(SAS_ERR_ARG, "null output buffer");
  if (n_batched) e = batch_launch_compact(B, flag, off, field_out, cand_out, s);
  // fields recomputed on the single-field path follow, each from its own result
  uint64_t n = n_batched;
  std::vector<std::pair<uint32_t, uint64_t>> fb_spans;  // (field, count) in output order
  for (uint32_t f = 0; f < b->n_fields && e == cudaSuccess; ++f) {
    if (!b->fallback[f]) continue;
    const CandView v = result_view(b->fallback[f]);
    if (v.n == 0) continue;
    uint32_t* idx = nullptr;
    if ((e = sc.alloc(&idx, v.n)) != cudaSuccess) break;
    uint64_t k = 0;
    if (int rc = select_owned(v, b->opts[f].n_low, idx, &k, s)) return rc;
    if (n + k > cap) return set_errorf(SAS_ERR_OVERFLOW, "room for %llu items, more needed", (unsigned long long)cap);
    if (k && (!field_out || !cand_out || !logit_out)) return set_error(SAS_ERR_ARG, "null output buffer");
    if (k) {
      k_fill_u32<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(field_out + n, k, f);
      note_launch();
      e = cudaMemcpyAsync(cand_out + n, idx, k * 4, cudaMemcpyDeviceToDevice, s);
    }
    fb_spans.push_back({f, k});
    n += k;
  }
  uint16_t* stamps = nullptr;
  if (e == cudaSuccess && n) e = sc.alloc(&stamps, n * 9 * 225);
  if (e == cudaSuccess && n_batched)
    e = launch_batch_stamps(B.fields, max_e, field_out, cand_out, n_batched, stamps, s);
  {
    uint64_t pos = n_batched;
    for (const auto& fs : fb_spans) {
      if (e != cudaSuccess) break;
      if (fs.second)
        e = launch_stamps(result_view(b->fallback[fs.first]), cand_out + pos, 0, fs.second, stamps + pos * 9 * 225, s);
      pos += fs.second;
    }
  }
  if (e == cudaSuccess && n) e = vet_forward_all(vt, stamps, n, logit_out, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(e, "batch vetting");
  *n_out = n;
  return SAS_OK;
}

int sas_batch_stats(const sas_batch* b, float* ms_last, uint64_t* fallbacks, uint64_t* rebuilds) {
  if (!b) return set_error(SAS_ERR_ARG, "null batch");
  if (ms_last) *ms_last = b->ms_last;
  if (fallbacks) *fallbacks = b->fallback_count;
  if (rebuilds) *rebuilds = b->rebuilds;
  return SAS_OK;
}

void sas_batch_destroy(sas_batch* b) { free_batch(b); }

int sas_autotune(const sas_grid* grid, const sas_catalog* cat, uint32_t n_min, const sas_opts* base,
                 uint32_t reps, void* stream, sas_opts* best, float* best_ms) {
  if (!grid || !cat || !best) return set_error(SAS_ERR_ARG, "null argument");
  if (reps == 0) reps = 3;
  sas_opts o0{};
  if (base) o0 = *base;
  float best_t = 1e30f;
  sas_opts best_o = o0;
  bool any = false;
  // the velocity tile (lattice points per tile) x the bin tile (super-bin side
  // and spatial tile width) x the velocity block, each where the caller left
  // it open; 0 leaves the choice to the planner
  std::vector<std::pair<uint32_t, uint32_t>> vtiles = {{8u, 8u}, {8u, 4u}};
  if (o0.tile_kx || o0.tile_ky) vtiles = {{o0.tile_kx, o0.tile_ky}};
  std::vector<uint32_t> sbs = {1u, 2u, 3u, 4u}, vbs = {0u, 2u, 4u}, bxs = {0u, 32u, 64u};
  if (o0.superbin) sbs = {o0.superbin};
  if (o0.velocity_block) vbs = {o0.velocity_block};
  if (o0.tile_bx || o0.tile_by) bxs = {o0.tile_bx};
  for (const auto& vt : vtiles)
  for (uint32_t sb : sbs)
  for (uint32_t bx : bxs)
    for (uint32_t vb : vbs) {
      sas_opts o = o0;
      o.tile_kx = vt.first;
      o.tile_ky = vt.second;
      o.superbin = sb;
      o.tile_bx = bx;
      o.velocity_block = vb;
      std::vector<float> ts;
      int rc = SAS_OK;
      for (uint32_t r = 0; r <= reps && rc == SAS_OK; ++r) {
        sas_result* res = nullptr;
        rc = sas_stack(grid, cat, n_min, &o, stream, &res);
        if (rc != SAS_OK) break;
        sas_result_info inf;
        sas_result_get_info(res, &inf);
        if (r > 0) ts.push_back(inf.ms_total);
        sas_result_free(res);
      }
      if (rc != SAS_OK) continue;  // a configuration the planner rejects for this field
      std::sort(ts.begin(), ts.end());
      const float med = ts[ts.size() / 2];
      if (med < best_t) {
        best_t = med;
        best_o = o;
        any = true;
      }
    }
  if (!any) return set_error(SAS_ERR_ARG, "no tile configuration fits this field");
  *best = best_o;
  if (best_ms) *best_ms = best_t;
  return SAS_OK;
}

}  // extern "C"
