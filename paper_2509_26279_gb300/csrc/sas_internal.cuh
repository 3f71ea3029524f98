// Internal declarations of the sm_103a shift-and-stack library.
// Shared by the library's translation units only.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>

#include "../../include/sas.h"

namespace sas {

// Exact-integer limits (see sas.h).
constexpr int64_t kLimPos = int64_t(1) << 29;     // |x|, |y|
constexpr int64_t kLimDomain = int64_t(1) << 28;  // |x_min|, nbx*bin, |shift|

// Device-side error flags (bitwise OR into one word).
enum : uint32_t {
  kFlagEpoch = 1u,       // an epoch index >= n_epochs
  kFlagPos = 2u,         // |x| or |y| >= 2^29
  kFlagShift = 4u,       // |shift| >= 2^28 for a used epoch
  kFlagCounter = 8u,     // a stack counter saturated (rerun with wider counters)
  kFlagTimeout = 16u,    // a bounded wait gave up
  kFlagInternal = 32u,   // invariant violated
  kFlagEmitCap = 64u,    // emission list capacity exceeded (rerun with more)
};

constexpr uint32_t kInvalidBucket = 0xFFFFFFFFu;

// A detection after bucketing: 16 bytes, so every bucket range is 16-byte aligned.
struct __align__(16) Det {
  int32_t x, y;
  uint32_t e;
  uint32_t id;
};

// Spatial buckets: detections sorted by (epoch, cy, cx) with coarse cells of
// `cell` mpx whose origin is (gx0, gy0).  Bucket b = (e*ncy + cy)*ncx + cx.
struct CoarseGeom {
  int32_t gx0, gy0;
  int32_t cell;
  int32_t ncx, ncy;
};

// Everything a search kernel needs to know about the lattice and domain.
struct SearchGeom {
  int32_t vx0, vy0, dvx, dvy;
  int32_t nvx, nvy;
  int32_t smin, smax;
  int32_t x_min, y_min;
  int32_t nbx, nby;
  int32_t bin;
  uint32_t E;
  int64_t tph;
  uint64_t v_begin, v_end;
};

// Emitted super-bin (threshold crossing of the stack counters); flags says why.
struct __align__(16) Emit {
  uint32_t v_idx, bx, by, flags;
};
// Which counters the stack kernel emits: every one at or over n_min (one
// threshold); those plus the tile-local peaks at or over n_low; or only the
// tile-local peaks at or over n_low.
enum : uint32_t { kSelectAll = 0u, kSelectPlainAndPeaks = 1u, kSelectPeaks = 2u };
enum : uint32_t {
  kEmitPlain = 1u,    // the super-bin's count reached n_min: its bins are counted against n_min
  kEmitLowPeak = 2u,  // count >= n_low and no neighbour of the tile larger: counted against n_low
};

// Candidate sort key, compared lexicographically (a, b, c):
//   a = (~distinct << 32) | ~raw,  b = (v_idx << 32) | by,  c = bx.
struct __align__(8) Key {
  uint64_t a, b;
  uint32_t c, pad;
};

// Stack kernel configuration.
struct TileCfg {
  int kx, ky;        // lattice points per velocity tile
  int bvx, bvy;      // velocity tiles per velocity block (share one staged detection set)
  int tx, ty;        // super-bins per spatial tile
  int s;             // bins per super-bin side
  int cb;            // counter bits: 8, 16, 32
  int nt;            // threads per CTA
  int ec;            // epochs per chunk (<= 256)
  int rows;          // bucket rows per epoch window (ec * rows <= seg_cap)
  int seg_cap;       // segment slots per chunk (= nt)
  int scap;          // staged detection records
  int emit_cap;      // per-CTA emission buffer entries
  int peak_cap;      // per-CTA list of counters awaiting the peak test (0: no peak selection)
  size_t smem;       // dynamic shared memory bytes
};

struct StackArgs {
  SearchGeom g;
  CoarseGeom cg;
  TileCfg tc;
  uint32_t magic;      // umulhi(X, magic) = X / (s*bin) for 0 <= X < tile extent
  int32_t bin_is_one;  // s*bin == 1: the quotient is X itself
  int32_t merge;       // the P columns of a counter word span at most two super-bins
  uint32_t n_min;
  uint32_t n_low;            // the counters' top bit means count >= n_low (n_low == n_min: one threshold)
  uint32_t select;           // kSelectAll, kSelectPlainAndPeaks or kSelectPeaks
  int32_t nvt_x, nvt_y;      // velocity blocks along kx, ky
  int32_t kx_lo, ky_lo;      // first lattice column/row covered by the blocks
  int32_t nst_x, nst_y;      // spatial tiles
  uint64_t n_tiles;          // work units = velocity blocks x spatial tiles
  const Det* dets;
  const uint8_t* w;          // [n] weight per detection id (weighted stacking), or null: all 1
  const uint32_t* boff;      // [E*ncy*ncx + 1]
  const uint32_t* ecount;    // [E] detections per epoch
  const int32_t* sxt;        // [nvx][E] shift in x
  const int32_t* syt;        // [nvy][E] shift in y
  Emit* emits;
  uint32_t emit_cap;
  uint32_t* n_emit;
  unsigned long long* n_pairs;
  unsigned long long* balance;  // sum over tiles of (counted - added); nonzero: a counter wrapped
  uint32_t* flags;
  unsigned long long* tile_counter;
};

// Process-wide count of kernels launched by the library (sas_kernel_launches).
void note_launch(uint32_t k = 1);

// Records the message of a failed call for sas_last_error() (printf-style) and
// returns code.
int set_errorf(int code, const char* fmt, ...);
inline int set_error(int code, const char* msg) { return set_errorf(code, "%s", msg); }

// ---- planning (sas_plan.cu) -------------------------------------------------

struct DevInfo {
  int sms = 0;
  int smem_optin = 0;
  int smem_per_sm = 0;
  bool ready = false;
};
int device_info(int dev, DevInfo* out);
uint32_t magic_for(int32_t bin);  // ceil(2^32 / bin)

// The plan of one field's search (sizes only; no device work).
struct FieldPlan {
  TileCfg tc;
  CoarseGeom cg;
  SearchGeom g;
  int kx, ky, cb, sb;
  int ky_lo, ky_hi, n_rows;
  uint64_t nb;  // buckets: E * ncy * ncx
  int64_t dT;   // max(t) - min(t)
};
// Super-bin side (1..4) for a search at threshold n_min (unit increments).
int choose_superbin(const sas_grid_desc& d, uint64_t n, uint32_t n_min, uint64_t nv);
int plan_field(const sas_grid_desc& d, uint64_t n, uint32_t E, const int64_t* t, int64_t tph,
               uint32_t n_min, uint64_t v_begin, uint64_t v_end, const sas_opts& o,
               const DevInfo& di, FieldPlan* fp);
// Same plan with counters twice as wide (after a counter wrapped).
int replan_wider(const sas_grid_desc& d, uint64_t n, uint32_t n_min, const sas_opts& o,
                 const DevInfo& di, FieldPlan* fp);
// Geometry, tiling and division parts of the stack kernel's arguments
// (n_low: the lower threshold of the tile-peak selection, 0 or n_min when off;
// peaks_only: emit the tile-local peaks alone).
struct StackArgs;
void fill_stack_args(const FieldPlan& fp, uint32_t n_min, uint32_t n_low, uint32_t peaks_only, StackArgs* sa);

// ---- launchers (defined in the .cu files) ----------------------------------

// sas_prep.cu
cudaError_t launch_ingest(const int32_t* x, const int32_t* y, const uint16_t* epoch, uint64_t n,
                          uint32_t E, CoarseGeom cg, uint32_t* bucket_count, uint32_t* ecount,
                          uint32_t* bucket_of, uint32_t* flags, cudaStream_t s);
cudaError_t launch_scatter(const int32_t* x, const int32_t* y, const uint16_t* epoch, uint64_t n,
                           const uint32_t* bucket_of, uint32_t* cursor, Det* dets, cudaStream_t s);
cudaError_t launch_epoch_setup(uint32_t E, const int64_t* t, const uint32_t* ecount, int64_t* dt,
                               int64_t* t0, cudaStream_t s);
cudaError_t launch_shift_tables(const SearchGeom& g, const int64_t* dt, const uint32_t* ecount,
                                int32_t* sxt, int32_t* syt, uint32_t* flags, cudaStream_t s);
// exclusive scan, out[i] = sum(in[0..i)), out has n+1 entries
cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* scratch,
                            cudaStream_t s);
cudaError_t launch_scan_u32_to_u64(const uint32_t* in, unsigned long long* out, uint64_t n,
                                   unsigned long long* scratch, cudaStream_t s);
size_t scan_scratch_elems(uint64_t n);

// sas_stack.cu (kernel: sas_stack_kernel.cuh)
bool stack_config_supported(int kx, int ky, int cb);
size_t stack_smem_bytes(const TileCfg& tc);
size_t stack_counter_bytes(const TileCfg& tc);
// Launches the instantiation with peak selection when a.select != kSelectAll.
cudaError_t launch_stack(const StackArgs& a, int grid, cudaStream_t s);
// One persistent launch over the units of several fields (per-field StackArgs in
// device memory; field f owns units [unit_base[f], unit_base[f+1]) of counter);
// peaks: the fields' select is not kSelectAll (all fields of a launch agree).
cudaError_t launch_stack_multi(int kx, int ky, int cb, bool peaks, const StackArgs* fargs,
                               const unsigned long long* unit_base, int n_fields,
                               unsigned long long* counter, size_t smem, int grid, cudaStream_t s);
// Sets the shared-memory limit of both instantiations.
cudaError_t stack_set_smem_attr(int kx, int ky, int cb, size_t smem);
// sas_stack_peaks.cu: the same with peak selection
cudaError_t launch_stack_peaks(const StackArgs& a, int grid, cudaStream_t s);
cudaError_t launch_stack_multi_peaks(int kx, int ky, int cb, const StackArgs* fargs,
                                     const unsigned long long* unit_base, int n_fields,
                                     unsigned long long* counter, size_t smem, int grid, cudaStream_t s);
cudaError_t stack_set_smem_attr_peaks(int kx, int ky, int cb, size_t smem);

// sas_post.cu
// Appends one key per bin of an emitted super-bin that lies in the domain and
// has >= n_min distinct epochs -- or, with weights wts (by detection id), a
// score >= n_min (keys needs room for s*s keys per emission).
cudaError_t launch_cell_count(const Emit* emits, uint32_t n_emit, int s_bins, const SearchGeom& g,
                              const CoarseGeom& cg, const Det* dets, const uint32_t* boff,
                              const uint32_t* ecount, const int32_t* sxt, const int32_t* syt,
                              uint32_t n_min, uint32_t n_low, Key* keys, uint32_t* n_valid,
                              unsigned long long* raw_total, const uint8_t* wts, cudaStream_t s);
cudaError_t launch_sort_keys(Key* keys, uint32_t n, uint32_t n_pad, cudaStream_t s);
// Sorts every aligned segment of `seg` keys (a power of two) of keys[0..n_total)
// ascending; n_total is a multiple of seg.
cudaError_t launch_sort_segments(Key* keys, uint32_t n_total, uint32_t seg, cudaStream_t s);
cudaError_t launch_key_raw(const Key* keys, uint32_t n, uint32_t* raw, cudaStream_t s);
cudaError_t launch_gather_ids(const Key* keys, uint32_t n, const unsigned long long* id_off,
                              const SearchGeom& g, const CoarseGeom& cg, const Det* dets,
                              const uint32_t* boff, const uint32_t* ecount, const int32_t* sxt,
                              const int32_t* syt, uint32_t* ids_tmp, uint32_t* ids,
                              uint32_t* flags, cudaStream_t s);
cudaError_t launch_write_candidates(const Key* keys, uint32_t n, const unsigned long long* id_off,
                                    sas_candidate* out, cudaStream_t s);

// A finished search's candidates together with what is needed to recount any
// cell of its lattice: bucketed catalog, per-epoch counts, shift tables.
struct CandView {
  const sas_candidate* cands;  // device, output order
  uint64_t n;
  SearchGeom g;
  CoarseGeom cg;
  const Det* dets;
  const uint32_t* boff;
  const uint32_t* ecount;
  const int32_t* sxt;
  const int32_t* syt;
  const uint32_t* ids;         // device, candidate i's ids at [id_off, id_off + id_len)
  uint64_t n_det;              // catalog size
};

// sas_stamps.cu: 9 x 15 x 15 distinct-epoch count stamps, u16 [count][9][15][15],
// of candidates idx[0..count) (idx NULL: candidates first..first+count).
cudaError_t launch_stamps(const CandView& v, const uint32_t* idx, uint64_t first, uint64_t count,
                          uint16_t* out, cudaStream_t s);

// sas_select.cu: ascending indices of the local peaks of v's candidates (no
// candidate within one lattice step and one bin precedes them in the output
// order) into idx (device, room for v.n); *n_peaks on the host; synchronizes s.
// Returns a sas_status.
int select_peaks(const CandView& v, uint32_t* idx, uint64_t* n_peaks, cudaStream_t s);

// sas_select.cu: ownership selection -- detection d belongs to the first
// candidate (output order) whose ids contain it; candidate i is kept when it
// owns at least half of its ids or (n_keep > 0) at least n_keep of them.  Same
// output convention as select_peaks.
int select_owned(const CandView& v, uint32_t n_keep, uint32_t* idx, uint64_t* n_kept, cudaStream_t s);

// sas_vet.cu: logits of n stamps (device), in batches of the vetter's
// max_batch; the device a vetter lives on.
cudaError_t vet_forward_all(sas_vet* vt, const uint16_t* stamps, uint64_t n, float* logits, cudaStream_t s);
int vet_device(const sas_vet* vt);

// sas_peel.cu: cluster finding (Sec. 2.1 step 3) over v's candidates with
// threshold n_min, at most max_clusters clusters; on success out holds device
// arrays (owned by the caller) of the clusters and their ids.
struct PeelOut {
  sas_candidate* cands = nullptr;
  uint32_t* ids = nullptr;
  uint64_t n = 0, n_ids = 0;
};
// sequential: run the loop as stated in one block instead of rounds of local maxima
int peel_clusters(const CandView& v, uint32_t n_min, uint32_t max_clusters, bool sequential, cudaStream_t s,
                  PeelOut* out);

// sas_refine.cu: refinement and gathering (Sec. 2.1 steps 4-6).
struct RefineIn {
  struct {
    const Det* dets;       // bucketed catalog, overflow bucket last
    const uint32_t* boff;  // [nb + 2]
    const int64_t* dt;     // [E] epoch time - t0, ticks
    SearchGeom g;
    CoarseGeom cg;
    uint64_t n_det;
  } search;
  struct {
    const sas_candidate* cands;
    uint64_t n;
    const uint32_t* ids;
  } clusters;
};
struct RefineOut {
  sas_track* tracks = nullptr;
  uint32_t* ids = nullptr;
  uint32_t n = 0, n_ids = 0;
};
int refine_tracks(const RefineIn& in, const sas_refine_opts& o, cudaStream_t s, RefineOut* out);

// sas_api.cu: the candidate view of a finished search.
CandView result_view(const sas_result* r);

// sas_probe.cu
cudaError_t run_atomic_probe(uint32_t iters, cudaStream_t s, double* ops_per_s, double* sm_mhz);
cudaError_t run_red_probe(uint32_t iters, cudaStream_t s, double* ops_per_s, double* sm_mhz);
cudaError_t run_or64_probe(uint32_t iters, cudaStream_t s, double* ops_per_s, double* sm_mhz);

// sas_noalloc.cu (returns a sas_status; *err gets the message on failure)
int noalloc_cell_counts(const sas_grid_desc& d, const sas_catalog* cat, const uint32_t* cells,
                        uint64_t n_cells, uint32_t* distinct, uint32_t* raw, void* stream,
                        std::string* err);

// ---- small device helpers ---------------------------------------------------

__host__ __device__ inline int64_t floor_div64(int64_t a, int64_t b) {  // b > 0
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

__host__ __device__ inline int32_t floor_div32(int32_t a, int32_t b) {  // b > 0
  int32_t q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

__host__ __device__ inline uint32_t div_ceil_u32(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

}  // namespace sas
