/*
 * sas.h -- C ABI of the GB300 (sm_103a) catalog shift-and-stack library.
 *
 * The operation (Stetzler et al., "An Efficient Shift-and-Stack Algorithm
 * Applied to Detection Catalogs", Sec. 2.1): given a detection catalog
 * C = [x_i, y_i, t_i], a set of hypothesis velocities V, a clustering radius
 * (bin size) Delta-x and a threshold N_min,
 *   1. Project every detection to the reference epoch t0 = the earliest time
 *      in the catalog:  x' = x - floor(vx (t - t0) / TPH),  y' likewise
 *      (linear motion model, Sec. 2 Eq. 1-2; residuals Eq. 3-8);
 *   2. Cluster: for every velocity build a 2-D histogram of the projected
 *      positions at resolution Delta-x; a cell counts the DISTINCT epochs of
 *      the detections in it (and the raw number of detections);
 *   3. Find clusters, in threshold form: every cell with at least N_min
 *      distinct epochs is a candidate, together with the ids of all the
 *      detections that contributed to it.
 * Candidates come out ordered by (distinct desc, raw desc, v_idx asc, by asc,
 * bx asc) -- Sec. 3.3 ranks clusters by their number of detections -- and may be
 * cut to the first K (the paper keeps the first 1000).
 *
 * Integer fixed point, so every step is exact:
 *   positions  int32 milli-pixels (mpx)      velocities  int32 mpx per hour
 *   times      int64 ticks, ticks_per_hour (TPH) > 0
 *   shift      floor(v * (t - t0) / TPH)     bin  floor((x' - x_min) / bin)
 * ("floor" is the mathematical floor, also for negative values; bins are
 * half-open.)
 *
 * Exact-integer limits (violations return SAS_ERR_RANGE, nothing is computed):
 *   |x|, |y| < 2^29 for every detection;  |x_min|, |y_min| < 2^28;
 *   nbx*bin < 2^28 and nby*bin < 2^28;    nvx*nvy < 2^31;
 *   |shift| < 2^28 for every lattice velocity and every epoch that has a
 *   detection;  (tile_kx - 1) * |dvx| * (max(t) - min(t)) / TPH < 2^23 and
 *   likewise for y (the shift spread inside one velocity tile);
 *   max(t) - min(t) < 2^32;  n < 2^31;  1 <= E <= SAS_MAX_EPOCHS.
 *
 * Threading and streams: every call enqueues its device work on the caller's
 * CUDA stream (NULL = the legacy default stream) and returns when its outputs
 * are complete.  Handles are not safe for concurrent use from several threads.
 * Errors: every entry point returns a sas_status; sas_last_error() gives a
 * message (thread-local, valid until the next call on that thread).
 */
#ifndef SAS_H_
#define SAS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAS_ABI_VERSION 2
#define SAS_MAX_EPOCHS 1024

typedef enum sas_status {
  SAS_OK = 0,
  SAS_ERR_ARG = 1,       /* null pointer, zero size or inconsistent descriptor      */
  SAS_ERR_RANGE = 2,     /* an input is outside the exact-integer limits above      */
  SAS_ERR_OVERFLOW = 3,  /* a caller buffer is too small; the needed sizes are set  */
  SAS_ERR_CUDA = 4,      /* CUDA runtime error (message in sas_last_error)          */
  SAS_ERR_OOM = 5,       /* device or host allocation failed                        */
  SAS_ERR_TIMEOUT = 6,   /* a bounded device-side wait gave up                      */
  SAS_ERR_INTERNAL = 7   /* internal invariant violated (a bug: please report)      */
} sas_status;

/* Velocity lattice and histogram domain (the set V and the bin size Delta-x of
 * Sec. 2.1; the lattice spacing follows the bound Delta-v <= Delta-x / Delta-t
 * of Sec. 2, Eq. 15-16).  Lattice point (kx, ky), 0 <= kx < nvx, 0 <= ky < nvy,
 * has velocity (vx0 + kx*dvx, vy0 + ky*dvy) mpx/h and index v_idx = ky*nvx + kx.
 * If speed_min or speed_max is nonzero only lattice points with
 * speed_min^2 <= vx^2 + vy^2 <= speed_max^2 are searched ("all on-sky angles"
 * over a rate range, Sec. 3.3); v_idx numbering is unchanged.  The histogram
 * covers [x_min, x_min + nbx*bin) x [y_min, y_min + nby*bin) mpx; projections
 * outside it are dropped. */
typedef struct sas_grid_desc {
  int32_t vx0, vy0;
  int32_t dvx, dvy;          /* any sign, zero allowed                            */
  uint32_t nvx, nvy;         /* >= 1                                              */
  int32_t speed_min;         /* mpx/h, >= 0                                       */
  int32_t speed_max;         /* mpx/h, >= speed_min (both 0 = whole lattice)      */
  int32_t x_min, y_min;      /* mpx                                               */
  uint32_t nbx, nby;         /* >= 1                                              */
  int32_t bin;               /* mpx, >= 1                                         */
} sas_grid_desc;

/* Detection catalog C = [x_i, y_i, t_i] (Sec. 2.1), structure of arrays.
 * Detection i was observed at time t[epoch[i]].  The caller owns every array.
 * With on_device = 1, x, y and epoch are device pointers (the library only
 * reads them, during the call); with on_device = 0 they are host pointers and
 * are copied.  t is always a host array of n_epochs entries. */
typedef struct sas_catalog {
  uint64_t n;
  const int32_t* x;          /* [n] mpx                                           */
  const int32_t* y;          /* [n] mpx                                           */
  const uint16_t* epoch;     /* [n] each < n_epochs                               */
  uint32_t n_epochs;         /* E                                                 */
  const int64_t* t;          /* [E] ticks, host memory                            */
  int64_t ticks_per_hour;    /* TPH                                               */
  int32_t on_device;
  int32_t reserved;
} sas_catalog;

/* Optional knobs of sas_stack (pass NULL for defaults).  Tile fields of 0 let
 * the library choose (built-in table or the autotuner cache). */
typedef struct sas_opts {
  uint64_t v_begin, v_end;   /* search only lattice indices [v_begin, v_end); 0,0 = all */
  uint64_t max_candidates;   /* keep the first K candidates in output order; 0 = all    */
  uint32_t tile_kx, tile_ky; /* lattice points per velocity tile: kx 4 or 8, ky 1, 2 or 4 */
  uint32_t tile_bx, tile_by; /* counters (super-bins) per spatial tile side             */
  uint32_t counter_bits;     /* 8, 16 or 32; 0 = choose                                 */
  uint32_t coarse_bins;      /* spatial bucket size in bins; 0 = choose                 */
  uint32_t superbin;         /* bins per counter side, 1..4; 0 = choose                 */
  uint32_t velocity_block;   /* velocity tiles per side sharing one staged detection
                                set, 1..8; 0 = choose                                   */
  uint32_t n_low;            /* 0: one threshold.  1 <= n_low <= n_min: also report the
                                cells with >= n_low distinct epochs whose super-bin is
                                a tile-local peak (see sas_stack); not with weights    */
  uint32_t peaks_only;       /* 1: report only the cells of tile-local peaks (>= n_low,
                                or >= n_min when n_low is 0); not with weights         */
} sas_opts;

/* One candidate trajectory: the cell (v_idx, bx, by) of the 3-D histogram with
 * count >= N_min distinct epochs, its raw number of detections and the range
 * [id_off, id_off + id_len) of its contributing detection ids (ascending
 * indices into the caller's catalog arrays) in the id array.  id_len == raw. */
typedef struct sas_candidate {
  uint32_t v_idx;
  uint32_t bx, by;
  uint32_t count;            /* distinct epochs                                   */
  uint32_t raw;              /* detections                                        */
  uint32_t id_len;
  uint64_t id_off;
} sas_candidate;

/* Summary of a finished search. */
typedef struct sas_result_info {
  uint64_t n_candidates;     /* after the optional top-K cut                      */
  uint64_t n_ids;            /* total contributing ids of those candidates        */
  uint64_t n_pairs;          /* in-domain (detection, velocity) pairs = detection-shifts */
  uint64_t n_emitted;        /* cells that crossed the counter threshold (superset) */
  int64_t t0;                /* reference epoch (ticks)                           */
  uint32_t counter_bits;     /* counter width the stack kernel ran with           */
  uint32_t tile_kx, tile_ky, tile_bx, tile_by;  /* the plan it ran with             */
  uint32_t superbin;         /* bins per counter side                             */
  uint32_t vblock_x, vblock_y;  /* velocity tiles per staged detection set          */
  uint32_t staged_cap;       /* staged detection records per CTA                  */
  uint32_t n_low;            /* lower threshold of the peak selection (n_min when off) */
  float ms_stack;            /* device time of the stack kernel (CUDA events)     */
  float ms_total;            /* device time of the whole call                     */
  float ms_prep;             /* ingest, buckets, reference epoch, shift tables    */
  float ms_count;            /* exact counts of emitted cells + ordering          */
  float ms_ids;              /* contributing ids + candidate records (+ host sync) */
  uint32_t peaks_only;       /* the selection it ran with (sas_opts.peaks_only)    */
} sas_result_info;

typedef struct sas_grid sas_grid;      /* opaque, owned by the library */
typedef struct sas_result sas_result;  /* opaque, owned by the library */

/* Library version string and the ABI version it implements. */
const char* sas_version(void);
int sas_abi_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads): a diagnostic for counting launches per search. */
uint64_t sas_kernel_launches(void);

/* Message of the last failed call on this thread ("" if none). */
const char* sas_last_error(void);

/* Validate a grid descriptor and return a handle (host memory only).
 * Errors: SAS_ERR_ARG (null, zero sizes, speed_max < speed_min),
 * SAS_ERR_RANGE (limits above).  *out is untouched on error. */
int sas_create_grid(const sas_grid_desc* desc, sas_grid** out);
void sas_destroy_grid(sas_grid* grid);
int sas_grid_get_desc(const sas_grid* grid, sas_grid_desc* desc);

/* Weighted stacking -- the likelihood accumulation the paper proposes for
 * future work (Sec. 5): detection i carries an integer weight w[i] in
 * [0, 255] (a fixed-point likelihood or S/N; uint8, in host or device memory
 * like the catalog arrays, indexed like them).  A cell's score is the sum over
 * epochs of the largest weight among that epoch's detections in the cell
 * (all weights 1: the distinct-epoch count); candidates are the cells with
 * score >= s_min, in the order (score desc, raw desc, v_idx, by, bx), and
 * sas_candidate.count holds the score.  Everything else as sas_stack; the
 * result supports sas_candidates, sas_stamps and sas_refine (not sas_peel,
 * whose recounts are distinct epochs).  s_min in [1, 2^31].
 * Errors: as sas_stack; SAS_ERR_ARG for null weights with n > 0, or for
 * opts->n_low or opts->peaks_only set (peak selection counts distinct epochs). */
int sas_stack_weighted(const sas_grid* grid, const sas_catalog* cat, const uint8_t* weights, uint32_t s_min,
                       const sas_opts* opts, void* stream, sas_result** out);

/* Run the search (Sec. 2.1 steps 1-3) on the current CUDA device.
 * grid, cat: see above.  n_min >= 1.  opts may be NULL.
 * With opts->n_low in [1, n_min) the list holds every cell with >= n_min
 * distinct epochs and, in addition, every cell with >= n_low distinct epochs
 * whose S x S super-bin (S = info.superbin) is a tile-local peak of the raw
 * counts: its raw count R(v, B) (detections whose projection at lattice point
 * v lands in one of B's bins) is >= n_low and no super-bin B' at a lattice
 * point v' of the same velocity tile (info.tile_kx x info.tile_ky lattice
 * points; tiles start at kx = 0 and at ky = v_begin / nvx) and of the same
 * spatial tile (info.tile_bx x info.tile_by super-bins from bin 0) with
 * |kx'-kx|, |ky'-ky|, |B'x-Bx|, |B'y-By| all <= 1 has R(v', B') > R(v, B)
 * (lattice points outside the searched set count 0).  This prunes the
 * neighbouring cells a mover or a noise alignment raises before they are
 * counted (an extension of the paper's threshold; the candidate list stays in
 * the same order).  With opts->peaks_only = 1 the list holds only the cells
 * with >= n_low distinct epochs (n_min when n_low is 0) whose super-bin is such
 * a peak: the cells at or above n_min elsewhere -- the neighbourhood every
 * mover raises around its best cell -- are pruned too, before counting, so
 * the list is no longer complete at n_min (sas_peel then refuses it).
 * stream: a
 * cudaStream_t (NULL = legacy default).  On success *out holds a new result
 * that the caller releases with sas_result_free; the result owns its device
 * memory.  The call synchronizes the stream before returning.
 * Errors: SAS_ERR_ARG (also n_low > n_min, peaks_only > 1, tile sides of
 * 4096 super-bins or more), SAS_ERR_RANGE (catalog or shifts out of limits, or an
 * epoch index >= n_epochs), SAS_ERR_OOM, SAS_ERR_CUDA; *out is untouched. */
int sas_stack(const sas_grid* grid, const sas_catalog* cat, uint32_t n_min,
              const sas_opts* opts, void* stream, sas_result** out);

int sas_result_get_info(const sas_result* result, sas_result_info* info);

/* Copy the candidates and their ids out of a result, in output order.
 * out[0..min(cap, n)) and ids[0..min(ids_cap, n_ids)) are written; *n_total
 * and *n_ids_total (either may be NULL) receive the full sizes.  With
 * on_device = 1 the destinations are device pointers.  Returns
 * SAS_ERR_OVERFLOW (after the partial copy) when cap or ids_cap is too small;
 * out or ids may be NULL with cap or ids_cap 0 to query sizes.  Both copies
 * are issued together and waited for once; page-locked host destinations
 * (reused from call to call) copy fastest. */
int sas_candidates(const sas_result* result, sas_candidate* out, uint64_t cap,
                   uint64_t* n_total, uint32_t* ids, uint64_t ids_cap,
                   uint64_t* n_ids_total, int on_device);

void sas_result_free(sas_result* result);

/* ---- Batched search: many fields in one graph-captured pass ---------------
 *
 * Many fields (CCDs) with uneven detection and epoch counts are searched by
 * one pass of every kernel -- one persistent stack launch per stack kernel
 * configuration (velocity tile and counter width) over the work units of its
 * fields -- recorded once as a CUDA graph by sas_batch_create and
 * replayed by sas_batch_run.  (The paper searches each CCD independently,
 * Sec. 3.3; batching is an implementation pattern with the same results.)
 *
 * grids[f], cats[f], n_min[f]: field f (catalogs in device memory, on_device
 * = 1, n >= 1; 1 <= n_min <= 128).  opts: NULL or an array of n_fields option
 * sets (v_begin/v_end are ignored; n_low and peaks_only as in sas_stack, per
 * field).  The
 * batch keeps the catalogs' device pointers:
 * the caller may rewrite their contents between runs (same sizes, same
 * epoch times) and must keep them alive until sas_batch_destroy.
 * sas_batch_run replays the pass on `stream` and synchronizes; a field that
 * exceeded the batch's fixed capacities (emissions, 32768 candidates, ids) or
 * whose counters wrapped is recomputed by sas_stack, so every field's result
 * equals sas_stack's.  Results stay valid until the next run.
 * Errors: as sas_stack; SAS_ERR_ARG for fields that cannot share a launch. */
typedef struct sas_batch sas_batch;
int sas_batch_create(const sas_grid* const* grids, const sas_catalog* cats, const uint32_t* n_min,
                     uint32_t n_fields, const sas_opts* opts, void* stream, sas_batch** out);
int sas_batch_run(sas_batch* batch, void* stream);
int sas_batch_field_info(const sas_batch* batch, uint32_t field, sas_result_info* info);
int sas_batch_candidates(const sas_batch* batch, uint32_t field, sas_candidate* out,
                         uint64_t cap, uint64_t* n_total, uint32_t* ids, uint64_t ids_cap,
                         uint64_t* n_ids_total, int on_device);
/* Device time (ms, CUDA events) of the last replayed pass, the number of field
 * fallbacks (fields recomputed on the single-field path: a counter wrapped, or
 * the grown capacities would not fit in device memory) and the number of
 * rebuilds so far (a replay that found a field over its key, emission or id
 * capacity grows those capacities to what the field reported, rebuilds the
 * arena and the graph, and replays).  Any output may be NULL. */
int sas_batch_stats(const sas_batch* batch, float* ms_last, uint64_t* fallbacks, uint64_t* rebuilds);
void sas_batch_destroy(sas_batch* batch);
/* sas_peaks, sas_stamps and sas_owned for field `field` of the last run (idx NULL in
 * sas_batch_stamps: candidates 0..count). */
int sas_batch_peaks(const sas_batch* batch, uint32_t field, uint32_t* idx, uint64_t* n_peaks,
                    void* stream);
int sas_batch_stamps(const sas_batch* batch, uint32_t field, const uint32_t* idx, uint64_t count,
                     uint16_t* out, void* stream);
int sas_batch_owned(const sas_batch* batch, uint32_t field, uint32_t n_keep, uint32_t* idx,
                    uint64_t* n_kept, void* stream);

typedef struct sas_vet sas_vet;

/* Vetting of every field of the last run in one pass: ownership selection
 * (as sas_owned with n_keep = the field's n_low, which is its n_min when the
 * field has no lower threshold), stamps of the kept candidates and their CNN logits (as
 * sas_vet_forward).  Writes one item per kept candidate: field_out[i],
 * cand_out[i] (its index in the field's candidate list) and logit_out[i]
 * (device arrays with room for `cap` items; the batch's total candidate count
 * always suffices), *n_out on the host.  Items are grouped by field, candidate
 * indices ascending within a field; the fields searched in the batch come
 * first in field order, then any field recomputed on the single-field path.
 * The vetter must live on the batch's device.  Synchronizes the stream.
 * Errors: SAS_ERR_ARG, SAS_ERR_OVERFLOW (cap too small), SAS_ERR_OOM,
 * SAS_ERR_CUDA. */
int sas_batch_vet(const sas_batch* batch, sas_vet* vetter, uint32_t* field_out, uint32_t* cand_out,
                  float* logit_out, uint64_t cap, uint64_t* n_out, void* stream);

/* Autotuner: times sas_stack on (grid, cat, n_min) for every combination of
 * the velocity tile (tile_kx x tile_ky in {8 x 8, 8 x 4}), the bin tile
 * (superbin in {1, 2, 3, 4} bins per super-bin side, tile_bx in {planner, 32,
 * 64} super-bins per spatial tile row, tile_by from the planner) and the
 * velocity block (velocity_block in {planner, 2, 4}); a field of *base that is
 * set (nonzero) is kept instead of swept, and combinations the planner
 * rejects for this field are skipped.  `reps` timed runs each after one
 * warm-up; *best gets the options with the lowest median device time of the
 * whole search (*best_ms).  Every combination gives the same candidates
 * (Sec. 2.1 steps 1-3 are independent of the tiling); only the speed differs. */
int sas_autotune(const sas_grid* grid, const sas_catalog* cat, uint32_t n_min,
                 const sas_opts* base, uint32_t reps, void* stream, sas_opts* best,
                 float* best_ms);

/* Exact counts of chosen cells without allocating device memory.
 *
 * The paper has no counterpart; this is a service for callers that cannot
 * allocate device memory while they run -- a process that has handed all of
 * its device memory to its own pool under a fixed budget, or code issuing work
 * from a loop that must never wait on the CUDA allocator.  For each cell
 * (v_idx, bx, by) it returns the same numbers as the exact-count step of
 * sas_stack: distinct[i] = number of distinct epochs and raw[i] = number of
 * detections of the catalog that project into the cell when shifted to the
 * earliest detection time.
 *
 * cells: device array of n_cells triples (v_idx, bx, by) as uint32.
 * distinct, raw: device arrays of n_cells uint32, owned by the caller.
 * cat: x, y and epoch must be device arrays (on_device = 1); t is host memory.
 * The call writes only distinct and raw; it allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call).  Its working state (epoch times and
 * flags) lives in one fixed 16 KiB array inside the library, which every GPU
 * that loads the library holds until the process exits; so n_epochs may not
 * exceed 1024 (SAS_ERR_RANGE otherwise).  The first call on a device does a
 * set-up (it looks up that array's device address and the device's SM count),
 * so make that first call before any stream capture.  All calls on a device
 * share the array: calls whose GPU work overlaps (other streams, other host
 * threads) race, and must be serialized by the caller.  Each call resets the
 * parts that must start at zero.  Before returning, the call synchronizes the
 * stream to read its status back.  Counting is exact in 64-bit arithmetic; the cost is
 * O(n_cells * n) (it scans the whole catalog per cell), meant for modest
 * numbers of cells.
 * Errors: SAS_ERR_ARG (nulls, host catalog, a cell outside the lattice or the
 * domain: its outputs are set to 0xffffffff), SAS_ERR_RANGE (n_epochs, an epoch
 * index >= n_epochs, |x| or |y| >= 2^29), SAS_ERR_CUDA. */
int sas_cell_counts_noalloc(const sas_grid* grid, const sas_catalog* cat, const uint32_t* cells,
                            uint64_t n_cells, uint32_t* distinct, uint32_t* raw, void* stream);

/* ---- Candidate vetter ---------------------------------------------------------
 *
 * Filtering the search results better is the paper's suggested route to fainter
 * objects (Sec. 5).  The vetter scores each candidate with a small CNN from
 * its count stamp, so the search can run at a lower n_min.
 *
 * Stamp of candidate (v_idx, bx, by), kx = v_idx % nvx, ky = v_idx / nvx: a
 * [9][15][15] uint16 array.  Plane q = (dy + 1) * 3 + (dx + 1), dx, dy in
 * {-1, 0, 1}, is the distinct-epoch histogram (Sec. 2.1 step 2) of lattice
 * point (kx + dx, ky + dy) over bins (bx - 7 + j, by - 7 + i) at element
 * (i, j).  Points off the lattice (the whole lattice, not only the searched
 * v range or annulus) and bins off the domain count 0.  Counts saturate at
 * 65535. */

/* Stamps of candidates [first, first + count) of a result, in output order,
 * into out: a device array of count * 9 * 15 * 15 uint16 owned by the
 * caller.  Runs on the current device (the result's) and is asynchronous on
 * `stream`.  Errors: SAS_ERR_ARG (null result, range beyond n_candidates,
 * null out with count > 0), SAS_ERR_CUDA. */
int sas_stamps(const sas_result* result, uint64_t first, uint64_t count, uint16_t* out,
               void* stream);
/* Stamps of candidates idx[0..count) (device uint32 indices into the result's
 * candidates, each < n_candidates) into out; otherwise as sas_stamps. */
int sas_stamps_indexed(const sas_result* result, const uint32_t* idx, uint64_t count,
                       uint16_t* out, void* stream);

/* Local peaks of a result's candidates: candidate i is a peak when no other
 * candidate within one lattice step in kx and in ky and one bin in bx and in
 * by precedes it in the output order.  A mover's cluster of neighbouring
 * threshold crossings (Sec. 2.2's velocity tolerance spans several lattice
 * steps) keeps its best cell; this is a cheap, order-defined stand-in for the
 * paper's peeling of clusters (Sec. 2.1 step 3).  Writes the ascending
 * indices of the peaks to idx (device uint32, room for n_candidates) and their
 * number to *n_peaks (host); synchronizes the stream.
 * Errors: SAS_ERR_ARG, SAS_ERR_OOM, SAS_ERR_CUDA. */
int sas_peaks(const sas_result* result, uint32_t* idx, uint64_t* n_peaks, void* stream);

/* Ownership selection of a result's candidates, a one-pass stand-in for the
 * paper's peeling of clusters (Sec. 2.1 step 3: the best cluster's detections
 * are removed before the next is taken).  Each detection belongs to the first
 * candidate, in output order, whose ids contain it; candidate i is kept when it
 * owns at least half of its ids, or, with n_keep > 0, at least n_keep of them
 * (what it alone holds would still pass a threshold of n_keep after the peel:
 * a fainter mover crossing a brighter one keeps its cell; pass the search's
 * n_min).  A mover's ghost cells (nearby velocities and bins that also collect
 * its detections) lose their detections to its best cell and drop out.
 * Output as sas_peaks.  Uses O(catalog size) scratch. */
int sas_owned(const sas_result* result, uint32_t n_keep, uint32_t* idx, uint64_t* n_kept,
              void* stream);

/* Cluster finding (Sec. 2.1 step 3): repeatedly take the cell with the largest
 * count (the search's total order on the current counts: distinct desc, raw
 * desc, v_idx, by, bx), stop when it is below n_min, else report its remaining
 * detections as a cluster and remove them from every cell; at most
 * max_clusters clusters (0: 1000, the paper's cut).  Removing detections only
 * lowers counts, so the loop runs over the search's candidate list; n_min must
 * be at least the search's threshold and the search must not have been cut to
 * its top candidates.
 * By default the loop runs as rounds that pick every local maximum at once (a
 * candidate whose key beats every live candidate it shares a detection with is
 * certain to be picked with its current detections); flags =
 * SAS_PEEL_SEQUENTIAL runs it one cluster at a time in a single block.  Both
 * give the same clusters in the same order.
 * On success *out is a new result (free it with sas_result_free) whose
 * candidates are the clusters in the order found, with their current counts
 * and ids (disjoint across clusters, ascending); sas_stamps and sas_peel do not
 * apply to it.  Synchronizes the stream.  Device scratch: about 30 bytes per
 * detection plus 40 per candidate.
 * Errors: SAS_ERR_ARG (null pointers, n_min below the search's, a top-K or
 * cluster result, unknown flags), SAS_ERR_RANGE (2^31 or more candidates or
 * detections), SAS_ERR_OOM, SAS_ERR_CUDA. */
#define SAS_PEEL_SEQUENTIAL 1u
int sas_peel(const sas_result* result, uint32_t n_min, uint32_t max_clusters, uint32_t flags, void* stream,
             sas_result** out);

/* ---- Refinement and gathering (Sec. 2.1 steps 4-6) -------------------------
 *
 * For each cluster (a candidate and its ids): fit a linear trajectory by
 * multivariate regression of (x, y) on t with the mean and covariance of the
 * Minimum Covariance Determinant subset of the points (t, x, y), found by
 * FAST-MCD (Rousseeuw & Van Driessen 1999); gather every detection of the
 * search's catalog whose distance to the line's position at its own epoch is at
 * most `radius`; repeat on the gathered set until it equals the fitted set.
 *   Points: t = epoch time - t0 in ticks, x and y in mpx.  h = floor((n + 4)/2);
 *   fewer than 5 points are fitted by least squares on all of them.  FAST-MCD:
 *   n_starts random 4-subsets (extended one point at a time while singular,
 *   up to h), the h nearest points, two C-steps (stopping at the first that
 *   does not lower det); the n_best lowest determinants continue for up to
 *   max_csteps C-steps; lowest determinant wins, ties to the lower start.
 *   Draws: start s of cluster k in round it uses key = mix(mix(mix(seed +
 *   (k+1)g) + (it+1)g) + (s+1)g) and draw j = mix(key + (j+1)g), SplitMix64's
 *   mix and g = 0x9E3779B97F4A7C15, mod 2^64; step j of the start's partial
 *   Fisher-Yates shuffle swaps positions j and j + draw_j mod (n - j).
 *   Arithmetic: exact integer moment sums; the scatter matrix rounded once to
 *   double; then fixed IEEE double expressions, so the result does not depend
 *   on how the GPU orders its reductions.
 * Output per cluster (in the clusters' order): the line (vx, vy in mpx/h; x0,
 * y0 in mpx at t0), the subset's residual covariance, det of its scatter
 * matrix (subset size^2 x covariance), status, and the ids (ascending) of the
 * last gathering -- of the fitted set for SAS_TRACK_TOO_MANY, of the cluster
 * when nothing was fitted.
 */
#define SAS_REFINE_MAX_POINTS 1024u
#define SAS_TRACK_CONVERGED 0u   /* the gathered set is the fitted set           */
#define SAS_TRACK_MAX_ITER 1u    /* max_iter fits without a fixed point          */
#define SAS_TRACK_DEGENERATE 2u  /* one epoch only (no slope), or < 2 gathered   */
#define SAS_TRACK_TOO_MANY 3u    /* more than SAS_REFINE_MAX_POINTS points        */

typedef struct sas_refine_opts {
  uint64_t seed;
  uint32_t n_starts;    /* 0: 500 (at most 4096)                           */
  uint32_t n_best;      /* 0: 10 (at most n_starts)                        */
  uint32_t max_csteps;  /* 0: 100                                          */
  uint32_t max_iter;    /* fits per cluster, 0: 10                         */
  int32_t radius;       /* gather radius in mpx, 0: the search's bin       */
  uint32_t reserved;
} sas_refine_opts;

typedef struct sas_track {
  double vx, vy;                  /* mpx per hour (NaN when no line)          */
  double x0, y0;                  /* mpx at t0                                */
  double res_xx, res_xy, res_yy;  /* residual covariance of the subset, mpx^2 */
  double det;                     /* det of the subset's scatter matrix       */
  uint32_t status;                /* SAS_TRACK_*                              */
  uint32_t iterations;            /* fits made                                */
  uint32_t h;                     /* points in the MCD subset                 */
  uint32_t n_points;              /* points of the last fit                   */
  uint64_t id_off;
  uint32_t id_len;
  uint32_t cluster;               /* index in the cluster list                */
} sas_track;

typedef struct sas_tracks sas_tracks;

/* search: a search result (its catalog is gathered from); clusters: a result
 * whose candidates are the clusters -- the output of sas_peel on `search`, or
 * `search` itself.  opts may be NULL (all defaults, seed 0).  Synchronizes the
 * stream.  Device scratch: about 8 KB per cluster plus 16 bytes per detection.
 * Errors: SAS_ERR_ARG (null pointers, a cluster list as `search`, catalogs of
 * different sizes, n_starts > 4096), SAS_ERR_OOM, SAS_ERR_CUDA. */
int sas_refine(const sas_result* search, const sas_result* clusters, const sas_refine_opts* opts, void* stream,
               sas_tracks** out);

/* Copy up to cap tracks and ids_cap ids (host or device buffers, on_device
 * selects); totals written when the pointers are non-NULL. */
int sas_tracks_get(const sas_tracks* tracks, sas_track* out, uint64_t cap, uint64_t* n_total, uint32_t* ids,
                   uint64_t ids_cap, uint64_t* n_ids_total, int on_device);
void sas_tracks_free(sas_tracks* tracks);

/* ---- Search parameters (Sec. 2.2) ------------------------------------------
 *
 * Host functions (no device): the relations the paper uses to choose the bin
 * size dx and the threshold N_min.  Lengths in one unit throughout (pixels or
 * arcsec), times in hours, velocities in length per hour, omega in length^2.
 * Each returns SAS_OK and writes its result, or SAS_ERR_ARG for a null output
 * or an argument outside its domain (non-positive dx, dt, a; negative rate),
 * or SAS_ERR_RANGE for a noise rate above 1e7 (choose_n_min, dx_scan) or more
 * than 65536 epochs (signal_tail).
 *
 * velocity_count: |V| = ((vmax_x - vmin_x) / dv)((vmax_y - vmin_y) / dv) with
 *   dv = dx / dt (Eq. v_size).
 * n_stacks: |V| omega / dx^2 (Eq. N_stacks).
 * peak_density(z, a): noise peaks per unit area per unit detection statistic
 *   for white noise under a Gaussian window of width a -- the Kac-Rice density
 *   of maxima of that Gaussian field (the paper's printed closed form is
 *   garbled; this is the quantity it stands for).  Integrates over z to
 *   1 / (4 sqrt(3) pi a^2).
 * peaks_above(nu_th, a): its integral above nu_th (Eq. n_pk_above).
 * noise_rate: Lambda = sum over epochs of peaks_above(nu_th, 1) (dx / a_i)^2,
 *   the mean noise count of a square bin of side dx.
 * poisson_sf: P(N >= k), N ~ Pois(lambda).
 * choose_n_min: the smallest N_min with P(N_noise >= N_min) <= eps.
 * p_signal: one epoch's probability that a source of S/N nu is detected above
 *   nu_th and falls in the bin of side dx centred on it:
 *   erfc((nu_th - nu) / sqrt 2) / 2 * erf(dx nu / (4 a))^2.
 * signal_tail: P(N_signal >= k) for independent epochs with probabilities p.
 * dx_scan: for each dx[j]: E[N_signal], E[N_noise] and the N_min that the
 *   budget eps = n_false / N_stacks requires, N_stacks from |V| = (dt dv / dx)^2
 *   (equal axis ranges dv) and the area omega.  An object is recoverable where
 *   E[N_signal] > E[N_noise] and E[N_signal] + E[N_noise] >= N_min.
 */
int sas_param_velocity_count(double vmin_x, double vmax_x, double vmin_y, double vmax_y, double dx, double dt,
                             double* out);
int sas_param_n_stacks(double n_velocities, double omega, double dx, double* out);
int sas_param_peak_density(double z, double a, double* out);
int sas_param_peaks_above(double nu_th, double a, double* out);
int sas_param_noise_rate(double nu_th, const double* a, uint32_t n_epochs, double dx, double* out);
int sas_param_poisson_sf(uint32_t k, double lambda, double* out);
int sas_param_choose_n_min(double lambda, double eps, uint32_t* out);
int sas_param_p_signal(double nu, double nu_th, double a, double dx, double* out);
int sas_param_signal_tail(const double* p, uint32_t n, uint32_t k, double* out);
int sas_param_dx_scan(double nu, double nu_th, const double* a, uint32_t n_epochs, const double* dx, uint32_t n_dx,
                      double dv, double dt, double omega, double n_false, double* e_signal, double* e_noise,
                      uint32_t* n_min);

/* The network (input = count / 16):
 *   conv1 9 -> 32 channels, 3x3 valid (15 -> 13), ReLU; conv2 32 -> 32 (13 -> 11),
 *   ReLU; conv3 32 -> 32 (11 -> 9), ReLU; flatten in (channel, row, column)
 *   order; fc1 2592 -> 64, ReLU; fc2 64 -> 1 = logit (score of a real mover).
 * Loss: mean binary cross-entropy with logits.
 * Parameters: 187,137 FP32 master values in this flat order:
 *   conv1.w [32][9][3][3], conv1.b [32], conv2.w [32][32][3][3], conv2.b [32],
 *   conv3.w [32][32][3][3], conv3.b [32], fc1.w [64][2592], fc1.b [64],
 *   fc2.w [64], fc2.b [1].
 * Arithmetic: the kernels use BF16 copies of the weights (round to nearest
 * even), round the input and every stored activation to BF16 and accumulate
 * in FP32.  The forward convolutions and fc1 run on the tensor cores (tcgen05,
 * BF16 operands); deltas and gradients are FP32, and the backward of conv2 and
 * conv3 runs on the tensor cores with TF32 operands (the deltas round to TF32
 * there).  Adam updates the FP32 masters and refreshes the BF16 copies.
 * Gradients are bit-reproducible for a batch.
 * A vetter lives on the device that was current at sas_vet_create; every call
 * makes that device current for its duration. */
#define SAS_VET_MAX_BATCH 32768u
typedef struct sas_vet sas_vet;

uint64_t sas_vet_num_params(void);

/* Allocate a vetter whose training batches hold up to max_batch stamps
 * (1..SAS_VET_MAX_BATCH; about 72 KB of device memory per stamp).  Parameters
 * start at zero; Adam starts with beta1 0.9, beta2 0.999, eps 1e-8.
 * Errors: SAS_ERR_ARG, SAS_ERR_OOM, SAS_ERR_CUDA. */
int sas_vet_create(int device, uint32_t max_batch, sas_vet** out);
int sas_vet_destroy(sas_vet* vetter);
/* Synchronizes the vetter's device and reports SAS_ERR_TIMEOUT when a wait of
 * the tensor-core forward gave up since the last check (the kernels never wait
 * without a limit; a wait that runs out leaves that call's logits incomplete). */
int sas_vet_check(sas_vet* vetter);
int sas_vet_set_adam(sas_vet* vetter, float beta1, float beta2, float eps);

/* Checkpoint: host arrays of sas_vet_num_params() floats.  set_state loads
 * the masters (and the Adam moments and step count, or resets them when m and
 * v are NULL) and synchronizes; get_state copies out any non-NULL argument. */
int sas_vet_set_state(sas_vet* vetter, const float* params, const float* m, const float* v,
                      uint64_t step);
int sas_vet_get_state(const sas_vet* vetter, float* params, float* m, float* v, uint64_t* step);
/* The BF16 working copy of the parameters (flat order, raw bits), to host. */
int sas_vet_get_bf16(const sas_vet* vetter, uint16_t* out);

/* The activations the last batch stored (BF16 raw bits, to host): layer 1, 2, 3
 * = the outputs of conv1, conv2, conv3 after ReLU, [n][32][h][h] with h = 13,
 * 11, 9 (channel-major, as the stored layout of conv3 is fc1's input); layer 4
 * = the fc1 output after ReLU, [n][64].  "The last batch" is the last forward
 * chunk or gradient batch of this vetter (sas_vet_forward runs in chunks of the
 * vetter's max_batch: its last chunk's activations are what remains).  n <=
 * max_batch samples are copied from the start of that batch.  Waits for the
 * device.  For inspection and tests (the backward of the network, Sec. 5's
 * learned filter, runs from exactly these values).
 * Errors: SAS_ERR_ARG (NULL, layer outside 1..4, n > max_batch), SAS_ERR_CUDA. */
int sas_vet_get_activations(const sas_vet* vetter, uint32_t layer, uint64_t n, uint16_t* out);

/* logits[i] of n stamps (device arrays: stamps [.][9][15][15] uint16,
 * logits [n] float); stamp i is stamps[index[i]] when index (device uint32
 * [n]) is given, else stamps[i]; any n, processed in batches of max_batch.
 * Asynchronous on `stream`. */
int sas_vet_forward(sas_vet* vetter, const uint16_t* stamps, const uint32_t* index, uint64_t n,
                    float* logits, void* stream);

/* Gradient (device float [sas_vet_num_params()]) of the mean BCE loss of n
 * (1..max_batch) stamps with labels (device float, parallel to stamps; 1 =
 * mover, 0 = not) at the current parameters; the batch is stamps[index[i]]
 * (and labels[index[i]]) when index (device uint32 [n]) is given, else the
 * first n.  The loss goes to *loss (device float, may be NULL).
 * Asynchronous on `stream`. */
int sas_vet_gradients(sas_vet* vetter, const uint16_t* stamps, const float* labels,
                      const uint32_t* index, uint32_t n, float* grad, float* loss, void* stream);

/* One Adam step (Kingma & Ba 2015) with a caller's gradient (device float
 * [sas_vet_num_params()]), learning rate lr >= 0.  Asynchronous. */
int sas_vet_apply_gradients(sas_vet* vetter, const float* grad, float lr, void* stream);

/* sas_vet_gradients followed by sas_vet_apply_gradients on an internal
 * gradient buffer.  Asynchronous. */
int sas_vet_train_step(sas_vet* vetter, const uint16_t* stamps, const float* labels,
                       const uint32_t* index, uint32_t n, float lr, float* loss, void* stream);

/* Measurement utility: throughput of conflict-free 32-bit shared-memory
 * atomicAdd whose old value is used (the returning form), on every SM of the
 * current device, in operations per second, measured with CUDA events over
 * `iters` operations per thread.  Reported beside the reduction peak below.
 * Also reports the SM clock (MHz) during the probe: clock64() cycles over the
 * global timer's nanoseconds on one SM, in the fastest repetition.
 * Not a paper operation (the roofline of Sec. 2.1 steps 1-2 on this GPU).
 * Errors: SAS_ERR_ARG (null output or iters == 0), SAS_ERR_CUDA. */
int sas_probe_shared_atomic_peak(uint32_t iters, void* stream, double* ops_per_s,
                                 double* sm_mhz);

/* Measurement utility: throughput of conflict-free 32-bit shared-memory
 * reductions (`red.shared.add.u32`, no value returned: the instruction the
 * stack kernel issues for Sec. 2.1 steps 1-2) on every SM of the current
 * device, in operations per second, over `iters` x 8 reductions per thread,
 * best of three timed repetitions after one warm-up.  This is the peak against
 * which the stack kernel's detection-shifts/s are compared.  *sm_mhz as above.
 * Errors: SAS_ERR_ARG (null output or iters == 0), SAS_ERR_CUDA. */
int sas_probe_shared_reduction_peak(uint32_t iters, void* stream, double* ops_per_s,
                                    double* sm_mhz);

/* Measurement utility: throughput of conflict-free 64-bit shared-memory
 * atomicOr whose old value is used -- the per-bin epoch-bitmask update that a
 * literal form of Sec. 2.1 step 2 would issue per (detection, velocity) pair,
 * which the stack kernel replaces by narrow counters -- in operations per
 * second on every SM, as above.  *sm_mhz as above.
 * Errors: SAS_ERR_ARG (null output or iters == 0), SAS_ERR_CUDA. */
int sas_probe_shared_or64_peak(uint32_t iters, void* stream, double* ops_per_s, double* sm_mhz);

#ifdef __cplusplus
}
#endif

#endif /* SAS_H_ */
