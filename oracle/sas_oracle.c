/*
 * CPU oracle for catalog shift-and-stack (Stetzler et al., Sec. 2.1, steps 1-3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header, table
 * or helper with the CUDA path and never calls it.
 *
 * What it computes (the plain definition, in int64, with mathematical floor
 * division):
 *   Step 1 "Project" (Sec. 2.1 step 1; motion model Eq. 1-2, residual Eq. 3-8):
 *       t0 = min_i t[epoch_i]                (reference epoch = earliest time in
 *                                             the catalog)
 *       sx = floor(vx * (t[e] - t0) / TPH),  sy = floor(vy * (t[e] - t0) / TPH)
 *       X  = x_i - sx - x_min,               Y  = y_i - sy - y_min
 *   Step 2 "Cluster" (Sec. 2.1 step 2): one 2-D histogram per hypothesis
 *       velocity with resolution Delta-x = w:  bx = floor(X / w), by = floor(Y / w),
 *       kept when 0 <= bx < nbx and 0 <= by < nby.  A cell counts the DISTINCT
 *       epochs of the detections that fall in it (and, separately, the raw number
 *       of detections).
 *   Step 3 "Find clusters" (Sec. 2.1 step 3), in its threshold form: every cell
 *       whose distinct-epoch count is >= N_min is a candidate; its contributing
 *       points are all detections that fell in it (ids ascending).
 *   Output order (Sec. 3.3: clusters ranked by their number of detections):
 *       distinct desc, raw desc, v_idx asc, by asc, bx asc.
 *
 * Velocity set (Sec. 2, Eq. for |V|): a regular lattice vx = vx0 + kx*dvx,
 * vy = vy0 + ky*dvy, v_idx = ky*nvx + kx, optionally restricted to the annulus
 * speed_min^2 <= vx^2 + vy^2 <= speed_max^2 (speed_min = speed_max = 0: all).
 *
 * Memory note: each velocity's histogram is a dense array over the domain; the
 * cells a velocity touched are remembered so that only they are reset before
 * the next velocity (nothing about the arithmetic changes).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
static int omp_default_threads(void) { return omp_get_max_threads(); }
#else
static int omp_default_threads(void) { return 1; }
#endif

typedef struct {
  int64_t v_idx;
  int32_t bx, by;
  int32_t distinct, raw;
  int64_t id_off, id_len;
} oracle_candidate;

enum { ORACLE_OK = 0, ORACLE_ERR_ARG = 1, ORACLE_ERR_OOM = 2, ORACLE_ERR_CAP = 3 };

/* Mathematical floor of a / b for b > 0 (C's '/' truncates toward zero). */
static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}

static int velocity_active(int64_t vx, int64_t vy, int32_t smin, int32_t smax) {
  if (smin == 0 && smax == 0) return 1;
  int64_t s2 = vx * vx + vy * vy;
  return s2 >= (int64_t)smin * smin && s2 <= (int64_t)smax * smax;
}

/* The reference epoch of step 1: the earliest observation time in the catalog. */
int64_t oracle_t0(int64_t n, const uint16_t* epoch, const int64_t* t) {
  int64_t t0 = INT64_MAX;
  for (int64_t i = 0; i < n; ++i)
    if (t[epoch[i]] < t0) t0 = t[epoch[i]];
  return t0;
}

/* Steps 1-2 for one detection at one velocity: the cell it lands in, or -1. */
static int64_t project_bin(int32_t xi, int32_t yi, int64_t sx, int64_t sy, int32_t x_min,
                           int32_t y_min, int32_t nbx, int32_t nby, int32_t w) {
  int64_t X = (int64_t)xi - sx - x_min;
  int64_t Y = (int64_t)yi - sy - y_min;
  int64_t bx = floor_div(X, w);
  int64_t by = floor_div(Y, w);
  if (bx < 0 || bx >= nbx || by < 0 || by >= nby) return -1;
  return by * (int64_t)nbx + bx;
}

static int cand_cmp(const void* pa, const void* pb) {
  const oracle_candidate* a = (const oracle_candidate*)pa;
  const oracle_candidate* b = (const oracle_candidate*)pb;
  if (a->distinct != b->distinct) return a->distinct > b->distinct ? -1 : 1;
  if (a->raw != b->raw) return a->raw > b->raw ? -1 : 1;
  if (a->v_idx != b->v_idx) return a->v_idx < b->v_idx ? -1 : 1;
  if (a->by != b->by) return a->by < b->by ? -1 : 1;
  if (a->bx != b->bx) return a->bx < b->bx ? -1 : 1;
  return 0;
}

/*
 * Full search over lattice indices [v_begin, v_end).
 * Outputs: candidates sorted in the order above (at most cap are written,
 * *n_cands = total), their ids concatenated (id_off/id_len index into ids; at
 * most ids_cap written, *n_ids = total), *n_pairs = number of in-domain
 * (detection, velocity) pairs.  If max_candidates > 0 the sorted list is cut to
 * its first max_candidates entries before ids are written.
 * Returns ORACLE_ERR_CAP when a capacity was too small (totals still reported).
 */
int oracle_stack(int64_t n, const int32_t* x, const int32_t* y, const uint16_t* epoch,
                 int32_t n_epochs, const int64_t* t, int64_t tph,
                 int32_t vx0, int32_t vy0, int32_t dvx, int32_t dvy, int32_t nvx, int32_t nvy,
                 int32_t speed_min, int32_t speed_max,
                 int32_t x_min, int32_t y_min, int32_t nbx, int32_t nby, int32_t w,
                 int32_t n_min, int64_t v_begin, int64_t v_end, int64_t max_candidates,
                 oracle_candidate* cands, int64_t cap, int64_t* n_cands,
                 int32_t* ids, int64_t ids_cap, int64_t* n_ids, int64_t* n_pairs) {
  if (n < 0 || n_epochs < 1 || tph <= 0 || w <= 0 || nbx <= 0 || nby <= 0 || nvx <= 0 ||
      nvy <= 0 || n_min < 1 || v_begin < 0 || v_end > (int64_t)nvx * nvy || v_begin > v_end)
    return ORACLE_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (epoch[i] >= n_epochs) return ORACLE_ERR_ARG;

  const int64_t nbins = (int64_t)nbx * nby;
  const int words = (n_epochs + 63) / 64;
  uint64_t* mask = (uint64_t*)calloc((size_t)(nbins * words), sizeof(uint64_t));
  int32_t* raw = (int32_t*)calloc((size_t)nbins, sizeof(int32_t));
  int64_t* cand_of = (int64_t*)malloc((size_t)nbins * sizeof(int64_t));
  int64_t* touched = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
  int64_t* sx = (int64_t*)malloc((size_t)n_epochs * sizeof(int64_t));
  int64_t* sy = (int64_t*)malloc((size_t)n_epochs * sizeof(int64_t));
  int64_t ccap = 1024, cn = 0, tcap = 4096, tn = 0;
  oracle_candidate* cl = (oracle_candidate*)malloc((size_t)ccap * sizeof(oracle_candidate));
  int32_t* tids = (int32_t*)malloc((size_t)tcap * sizeof(int32_t)); /* ids, by candidate */
  if (!mask || !raw || !cand_of || !touched || !sx || !sy || !cl || !tids) {
    free(mask); free(raw); free(cand_of); free(touched); free(sx); free(sy); free(cl); free(tids);
    return ORACLE_ERR_OOM;
  }
  for (int64_t b = 0; b < nbins; ++b) cand_of[b] = -1;

  const int64_t t0 = oracle_t0(n, epoch, t);
  int64_t pairs = 0;
  int status = ORACLE_OK;

  for (int64_t v = v_begin; v < v_end; ++v) {
    const int64_t kx = v % nvx, ky = v / nvx;
    const int64_t vx = (int64_t)vx0 + kx * dvx, vy = (int64_t)vy0 + ky * dvy;
    if (!velocity_active(vx, vy, speed_min, speed_max)) continue;
    /* Step 1: the shift of every epoch for this hypothesis velocity. */
    for (int e = 0; e < n_epochs; ++e) {
      sx[e] = floor_div(vx * (t[e] - t0), tph);
      sy[e] = floor_div(vy * (t[e] - t0), tph);
    }
    /* Step 2: histogram of projected positions (epoch sets and raw counts). */
    tn = 0;
    for (int64_t i = 0; i < n; ++i) {
      const int e = epoch[i];
      const int64_t b = project_bin(x[i], y[i], sx[e], sy[e], x_min, y_min, nbx, nby, w);
      if (b < 0) continue;
      ++pairs;
      if (raw[b] == 0) touched[tn++] = b;
      raw[b] += 1;
      mask[b * words + e / 64] |= (uint64_t)1 << (e % 64);
    }
    /* Step 3 (threshold form): every cell with >= n_min distinct epochs. */
    int64_t first = cn;
    for (int64_t k = 0; k < tn; ++k) {
      const int64_t b = touched[k];
      int32_t d = 0;
      for (int q = 0; q < words; ++q) d += __builtin_popcountll(mask[b * words + q]);
      if (d < n_min) continue;
      if (cn == ccap) {
        ccap *= 2;
        oracle_candidate* p = (oracle_candidate*)realloc(cl, (size_t)ccap * sizeof(*cl));
        if (!p) { status = ORACLE_ERR_OOM; goto done; }
        cl = p;
      }
      oracle_candidate* c = &cl[cn];
      c->v_idx = v; c->bx = (int32_t)(b % nbx); c->by = (int32_t)(b / nbx);
      c->distinct = d; c->raw = raw[b]; c->id_off = 0; c->id_len = 0;
      cand_of[b] = cn++;
    }
    if (cn > first) {
      /* Contributing points: reserve raw[b] slots per candidate, then fill in
         ascending detection order. */
      int64_t need = 0;
      for (int64_t c = first; c < cn; ++c) need += cl[c].raw;
      int64_t base = 0;
      for (int64_t c = 0; c < first; ++c) base += cl[c].raw;
      if (base + need > tcap) {
        while (base + need > tcap) tcap *= 2;
        int32_t* p = (int32_t*)realloc(tids, (size_t)tcap * sizeof(int32_t));
        if (!p) { status = ORACLE_ERR_OOM; goto done; }
        tids = p;
      }
      int64_t off = base;
      for (int64_t c = first; c < cn; ++c) { cl[c].id_off = off; off += cl[c].raw; }
      for (int64_t i = 0; i < n; ++i) {
        const int e = epoch[i];
        const int64_t b = project_bin(x[i], y[i], sx[e], sy[e], x_min, y_min, nbx, nby, w);
        if (b < 0 || cand_of[b] < 0) continue;
        oracle_candidate* c = &cl[cand_of[b]];
        tids[c->id_off + c->id_len++] = (int32_t)i;
      }
    }
    /* Reset the cells this velocity touched. */
    for (int64_t k = 0; k < tn; ++k) {
      const int64_t b = touched[k];
      raw[b] = 0; cand_of[b] = -1;
      memset(&mask[b * words], 0, (size_t)words * sizeof(uint64_t));
    }
  }

  qsort(cl, (size_t)cn, sizeof(oracle_candidate), cand_cmp);
  if (max_candidates > 0 && cn > max_candidates) cn = max_candidates;
  {
    int64_t total_ids = 0;
    for (int64_t c = 0; c < cn; ++c) total_ids += cl[c].id_len;
    *n_cands = cn;
    *n_ids = total_ids;
    if (cn > cap || total_ids > ids_cap) status = ORACLE_ERR_CAP;
    int64_t off = 0;
    for (int64_t c = 0; c < cn && c < cap; ++c) {
      oracle_candidate o = cl[c];
      int64_t src = o.id_off;
      o.id_off = off;
      if (off + o.id_len <= ids_cap)
        memcpy(&ids[off], &tids[src], (size_t)o.id_len * sizeof(int32_t));
      off += o.id_len;
      cands[c] = o;
    }
  }
  *n_pairs = pairs;
done:
  free(mask); free(raw); free(cand_of); free(touched); free(sx); free(sy); free(cl); free(tids);
  return status;
}

/*
 * One cell, computed on its own from the definition: the distinct epochs, the raw
 * count and the (ascending) ids of the detections that land in bin (bx, by) at
 * lattice index v_idx.  Used to check single outputs of full-size searches.
 * Writes at most ids_cap ids; *n_ids is the total.
 */
int oracle_cell(int64_t n, const int32_t* x, const int32_t* y, const uint16_t* epoch,
                int32_t n_epochs, const int64_t* t, int64_t tph,
                int32_t vx0, int32_t vy0, int32_t dvx, int32_t dvy, int32_t nvx,
                int32_t x_min, int32_t y_min, int32_t nbx, int32_t nby, int32_t w,
                int64_t v_idx, int32_t bx, int32_t by,
                int32_t* distinct, int32_t* raw, int32_t* ids, int64_t ids_cap, int64_t* n_ids) {
  if (n_epochs < 1 || n_epochs > 65536 || w <= 0 || tph <= 0 || nvx <= 0) return ORACLE_ERR_ARG;
  const int64_t t0 = oracle_t0(n, epoch, t);
  const int64_t kx = v_idx % nvx, ky = v_idx / nvx;
  const int64_t vx = (int64_t)vx0 + kx * dvx, vy = (int64_t)vy0 + ky * dvy;
  uint64_t seen[1024];
  memset(seen, 0, sizeof(seen));
  int32_t r = 0;
  int64_t k = 0;
  const int64_t want = (int64_t)by * nbx + bx;
  for (int64_t i = 0; i < n; ++i) {
    const int e = epoch[i];
    const int64_t sxe = floor_div(vx * (t[e] - t0), tph);
    const int64_t sye = floor_div(vy * (t[e] - t0), tph);
    if (project_bin(x[i], y[i], sxe, sye, x_min, y_min, nbx, nby, w) != want) continue;
    seen[e / 64] |= (uint64_t)1 << (e % 64);
    ++r;
    if (k < ids_cap) ids[k] = (int32_t)i;
    ++k;
  }
  int32_t d = 0;
  for (int q = 0; q < 1024; ++q) d += __builtin_popcountll(seen[q]);
  *distinct = d;
  *raw = r;
  *n_ids = k;
  return ORACLE_OK;
}

/*
 * The full 2-D histogram of one velocity (steps 1-2 only): distinct[b] and
 * raw[b] for every bin b = by*nbx + bx.  Used by invariant checks.
 */
int oracle_histogram(int64_t n, const int32_t* x, const int32_t* y, const uint16_t* epoch,
                     int32_t n_epochs, const int64_t* t, int64_t tph, int64_t vx, int64_t vy,
                     int32_t x_min, int32_t y_min, int32_t nbx, int32_t nby, int32_t w,
                     int32_t* distinct, int32_t* raw) {
  if (n_epochs < 1 || w <= 0 || tph <= 0) return ORACLE_ERR_ARG;
  const int64_t nbins = (int64_t)nbx * nby;
  const int words = (n_epochs + 63) / 64;
  uint64_t* mask = (uint64_t*)calloc((size_t)(nbins * words), sizeof(uint64_t));
  if (!mask) return ORACLE_ERR_OOM;
  const int64_t t0 = oracle_t0(n, epoch, t);
  for (int64_t b = 0; b < nbins; ++b) raw[b] = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int e = epoch[i];
    const int64_t sxe = floor_div(vx * (t[e] - t0), tph);
    const int64_t sye = floor_div(vy * (t[e] - t0), tph);
    const int64_t b = project_bin(x[i], y[i], sxe, sye, x_min, y_min, nbx, nby, w);
    if (b < 0) continue;
    raw[b] += 1;
    mask[b * words + e / 64] |= (uint64_t)1 << (e % 64);
  }
  for (int64_t b = 0; b < nbins; ++b) {
    int32_t d = 0;
    for (int q = 0; q < words; ++q) d += __builtin_popcountll(mask[b * words + q]);
    distinct[b] = d;
  }
  free(mask);
  return ORACLE_OK;
}

/*
 * The same search with the lattice range split into chunks that run in an
 * OpenMP loop over velocities (each chunk is one oracle_stack call, with its
 * own private histograms), then merged: every chunk's candidates concatenated
 * and sorted by the same total order, the optional top-K cut applied, ids
 * copied in that order.  The velocities' histograms are independent (Sec. 2.1
 * step 2), so the output equals oracle_stack's byte for byte.  n_threads <= 0:
 * OpenMP's default team.  Same outputs and statuses as oracle_stack.
 */
typedef struct {
  oracle_candidate* cands;
  int32_t* ids;
  int64_t n_cands, n_ids, n_pairs;
  int status;
} oracle_chunk;

int oracle_stack_mt(int64_t n, const int32_t* x, const int32_t* y, const uint16_t* epoch,
                    int32_t n_epochs, const int64_t* t, int64_t tph,
                    int32_t vx0, int32_t vy0, int32_t dvx, int32_t dvy, int32_t nvx, int32_t nvy,
                    int32_t speed_min, int32_t speed_max,
                    int32_t x_min, int32_t y_min, int32_t nbx, int32_t nby, int32_t w,
                    int32_t n_min, int64_t v_begin, int64_t v_end, int64_t max_candidates,
                    oracle_candidate* cands, int64_t cap, int64_t* n_cands,
                    int32_t* ids, int64_t ids_cap, int64_t* n_ids, int64_t* n_pairs,
                    int32_t n_threads) {
  if (v_begin < 0 || v_end > (int64_t)nvx * nvy || v_begin > v_end) return ORACLE_ERR_ARG;
  const int64_t nv = v_end - v_begin;
  const int team = n_threads > 0 ? n_threads : omp_default_threads();
  /* chunks of at least 8 velocities (each chunk allocates its own histograms),
     at most 256, and at least two per thread where the range allows it */
  int64_t n_chunks = nv / 8;
  if (n_chunks > 256) n_chunks = 256;
  if (n_chunks < 2 * (int64_t)team) n_chunks = 2 * (int64_t)team;
  if (n_chunks > nv) n_chunks = nv;
  if (n_chunks < 1) n_chunks = 1;
  oracle_chunk* ch = (oracle_chunk*)calloc((size_t)n_chunks, sizeof(oracle_chunk));
  if (!ch) return ORACLE_ERR_OOM;
  (void)team;
#pragma omp parallel for schedule(dynamic, 1) num_threads(team)
  for (int64_t k = 0; k < n_chunks; ++k) {
    const int64_t a = v_begin + nv * k / n_chunks, b = v_begin + nv * (k + 1) / n_chunks;
    int64_t ccap = 256, icap = 4096;
    for (;;) {
      ch[k].cands = (oracle_candidate*)malloc((size_t)ccap * sizeof(oracle_candidate));
      ch[k].ids = (int32_t*)malloc((size_t)icap * sizeof(int32_t));
      if (!ch[k].cands || !ch[k].ids) { ch[k].status = ORACLE_ERR_OOM; break; }
      ch[k].status = oracle_stack(n, x, y, epoch, n_epochs, t, tph, vx0, vy0, dvx, dvy, nvx, nvy,
                                  speed_min, speed_max, x_min, y_min, nbx, nby, w, n_min, a, b, 0,
                                  ch[k].cands, ccap, &ch[k].n_cands, ch[k].ids, icap, &ch[k].n_ids,
                                  &ch[k].n_pairs);
      if (ch[k].status != ORACLE_ERR_CAP) break;
      free(ch[k].cands); free(ch[k].ids);
      ch[k].cands = NULL; ch[k].ids = NULL;
      if (ch[k].n_cands > ccap) ccap = ch[k].n_cands;
      if (ch[k].n_ids > icap) icap = ch[k].n_ids;
    }
  }
  int status = ORACLE_OK;
  int64_t total_c = 0, total_i = 0, pairs = 0;
  for (int64_t k = 0; k < n_chunks; ++k) {
    if (ch[k].status != ORACLE_OK && status == ORACLE_OK) status = ch[k].status;
    total_c += ch[k].n_cands;
    total_i += ch[k].n_ids;
    pairs += ch[k].n_pairs;
  }
  oracle_candidate* all = NULL;
  int32_t* all_ids = NULL;
  if (status == ORACLE_OK) {
    all = (oracle_candidate*)malloc((size_t)(total_c > 0 ? total_c : 1) * sizeof(oracle_candidate));
    all_ids = (int32_t*)malloc((size_t)(total_i > 0 ? total_i : 1) * sizeof(int32_t));
    if (!all || !all_ids) status = ORACLE_ERR_OOM;
  }
  if (status == ORACLE_OK) {
    /* concatenate, with id_off pointing into the concatenated id array */
    int64_t pc = 0, pi = 0;
    for (int64_t k = 0; k < n_chunks; ++k) {
      for (int64_t c = 0; c < ch[k].n_cands; ++c) {
        all[pc] = ch[k].cands[c];
        all[pc].id_off += pi;
        ++pc;
      }
      memcpy(all_ids + pi, ch[k].ids, (size_t)ch[k].n_ids * sizeof(int32_t));
      pi += ch[k].n_ids;
    }
    qsort(all, (size_t)total_c, sizeof(oracle_candidate), cand_cmp);
    int64_t cn = total_c;
    if (max_candidates > 0 && cn > max_candidates) cn = max_candidates;
    int64_t kept_ids = 0;
    for (int64_t c = 0; c < cn; ++c) kept_ids += all[c].id_len;
    *n_cands = cn;
    *n_ids = kept_ids;
    *n_pairs = pairs;
    if (cn > cap || kept_ids > ids_cap) status = ORACLE_ERR_CAP;
    int64_t off = 0;
    for (int64_t c = 0; c < cn && c < cap; ++c) {
      oracle_candidate o = all[c];
      const int64_t src = o.id_off;
      o.id_off = off;
      if (off + o.id_len <= ids_cap)
        memcpy(&ids[off], &all_ids[src], (size_t)o.id_len * sizeof(int32_t));
      off += o.id_len;
      cands[c] = o;
    }
  }
  for (int64_t k = 0; k < n_chunks; ++k) { free(ch[k].cands); free(ch[k].ids); }
  free(ch); free(all); free(all_ids);
  return status;
}

/* Number of threads the OpenMP loop above uses by default (1 without OpenMP). */
int32_t oracle_threads(void) { return omp_default_threads(); }
