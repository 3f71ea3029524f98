// Ingest, bucketing, reference epoch, shift tables and scans (Sec. 2.1 step 1).
#include <climits>

#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr int kPrepThreads = 256;

// a1 + a2 (count phase): validate each detection, count detections per epoch
// (for the reference epoch t0, which is taken over the whole catalog) and per
// spatial bucket.  Detections whose coarse cell lies outside the bucket grid can
// never project into the histogram domain and get no bucket.
__global__ void k_ingest(const int32_t* __restrict__ x, const int32_t* __restrict__ y,
                         const uint16_t* __restrict__ epoch, uint64_t n, uint32_t E,
                         CoarseGeom cg, uint32_t* __restrict__ bucket_count,
                         uint32_t* __restrict__ ecount, uint32_t* __restrict__ bucket_of,
                         uint32_t* __restrict__ flags) {
  extern __shared__ uint32_t s_hist[];  // [E] per-block epoch histogram
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x) s_hist[e] = 0;
  __syncthreads();
  uint32_t fl = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t e = epoch[i];
    const int32_t xi = x[i], yi = y[i];
    uint32_t b = kInvalidBucket;
    if (e >= E) {
      fl |= kFlagEpoch;
    } else {
      atomicAdd(&s_hist[e], 1u);
      if (xi <= -kLimPos || xi >= kLimPos || yi <= -kLimPos || yi >= kLimPos) {
        fl |= kFlagPos;
      } else {
        const int64_t cx = floor_div64((int64_t)xi - cg.gx0, cg.cell);
        const int64_t cy = floor_div64((int64_t)yi - cg.gy0, cg.cell);
        if (cx >= 0 && cx < cg.ncx && cy >= 0 && cy < cg.ncy) {
          b = (uint32_t)(((uint64_t)e * cg.ncy + (uint64_t)cy) * cg.ncx + (uint64_t)cx);
        } else {
          b = (uint32_t)((uint64_t)E * cg.ncy * cg.ncx);  // overflow bucket: outside the grid
        }
        atomicAdd(&bucket_count[b], 1u);
      }
    }
    bucket_of[i] = b;
  }
  if (fl) atomicOr(flags, fl);
  __syncthreads();
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x)
    if (s_hist[e]) atomicAdd(&ecount[e], s_hist[e]);
}

// a2 (scatter phase): place each bucketed detection at its bucket's cursor.
__global__ void k_scatter(const int32_t* __restrict__ x, const int32_t* __restrict__ y,
                          const uint16_t* __restrict__ epoch, uint64_t n,
                          const uint32_t* __restrict__ bucket_of, uint32_t* __restrict__ cursor,
                          Det* __restrict__ dets) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t b = bucket_of[i];
    if (b == kInvalidBucket) continue;
    const uint32_t pos = atomicAdd(&cursor[b], 1u);
    Det d;
    d.x = x[i];
    d.y = y[i];
    d.e = epoch[i];
    d.id = (uint32_t)i;
    dets[pos] = d;
  }
}

// Sec. 2.1 step 1: the reference epoch t0 is the earliest observation time of
// the catalog (over epochs that hold at least one detection); dt[e] = t[e] - t0.
__global__ void k_epoch_setup(uint32_t E, const int64_t* __restrict__ t,
                              const uint32_t* __restrict__ ecount, int64_t* __restrict__ dt,
                              int64_t* __restrict__ t0_out) {
  __shared__ long long s_min[32];
  long long m = LLONG_MAX;
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x)
    if (ecount[e] > 0 && t[e] < m) m = t[e];
  for (int o = 16; o > 0; o >>= 1) {
    long long other = __shfl_xor_sync(0xffffffffu, m, o);
    m = other < m ? other : m;
  }
  if ((threadIdx.x & 31) == 0) s_min[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x + 31) / 32 ? s_min[threadIdx.x] : LLONG_MAX;
    for (int o = 16; o > 0; o >>= 1) {
      long long other = __shfl_xor_sync(0xffffffffu, m, o);
      m = other < m ? other : m;
    }
    if (threadIdx.x == 0) s_min[0] = m;
  }
  __syncthreads();
  const long long t0 = s_min[0];
  for (uint32_t e = threadIdx.x; e < E; e += blockDim.x)
    dt[e] = ecount[e] > 0 ? (int64_t)(t[e] - t0) : 0;
  if (threadIdx.x == 0) *t0_out = t0;
}

// Sec. 2 Eq. 1-2: the shift of lattice column k at epoch e,
// s[k][e] = floor((v0 + k*dv) * dt[e] / TPH), exact in int64.
__global__ void k_shift_table(int32_t v0, int32_t dv, int32_t nk, uint32_t E, int64_t tph,
                              const int64_t* __restrict__ dt, const uint32_t* __restrict__ ecount,
                              int32_t* __restrict__ out, uint32_t* __restrict__ flags) {
  const uint64_t total = (uint64_t)nk * E;
  uint32_t fl = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = (uint32_t)(i / E), e = (uint32_t)(i % E);
    const int64_t v = (int64_t)v0 + (int64_t)k * dv;
    const int64_t s = floor_div64(v * dt[e], tph);
    int32_t sv = 0;
    if (s <= -kLimDomain || s >= kLimDomain) {
      if (ecount[e] > 0) fl |= kFlagShift;
    } else {
      sv = (int32_t)s;
    }
    out[i] = sv;
  }
  if (fl) atomicOr(flags, fl);
}

// ---- exclusive scan (three passes: block sums, scan of sums, apply) ---------

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ T block_exclusive_scan(T v, T* s_warp, T* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += n;
  }
  if (lane == 31) s_warp[w] = inc;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    T s = lane < nw ? s_warp[lane] : T(0);
    T si = s;
    for (int o = 1; o < 32; o <<= 1) {
      T n = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += n;
    }
    if (lane < nw) s_warp[lane] = si - s;
    if (lane == nw - 1) s_warp[32] = si;
  }
  __syncthreads();
  const T r = s_warp[w] + inc - v;
  if (total) *total = s_warp[32];
  __syncthreads();
  return r;
}

template <typename Tin, typename Tout>
__global__ void k_scan_reduce(const Tin* __restrict__ in, uint64_t n, Tout* __restrict__ sums) {
  __shared__ Tout s_warp[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  Tout acc = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + k;
    if (i < n) acc += (Tout)in[i];
  }
  Tout total;
  block_exclusive_scan<Tout>(acc, s_warp, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block scans the block sums in place (any count, carried across rounds).
template <typename Tout>
__global__ void k_scan_top(Tout* __restrict__ sums, uint64_t nb) {
  __shared__ Tout s_warp[33];
  Tout carry = 0;
  for (uint64_t base = 0; base < nb; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    const Tout v = i < nb ? sums[i] : Tout(0);
    Tout total;
    const Tout ex = block_exclusive_scan<Tout>(v, s_warp, &total);
    if (i < nb) sums[i] = carry + ex;
    carry += total;
  }
}

template <typename Tin, typename Tout>
__global__ void k_scan_apply(const Tin* __restrict__ in, uint64_t n, const Tout* __restrict__ sums,
                             Tout* __restrict__ out) {
  __shared__ Tout s_warp[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  Tout v[kScanItems];
  Tout acc = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + k;
    v[k] = i < n ? (Tout)in[i] : Tout(0);
    acc += v[k];
  }
  Tout total;
  Tout run = block_exclusive_scan<Tout>(acc, s_warp, &total) + sums[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    const uint64_t i = base + (uint64_t)threadIdx.x * kScanItems + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

template <typename Tin, typename Tout>
cudaError_t scan_impl(const Tin* in, Tout* out, uint64_t n, Tout* scratch, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(Tout), s);
  const uint64_t nb = (n + kScanTile - 1) / kScanTile;
  k_scan_reduce<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, scratch);
  k_scan_top<Tout><<<1, kScanThreads, 0, s>>>(scratch, nb);
  k_scan_apply<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, scratch, out);
  note_launch(3);
  return cudaGetLastError();
}

unsigned grid_for(uint64_t n, int threads) {
  uint64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152ull * 64) b = 152ull * 64;
  return (unsigned)b;
}

}  // namespace

size_t scan_scratch_elems(uint64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

cudaError_t launch_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* scratch,
                            cudaStream_t s) {
  return scan_impl<uint32_t, uint32_t>(in, out, n, scratch, s);
}

cudaError_t launch_scan_u32_to_u64(const uint32_t* in, unsigned long long* out, uint64_t n,
                                   unsigned long long* scratch, cudaStream_t s) {
  return scan_impl<uint32_t, unsigned long long>(in, out, n, scratch, s);
}

cudaError_t launch_ingest(const int32_t* x, const int32_t* y, const uint16_t* epoch, uint64_t n,
                          uint32_t E, CoarseGeom cg, uint32_t* bucket_count, uint32_t* ecount,
                          uint32_t* bucket_of, uint32_t* flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_ingest<<<grid_for(n, kPrepThreads), kPrepThreads, E * sizeof(uint32_t), s>>>(
      x, y, epoch, n, E, cg, bucket_count, ecount, bucket_of, flags);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_scatter(const int32_t* x, const int32_t* y, const uint16_t* epoch, uint64_t n,
                           const uint32_t* bucket_of, uint32_t* cursor, Det* dets,
                           cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_scatter<<<grid_for(n, kPrepThreads), kPrepThreads, 0, s>>>(x, y, epoch, n, bucket_of, cursor,
                                                                dets);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_epoch_setup(uint32_t E, const int64_t* t, const uint32_t* ecount, int64_t* dt,
                               int64_t* t0, cudaStream_t s) {
  k_epoch_setup<<<1, 1024, 0, s>>>(E, t, ecount, dt, t0);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_shift_tables(const SearchGeom& g, const int64_t* dt, const uint32_t* ecount,
                                int32_t* sxt, int32_t* syt, uint32_t* flags, cudaStream_t s) {
  k_shift_table<<<grid_for((uint64_t)g.nvx * g.E, kPrepThreads), kPrepThreads, 0, s>>>(
      g.vx0, g.dvx, g.nvx, g.E, g.tph, dt, ecount, sxt, flags);
  k_shift_table<<<grid_for((uint64_t)g.nvy * g.E, kPrepThreads), kPrepThreads, 0, s>>>(
      g.vy0, g.dvy, g.nvy, g.E, g.tph, dt, ecount, syt, flags);
  note_launch(2);
  return cudaGetLastError();
}

}  // namespace sas
