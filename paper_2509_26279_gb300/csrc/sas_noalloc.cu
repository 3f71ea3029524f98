// sas_cell_counts_noalloc: exact counts of caller-chosen cells with no device
// allocation.
//
// Some callers cannot allocate device memory while they run: code that has
// handed all device memory to its own pool ahead of time (a serving process
// with a fixed memory budget), code that runs where allocating CUDA calls are
// not allowed or would stall it (for example inside work that is being placed
// on a stream by a real-time loop that must never wait on the allocator).  For
// them this entry point computes the same per-cell numbers as the exact-count
// step of sas_stack (distinct epochs and raw detections of a histogram cell),
// reading the catalog where the caller keeps it, writing only the caller's
// output arrays, and keeping its small working state in a fixed array that is
// part of the library image.
#include <algorithm>
#include <climits>
#include <mutex>
#include <string>

#include "sas_internal.cuh"

namespace sas {

namespace {

// Fixed working state, 16 KiB, shared by every call on a device: the epoch
// times [0, 8 KiB), one presence word per epoch [8 KiB, 12 KiB) and a status
// word at 12 KiB.  Every GPU that loads the library holds it until exit.
constexpr size_t kNoAllocScratchBytes = 16384;
constexpr size_t kOffT = 0, kOffPresent = 8192, kOffStatus = 12288;
static_assert(SAS_MAX_EPOCHS * 8 <= kOffPresent, "epoch times must fit");
static_assert(kOffPresent + SAS_MAX_EPOCHS * 4 <= kOffStatus, "presence words must fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[64] = {};
int g_sms[64] = {};  // multiprocessors of each device (grid sizes)

constexpr int kCountThreads = 256;

// Marks the epochs that hold a detection (the reference epoch is the earliest
// of those, Sec. 2.1 step 1) and checks the catalog against the library's
// exact-integer limits.
__global__ void k_mark_epochs(const uint16_t* __restrict__ epoch, const int32_t* __restrict__ x,
                              const int32_t* __restrict__ y, uint64_t n, uint32_t E,
                              unsigned char* scratch) {
  uint32_t* present = reinterpret_cast<uint32_t*>(scratch + kOffPresent);
  uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kOffStatus);
  uint32_t fl = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t e = epoch[i];
    if (e >= E) {
      fl |= kFlagEpoch;
      continue;
    }
    if (x[i] <= -kLimPos || x[i] >= kLimPos || y[i] <= -kLimPos || y[i] >= kLimPos) fl |= kFlagPos;
    if (present[e] == 0) present[e] = 1;
  }
  if (fl) atomicOr(status, fl);
}

// One block per cell: the block computes t0 and the cell's shift at every
// epoch (Sec. 2 Eq. 1-2), then scans the whole catalog for detections whose
// projection falls in the cell (Sec. 2.1 step 2), marking their epochs in a
// bitmask whose popcount is the distinct-epoch count.
__global__ void __launch_bounds__(kCountThreads) k_count_cells(
    const int32_t* __restrict__ x, const int32_t* __restrict__ y,
    const uint16_t* __restrict__ epoch, uint64_t n, uint32_t E, int64_t tph, SearchGeom g,
    const uint32_t* __restrict__ cells, uint64_t n_cells, uint32_t* __restrict__ distinct,
    uint32_t* __restrict__ raw, unsigned char* scratch) {
  __shared__ int64_t s_sx[SAS_MAX_EPOCHS], s_sy[SAS_MAX_EPOCHS];
  __shared__ uint32_t s_mask[SAS_MAX_EPOCHS / 32];
  __shared__ long long s_min[kCountThreads / 32];
  __shared__ uint32_t s_raw;
  const int64_t* t = reinterpret_cast<const int64_t*>(scratch + kOffT);
  const uint32_t* present = reinterpret_cast<const uint32_t*>(scratch + kOffPresent);
  uint32_t* status = reinterpret_cast<uint32_t*>(scratch + kOffStatus);
  const int tid = threadIdx.x;

  long long m = LLONG_MAX;
  for (uint32_t e = tid; e < E; e += blockDim.x)
    if (present[e] && t[e] < m) m = t[e];
  for (int o = 16; o > 0; o >>= 1) {
    const long long other = __shfl_xor_sync(0xffffffffu, m, o);
    m = other < m ? other : m;
  }
  if ((tid & 31) == 0) s_min[tid >> 5] = m;
  __syncthreads();
  long long t0 = s_min[0];
  for (int w = 1; w < kCountThreads / 32; ++w) t0 = s_min[w] < t0 ? s_min[w] : t0;

  for (uint64_t c = blockIdx.x; c < n_cells; c += gridDim.x) {
    const uint32_t v_idx = cells[3 * c], bx = cells[3 * c + 1], by = cells[3 * c + 2];
    if (v_idx >= (uint32_t)g.nvx * (uint32_t)g.nvy || bx >= (uint32_t)g.nbx ||
        by >= (uint32_t)g.nby) {
      if (tid == 0) {
        distinct[c] = 0xffffffffu;
        raw[c] = 0xffffffffu;
        atomicOr(status, kFlagInternal);
      }
      continue;
    }
    const int64_t vx = (int64_t)g.vx0 + (int64_t)(v_idx % (uint32_t)g.nvx) * g.dvx;
    const int64_t vy = (int64_t)g.vy0 + (int64_t)(v_idx / (uint32_t)g.nvx) * g.dvy;
    for (uint32_t e = tid; e < E; e += blockDim.x) {
      const int64_t dt = present[e] ? (int64_t)(t[e] - t0) : 0;
      s_sx[e] = (int64_t)g.x_min + (int64_t)bx * g.bin + floor_div64(vx * dt, tph);
      s_sy[e] = (int64_t)g.y_min + (int64_t)by * g.bin + floor_div64(vy * dt, tph);
    }
    for (uint32_t q = tid; q < SAS_MAX_EPOCHS / 32; q += blockDim.x) s_mask[q] = 0;
    if (tid == 0) s_raw = 0;
    __syncthreads();
    uint32_t r = 0;
    for (uint64_t i = tid; i < n; i += blockDim.x) {
      const uint32_t e = epoch[i];
      if (e >= E) continue;
      const int64_t X = (int64_t)x[i] - s_sx[e], Y = (int64_t)y[i] - s_sy[e];
      if (X >= 0 && X < g.bin && Y >= 0 && Y < g.bin) {
        atomicOr(&s_mask[e >> 5], 1u << (e & 31));
        ++r;
      }
    }
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if ((tid & 31) == 0 && r) atomicAdd(&s_raw, r);
    __syncthreads();
    if (tid < 32) {
      uint32_t d = 0;
      for (uint32_t q = tid; q < SAS_MAX_EPOCHS / 32; q += 32) d += __popc(s_mask[q]);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
      if (tid == 0) {
        distinct[c] = d;
        raw[c] = s_raw;
      }
    }
    __syncthreads();
  }
}

// The device address of the fixed array, looked up once per device with that
// device current.  In host code the array's name is only a host-side stand-in,
// so kernels are given this address instead.  The same set-up reads the
// device's multiprocessor count, which sizes the grids.
int scratch_for_device(int dev, unsigned char** out, int* sms) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= 64) return SAS_ERR_ARG;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return SAS_ERR_CUDA;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n < 1) return SAS_ERR_CUDA;
    g_sms[dev] = n;
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  *sms = g_sms[dev];
  return SAS_OK;
}

}  // namespace

int noalloc_cell_counts(const sas_grid_desc& d, const sas_catalog* cat, const uint32_t* cells,
                        uint64_t n_cells, uint32_t* distinct, uint32_t* raw, void* stream,
                        std::string* err) {
  const uint32_t E = cat->n_epochs;
  if (E < 1 || E > SAS_MAX_EPOCHS) {
    *err = "n_epochs must be in [1, 1024] (the fixed working array holds 1024 epochs)";
    return SAS_ERR_RANGE;
  }
  if (!cat->on_device) {
    *err = "the catalog must be in device memory (on_device = 1)";
    return SAS_ERR_ARG;
  }
  if (cat->ticks_per_hour <= 0 || !cat->t) {
    *err = "bad epoch time table";
    return SAS_ERR_ARG;
  }
  if (cat->n >= ((uint64_t)1 << 31)) {
    *err = "n must be < 2^31";
    return SAS_ERR_RANGE;
  }
  if (cat->n > 0 && (!cat->x || !cat->y || !cat->epoch)) {
    *err = "null catalog array";
    return SAS_ERR_ARG;
  }
  if (n_cells > 0 && (!cells || !distinct || !raw)) {
    *err = "null cell or output array";
    return SAS_ERR_ARG;
  }
  int64_t tmin = cat->t[0], tmax = cat->t[0];
  for (uint32_t e = 1; e < E; ++e) {
    tmin = cat->t[e] < tmin ? cat->t[e] : tmin;
    tmax = cat->t[e] > tmax ? cat->t[e] : tmax;
  }
  if ((__int128)tmax - tmin >= ((__int128)1 << 32)) {
    *err = "time span must be < 2^32 ticks";
    return SAS_ERR_RANGE;
  }
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) {
    *err = cudaGetErrorString(ce);
    return SAS_ERR_CUDA;
  }
  unsigned char* scratch = nullptr;
  int sms = 0;
  if (scratch_for_device(dev, &scratch, &sms) != SAS_OK) {
    *err = "set-up failed (cudaGetSymbolAddress of the fixed working array, or the device's SM count)";
    return SAS_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // The array keeps the previous call's contents: reset what must start at zero.
  ce = cudaMemcpyAsync(scratch + kOffT, cat->t, E * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(scratch + kOffPresent, 0, SAS_MAX_EPOCHS * 4, s);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(scratch + kOffStatus, 0, 4, s);
  if (ce != cudaSuccess) {
    *err = cudaGetErrorString(ce);
    return SAS_ERR_CUDA;
  }
  SearchGeom g{};
  g.vx0 = d.vx0; g.vy0 = d.vy0; g.dvx = d.dvx; g.dvy = d.dvy;
  g.nvx = (int32_t)d.nvx; g.nvy = (int32_t)d.nvy;
  g.x_min = d.x_min; g.y_min = d.y_min;
  g.nbx = (int32_t)d.nbx; g.nby = (int32_t)d.nby; g.bin = d.bin;
  g.E = E; g.tph = cat->ticks_per_hour;
  if (cat->n > 0) {
    const unsigned blocks = (unsigned)std::min<uint64_t>((cat->n + 255) / 256, (uint64_t)sms * 16);
    k_mark_epochs<<<blocks, 256, 0, s>>>(cat->epoch, cat->x, cat->y, cat->n, E, scratch);
    note_launch();
  }
  if (n_cells > 0) {
    const unsigned blocks = (unsigned)std::min<uint64_t>(n_cells, (uint64_t)sms * 8);
    k_count_cells<<<blocks, kCountThreads, 0, s>>>(cat->x, cat->y, cat->epoch, cat->n, E,
                                                   cat->ticks_per_hour, g, cells, n_cells,
                                                   distinct, raw, scratch);
    note_launch();
  }
  uint32_t status = 0;
  ce = cudaGetLastError();
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(&status, scratch + kOffStatus, 4, cudaMemcpyDeviceToHost, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    *err = cudaGetErrorString(ce);
    return SAS_ERR_CUDA;
  }
  if (status & kFlagEpoch) { *err = "an epoch index is >= n_epochs"; return SAS_ERR_RANGE; }
  if (status & kFlagPos) { *err = "a detection has |x| or |y| >= 2^29"; return SAS_ERR_RANGE; }
  if (status & kFlagInternal) { *err = "a cell lies outside the lattice or the domain"; return SAS_ERR_ARG; }
  return SAS_OK;
}

}  // namespace sas
