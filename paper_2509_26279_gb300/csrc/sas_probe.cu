// Shared-memory atomic throughput probes: the roofline peak of the stack kernel.
//
// Every thread of every resident CTA issues `iters` x 8 atomic updates to
// shared memory: 32-bit `red.shared.add.u32` (no value returned: the
// instruction the stack kernel's hot loop issues), 32-bit atomicAdd whose old
// value is used, or 64-bit `atom.shared.or.b64` whose old value is used (the
// epoch-bitmask update the stack kernel does not use; measured to justify the
// counters).  Lane l of warp w always touches word (w*32 + l) + k*blockDim,
// so the 32 lanes of a warp hit 32 distinct banks (conflict-free) and the
// addresses are compile-time offsets of one base register: the loop is bound by
// the shared-memory atomic unit, not by address arithmetic.
#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeUnroll = 8;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// clk[0], clk[1]: SM cycles and nanoseconds (global timer) over block 0's loop,
// from which the SM clock during the probe follows.
// MODE 0: atomicAdd (old value used); 1: red.shared.add.u32; 2: 64-bit atomicOr
// (old value used).  Lane l of warp w uses word (w * 32 + l) + k * blockDim of
// 32-bit words, or word (w * 32 + l) + (k % 4) * blockDim of 64-bit words (a
// warp's 32 lanes cover the 32 banks twice: the conflict-free 64-bit pattern).
template <int MODE>
__global__ void __launch_bounds__(kProbeThreads, 2)
    k_atomic_probe(uint32_t iters, uint32_t* sink, unsigned long long* clk) {
  // 64-bit words: four per thread (32 KB), each reused every fourth update
  __shared__ unsigned long long s64[MODE == 2 ? kProbeThreads * 4 : 1];
  __shared__ uint32_t s[MODE == 2 ? 1 : kProbeThreads * kProbeUnroll];
  if constexpr (MODE == 2) {
    for (int i = threadIdx.x; i < kProbeThreads * 4; i += blockDim.x) s64[i] = 0;
  } else {
    for (int i = threadIdx.x; i < kProbeThreads * kProbeUnroll; i += blockDim.x) s[i] = 0;
  }
  __syncthreads();
  const long long c0 = clock64();
  const unsigned long long t0 = global_ns();
  uint32_t* base = s + (MODE == 2 ? 0 : threadIdx.x);
  unsigned long long* base64 = s64 + (MODE == 2 ? threadIdx.x : 0);
  const uint32_t base_s = (uint32_t)__cvta_generic_to_shared(base);
  uint32_t acc = 0;
  unsigned long long acc64 = 0;
  for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kProbeUnroll; ++k) {
      if constexpr (MODE == 1)
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(base_s + 4u * (uint32_t)(k * kProbeThreads)), "r"(1u));
      else if constexpr (MODE == 2)
        acc64 |= atomicOr(base64 + (k & 3) * kProbeThreads, 1ull << ((it + k) & 63));
      else
        acc += atomicAdd(base + k * kProbeThreads, 1u);
    }
  }
  __syncthreads();
  const long long c1 = clock64();
  const unsigned long long t1 = global_ns();
  if (threadIdx.x == 0) {
    if (blockIdx.x == 0) {
      clk[0] = (unsigned long long)(c1 - c0);
      clk[1] = t1 - t0;
    }
    if constexpr (MODE == 2)
      sink[blockIdx.x] = (uint32_t)(s64[0] ^ acc64);
    else
      sink[blockIdx.x] = s[0] + acc;
  }
}

template <int MODE>
cudaError_t run_probe(uint32_t iters, cudaStream_t st, double* ops_per_s, double* sm_mhz) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_atomic_probe<MODE>, kProbeThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int blocks = sms * per_sm;
  uint32_t* sink = nullptr;
  unsigned long long* cycles = nullptr;
  if ((e = cudaMallocAsync(&sink, blocks * sizeof(uint32_t), st)) != cudaSuccess) return e;
  if ((e = cudaMallocAsync(&cycles, 2 * sizeof(unsigned long long), st)) != cudaSuccess) return e;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best_ms = 1e30f;
  double mhz = 0;
  for (int rep = 0; rep < 4; ++rep) {  // rep 0 warms up
    cudaMemsetAsync(cycles, 0, 2 * sizeof(unsigned long long), st);
    cudaEventRecord(a, st);
    k_atomic_probe<MODE><<<blocks, kProbeThreads, 0, st>>>(iters, sink, cycles);
    note_launch();
    cudaEventRecord(b, st);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    unsigned long long cyc[2] = {0, 0};
    cudaMemcpy(cyc, cycles, sizeof(cyc), cudaMemcpyDeviceToHost);
    if (rep > 0 && ms < best_ms) {
      best_ms = ms;
      mhz = cyc[1] ? (double)cyc[0] / ((double)cyc[1] * 1e-3) : 0.0;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(sink, st);
  cudaFreeAsync(cycles, st);
  if (e != cudaSuccess) return e;
  const double ops = (double)blocks * kProbeThreads * (double)iters * kProbeUnroll;
  *ops_per_s = ops / (best_ms * 1e-3);
  *sm_mhz = mhz;
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_atomic_probe(uint32_t iters, cudaStream_t s, double* ops_per_s, double* sm_mhz) {
  return run_probe<0>(iters, s, ops_per_s, sm_mhz);
}

cudaError_t run_red_probe(uint32_t iters, cudaStream_t s, double* ops_per_s, double* sm_mhz) {
  return run_probe<1>(iters, s, ops_per_s, sm_mhz);
}

cudaError_t run_or64_probe(uint32_t iters, cudaStream_t s, double* ops_per_s, double* sm_mhz) {
  return run_probe<2>(iters, s, ops_per_s, sm_mhz);
}

}  // namespace sas
