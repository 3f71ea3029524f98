// Candidate vetter: a small CNN that scores a candidate from its count stamp,
// trained and run on the GPU (BF16 weights and activations, FP32 accumulation).
//
// Filtering the search results better is the paper's own suggestion for going
// fainter (Sec. 5); this network is that filter.  Network (input = count / 16):
//   conv1 9->32 3x3 valid + ReLU (15 -> 13), conv2 32->32 (13 -> 11) + ReLU,
//   conv3 32->32 (11 -> 9) + ReLU, flatten (channel, row, column),
//   fc1 2592 -> 64 + ReLU, fc2 64 -> 1 = logit;  loss: mean BCE with logits.
// Flat parameter order: conv1.w [32,9,3,3], conv1.b, conv2.w [32,32,3,3],
// conv2.b, conv3.w, conv3.b, fc1.w [64,2592], fc1.b, fc2.w [64], fc2.b.
//
// Numerics: weights are used as BF16 copies of FP32 master values; every stored
// activation (input, conv outputs, fc1 output) is rounded to BF16; products are
// exact in FP32 and accumulate in FP32.  Back-propagated deltas and weight
// gradients are FP32.  Weight gradients are summed per block over a fixed
// stamp-to-block assignment and then over blocks in a fixed order, so a
// gradient is bit-reproducible for a given batch.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sas_internal.cuh"
#include "sas_tc.cuh"

struct sas_vet {
  int device;
  uint32_t max_batch;
  uint64_t step;
  float beta1, beta2, eps;
  // parameters
  float* master;
  float* m;
  float* v;
  float* grad;
  __nv_bfloat16* wb;     // BF16 copy in the flat order
  // activations and deltas of one batch
  __nv_bfloat16* a1;     // [B][32][13][13]
  __nv_bfloat16* a2;     // [B][32][11][11]
  __nv_bfloat16* a3;     // [B][2592]
  __nv_bfloat16* a4;     // [B][64]
  float* logits;         // [B]
  float* fcpart;         // [kFcSplit][64][B rounded up to 128] fc1 partial sums
  float* glogit;         // [B]
  float* g4;             // [B][64]
  float* g3;             // [B][2592]
  float* g2;             // [B][32][11][11]
  float* g1;             // [B][32][13][13]
  float* partial;        // per-block weight-gradient partial sums
  float* loss;           // [1]
  uint32_t* status;      // [1] nonzero: a tensor-core wait gave up (sas_vet_check)
};

namespace sas {
namespace vet {

constexpr int kS = 15, kQ = 9, kCh = 32;
constexpr int kH1 = 13, kH2 = 11, kH3 = 9;
constexpr int kF = kCh * kH3 * kH3;  // 2592
constexpr int kHid = 64;
constexpr int kW1 = 0, kB1 = kW1 + kCh * kQ * 9, kW2 = kB1 + kCh, kB2 = kW2 + kCh * kCh * 9;
constexpr int kW3 = kB2 + kCh, kB3 = kW3 + kCh * kCh * 9, kWf1 = kB3 + kCh, kBf1 = kWf1 + kHid * kF;
constexpr int kWf2 = kBf1 + kHid, kBf2 = kWf2 + kHid, kNParams = kBf2 + 1;
static_assert(kNParams == 187137, "parameter layout");

constexpr int kBackBlocks = 256;      // blocks (and partial sums) of the conv backward kernels
constexpr int kPartialStride = kCh * kCh * 9 + kCh;  // >= parts * weights + biases of any layer
constexpr uint32_t kFc1Slices = 8;                   // stamp slices of the fc1 weight gradient
static_assert((size_t)kFc1Slices * (kHid * kF + kHid) <= (size_t)kBackBlocks * kPartialStride,
              "fc1 slices fit the partial buffer");
static_assert(kPartialStride >= 3 * kCh * kQ * 9 + kCh, "partial stride");

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// ---- forward on the tensor cores: the three convolutions as implicit GEMMs ---
//
// Per stamp and layer: D[pixel][out] = sum over taps (dy, dx) and input channels
// c of A[pixel + dy * W + dx][c] * w[out][c][dy][dx], with A the layer's input
// (W x W pixels, row r = y * W + x) and D computed over the padded output grid
// (rows y * W + x for x < W; the columns x >= W - 2 are not outputs and are
// dropped).  A sits in shared memory as [8-channel chunk][row][8 channels], so
// its rows are 16 bytes apart and the operand of tap (dy, dx) is the same
// buffer started dy * W + dx rows later: no im2col is built.  Each tap of each
// 128-row tile is one tcgen05.mma per 16 input channels (BF16 x BF16 -> FP32 in
// TMEM), all issued by one thread; every warp then reads its TMEM lanes back for
// bias + ReLU + BF16 rounding straight into the next layer's input layout.
// Products are exact in FP32 and the sums accumulate in FP32.

constexpr int kTcThreads = 512;   // 16 warps: 4 TMEM lane quadrants x 4 eight-channel slices
constexpr int kTcRows0 = 288;     // x0: 15 x 15 pixels; tiles read up to row 2 * 128 - 1 + 2 * 15 + 2
constexpr int kTcRows1 = 288;     // a1: 13 x 13 pixels; up to row 2 * 128 - 1 + 2 * 13 + 2
constexpr int kTcRows2 = 160;     // a2: 11 x 11 pixels; up to row 127 + 2 * 11 + 2
constexpr int kTcW1 = 9 * kCh * 16 * 2;   // per tap: 32 outputs x 16 input channels (9 real)
constexpr int kTcW23 = 9 * kCh * kCh * 2; // per tap: 32 x 32
constexpr int kSmX0 = 0;
constexpr int kSmA1 = kSmX0 + 2 * kTcRows0 * 16;
constexpr int kSmA2 = kSmA1 + 4 * kTcRows1 * 16;
constexpr int kSmW1 = kSmA2 + 4 * kTcRows2 * 16;
constexpr int kSmW2 = kSmW1 + kTcW1;
constexpr int kSmW3 = kSmW2 + kTcW23;
constexpr int kSmBias = kSmW3 + kTcW23;
constexpr int kSmBar = kSmBias + 3 * kCh * 4;
constexpr int kTcSmem = kSmBar + 16;
constexpr int kTcTmemCols = 256;  // conv1 tiles at columns 0, 32; conv2 at 64, 96; conv3 at 128
static_assert(2 * kTcRows0 >= 2 * 128 + 2 * kS + 2 && kTcRows1 >= 2 * 128 + 2 * kH1 + 2 &&
                  kTcRows2 >= 128 + 2 * kH2 + 2, "shifted windows stay inside the buffers");
static_assert(kTcRows0 >= 2 * 128 + 2 * kS + 2, "conv1 windows");
static_assert(kSmW1 % 128 == 0 && kSmW2 % 128 == 0 && kSmW3 % 128 == 0 && kSmA1 % 16 == 0 &&
                  kSmA2 % 16 == 0, "operand alignment");
static_assert(2 * kTcSmem <= 227 * 1024, "two CTAs per SM");

// Per-tap weights of a layer as the B operand: B_t[o][c] = w[o][c][t] (c < cin),
// zero for c >= cin; kc 16-byte chunks per row (K = 8 kc).
__device__ void tc_load_w_taps(const __nv_bfloat16* __restrict__ w, int cin, int kc, unsigned char* dst) {
  const int per_tap = kCh * kc * 8;
  for (int i = threadIdx.x; i < 9 * per_tap; i += blockDim.x) {
    const int t = i / per_tap, j = i - t * per_tap, o = j / (kc * 8), c = j - o * (kc * 8);
    const __nv_bfloat16 v = c < cin ? w[(o * cin + c) * 9 + t] : __float2bfloat16_rn(0.f);
    *reinterpret_cast<__nv_bfloat16*>(dst + t * per_tap * 2 + tc::cm_offset(o, c, kc)) = v;
  }
}

// The MMAs of one layer (thread 0): NT tiles of 128 output rows, 9 taps, KS
// steps of 16 input channels; input rows R per chunk, input width W.
template <int NT, int KS, int R, int W>
__device__ __forceinline__ void tc_conv_mma(uint32_t a_base, uint32_t w_base, uint32_t tmem_col) {
  constexpr uint32_t idesc = tc::idesc_bf16(128, 32);
  constexpr uint32_t per_tap = kCh * KS * 2 * 16;  // bytes of one tap's B operand
#pragma unroll
  for (int t = 0; t < NT; ++t)
    for (int tap = 0; tap < 9; ++tap) {
      const uint32_t shift = (uint32_t)((tap / 3) * W + (tap % 3));
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const uint64_t ad = tc::smem_desc_strided(a_base + (uint32_t)(2 * ks * R * 16) + (t * 128u + shift) * 16u,
                                                  (uint32_t)(R * 16), 128u);
        const uint64_t bd = tc::smem_desc(w_base + (uint32_t)tap * per_tap + (uint32_t)(2 * ks * 128), 2 * KS);
        tc::mma_bf16(tmem_col + (uint32_t)(t * 32), ad, bd, idesc, (tap | ks) != 0);
      }
    }
}

// Bias, ReLU and BF16 rounding of a layer's D (NT tiles at TMEM column tmem_col)
// over the padded grid of width W (outputs: W - 2 x W - 2) into the next layer's
// input layout (rows (W - 2) * y + x, Rn rows per chunk) and, optionally, the
// global activation [ch][W-2][W-2].
template <int NT, int W, int Rn>
__device__ __forceinline__ void tc_conv_epi(uint32_t tmem_col, const float* bias, unsigned char* next,
                                            __nv_bfloat16* out_g) {
  constexpr int HO = W - 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3, h = warp >> 2;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    float v[8];
    tc::ld8(tmem_col + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * 32 + h * 8), v);
    const int m = t * 128 + q * 32 + lane, y = m / W, x = m - y * W;
    if (y < HO && x < HO) {
      const int p = y * HO + x;
      uint32_t pk[4];
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const __nv_bfloat16 r0 = __float2bfloat16_rn(fmaxf(v[j] + bias[h * 8 + j], 0.f));
        const __nv_bfloat16 r1 = __float2bfloat16_rn(fmaxf(v[j + 1] + bias[h * 8 + j + 1], 0.f));
        pk[j / 2] = (uint32_t)__bfloat16_as_ushort(r0) | ((uint32_t)__bfloat16_as_ushort(r1) << 16);
        if (out_g) {
          out_g[(h * 8 + j) * HO * HO + p] = r0;
          out_g[(h * 8 + j + 1) * HO * HO + p] = r1;
        }
      }
      if (next)
        *reinterpret_cast<uint4*>(next + (h * Rn + p) * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

// One layer: operand visible to the tensor core, MMAs by thread 0, bounded
// wait, epilogue.  Returns false (block-uniform) when the wait gave up.
template <int NT, int KS, int R, int W, int Rn>
__device__ __forceinline__ bool tc_conv_layer(unsigned char* smc, int a_off, int w_off, uint32_t tmem_col,
                                              uint64_t* bar, uint32_t& phase, const float* bias, int next_off,
                                              __nv_bfloat16* out_g) {
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0) {
    tc::fence_after_sync();
    tc_conv_mma<NT, KS, R, W>(tc::smem_u32(smc + a_off), tc::smem_u32(smc + w_off), tmem_col);
    tc::commit(bar);
  }
  const bool ok = tc::mbar_wait(bar, phase, 1u << 22);
  phase ^= 1u;
  if (__syncthreads_or(!ok)) return false;
  tc::fence_after_sync();
  tc_conv_epi<NT, W, Rn>(tmem_col, bias, next_off >= 0 ? smc + next_off : nullptr, out_g);
  tc::fence_before_sync();
  return true;
}

__global__ void __launch_bounds__(kTcThreads, 2) k_conv_fwd_tc(const uint16_t* __restrict__ stamps,
                                                               const uint32_t* __restrict__ idx, uint32_t n,
                                                               const __nv_bfloat16* __restrict__ wb,
                                                               __nv_bfloat16* a1g, __nv_bfloat16* a2g,
                                                               __nv_bfloat16* __restrict__ a3g,
                                                               uint32_t* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smc[];
  float* bias = reinterpret_cast<float*>(smc + kSmBias);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smc + kSmBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smc + kSmBar + 8);
  uint16_t* x0 = reinterpret_cast<uint16_t*>(smc + kSmX0);
  const int tid = threadIdx.x;
  if (tid < 32) tc::tmem_alloc(tslot, kTcTmemCols);
  if (tid == 0) tc::mbar_init(bar, 1);
  // activation buffers: rows that are never written (input padding, channel
  // padding of x0) stay zero
  for (int i = tid; i < kSmW1 / 16; i += kTcThreads) reinterpret_cast<uint4*>(smc)[i] = make_uint4(0, 0, 0, 0);
  tc_load_w_taps(wb + kW1, kQ, 2, smc + kSmW1);
  tc_load_w_taps(wb + kW2, kCh, 4, smc + kSmW2);
  tc_load_w_taps(wb + kW3, kCh, 4, smc + kSmW3);
  if (tid < 3 * kCh) {
    const int l = tid / kCh, o = tid % kCh;
    bias[tid] = ld(wb + (l == 0 ? kB1 : l == 1 ? kB2 : kB3) + o);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  // each thread holds its share of the next stamp while the current one runs
  constexpr int kPer = (kQ * kS * kS + kTcThreads - 1) / kTcThreads;
  uint16_t nxt[kPer];
  auto fetch = [&](uint32_t b) {
    if (b >= n) return;
    const uint16_t* st = stamps + (size_t)(idx ? idx[b] : b) * kQ * kS * kS;
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int i = tid + r * kTcThreads;
      nxt[r] = i < kQ * kS * kS ? st[i] : (uint16_t)0;
    }
  };
  fetch(blockIdx.x);
  for (uint32_t b = blockIdx.x; b < n; b += gridDim.x) {
    // x0[chunk c / 8][row][c % 8] = count / 16 in BF16 (exact for counts <= 256 * 16)
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int i = tid + r * kTcThreads;
      if (i < kQ * kS * kS) {
        const int c = i / (kS * kS), p = i - c * (kS * kS);
        x0[((c >> 3) * kTcRows0 + p) * 8 + (c & 7)] =
            __bfloat16_as_ushort(__float2bfloat16_rn((float)nxt[r] * 0.0625f));
      }
    }
    fetch(b + gridDim.x);
    if (!tc_conv_layer<2, 1, kTcRows0, kS, kTcRows1>(smc, kSmX0, kSmW1, tmem, bar, phase, bias, kSmA1,
                                                     a1g ? a1g + (size_t)b * kCh * kH1 * kH1 : nullptr) ||
        !tc_conv_layer<2, 2, kTcRows1, kH1, kTcRows2>(smc, kSmA1, kSmW2, tmem + 64, bar, phase, bias + kCh, kSmA2,
                                                      a2g ? a2g + (size_t)b * kCh * kH2 * kH2 : nullptr) ||
        !tc_conv_layer<1, 2, kTcRows2, kH2, 1>(smc, kSmA2, kSmW3, tmem + 128, bar, phase, bias + 2 * kCh, -1,
                                               a3g + (size_t)b * kF)) {
      if (tid == 0) atomicOr(status, 1u);
      break;
    }
    __syncthreads();  // the next stamp's input overwrites x0, which the MMAs above read
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_free(tmem, kTcTmemCols);
}

// ---- forward: fc1 on the tensor cores, fc2 in the epilogue --------------------
//
// D[stamp][j] = sum_k a3[stamp][k] * fc1.w[j][k]: M = 128 stamps per block,
// N = 64, K = 2592 in 27 blocks of 96, split over kFcSplit blocks along K so
// that a batch of 4096 stamps keeps 128 SMs busy.  Both operands are
// K-contiguous in global memory; every thread copies 16-byte rows of core
// matrices into the no-swizzle K-major layout of one of three stages while the
// MMAs of the others run (one mbarrier per stage, bounded waits).  Each block
// writes its FP32 partial D column-major; k_fc_epi adds the kFcSplit partials
// in a fixed order, adds the bias, applies ReLU, rounds to BF16, stores a4 and
// forms the logit with fc2 in a fixed order.
constexpr int kFcTcRows = 128, kFcTcKB = 96, kFcTcKC = kFcTcKB / 8, kFcTcNB = kF / kFcTcKB;
constexpr int kFcTcThreads = 256, kFcTcStages = 3, kFcSplit = 4;
constexpr int kFcTcA = kFcTcRows * kFcTcKB * 2, kFcTcB = kHid * kFcTcKB * 2;
constexpr int kFcTcStage = kFcTcA + kFcTcB;
constexpr int kFcTcSmem = kFcTcStages * kFcTcStage + 8 * kFcTcStages + 16;
static_assert(kF % kFcTcKB == 0, "fc1 K blocks");

// part[s][j][stamp] (stamps padded to whole 128-row tiles: ld = tiles * 128)
__global__ void __launch_bounds__(kFcTcThreads) k_fc_fwd_tc(const __nv_bfloat16* __restrict__ a3g, uint32_t n,
                                                            const __nv_bfloat16* __restrict__ wb,
                                                            float* __restrict__ part, uint32_t ldp,
                                                            uint32_t* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smf[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smf + kFcTcStages * kFcTcStage);  // [kFcTcStages]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + kFcTcStages);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t b0 = blockIdx.x * kFcTcRows;
  const int sp = blockIdx.y;
  const int kb_lo = sp * kFcTcNB / kFcSplit, kb_hi = (sp + 1) * kFcTcNB / kFcSplit;
  if (tid < 32) tc::tmem_alloc(tslot, kHid);
  if (tid == 0)
    for (int st = 0; st < kFcTcStages; ++st) tc::mbar_init(bar + st, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint4* a3v = reinterpret_cast<const uint4*>(a3g);
  const uint4* w1v = reinterpret_cast<const uint4*>(wb + kWf1);
  constexpr uint32_t idesc = tc::idesc_bf16(kFcTcRows, kHid);
  uint32_t ph[kFcTcStages] = {};
  bool ok = true;
  for (int kb = kb_lo; kb < kb_hi && ok; ++kb) {
    const int l = kb - kb_lo, st = l % kFcTcStages;
    unsigned char* A = smf + st * kFcTcStage;
    unsigned char* B = A + kFcTcA;
    if (l >= kFcTcStages) {  // the MMAs that read this stage kFcTcStages blocks ago are done
      ok = tc::mbar_wait(bar + st, ph[st], 1u << 22);
      ph[st] ^= 1u;
      if (__syncthreads_or(!ok)) break;
    }
    const int k8 = kb * kFcTcKC;  // first 16-byte chunk of the block along K
    for (int i = tid; i < kFcTcRows * kFcTcKC; i += kFcTcThreads) {
      const int r = i / kFcTcKC, c = i - r * kFcTcKC;
      const uint4 v = b0 + r < n ? a3v[(size_t)(b0 + r) * (kF / 8) + k8 + c] : make_uint4(0, 0, 0, 0);
      *reinterpret_cast<uint4*>(A + tc::cm_offset(r, c * 8, kFcTcKC)) = v;
    }
    for (int i = tid; i < kHid * kFcTcKC; i += kFcTcThreads) {
      const int r = i / kFcTcKC, c = i - r * kFcTcKC;
      *reinterpret_cast<uint4*>(B + tc::cm_offset(r, c * 8, kFcTcKC)) = w1v[(size_t)r * (kF / 8) + k8 + c];
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a0 = tc::smem_u32(A), w0 = tc::smem_u32(B);
#pragma unroll
      for (int ks = 0; ks < kFcTcKC / 2; ++ks)
        tc::mma_bf16(tmem, tc::smem_desc(a0 + (uint32_t)(2 * ks * 128), kFcTcKC),
                     tc::smem_desc(w0 + (uint32_t)(2 * ks * 128), kFcTcKC), idesc, (l > 0 || ks > 0) ? 1u : 0u);
      tc::commit(bar + st);
    }
  }
  if (ok) {  // one commit outstanding on every stage that was used
    const int used = min(kb_hi - kb_lo, kFcTcStages);
    for (int st = 0; st < used && ok; ++st) {
      ok = tc::mbar_wait(bar + st, ph[st], 1u << 22);
      ph[st] ^= 1u;
    }
    ok = !__syncthreads_or(!ok);
  }
  if (!ok) {
    if (tid == 0) atomicOr(status, 1u);
  } else {
    tc::fence_after_sync();
    const int q = warp & 3, h = warp >> 2;  // lane quadrant, column half
    const uint32_t b = b0 + (uint32_t)(q * 32 + lane);
    float* out = part + (size_t)sp * kHid * ldp;
#pragma unroll
    for (int c = h * 32; c < h * 32 + 32; c += 16) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) out[(size_t)(c + jj) * ldp + b] = v[jj];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (tid < 32) tc::tmem_free(tmem, kHid);
}

// One thread per stamp: the partial sums in split order, bias, ReLU, BF16,
// then fc2 in j order.
__global__ void __launch_bounds__(256) k_fc_epi(const float* __restrict__ part, uint32_t ldp, uint32_t n,
                                                const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* a4g,
                                                float* __restrict__ logits) {
  __shared__ float b1[kHid], w2[kHid];
  if (threadIdx.x < kHid) {
    b1[threadIdx.x] = ld(wb + kBf1 + threadIdx.x);
    w2[threadIdx.x] = ld(wb + kWf2 + threadIdx.x);
  }
  __syncthreads();
  const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  float logit = 0.f;
  for (int j = 0; j < kHid; ++j) {
    float acc = part[(size_t)j * ldp + b];
#pragma unroll
    for (int sp = 1; sp < kFcSplit; ++sp) acc += part[((size_t)sp * kHid + j) * ldp + b];
    const float a = bf(fmaxf(acc + b1[j], 0.f));
    if (a4g) a4g[(size_t)b * kHid + j] = __float2bfloat16_rn(a);
    logit = fmaf(a, w2[j], logit);
  }
  logits[b] = logit + ld(wb + kBf2);
}

// ---- loss, fc2 gradients, fc1 output deltas ------------------------------------

// One block: per-stamp loss and d loss / d logit; loss mean; fc2 gradients.
constexpr int kLossThreads = 1024;

__global__ void __launch_bounds__(kLossThreads) k_loss(const float* __restrict__ logits,
                                                       const float* __restrict__ labels,
                                                       const uint32_t* __restrict__ idx, uint32_t n,
                                                       const __nv_bfloat16* __restrict__ a4g,
                                                       float* __restrict__ glogit,
                                                       float* __restrict__ grad, float* __restrict__ loss) {
  __shared__ float red[kLossThreads];
  const int t = threadIdx.x;
  const float inv_n = 1.f / (float)n;
  float l = 0.f;
  for (uint32_t b = t; b < n; b += blockDim.x) {
    const float z = logits[b], y = labels[idx ? idx[b] : b];
    l += fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)));
    glogit[b] = (1.f / (1.f + expf(-z)) - y) * inv_n;
  }
  red[t] = l;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) *loss = red[0] * inv_n;
  __syncthreads();
  // fc2.w[j] = sum_b glogit[b] * a4[b][j]; fc2.b = sum_b glogit[b]
  // 16 parts of the batch per hidden unit, combined in a fixed order
  const int j = t & 63, part = t >> 6;
  float acc = 0.f, accb = 0.f;
  for (uint32_t b = part; b < n; b += 16) {
    const float g = glogit[b];
    acc = fmaf(g, ld(a4g + (size_t)b * kHid + j), acc);
    accb += g;
  }
  red[t] = acc;
  __syncthreads();
  if (t < 64) {
    float s = 0.f;
    for (int p = 0; p < 16; ++p) s += red[p * 64 + t];
    grad[kWf2 + t] = s;
  }
  __syncthreads();
  red[t] = (j == 0) ? accb : 0.f;
  __syncthreads();
  if (t == 0) {
    float s = 0.f;
    for (int p = 0; p < 16; ++p) s += red[p * 64];
    grad[kBf2] = s;
  }
}

// g4[b][j] = glogit[b] * w2[j] * (a4[b][j] > 0)
__global__ void k_g4(const float* __restrict__ glogit, const __nv_bfloat16* __restrict__ a4g,
                     const __nv_bfloat16* __restrict__ wb, uint32_t n, float* __restrict__ g4) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= (uint64_t)n * kHid) return;
  const int j = (int)(i % kHid);
  g4[i] = ld(a4g + i) > 0.f ? glogit[i / kHid] * ld(wb + kWf2 + j) : 0.f;
}

// fc1.w[j][k] = sum_b g4[b][j] * a3[b][k];  fc1.b[j] = sum_b g4[b][j].
// Block: 32 columns k, all 64 rows j, whole batch.
// Grid (columns / 32, slices): slice s adds the stamps [s n / S, (s + 1) n / S)
// and writes its partial sums to part[s][j][k] (weights) and part[S * 64 * kF +
// s * 64 + j] (biases); k_fc1_sum adds the slices in a fixed order.
__global__ void __launch_bounds__(256) k_fc1_dw(const float* __restrict__ g4,
                                                const __nv_bfloat16* __restrict__ a3g, uint32_t n,
                                                float* __restrict__ part) {
  __shared__ __align__(16) float Gs[32][kHid];
  __shared__ float Fs[32][33];
  const int t = threadIdx.x, jq = t & 15, kp = t >> 4;
  const int k0 = blockIdx.x * 32;
  const uint32_t S = gridDim.y, s = blockIdx.y;
  const uint32_t lo = (uint32_t)((uint64_t)n * s / S), hi = (uint32_t)((uint64_t)n * (s + 1) / S);
  float* pw = part + (size_t)s * kHid * kF;                 // [j][k] of this slice
  float* pb = part + (size_t)S * kHid * kF + (size_t)s * kHid;  // [j] of this slice
  float acc[4][2] = {}, accb[4] = {};
  for (uint32_t b0 = lo; b0 < hi; b0 += 32) {
    for (int i = t; i < 32 * kHid; i += 256) {
      const uint32_t b = b0 + i / kHid;
      Gs[i / kHid][i % kHid] = b < hi ? g4[(size_t)b * kHid + i % kHid] : 0.f;
    }
    for (int i = t; i < 32 * 32; i += 256) {
      const uint32_t b = b0 + i / 32;
      const int k = k0 + i % 32;
      Fs[i / 32][i % 32] = (b < hi && k < kF) ? ld(a3g + (size_t)b * kF + k) : 0.f;
    }
    __syncthreads();
    for (int bb = 0; bb < 32; ++bb) {
      const float4 g = *reinterpret_cast<const float4*>(&Gs[bb][jq * 4]);
      const float f0 = Fs[bb][kp * 2], f1 = Fs[bb][kp * 2 + 1];
      acc[0][0] = fmaf(g.x, f0, acc[0][0]); acc[0][1] = fmaf(g.x, f1, acc[0][1]);
      acc[1][0] = fmaf(g.y, f0, acc[1][0]); acc[1][1] = fmaf(g.y, f1, acc[1][1]);
      acc[2][0] = fmaf(g.z, f0, acc[2][0]); acc[2][1] = fmaf(g.z, f1, acc[2][1]);
      acc[3][0] = fmaf(g.w, f0, acc[3][0]); acc[3][1] = fmaf(g.w, f1, acc[3][1]);
      accb[0] += g.x; accb[1] += g.y; accb[2] += g.z; accb[3] += g.w;
    }
    __syncthreads();
  }
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int j = jq * 4 + jj;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const int k = k0 + kp * 2 + kk;
      if (k < kF) pw[(size_t)j * kF + k] = acc[jj][kk];
    }
    if (blockIdx.x == 0 && kp == 0) pb[j] = accb[jj];
  }
}

// grad[fc1.w] and grad[fc1.b]: the S slices of k_fc1_dw added in slice order.
__global__ void k_fc1_sum(const float* __restrict__ part, uint32_t S, float* __restrict__ grad) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (uint32_t)(kHid * kF)) {
    float v = 0.f;
    for (uint32_t s = 0; s < S; ++s) v += part[(size_t)s * kHid * kF + i];
    grad[kWf1 + i] = v;
  } else if (i < (uint32_t)(kHid * kF + kHid)) {
    const uint32_t j = i - kHid * kF;
    float v = 0.f;
    for (uint32_t s = 0; s < S; ++s) v += part[(size_t)S * kHid * kF + s * kHid + j];
    grad[kBf1 + j] = v;
  }
}

// g3[b][k] = (sum_j g4[b][j] * fc1.w[j][k]) * (a3[b][k] > 0).
// Block: 64 columns k x 32 stamps.
__global__ void __launch_bounds__(256) k_fc1_dx(const float* __restrict__ g4,
                                                const __nv_bfloat16* __restrict__ wb,
                                                const __nv_bfloat16* __restrict__ a3g, uint32_t n,
                                                float* __restrict__ g3) {
  __shared__ float Gs[32][kHid + 1];
  __shared__ float Ws[kHid][64];
  const int t = threadIdx.x, kk = t & 63, bg = t >> 6;
  const int k0 = blockIdx.x * 64;
  const uint32_t b0 = blockIdx.y * 32;
  for (int i = t; i < 32 * kHid; i += 256) {
    const uint32_t b = b0 + i / kHid;
    Gs[i / kHid][i % kHid] = b < n ? g4[(size_t)b * kHid + i % kHid] : 0.f;
  }
  for (int i = t; i < kHid * 64; i += 256) {
    const int j = i / 64, k = k0 + i % 64;
    Ws[j][i % 64] = k < kF ? ld(wb + kWf1 + (size_t)j * kF + k) : 0.f;
  }
  __syncthreads();
  float acc[8] = {};
  for (int j = 0; j < kHid; ++j) {
    const float w = Ws[j][kk];
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[s] = fmaf(Gs[bg * 8 + s][j], w, acc[s]);
  }
  const int k = k0 + kk;
  if (k >= kF) return;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const uint32_t b = b0 + bg * 8 + s;
    if (b < n) g3[(size_t)b * kF + k] = ld(a3g + (size_t)b * kF + k) > 0.f ? acc[s] : 0.f;
  }
}

// ---- conv1 weight gradient (CUDA cores) -----------------------------------------

constexpr int kBackThreads = 256;

// The first layer (C = 9 input channels of HI x HI, output 32 x HO x HO): gin
// is the masked delta of its output [n][32][HO*HO], its input the stamps (no
// input delta is needed).  Block partial (at partial + blockIdx.x *
// kPartialStride): [parts][32][C][9] weight sums, then [32] bias sums.
template <int C, int HI>
__global__ void __launch_bounds__(kBackThreads) k_conv1_dw(const float* __restrict__ gin,
                                                           const uint16_t* __restrict__ stamps,
                                                           const uint32_t* __restrict__ idx, uint32_t n,
                                                           float* __restrict__ partial) {
  constexpr int HO = HI - 2, P = HO * HO, Q = HI * HI;
  constexpr int PARTS = kBackThreads / (8 * C);  // 3 for C = 9
  static_assert(PARTS >= 1, "too many channels");
  extern __shared__ __align__(16) float sm[];
  float* g_s = sm;             // [32][P]
  float* a_s = g_s + kCh * P;  // [C][Q]
  const int t = threadIdx.x;
  // weight-gradient ownership: (4 output channels, 1 input channel, 1 pixel part)
  const int c_own = t % C, oq = (t / C) % 8, part = t / (8 * C);
  const bool owner = part < PARTS;
  float acc[4][9];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) acc[j][tap] = 0.f;
  float accb = 0.f;
  for (uint32_t b = blockIdx.x; b < n; b += gridDim.x) {
    __syncthreads();
    for (int i = t; i < kCh * P; i += blockDim.x) g_s[i] = gin[(size_t)b * kCh * P + i];
    for (int i = t; i < C * Q; i += blockDim.x)
      a_s[i] = bf((float)stamps[(size_t)(idx ? idx[b] : b) * C * Q + i] * 0.0625f);
    __syncthreads();
    if (owner) {
      for (int p = part; p < P; p += PARTS) {
        const int y = p / HO, x = p - y * HO;
        float g[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) g[j] = g_s[(oq * 4 + j) * P + p];
        const float* ap = a_s + c_own * Q + y * HI + x;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const float a = ap[(tap / 3) * HI + tap % 3];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[j][tap] = fmaf(g[j], a, acc[j][tap]);
        }
      }
    }
    if (t < kCh) {
      for (int p = 0; p < P; ++p) accb += g_s[t * P + p];
    }
  }
  float* out = partial + (size_t)blockIdx.x * kPartialStride;
  if (owner) {
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int tap = 0; tap < 9; ++tap)
        out[(size_t)part * kCh * C * 9 + ((oq * 4 + j) * C + c_own) * 9 + tap] = acc[j][tap];
  }
  if (t < kCh) out[PARTS * kCh * C * 9 + t] = accb;
}

// ---- conv backward on the tensor cores (TF32) for the 32-channel layers ------
//
// Per block (a fixed set of stamps, so gradients stay bit-reproducible):
//   dW[k = (c, tap)][o] += sum_p im2col(a)[k][p] * g[o][p]: M = 288 rows of k
//     (three 128-row tiles, the last padded), N = 32, K = output pixels in
//     chunks of 32; accumulated in TMEM across the block's stamps.
//   dX[q][c] = sum_(o, tap) g[o][q - tap] * w[o][c][tap]: M = input pixels in
//     128-row tiles, N = 32, K = 288 in chunks of 32; masked by the ReLU of the
//     layer's input and written per stamp.
// Operands are FP32 read as TF32 (activations and weights are BF16 values, so
// exact; deltas round to TF32) in the no-swizzle K-major layout with 4-byte
// elements; one thread issues the MMAs, completion through an mbarrier with a
// bounded wait.  Bias gradients stay on the CUDA cores.
constexpr int kBtThreads = 256;
constexpr int kBtKCX = 9 * kCh / 4;                 // dX K (o, tap) = 288: 72 core matrices
constexpr int kBtSmWb = 0;                           // [32 c][288] dX B operand (resident)
constexpr int kBtSmA = kBtSmWb + kCh * 9 * kCh * 4;  // A chunk: 384 x 32 (dW) or up to 256 x 32 (dX)
constexpr int kBtSmB = kBtSmA + 384 * 32 * 4;        // dW B chunk: 32 x 32
constexpr int kBtSmG = kBtSmB + kCh * 32 * 4;        // g [32][P], then a [32][Q], then barrier

// Position i of a 4-byte-element operand with 32 K per row (8 core matrices
// per row group) in the no-swizzle K-major layout: its row and k, so that
// cm_offset4(cm_row(i), cm_k(i), 8) == 4 i.
__device__ __forceinline__ int cm_row(int i) { return (i >> 8) * 8 + ((i >> 2) & 7); }
__device__ __forceinline__ int cm_k(int i) { return ((i >> 5) & 7) * 4 + (i & 3); }

template <int HI>
constexpr size_t back_tc_smem() {
  return (size_t)kBtSmG + (size_t)kCh * (HI - 2) * (HI - 2) * 4 + (size_t)kCh * HI * HI * 4 + 16;
}

template <int HI>
__global__ void __launch_bounds__(kBtThreads, 1) k_conv_back_tc(
    const float* __restrict__ gin, const __nv_bfloat16* __restrict__ ain, uint32_t n,
    const __nv_bfloat16* __restrict__ w, float* __restrict__ gout, float* __restrict__ partial,
    uint32_t* __restrict__ status) {
  constexpr int C = kCh, HO = HI - 2, P = HO * HO, Q = HI * HI;
  constexpr int NCW = (P + 31) / 32, MQ = (Q + 127) / 128, KC = 8;
  static_assert(MQ * 128 <= 384, "dX tile fits the A buffer");
  extern __shared__ __align__(1024) unsigned char smb[];
  unsigned char* Wb = smb + kBtSmWb;
  unsigned char* Ab = smb + kBtSmA;
  unsigned char* Bb = smb + kBtSmB;
  float* g_s = reinterpret_cast<float*>(smb + kBtSmG);
  float* a_s = g_s + C * P;
  uint64_t* bar = reinterpret_cast<uint64_t*>(a_s + C * Q);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(tslot, 256);  // dW: columns [0, 96), dX: [128, 128 + 32 MQ)
  if (tid == 0) tc::mbar_init(bar, 1);
  for (int i = tid; i < C * 9 * C; i += kBtThreads) {  // Wb[c][(o, tap)] = w[o][c][tap]
    const int c = i / (9 * C), K = i - c * 9 * C, o = K / 9, tap = K - o * 9;
    *reinterpret_cast<float*>(Wb + tc::cm_offset4(c, K, kBtKCX)) = ld(w + (o * C + c) * 9 + tap);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t a0 = tc::smem_u32(Ab), b0 = tc::smem_u32(Bb), wb0 = tc::smem_u32(Wb);
  constexpr uint32_t idesc = tc::idesc_tf32(128, 32);
  uint32_t phase = 0;
  float accb = 0.f;
  bool any = false, ok = true;
  // one chunk of MMAs issued by thread 0, then everyone waits for them
  auto run = [&](auto issue) -> bool {
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      issue();
      tc::commit(bar);
    }
    const bool done = tc::mbar_wait(bar, phase, 1u << 22);
    phase ^= 1u;
    return !__syncthreads_or(!done);
  };
  for (uint32_t b = blockIdx.x; b < n && ok; b += gridDim.x) {
    for (int i = tid; i < C * P; i += kBtThreads) g_s[i] = gin[(size_t)b * C * P + i];
    for (int i = tid; i < C * Q; i += kBtThreads) a_s[i] = ld(ain + (size_t)b * C * Q + i);
    __syncthreads();
    if (tid < C)
      for (int p = 0; p < P; ++p) accb += g_s[tid * P + p];
    // dW: im2col(a)^T x g over chunks of 32 output pixels
    for (int ch = 0; ch < NCW && ok; ++ch) {
      const int p0 = ch * 32;
      // buffers are filled in memory order (a warp writes one 128-byte core
      // matrix): element i is (row, k) = cm_row(i), cm_k(i)
      for (int i = tid; i < 384 * 32; i += kBtThreads) {
        const int k = cm_row(i), kk = cm_k(i), p = p0 + kk;
        float v = 0.f;
        if (k < 9 * C && p < P) {
          const int c = k / 9, tap = k - c * 9, y = p / HO, x = p - y * HO;
          v = a_s[c * Q + (y + tap / 3) * HI + x + tap % 3];
        }
        reinterpret_cast<float*>(Ab)[i] = v;
      }
      for (int i = tid; i < C * 32; i += kBtThreads) {
        const int o = cm_row(i), p = p0 + cm_k(i);
        reinterpret_cast<float*>(Bb)[i] = p < P ? g_s[o * P + p] : 0.f;
      }
      const uint32_t acc0 = (any || ch > 0) ? 1u : 0u;
      ok = run([&] {
        for (int mt = 0; mt < 3; ++mt)
          for (int ks = 0; ks < 4; ++ks)
            tc::mma_tf32(tmem + (uint32_t)(mt * 32), tc::smem_desc(a0 + (uint32_t)(mt * 16 * KC * 128 + ks * 256), KC),
                         tc::smem_desc(b0 + (uint32_t)(ks * 256), KC), idesc, (acc0 | (uint32_t)ks) ? 1u : 0u);
      });
    }
    any = true;
    // dX: im2col(g) x w over chunks of 32 of (o, tap)
    for (int ch = 0; ch < 9 && ok; ++ch) {
      for (int i = tid; i < MQ * 128 * 32; i += kBtThreads) {
        const int q = cm_row(i), K = ch * 32 + cm_k(i), o = K / 9, tap = K - o * 9;
        float v = 0.f;
        if (q < Q) {
          const int yi = q / HI, xi = q - yi * HI, yo = yi - tap / 3, xo = xi - tap % 3;
          if (yo >= 0 && yo < HO && xo >= 0 && xo < HO) v = g_s[o * P + yo * HO + xo];
        }
        reinterpret_cast<float*>(Ab)[i] = v;
      }
      ok = run([&] {
        for (int mt = 0; mt < MQ; ++mt)
          for (int ks = 0; ks < 4; ++ks)
            tc::mma_tf32(tmem + (uint32_t)(128 + mt * 32),
                         tc::smem_desc(a0 + (uint32_t)(mt * 16 * KC * 128 + ks * 256), KC),
                         tc::smem_desc(wb0 + (uint32_t)(ch * 8 * 128 + ks * 256), kBtKCX), idesc,
                         (ch > 0 || ks > 0) ? 1u : 0u);
      });
    }
    if (!ok) break;
    tc::fence_after_sync();
    {  // dX epilogue: warp w reads lane quadrant w % 4, columns 16 (w / 4) .. + 15
      const int q4 = warp & 3, h = warp >> 2;
      float* go = gout + (size_t)b * C * Q;
      for (int mt = 0; mt < MQ; ++mt) {
        float v[16];
        tc::ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(128 + mt * 32 + h * 16), v);
        const int q = mt * 128 + q4 * 32 + lane;
        if (q < Q) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = h * 16 + j;
            go[c * Q + q] = a_s[c * Q + q] > 0.f ? v[j] : 0.f;
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // g_s, a_s and the dX columns are free for the next stamp
  }
  if (!ok && tid == 0) atomicOr(status, 1u);
  tc::fence_after_sync();
  float* out = partial + (size_t)blockIdx.x * kPartialStride;  // [32 o][C][9], then [32] biases
  if (ok) {
    const int q4 = warp & 3, h = warp >> 2;
    for (int mt = 0; mt < 3; ++mt) {
      float v[16];
      tc::ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(mt * 32 + h * 16), v);
      const int k = mt * 128 + q4 * 32 + lane;
      if (k < 9 * C) {
        const int c = k / 9, tap = k - c * 9;
#pragma unroll
        for (int j = 0; j < 16; ++j) out[((h * 16 + j) * C + c) * 9 + tap] = any ? v[j] : 0.f;
      }
    }
  }
  if (tid < C) out[C * C * 9 + tid] = accb;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 256);
}

// grad[w_off + i] = sum over blocks and parts of the partial weight sums;
// grad[b_off + o] likewise for the biases.  Fixed summation order.
// One warp per element: lane l adds blocks l, l + 32, ... in order, then the
// lanes combine in a fixed xor pattern.
__global__ void k_reduce_partials(const float* __restrict__ partial, int n_blocks, int parts, int nw,
                                  float* __restrict__ grad, int w_off, int b_off) {
  const int i = (int)((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (i >= nw + kCh) return;  // whole warps leave together
  float s = 0.f;
  for (int blk = lane; blk < n_blocks; blk += 32) {
    const float* p = partial + (size_t)blk * kPartialStride;
    if (i < nw) {
      for (int q = 0; q < parts; ++q) s += p[(size_t)q * nw + i];
    } else {
      s += p[(size_t)parts * nw + (i - nw)];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) grad[i < nw ? w_off + i : b_off + (i - nw)] = s;
}

// ---- parameters --------------------------------------------------------------

__global__ void k_cast(const float* __restrict__ master, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  wb[i] = __float2bfloat16_rn(master[i]);
}

// Adam (Kingma & Ba 2015) on the FP32 master values; refreshes the BF16 copies.
__global__ void k_adam(float* __restrict__ master, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, float lr, float beta1, float beta2, float eps,
                       float bc1, float bc2, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNParams) return;
  const float g = grad[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * g;
  const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float p = master[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  master[i] = p;
  wb[i] = __float2bfloat16_rn(p);
}

// ---- host side -----------------------------------------------------------------

template <int C, int HI>
constexpr size_t conv1_dw_smem() {
  return sizeof(float) * ((size_t)kCh * (HI - 2) * (HI - 2) + (size_t)C * HI * HI);
}

cudaError_t set_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_conv_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fc_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kFcTcSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_back_tc<kH2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)back_tc_smem<kH2>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_back_tc<kH1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)back_tc_smem<kH1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv1_dw<kQ, kS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)conv1_dw_smem<kQ, kS>());
  if (e == cudaSuccess) done = true;
  return e;
}

int fwd_blocks() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    n = sms > 0 ? sms : 152;
  }
  return n;
}

// Forward of n <= max_batch stamps; with keep, stores the activations training needs.
cudaError_t forward(sas_vet* vt, const uint16_t* stamps, const uint32_t* idx, uint32_t n, bool keep,
                    float* logits, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<uint32_t>(n, 2u * (uint32_t)fwd_blocks());  // two CTAs per SM
  k_conv_fwd_tc<<<blocks, kTcThreads, kTcSmem, s>>>(stamps, idx, n, vt->wb, keep ? vt->a1 : nullptr,
                                                   keep ? vt->a2 : nullptr, vt->a3, vt->status);
  const uint32_t tiles = (n + kFcTcRows - 1) / kFcTcRows, ldp = tiles * kFcTcRows;
  k_fc_fwd_tc<<<dim3(tiles, kFcSplit), kFcTcThreads, kFcTcSmem, s>>>(vt->a3, n, vt->wb, vt->fcpart, ldp,
                                                                     vt->status);
  k_fc_epi<<<(n + 255) / 256, 256, 0, s>>>(vt->fcpart, ldp, n, vt->wb, keep ? vt->a4 : nullptr, logits);
  note_launch();
  note_launch(2);
  return cudaGetLastError();
}

cudaError_t gradients(sas_vet* vt, const uint16_t* stamps, const float* labels, const uint32_t* idx,
                      uint32_t n, float* grad, cudaStream_t s) {
  cudaError_t e = forward(vt, stamps, idx, n, true, vt->logits, s);
  if (e != cudaSuccess) return e;
  k_loss<<<1, kLossThreads, 0, s>>>(vt->logits, labels, idx, n, vt->a4, vt->glogit, grad, vt->loss);
  k_g4<<<(unsigned)(((uint64_t)n * kHid + 255) / 256), 256, 0, s>>>(vt->glogit, vt->a4, vt->wb, n, vt->g4);
  {
    // stamp slices of about 512 (at most the partial buffer's room), summed in order
    const uint32_t S = std::max<uint32_t>(1, std::min<uint32_t>(kFc1Slices, n / 512));
    k_fc1_dw<<<dim3((kF + 31) / 32, S), 256, 0, s>>>(vt->g4, vt->a3, n, vt->partial);
    k_fc1_sum<<<(kHid * kF + kHid + 255) / 256, 256, 0, s>>>(vt->partial, S, grad);
    note_launch();
  }
  k_fc1_dx<<<dim3((kF + 63) / 64, (n + 31) / 32), 256, 0, s>>>(vt->g4, vt->wb, vt->a3, n, vt->g3);
  const int nb = (int)std::min<uint32_t>(n, kBackBlocks);
  k_conv_back_tc<kH2><<<nb, kBtThreads, back_tc_smem<kH2>(), s>>>(vt->g3, vt->a2, n, vt->wb + kW3, vt->g2,
                                                                   vt->partial, vt->status);
  k_reduce_partials<<<(kCh * kCh * 9 + kCh + 7) / 8, 256, 0, s>>>(vt->partial, nb, 1, kCh * kCh * 9,
                                                                      grad, kW3, kB3);
  k_conv_back_tc<kH1><<<nb, kBtThreads, back_tc_smem<kH1>(), s>>>(vt->g2, vt->a1, n, vt->wb + kW2, vt->g1,
                                                                   vt->partial, vt->status);
  k_reduce_partials<<<(kCh * kCh * 9 + kCh + 7) / 8, 256, 0, s>>>(vt->partial, nb, 1, kCh * kCh * 9,
                                                                      grad, kW2, kB2);
  k_conv1_dw<kQ, kS><<<nb, kBackThreads, conv1_dw_smem<kQ, kS>(), s>>>(vt->g1, stamps, idx, n, vt->partial);
  k_reduce_partials<<<(kCh * kQ * 9 + kCh + 7) / 8, 256, 0, s>>>(
      vt->partial, nb, kBackThreads / (8 * kQ), kCh * kQ * 9, grad, kW1, kB1);
  note_launch(10);
  return cudaGetLastError();
}

cudaError_t adam(sas_vet* vt, const float* grad, float lr, cudaStream_t s) {
  vt->step += 1;
  const double bc1 = 1.0 - std::pow((double)vt->beta1, (double)vt->step);
  const double bc2 = 1.0 - std::pow((double)vt->beta2, (double)vt->step);
  k_adam<<<(kNParams + 255) / 256, 256, 0, s>>>(vt->master, vt->m, vt->v, grad, lr, vt->beta1, vt->beta2,
                                               vt->eps, (float)bc1, (float)bc2, vt->wb);
  note_launch();
  return cudaGetLastError();
}

}  // namespace vet

cudaError_t vet_forward_all(sas_vet* vt, const uint16_t* stamps, uint64_t n, float* logits, cudaStream_t s) {
  for (uint64_t b0 = 0; b0 < n; b0 += vt->max_batch) {
    const uint32_t nb = (uint32_t)std::min<uint64_t>(vt->max_batch, n - b0);
    cudaError_t e = vet::forward(vt, stamps + b0 * 9 * 225, nullptr, nb, false, logits + b0, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int vet_device(const sas_vet* vt) { return vt->device; }

}  // namespace sas

// ---- C ABI -----------------------------------------------------------------------

using namespace sas;

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int cuda_fail(cudaError_t e, const char* what) {
  return set_errorf(SAS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void free_vet(sas_vet* vt) {
  void* ptrs[] = {vt->master, vt->m, vt->v, vt->grad, vt->wb, vt->a1, vt->a2, vt->a3,
                  vt->a4, vt->logits, vt->glogit, vt->g4, vt->g3, vt->g2, vt->g1, vt->partial, vt->loss,
                  vt->status, vt->fcpart};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete vt;
}

}  // namespace

extern "C" {

uint64_t sas_vet_num_params(void) { return (uint64_t)vet::kNParams; }

int sas_vet_create(int device, uint32_t max_batch, sas_vet** out) {
  if (!out) return set_error(SAS_ERR_ARG, "sas_vet_create: out is NULL");
  *out = nullptr;
  if (max_batch == 0 || max_batch > SAS_VET_MAX_BATCH)
    return set_errorf(SAS_ERR_ARG, "sas_vet_create: max_batch must be 1..%u", (unsigned)SAS_VET_MAX_BATCH);
  DeviceGuard guard(device);
  if (cudaError_t e = vet::set_attrs(); e != cudaSuccess) return cuda_fail(e, "sas_vet_create");
  sas_vet* vt = new sas_vet();
  std::memset(vt, 0, sizeof(*vt));
  vt->device = device;
  vt->max_batch = max_batch;
  vt->beta1 = 0.9f;
  vt->beta2 = 0.999f;
  vt->eps = 1e-8f;
  const size_t B = max_batch, N = vet::kNParams;
  struct Req {
    void** p;
    size_t bytes;
  } reqs[] = {
      {(void**)&vt->master, N * 4}, {(void**)&vt->m, N * 4}, {(void**)&vt->v, N * 4},
      {(void**)&vt->grad, N * 4}, {(void**)&vt->wb, N * 2},
      {(void**)&vt->a1, B * vet::kCh * vet::kH1 * vet::kH1 * 2}, {(void**)&vt->a2, B * vet::kCh * vet::kH2 * vet::kH2 * 2},
      {(void**)&vt->a3, B * vet::kF * 2}, {(void**)&vt->a4, B * vet::kHid * 2}, {(void**)&vt->logits, B * 4},
      {(void**)&vt->glogit, B * 4}, {(void**)&vt->g4, B * vet::kHid * 4}, {(void**)&vt->g3, B * vet::kF * 4},
      {(void**)&vt->g2, B * vet::kCh * vet::kH2 * vet::kH2 * 4}, {(void**)&vt->g1, B * vet::kCh * vet::kH1 * vet::kH1 * 4},
      {(void**)&vt->partial, (size_t)vet::kBackBlocks * vet::kPartialStride * 4}, {(void**)&vt->loss, 4},
      {(void**)&vt->status, 4},
      {(void**)&vt->fcpart, (size_t)vet::kFcSplit * vet::kHid * ((B + 127) / 128 * 128) * 4},
  };
  for (auto& r : reqs) {
    if (cudaError_t e = cudaMalloc(r.p, r.bytes); e != cudaSuccess) {
      free_vet(vt);
      return cuda_fail(e, "sas_vet_create: cudaMalloc");
    }
  }
  cudaMemset(vt->status, 0, 4);
  cudaMemset(vt->master, 0, N * 4);
  cudaMemset(vt->m, 0, N * 4);
  cudaMemset(vt->v, 0, N * 4);
  vet::k_cast<<<(vet::kNParams + 255) / 256, 256>>>(vt->master, vt->wb);
  note_launch();
  if (cudaError_t e = cudaDeviceSynchronize(); e != cudaSuccess) {
    free_vet(vt);
    return cuda_fail(e, "sas_vet_create");
  }
  *out = vt;
  return SAS_OK;
}

int sas_vet_destroy(sas_vet* vt) {
  if (!vt) return SAS_OK;
  DeviceGuard guard(vt->device);
  cudaDeviceSynchronize();
  free_vet(vt);
  return SAS_OK;
}

int sas_vet_check(sas_vet* vt) {
  if (!vt) return set_error(SAS_ERR_ARG, "sas_vet_check: NULL vetter");
  DeviceGuard guard(vt->device);
  uint32_t st = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, vt->status, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st) e = cudaMemset(vt->status, 0, 4);
  if (e != cudaSuccess) return cuda_fail(e, "sas_vet_check");
  if (st) return set_error(SAS_ERR_TIMEOUT, "sas_vet_check: a tensor-core wait gave up; logits are incomplete");
  return SAS_OK;
}

int sas_vet_set_adam(sas_vet* vt, float beta1, float beta2, float eps) {
  if (!vt) return set_error(SAS_ERR_ARG, "sas_vet_set_adam: NULL vetter");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f))
    return set_error(SAS_ERR_ARG, "sas_vet_set_adam: need 0 <= beta < 1 and eps > 0");
  vt->beta1 = beta1;
  vt->beta2 = beta2;
  vt->eps = eps;
  return SAS_OK;
}

int sas_vet_set_state(sas_vet* vt, const float* params, const float* m, const float* v, uint64_t step) {
  if (!vt || !params) return set_error(SAS_ERR_ARG, "sas_vet_set_state: NULL argument");
  if ((m == nullptr) != (v == nullptr))
    return set_error(SAS_ERR_ARG, "sas_vet_set_state: give both Adam moments or neither");
  DeviceGuard guard(vt->device);
  const size_t bytes = (size_t)vet::kNParams * 4;
  cudaError_t e = cudaMemcpy(vt->master, params, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = m ? cudaMemcpy(vt->m, m, bytes, cudaMemcpyHostToDevice) : cudaMemset(vt->m, 0, bytes);
  if (e == cudaSuccess) e = v ? cudaMemcpy(vt->v, v, bytes, cudaMemcpyHostToDevice) : cudaMemset(vt->v, 0, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "sas_vet_set_state");
  vt->step = m ? step : 0;
  vet::k_cast<<<(vet::kNParams + 255) / 256, 256>>>(vt->master, vt->wb);
  note_launch();
  e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SAS_OK : cuda_fail(e, "sas_vet_set_state");
}

int sas_vet_get_state(const sas_vet* vt, float* params, float* m, float* v, uint64_t* step) {
  if (!vt) return set_error(SAS_ERR_ARG, "sas_vet_get_state: NULL vetter");
  DeviceGuard guard(vt->device);
  const size_t bytes = (size_t)vet::kNParams * 4;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && params) e = cudaMemcpy(params, vt->master, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && m) e = cudaMemcpy(m, vt->m, bytes, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemcpy(v, vt->v, bytes, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "sas_vet_get_state");
  if (step) *step = vt->step;
  return SAS_OK;
}

int sas_vet_get_bf16(const sas_vet* vt, uint16_t* out) {
  if (!vt || !out) return set_error(SAS_ERR_ARG, "sas_vet_get_bf16: NULL argument");
  DeviceGuard guard(vt->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(out, vt->wb, (size_t)vet::kNParams * 2, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SAS_OK : cuda_fail(e, "sas_vet_get_bf16");
}

int sas_vet_get_activations(const sas_vet* vt, uint32_t layer, uint64_t n, uint16_t* out) {
  if (!vt || (n && !out)) return set_error(SAS_ERR_ARG, "sas_vet_get_activations: NULL argument");
  if (layer < 1 || layer > 4) return set_error(SAS_ERR_ARG, "sas_vet_get_activations: layer must be 1..4");
  if (n > vt->max_batch) return set_error(SAS_ERR_ARG, "sas_vet_get_activations: n exceeds the vetter's batch");
  const size_t per = layer == 1 ? (size_t)vet::kCh * vet::kH1 * vet::kH1
                   : layer == 2 ? (size_t)vet::kCh * vet::kH2 * vet::kH2
                   : layer == 3 ? (size_t)vet::kF : (size_t)vet::kHid;
  const __nv_bfloat16* src = layer == 1 ? vt->a1 : layer == 2 ? vt->a2 : layer == 3 ? vt->a3 : vt->a4;
  DeviceGuard guard(vt->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && n) e = cudaMemcpy(out, src, n * per * 2, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SAS_OK : cuda_fail(e, "sas_vet_get_activations");
}

int sas_vet_forward(sas_vet* vt, const uint16_t* stamps, const uint32_t* index, uint64_t n, float* logits,
                    void* stream) {
  if (!vt) return set_error(SAS_ERR_ARG, "sas_vet_forward: NULL vetter");
  if (n && (!stamps || !logits)) return set_error(SAS_ERR_ARG, "sas_vet_forward: NULL buffer");
  DeviceGuard guard(vt->device);
  cudaStream_t s = (cudaStream_t)stream;
  for (uint64_t b0 = 0; b0 < n; b0 += vt->max_batch) {
    const uint32_t nb = (uint32_t)std::min<uint64_t>(vt->max_batch, n - b0);
    const uint16_t* st = index ? stamps : stamps + b0 * 9 * 225;
    if (cudaError_t e = vet::forward(vt, st, index ? index + b0 : nullptr, nb, false, logits + b0, s);
        e != cudaSuccess)
      return cuda_fail(e, "sas_vet_forward");
  }
  return SAS_OK;
}

int sas_vet_gradients(sas_vet* vt, const uint16_t* stamps, const float* labels, const uint32_t* index,
                      uint32_t n, float* grad, float* loss, void* stream) {
  if (!vt) return set_error(SAS_ERR_ARG, "sas_vet_gradients: NULL vetter");
  if (n == 0 || n > vt->max_batch)
    return set_errorf(SAS_ERR_ARG, "sas_vet_gradients: n must be 1..%u", vt->max_batch);
  if (!stamps || !labels || !grad) return set_error(SAS_ERR_ARG, "sas_vet_gradients: NULL buffer");
  DeviceGuard guard(vt->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = vet::gradients(vt, stamps, labels, index, n, grad, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, vt->loss, 4, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? SAS_OK : cuda_fail(e, "sas_vet_gradients");
}

int sas_vet_apply_gradients(sas_vet* vt, const float* grad, float lr, void* stream) {
  if (!vt || !grad) return set_error(SAS_ERR_ARG, "sas_vet_apply_gradients: NULL argument");
  if (!(lr >= 0.f)) return set_error(SAS_ERR_ARG, "sas_vet_apply_gradients: lr must be >= 0");
  DeviceGuard guard(vt->device);
  cudaError_t e = vet::adam(vt, grad, lr, (cudaStream_t)stream);
  return e == cudaSuccess ? SAS_OK : cuda_fail(e, "sas_vet_apply_gradients");
}

int sas_vet_train_step(sas_vet* vt, const uint16_t* stamps, const float* labels, const uint32_t* index,
                       uint32_t n, float lr, float* loss, void* stream) {
  if (!vt) return set_error(SAS_ERR_ARG, "sas_vet_train_step: NULL vetter");
  if (n == 0 || n > vt->max_batch)
    return set_errorf(SAS_ERR_ARG, "sas_vet_train_step: n must be 1..%u", vt->max_batch);
  if (!stamps || !labels) return set_error(SAS_ERR_ARG, "sas_vet_train_step: NULL buffer");
  if (!(lr >= 0.f)) return set_error(SAS_ERR_ARG, "sas_vet_train_step: lr must be >= 0");
  DeviceGuard guard(vt->device);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = vet::gradients(vt, stamps, labels, index, n, vt->grad, s);
  if (e == cudaSuccess) e = vet::adam(vt, vt->grad, lr, s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, vt->loss, 4, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? SAS_OK : cuda_fail(e, "sas_vet_train_step");
}

}  // extern "C"
