// Refinement and gathering (Sec. 2.1 steps 4-6).
//
// Every cluster's detections are points z = (t, x, y): t the epoch's time minus
// t0 in ticks, x and y in mpx.  Step 4 fits a linear trajectory by regressing
// (x, y) on t with the mean and covariance of the Minimum Covariance
// Determinant subset, found by FAST-MCD (Rousseeuw & Van Driessen 1999: random
// (d+1)-subsets, C-steps, the best starts iterated to convergence).  Step 5
// gathers every detection of the catalog within the radius of the fitted line
// at its epoch; step 6 repeats the two until the gathered set is the fitted one.
//
// Arithmetic.  Moment sums of a subset are exact (int64 first moments, int128
// second moments), so the warp reductions that form them may run in any order.
// The exact scatter matrix S = m sum(z z^T) - sum(z) sum(z)^T is rounded to
// double once (correctly rounded), and every later quantity -- adjugate,
// determinant, ranks q = u^T adj(S) u with u = m z - sum(z), the line, the
// gather distance -- is a fixed expression of IEEE double operations written
// with explicit round-to-nearest intrinsics (never fused), so each decision
// (which points a C-step keeps, which start wins, which detections are
// gathered) does not depend on the order of a parallel reduction.
//
// Random draws: counter-based SplitMix64 (Steele, Lea & Flood 2014).  Start s
// of cluster k in iteration it takes key = mix(mix(mix(seed + (k+1)g) + (it+1)g)
// + (s+1)g) and draw j = mix(key + (j+1)g); a start's subset is a partial
// Fisher-Yates shuffle whose step j swaps position j with j + draw_j mod (n-j).
//
// Layout: one block (8 warps) per cluster fits; each warp runs whole starts.
// A warp holds subset membership as one 32-bit word per lane (bit c = point
// 32c + lane), its points' rank keys and its shuffle in shared memory.
#include <algorithm>
#include <vector>

#include "sas_internal.cuh"

namespace sas {

namespace {

constexpr int kFitWarps = 8;
constexpr int kFitThreads = kFitWarps * 32;
constexpr uint32_t kRunning = 0xFFu;
constexpr int kDim = 3;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t start_key(uint64_t seed, uint32_t k, uint32_t it, uint32_t s) {
  const uint64_t a = mix64(seed + (uint64_t)(k + 1) * kGolden);
  const uint64_t b = mix64(a + (uint64_t)(it + 1) * kGolden);
  return mix64(b + (uint64_t)(s + 1) * kGolden);
}

__device__ __forceinline__ uint64_t draw_word(uint64_t key, uint32_t j) {
  return mix64(key + (uint64_t)(j + 1) * kGolden);
}

// Correctly rounded (to nearest even) int128 -> double: the top 64 bits with a
// sticky bit for the rest, converted by the hardware's rounding, then scaled
// by a power of two (exact).
__device__ __forceinline__ double i128_to_double(__int128 v) {
  if (v == 0) return 0.0;
  const bool neg = v < 0;
  const unsigned __int128 a = neg ? (unsigned __int128)(-(v + 1)) + 1u : (unsigned __int128)v;
  const uint64_t hi = (uint64_t)(a >> 64), lo = (uint64_t)a;
  double r;
  if (hi == 0) {
    r = __ull2double_rn(lo);
  } else {
    const int sh = 64 - __clzll((long long)hi);  // 1..63
    uint64_t m = (uint64_t)(a >> sh);
    m |= (lo & ((1ull << sh) - 1ull)) != 0 ? 1ull : 0ull;
    r = ldexp(__ull2double_rn(m), sh);
  }
  return neg ? -r : r;
}

__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dvd(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int o) {
  const uint64_t lo = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)v, o);
  const uint64_t hi = __shfl_xor_sync(0xffffffffu, (unsigned long long)(uint64_t)(v >> 64), o);
  return (__int128)(((unsigned __int128)hi << 64) | lo);
}

// A subset's exact sums and the fixed double expressions derived from them.
struct WFit {
  uint32_t m;
  int64_t T, X, Y;
  __int128 Stt;                       // exact S_tt (zero <=> one epoch)
  double s00, s01, s02, s11, s12, s22;
  double a00, a01, a02, a11, a12, a22;
  double det;
};

struct Pts {
  const int64_t* t;
  const int32_t* x;
  const int32_t* y;
  uint32_t n, nc;  // points, 32-point chunks
};

// Exact moments of the subset (bits: lane's membership word), then S, adj, det.
__device__ __noinline__ WFit wfit(const Pts& p, uint32_t bits, int lane) {
  int64_t T = 0, X = 0, Y = 0;
  __int128 tt = 0, tx = 0, ty = 0, xx = 0, xy = 0, yy = 0;
  for (uint32_t c = 0; c < p.nc; ++c) {
    if (!((bits >> c) & 1u)) continue;
    const uint32_t i = c * 32 + lane;
    const int64_t t = p.t[i], x = p.x[i], y = p.y[i];
    T += t;
    X += x;
    Y += y;
    tt += (__int128)t * t;
    tx += (__int128)t * x;
    ty += (__int128)t * y;
    xx += (__int128)x * x;
    xy += (__int128)x * y;
    yy += (__int128)y * y;
  }
  uint32_t m = __popc(bits);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T += __shfl_xor_sync(0xffffffffu, (long long)T, o);
    X += __shfl_xor_sync(0xffffffffu, (long long)X, o);
    Y += __shfl_xor_sync(0xffffffffu, (long long)Y, o);
    tt += shfl_xor_i128(tt, o);
    tx += shfl_xor_i128(tx, o);
    ty += shfl_xor_i128(ty, o);
    xx += shfl_xor_i128(xx, o);
    xy += shfl_xor_i128(xy, o);
    yy += shfl_xor_i128(yy, o);
    m += __shfl_xor_sync(0xffffffffu, m, o);
  }
  WFit f;
  f.m = m;
  f.T = T;
  f.X = X;
  f.Y = Y;
  const __int128 M = m;
  f.Stt = M * tt - (__int128)T * T;
  f.s00 = i128_to_double(f.Stt);
  f.s01 = i128_to_double(M * tx - (__int128)T * X);
  f.s02 = i128_to_double(M * ty - (__int128)T * Y);
  f.s11 = i128_to_double(M * xx - (__int128)X * X);
  f.s12 = i128_to_double(M * xy - (__int128)X * Y);
  f.s22 = i128_to_double(M * yy - (__int128)Y * Y);
  f.a00 = sub(mul(f.s11, f.s22), mul(f.s12, f.s12));
  f.a01 = sub(mul(f.s02, f.s12), mul(f.s01, f.s22));
  f.a02 = sub(mul(f.s01, f.s12), mul(f.s02, f.s11));
  f.a11 = sub(mul(f.s00, f.s22), mul(f.s02, f.s02));
  f.a12 = sub(mul(f.s01, f.s02), mul(f.s00, f.s12));
  f.a22 = sub(mul(f.s00, f.s11), mul(f.s01, f.s01));
  f.det = add(add(mul(f.s00, f.a00), mul(f.s01, f.a01)), mul(f.s02, f.a02));
  return f;
}

__device__ __forceinline__ uint64_t order_key(double q) {
  const uint64_t b = (uint64_t)__double_as_longlong(q);
  return (b >> 63) ? ~b : (b | (1ull << 63));
}

// Membership bits of the h smallest (key, index) among n <= 32 NC points:
// each lane counts its NC points' ranks against every key (no dependent
// reductions).
template <int NC>
__device__ __forceinline__ uint32_t rank_select(const uint64_t* keys, uint32_t n, uint32_t h, int lane) {
  uint64_t mine[NC];
  uint32_t rank[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const uint32_t i = c * 32 + lane;
    mine[c] = i < n ? keys[i] : ~0ull;
    rank[c] = 0;
  }
  for (uint32_t j = 0; j < n; ++j) {
    const uint64_t kj = keys[j];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const uint32_t i = c * 32 + lane;
      rank[c] += (kj < mine[c] || (kj == mine[c] && j < i)) ? 1u : 0u;
    }
  }
  uint32_t bits = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const uint32_t i = c * 32 + lane;
    if (i < n && rank[c] < h) bits |= 1u << c;
  }
  return bits;
}

// C-step: the h points of smallest (q, index) under the fit's (mean, adj).
// Up to 256 points: each point's rank is counted against every key (no
// dependent reductions), for the cluster's number of 32-point chunks; more:
// the h-th smallest key by binary descent.
__device__ __noinline__ uint32_t wselect(const Pts& p, const WFit& f, uint32_t h, uint64_t* keys, int lane) {
  const int64_t m = f.m;
  for (uint32_t c = 0; c < p.nc; ++c) {
    const uint32_t i = c * 32 + lane;
    if (i >= p.n) break;
    const double u0 = (double)(m * p.t[i] - f.T);  // |u| < 2^53: exact
    const double u1 = (double)(m * (int64_t)p.x[i] - f.X);
    const double u2 = (double)(m * (int64_t)p.y[i] - f.Y);
    const double w0 = add(add(mul(f.a00, u0), mul(f.a01, u1)), mul(f.a02, u2));
    const double w1 = add(add(mul(f.a01, u0), mul(f.a11, u1)), mul(f.a12, u2));
    const double w2 = add(add(mul(f.a02, u0), mul(f.a12, u1)), mul(f.a22, u2));
    keys[i] = order_key(add(add(mul(u0, w0), mul(u1, w1)), mul(u2, w2)));
  }
  __syncwarp();
  uint32_t bits = 0;
  if (p.n <= 256) {
    switch (p.nc) {
      case 1: bits = rank_select<1>(keys, p.n, h, lane); break;
      case 2: bits = rank_select<2>(keys, p.n, h, lane); break;
      case 3: bits = rank_select<3>(keys, p.n, h, lane); break;
      case 4: bits = rank_select<4>(keys, p.n, h, lane); break;
      default: bits = rank_select<8>(keys, p.n, h, lane); break;
    }
    __syncwarp();
    return bits;
  }
  uint64_t K = 0;
  for (int b = 63; b >= 0; --b) {
    const uint64_t test = K | (1ull << b);
    uint32_t cnt = 0;
    for (uint32_t c = 0; c < p.nc; ++c) {
      const uint32_t i = c * 32 + lane;
      if (i < p.n) cnt += keys[i] < test;
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (cnt < h) K = test;
  }
  uint32_t below = 0;
  for (uint32_t c = 0; c < p.nc; ++c) {
    const uint32_t i = c * 32 + lane;
    if (i < p.n) below += keys[i] < K;
  }
  int32_t need = (int32_t)h - (int32_t)__reduce_add_sync(0xffffffffu, below);
  for (uint32_t c = 0; c < p.nc; ++c) {
    const uint32_t i = c * 32 + lane;
    const uint64_t k = i < p.n ? keys[i] : ~0ull;
    const bool eq = i < p.n && k == K;
    const uint32_t ball = __ballot_sync(0xffffffffu, eq);
    const int32_t rank = __popc(ball & ((1u << lane) - 1u));
    if ((i < p.n && k < K) || (eq && rank < need)) bits |= 1u << c;
    need = max(0, need - __popc(ball));
  }
  __syncwarp();
  return bits;
}

struct StartOut {
  double det;
  uint32_t bits;
};

// One FAST-MCD start: draws while singular (up to h points), the h nearest,
// then C-steps while det decreases (at most max_steps).
__device__ __noinline__ StartOut run_start(const Pts& p, uint32_t h, uint64_t key, uint32_t max_steps,
                                           uint64_t* keys, uint16_t* perm, int lane) {
  for (uint32_t i = lane; i < p.n; i += 32) perm[i] = (uint16_t)i;
  __syncwarp();
  uint32_t bits = 0, j = 0;
  auto draw = [&]() {
    uint32_t e = 0;
    if (lane == 0) {
      const uint32_t r = j + (uint32_t)(draw_word(key, j) % (uint64_t)(p.n - j));
      const uint16_t a = perm[j], b = perm[r];
      perm[j] = b;
      perm[r] = a;
      e = b;
    }
    e = __shfl_sync(0xffffffffu, e, 0);
    if ((int)(e & 31) == lane) bits |= 1u << (e >> 5);
    ++j;
    __syncwarp();
  };
  for (int q = 0; q < kDim + 1; ++q) draw();
  WFit f = wfit(p, bits, lane);
  while (f.det <= 0.0 && j < h) {
    draw();
    f = wfit(p, bits, lane);
  }
  if (f.det <= 0.0) return StartOut{f.det, bits};
  bits = wselect(p, f, h, keys, lane);
  f = wfit(p, bits, lane);
  for (uint32_t step = 0; step < max_steps; ++step) {
    if (f.det <= 0.0) break;
    const uint32_t b2 = wselect(p, f, h, keys, lane);
    if (__all_sync(0xffffffffu, b2 == bits)) break;  // same subset: same det, no decrease
    const WFit f2 = wfit(p, b2, lane);
    if (!(f2.det < f.det)) break;
    bits = b2;
    f = f2;
  }
  return StartOut{f.det, bits};
}

__device__ __forceinline__ bool det_before(double da, uint32_t sa, double db, uint32_t sb) {
  return da < db || (da == db && sa < sb);
}

struct BestOut {
  double det;
  uint32_t s;
  uint32_t bits[32];
  uint32_t pad;
};

struct FitArgs {
  const Det* pt;        // [n_det] by detection id (x, y, e)
  const int64_t* dt;    // [E] epoch time - t0, ticks
  const uint32_t* P;    // [k][cap] current point ids
  const uint32_t* Pn;
  uint32_t cap, iter;
  uint64_t seed;
  uint32_t n_starts, n_best, max_csteps, npad;
  double* det3;         // [k][n_starts] det after the first two C-steps
  BestOut* best;        // [k][n_best]
  sas_track* tracks;
  uint32_t* status;
};

// Shared layout of the fit kernels: points, then per-warp keys and shuffles.
struct FitSmem {
  int64_t* t;
  int32_t* x;
  int32_t* y;
  uint64_t* keys;
  uint16_t* perm;
  uint32_t* best;  // n_best selected starts
};

__device__ FitSmem carve(unsigned char* smem, uint32_t npad, uint32_t n_best) {
  FitSmem m;
  m.t = (int64_t*)smem;
  m.keys = (uint64_t*)(m.t + npad);
  m.x = (int32_t*)(m.keys + (size_t)kFitWarps * npad);
  m.y = m.x + npad;
  m.best = (uint32_t*)(m.y + npad);
  m.perm = (uint16_t*)(m.best + n_best);
  return m;
}

__device__ uint32_t load_points(const FitArgs& a, uint32_t k, const FitSmem& m, int tid, int nthreads) {
  const uint32_t n = a.Pn[k];
  for (uint32_t i = tid; i < n; i += nthreads) {
    const Det d = a.pt[a.P[(size_t)k * a.cap + i]];
    m.t[i] = a.dt[d.e];
    m.x[i] = d.x;
    m.y[i] = d.y;
  }
  return n;
}

// Phase 1: every start takes two C-steps; blockIdx.x splits a cluster's starts.
__global__ void __launch_bounds__(kFitThreads) k_fit_starts(FitArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t k = blockIdx.y;
  if (a.status[k] != kRunning) return;
  if (a.Pn[k] < (uint32_t)kDim + 2) return;
  const FitSmem m = carve(smem, a.npad, a.n_best);
  const uint32_t n = load_points(a, k, m, threadIdx.x, kFitThreads);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Pts p{m.t, m.x, m.y, n, (n + 31) / 32};
  const uint32_t h = (n + kDim + 1) / 2;
  const uint32_t stride = gridDim.x * kFitWarps;
  for (uint32_t s = blockIdx.x * kFitWarps + warp; s < a.n_starts; s += stride) {
    const StartOut o = run_start(p, h, start_key(a.seed, k, a.iter, s), 2, m.keys + (size_t)warp * a.npad,
                                 m.perm + (size_t)warp * a.npad, lane);
    if (lane == 0) a.det3[(size_t)k * a.n_starts + s] = o.det;
  }
}

// Phase 2: the n_best lowest (det, start) continue for up to max_csteps.
__global__ void __launch_bounds__(kFitThreads) k_fit_best(FitArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t k = blockIdx.y;
  if (a.status[k] != kRunning) return;
  if (a.Pn[k] < (uint32_t)kDim + 2) return;
  const FitSmem m = carve(smem, a.npad, a.n_best);
  const uint32_t n = load_points(a, k, m, threadIdx.x, kFitThreads);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double* det3 = a.det3 + (size_t)k * a.n_starts;
  if (warp == 0) {  // the n_best lowest (det, start), in order
    for (uint32_t b = 0; b < a.n_best; ++b) {
      double bd = 0.0;
      uint32_t bs = 0xFFFFFFFFu;
      for (uint32_t s = lane; s < a.n_starts; s += 32) {
        const double d = det3[s];
        bool taken = false;
        for (uint32_t q = 0; q < b; ++q) taken |= m.best[q] == s;
        if (!taken && (bs == 0xFFFFFFFFu || det_before(d, s, bd, bs))) {
          bd = d;
          bs = s;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const uint32_t os = __shfl_xor_sync(0xffffffffu, bs, o);
        if (os != 0xFFFFFFFFu && (bs == 0xFFFFFFFFu || det_before(od, os, bd, bs))) {
          bd = od;
          bs = os;
        }
      }
      if (lane == 0) m.best[b] = bs;
      __syncwarp();
    }
  }
  __syncthreads();
  const Pts p{m.t, m.x, m.y, n, (n + 31) / 32};
  const uint32_t h = (n + kDim + 1) / 2;
  const uint32_t b = blockIdx.x * kFitWarps + warp;
  if (b >= a.n_best) return;
  const uint32_t s = m.best[b];
  const StartOut o = run_start(p, h, start_key(a.seed, k, a.iter, s), a.max_csteps, m.keys + (size_t)warp * a.npad,
                               m.perm + (size_t)warp * a.npad, lane);
  BestOut& r = a.best[(size_t)k * a.n_best + b];
  r.bits[lane] = o.bits;
  if (lane == 0) {
    r.det = o.det;
    r.s = s;
  }
}

// Phase 3 (one warp per cluster): the winning subset and its line.
__global__ void __launch_bounds__(32) k_fit_final(FitArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t k = blockIdx.x;
  if (a.status[k] != kRunning) return;
  const FitSmem m = carve(smem, a.npad, 0);
  const uint32_t n = load_points(a, k, m, threadIdx.x, 32);
  __syncwarp();
  const int lane = threadIdx.x;
  const Pts p{m.t, m.x, m.y, n, (n + 31) / 32};
  uint32_t bits;
  if (n < (uint32_t)kDim + 2) {
    bits = lane < (int)n ? 1u : 0u;  // n < 32: every point, one chunk
  } else {
    const BestOut* bo = a.best + (size_t)k * a.n_best;
    uint32_t w = 0;
    for (uint32_t b = 1; b < a.n_best; ++b)
      if (det_before(bo[b].det, bo[b].s, bo[w].det, bo[w].s)) w = b;
    bits = bo[w].bits[lane];
  }
  const WFit f = wfit(p, bits, lane);
  if (lane != 0) return;
  sas_track& tr = a.tracks[k];
  tr.iterations = a.iter + 1;
  tr.det = f.det;
  tr.h = f.m;
  tr.n_points = n;
  if (f.Stt == 0) {
    a.status[k] = SAS_TRACK_DEGENERATE;
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    tr.vx = tr.vy = tr.x0 = tr.y0 = tr.res_xx = tr.res_xy = tr.res_yy = nan;
    return;
  }
  const double vxt = dvd(f.s01, f.s00), vyt = dvd(f.s02, f.s00);
  const double md = (double)f.m, mm = mul(md, md);
  tr.x0 = dvd(sub((double)f.X, mul(vxt, (double)f.T)), md);
  tr.y0 = dvd(sub((double)f.Y, mul(vyt, (double)f.T)), md);
  tr.vx = vxt;  // per tick until the output pass converts
  tr.vy = vyt;
  tr.res_xx = dvd(sub(f.s11, mul(vxt, f.s01)), mm);
  tr.res_xy = dvd(sub(f.s12, mul(vxt, f.s02)), mm);
  tr.res_yy = dvd(sub(f.s22, mul(vyt, f.s02)), mm);
}

// Step 5: per (cluster, epoch) warp, the buckets around the line's position
// at that epoch; blockIdx.x covers 4 epochs, epoch E is the overflow bucket.
__global__ void k_gather(const sas_track* __restrict__ tracks, const uint32_t* __restrict__ status,
                         const Det* __restrict__ dets, const uint32_t* __restrict__ boff,
                         const int64_t* __restrict__ dt, SearchGeom g, CoarseGeom cg, int32_t radius,
                         uint32_t cap, uint32_t* __restrict__ G, uint32_t* __restrict__ Gn) {
  const uint32_t k = blockIdx.y;
  if (status[k] != kRunning) return;
  const uint32_t e = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e > g.E) return;
  const sas_track tr = tracks[k];
  const double r2 = mul((double)radius, (double)radius);
  const uint64_t nb = (uint64_t)g.E * cg.ncy * cg.ncx;
  auto test = [&](const Det& d) {
    const double t = (double)dt[d.e];
    const double px = add(tr.x0, mul(tr.vx, t)), py = add(tr.y0, mul(tr.vy, t));
    const double rx = sub((double)d.x, px), ry = sub((double)d.y, py);
    if (add(mul(rx, rx), mul(ry, ry)) <= r2) {
      const uint32_t slot = atomicAdd(&Gn[k], 1u);
      if (slot < cap) G[(size_t)k * cap + slot] = d.id;
    }
  };
  if (e == g.E) {
    for (uint32_t i = boff[nb] + lane; i < boff[nb + 1]; i += 32) test(dets[i]);
    return;
  }
  const double t = (double)dt[e];
  const double px = add(tr.x0, mul(tr.vx, t)), py = add(tr.y0, mul(tr.vy, t));
  // cells that can hold a point within the radius (one extra mpx of margin)
  double cx0 = floor((px - radius - 1.0 - cg.gx0) / cg.cell), cx1 = floor((px + radius + 1.0 - cg.gx0) / cg.cell);
  double cy0 = floor((py - radius - 1.0 - cg.gy0) / cg.cell), cy1 = floor((py + radius + 1.0 - cg.gy0) / cg.cell);
  if (!(cx1 >= 0.0 && cy1 >= 0.0 && cx0 < (double)cg.ncx && cy0 < (double)cg.ncy)) return;
  const int ax = (int)fmax(cx0, 0.0), bx = (int)fmin(cx1, (double)(cg.ncx - 1));
  const int ay = (int)fmax(cy0, 0.0), by = (int)fmin(cy1, (double)(cg.ncy - 1));
  for (int cy = ay; cy <= by; ++cy) {
    const uint64_t b0 = ((uint64_t)e * cg.ncy + cy) * cg.ncx;
    const uint32_t k1 = boff[b0 + bx + 1];
    for (uint32_t i = boff[b0 + ax] + lane; i < k1; i += 32) test(dets[i]);
  }
}

// Step 6: sort the gathered ids, compare with the fitted set, decide.
__global__ void __launch_bounds__(512) k_settle(uint32_t* __restrict__ status, sas_track* __restrict__ tracks,
                                                uint32_t* __restrict__ P, uint32_t* __restrict__ Pn,
                                                const uint32_t* __restrict__ G, uint32_t* __restrict__ Gn,
                                                uint32_t cap, uint32_t iter, uint32_t max_iter) {
  __shared__ uint32_t s_g[1024];
  __shared__ int s_same;
  const uint32_t k = blockIdx.x;
  if (status[k] != kRunning) return;
  const uint32_t gn = Gn[k], pn = Pn[k];
  __syncthreads();
  if (threadIdx.x == 0) Gn[k] = 0;
  if (gn > cap) {
    if (threadIdx.x == 0) status[k] = SAS_TRACK_TOO_MANY;
    return;
  }
  uint32_t n2 = 1;
  while (n2 < gn) n2 <<= 1;
  for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) s_g[i] = i < gn ? G[(size_t)k * cap + i] : 0xFFFFFFFFu;
  if (threadIdx.x == 0) s_same = gn == pn;
  __syncthreads();
  for (uint32_t len = 2; len <= n2; len <<= 1) {
    for (uint32_t j = len >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const bool asc = (i & len) == 0;
          const uint32_t a = s_g[i], b = s_g[l];
          if ((a > b) == asc) {
            s_g[i] = b;
            s_g[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  if (gn == pn)
    for (uint32_t i = threadIdx.x; i < gn; i += blockDim.x)
      if (s_g[i] != P[(size_t)k * cap + i]) s_same = 0;
  __syncthreads();
  if (s_same) {
    if (threadIdx.x == 0) status[k] = SAS_TRACK_CONVERGED;
    return;
  }
  for (uint32_t i = threadIdx.x; i < gn; i += blockDim.x) P[(size_t)k * cap + i] = s_g[i];
  if (threadIdx.x == 0) {
    Pn[k] = gn;
    if (gn < 2)
      status[k] = SAS_TRACK_DEGENERATE;
    else if (iter + 1 >= max_iter)
      status[k] = SAS_TRACK_MAX_ITER;
  }
}

__global__ void k_pt_of(const Det* __restrict__ dets, const uint32_t* __restrict__ n_ptr, Det* __restrict__ pt) {
  const uint32_t n = *n_ptr;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) pt[dets[i].id] = dets[i];
}

// The clusters' ids become the first point sets; too large ones stop here.
__global__ void k_refine_init(const sas_candidate* __restrict__ c, uint32_t n, const uint32_t* __restrict__ ids,
                              uint32_t cap, uint32_t* __restrict__ P, uint32_t* __restrict__ Pn,
                              uint32_t* __restrict__ status, sas_track* __restrict__ tracks,
                              uint32_t* __restrict__ max_n) {
  const uint32_t k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const sas_candidate ck = c[k];
  if (lane == 0) {
    sas_track tr{};
    const double nan = __longlong_as_double(0x7FF8000000000000ll);
    tr.vx = tr.vy = tr.x0 = tr.y0 = tr.res_xx = tr.res_xy = tr.res_yy = nan;
    tr.det = 0.0;
    tr.n_points = ck.id_len;
    tr.cluster = k;
    tracks[k] = tr;
    status[k] = ck.id_len > cap ? (uint32_t)SAS_TRACK_TOO_MANY : kRunning;
    Pn[k] = ck.id_len > cap ? 0u : ck.id_len;
    if (ck.id_len <= cap) atomicMax(max_n, ck.id_len);
  }
  if (ck.id_len <= cap)
    for (uint32_t i = lane; i < ck.id_len; i += 32) P[(size_t)k * cap + i] = ids[ck.id_off + i];
}

__global__ void k_refine_count(const uint32_t* __restrict__ status, const uint32_t* __restrict__ Pn, uint32_t n,
                               uint32_t* __restrict__ ctl) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || status[k] != kRunning) return;
  atomicAdd(&ctl[0], 1u);
  atomicMax(&ctl[1], Pn[k]);
}

__global__ void k_track_len(const uint32_t* __restrict__ status, const uint32_t* __restrict__ Pn,
                            const sas_track* __restrict__ tracks, uint32_t n, uint32_t* __restrict__ len) {
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  len[k] = (status[k] == SAS_TRACK_TOO_MANY && tracks[k].iterations == 0) ? tracks[k].n_points : Pn[k];
}

__global__ void k_track_write(const sas_candidate* __restrict__ c, const uint32_t* __restrict__ ids,
                              const uint32_t* __restrict__ status, const uint32_t* __restrict__ P,
                              const uint32_t* __restrict__ len, const uint32_t* __restrict__ off, uint32_t cap,
                              uint32_t n, double tph, sas_track* __restrict__ tracks, uint32_t* __restrict__ out_ids) {
  const uint32_t k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= n) return;
  const uint32_t l = len[k], o = off[k];
  const bool orig = status[k] == SAS_TRACK_TOO_MANY && tracks[k].iterations == 0;
  for (uint32_t i = lane; i < l; i += 32) out_ids[o + i] = orig ? ids[c[k].id_off + i] : P[(size_t)k * cap + i];
  if (lane == 0) {
    sas_track& tr = tracks[k];
    tr.status = status[k];
    tr.id_off = o;
    tr.id_len = l;
    tr.vx = mul(tr.vx, tph);  // mpx per tick -> per hour
    tr.vy = mul(tr.vy, tph);
  }
}

unsigned nblocks(uint64_t n, unsigned per) { return (unsigned)std::max<uint64_t>(1, (n + per - 1) / per); }

}  // namespace

size_t refine_fit_smem(uint32_t npad, uint32_t n_best) {
  return (size_t)npad * 8 + (size_t)kFitWarps * npad * 8 + (size_t)npad * 8 + (size_t)n_best * 4 +
         (size_t)kFitWarps * npad * 2;
}

int refine_tracks(const RefineIn& in, const sas_refine_opts& o, cudaStream_t s, RefineOut* out) {
  *out = RefineOut{};
  const uint32_t nc = (uint32_t)in.clusters.n;
  if (nc == 0) return SAS_OK;
  const uint32_t cap = SAS_REFINE_MAX_POINTS;
  const uint64_t nd = in.search.n_det;
  const uint64_t nb = (uint64_t)in.search.g.E * in.search.cg.ncy * in.search.cg.ncx;
  std::vector<void*> ptrs;
  auto get = [&](auto** p, uint64_t bytes) {
    cudaError_t e = cudaMallocAsync((void**)p, std::max<uint64_t>(bytes, 16), s);
    if (e == cudaSuccess) ptrs.push_back((void*)*p);
    return e;
  };
  Det* pt = nullptr;
  uint32_t *P = nullptr, *Pn = nullptr, *G = nullptr, *Gn = nullptr, *status = nullptr, *ctl = nullptr,
           *len = nullptr, *off = nullptr, *scr = nullptr;
  sas_track* tracks = nullptr;
  uint32_t* out_ids = nullptr;
  double* det3 = nullptr;
  BestOut* best = nullptr;
  cudaError_t e = get(&pt, nd * sizeof(Det));
  if (e == cudaSuccess) e = get(&det3, (uint64_t)nc * o.n_starts * 8);
  if (e == cudaSuccess) e = get(&best, (uint64_t)nc * o.n_best * sizeof(BestOut));
  if (e == cudaSuccess) e = get(&P, (uint64_t)nc * cap * 4);
  if (e == cudaSuccess) e = get(&G, (uint64_t)nc * cap * 4);
  if (e == cudaSuccess) e = get(&Pn, nc * 4ull);
  if (e == cudaSuccess) e = get(&Gn, nc * 4ull);
  if (e == cudaSuccess) e = get(&status, nc * 4ull);
  if (e == cudaSuccess) e = get(&ctl, 16);
  if (e == cudaSuccess) e = get(&len, (nc + 1) * 4ull);
  if (e == cudaSuccess) e = get(&off, (nc + 1) * 4ull);
  if (e == cudaSuccess) e = get(&scr, scan_scratch_elems(nc + 1) * 4);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&tracks, nc * sizeof(sas_track), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(Gn, 0, nc * 4ull, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, 16, s);
  if (e == cudaSuccess) {
    k_pt_of<<<152 * 8, 256, 0, s>>>(in.search.dets, in.search.boff + nb + 1, pt);
    k_refine_init<<<nblocks(nc, 8), 256, 0, s>>>(in.clusters.cands, nc, in.clusters.ids, cap, P, Pn, status, tracks,
                                                 &ctl[1]);
    note_launch(2);
    e = cudaGetLastError();
  }
  uint32_t h_ctl[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_ctl, ctl, 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  uint32_t running = nc, max_n = h_ctl[1];
  for (uint32_t it = 0; e == cudaSuccess && it < o.max_iter && running > 0; ++it) {
    FitArgs fa;
    fa.pt = pt;
    fa.dt = in.search.dt;
    fa.P = P;
    fa.Pn = Pn;
    fa.cap = cap;
    fa.iter = it;
    fa.seed = o.seed;
    fa.n_starts = o.n_starts;
    fa.n_best = o.n_best;
    fa.max_csteps = o.max_csteps;
    fa.npad = std::max<uint32_t>(32, (max_n + 31) / 32 * 32);
    fa.det3 = det3;
    fa.best = best;
    fa.tracks = tracks;
    fa.status = status;
    const size_t smem = refine_fit_smem(fa.npad, o.n_best);
    // split each cluster's starts over enough blocks to fill the GPU twice
    const uint32_t split = std::max<uint32_t>(
        1, std::min<uint32_t>((o.n_starts + kFitWarps - 1) / kFitWarps, (4 * 152 + running - 1) / running));
    e = cudaFuncSetAttribute(k_fit_starts, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fit_best, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fit_final, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) break;
    k_fit_starts<<<dim3(split, nc), kFitThreads, smem, s>>>(fa);
    k_fit_best<<<dim3((o.n_best + kFitWarps - 1) / kFitWarps, nc), kFitThreads, smem, s>>>(fa);
    k_fit_final<<<nc, 32, smem, s>>>(fa);
    note_launch(3);
    k_gather<<<dim3((in.search.g.E + 1 + 3) / 4, nc), 128, 0, s>>>(tracks, status, in.search.dets, in.search.boff,
                                                                   in.search.dt, in.search.g, in.search.cg, o.radius,
                                                                   cap, G, Gn);
    k_settle<<<nc, 512, 0, s>>>(status, tracks, P, Pn, G, Gn, cap, it, o.max_iter);
    note_launch(2);
    if ((e = cudaMemsetAsync(ctl, 0, 8, s)) != cudaSuccess) break;
    k_refine_count<<<nblocks(nc, 256), 256, 0, s>>>(status, Pn, nc, ctl);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(h_ctl, ctl, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    running = h_ctl[0];
    max_n = h_ctl[1];
  }
  uint32_t n_ids = 0;
  if (e == cudaSuccess) {
    k_track_len<<<nblocks(nc, 256), 256, 0, s>>>(status, Pn, tracks, nc, len);
    note_launch();
    e = launch_scan_u32(len, off, nc, scr, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n_ids, off + nc, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&out_ids, std::max<size_t>(n_ids, 1) * 4, s);
  if (e == cudaSuccess) {
    k_track_write<<<nblocks(nc, 8), 256, 0, s>>>(in.clusters.cands, in.clusters.ids, status, P, len, off, cap, nc,
                                                 (double)in.search.g.tph, tracks, out_ids);
    note_launch();
    e = cudaGetLastError();
  }
  for (void* p : ptrs) cudaFreeAsync(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (tracks) cudaFree(tracks);
    if (out_ids) cudaFree(out_ids);
    return set_errorf(e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA, "refine: %s",
                      cudaGetErrorString(e));
  }
  out->tracks = tracks;
  out->ids = out_ids;
  out->n = nc;
  out->n_ids = n_ids;
  return SAS_OK;
}

}  // namespace sas
