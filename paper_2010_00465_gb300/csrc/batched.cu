// batched.cu -- cos/sin of many FP32 matrices of uneven order and norm, each
// with its own (2m, s), in one persistent launch with the products on the
// tensor cores.
//
// Every CTA (one per SM) takes matrices from a device work queue (largest
// order first: the host orders the batch by n), computes ||A||_1 (FP64 sums,
// warp-shuffle maximum), chooses (2m, s) from Table 2 on the device and runs
// the same product plan as the single-matrix path: the Pi_2m products of the
// factorised scheme with its linear combinations fused into each product's
// epilogue, then s double-angle products [C; S] C.
//
// Precision.  The double-angle recurrence C <- 2C^2 - I amplifies the
// rounding of the chain's stored results by two orders of magnitude at
// ||A||_1 near 64 (FP32 storage with exactly rounded products ends 1.3e-5
// from the FP64 result on a 1 x 1 matrix, 8e-6 at n = 128).  So the chain
// keeps its intermediates as double-float pairs (hi, lo) of FP32 values
// (about 48 bits) with double-float epilogue arithmetic on the FP32 pipes
// (GB300's FP64 rate is 1/64 of FP32's), and the double-angle steps, whose
// own rounding is amplified far less, store FP32.
//
// Products on the tensor cores.  Each operand is cut into four 7-bit
// fixed-point slices, rows of X scaled by 2^-e_r and columns of Y by 2^-f_c
// (powers of two from a pre-pass over the operands):
//   X[r][k] 2^(7-e_r) = a_0 + a_1 2^-7 + a_2 2^-14 + a_3 2^-21 (+ < 2^-22),
// with integer digits |a_0| <= 128, |a_p| <= 64, exact in BF16.  The ten
// slice products with p + q <= 3 run as kind::f16 tcgen05 MMAs (M = 128,
// N <= 128, K = 16) into one FP32 TMEM accumulator per level L = p + q; every
// term is an integer and for K <= 256 every level stays below 2^24, so each
// level sum is exact.  The epilogue combines the levels (double-float for the
// chain, FP32 for the squaring) and applies 2^(e_r + f_c - 14).  The dropped
// digits leave at most 2^-28 K max|X[r][.]| max|Y[.][c]| per entry.  The
// chain's matrices are often dominated by their diagonal (C_j = a_0 I + ...),
// which would set the fixed-point grid of the whole row, so X[r][r mod K] is
// left out of the slices of X and X[r][d] Y[d][c] (d = r mod K) is added in
// the epilogue; one operand suffices, since the error is then relative to
// the off-diagonal maxima of X's rows.
//
// Data movement.  The operands live in the CTA's workspace slice (L2-hot for
// the common orders); the slicing warps read them with coalesced loads and
// write the slices into 64-byte-swizzled K-major shared memory (two stages
// of 32 k, each written while the tensor core reads the other), one thread
// issues the MMAs, and the eight warps drain TMEM through per-warp
// shared-memory tiles so that the epilogue's loads and stores walk rows.
//
// Graph capture: the plan records the queue reset and the persistent launch
// in a CUDA graph once; each replay is one graph launch.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"
#include "plan.h"
#include "sm100_ptx.cuh"
#include "tc_gemm.h"
#include "theta_table.cuh"

namespace cs {
namespace bt {

using namespace ptx;

constexpr int kMaxWarps = 16;
constexpr int kMaxOrder = 256;
constexpr int kMaxM = 2 * kMaxOrder;  // rows of the stacked double-angle operand
constexpr int kBM = 128;              // tile rows = TMEM lanes
constexpr int kKc = 32;               // k per stage (rows of 64 bytes of BF16)
constexpr int kSlices = 4;
constexpr int kDfSlots = 10;          // W0..W7, C, S as double-float pairs
constexpr int kFloatsPerN2 = 2 * kDfSlots + 4;  // + two stacked FP32 [C; S] buffers

// Tiles of 128 x NT: four level accumulators of NT columns fill 4 NT TMEM
// columns, so NT = 128 runs one CTA per SM and NT = 64 two.  The epilogue
// stages a tile's product (two planes of 128 x NT floats) in the stages,
// which are idle once the tile's MMAs are done.
template <int NT, int TH>
struct Cfg {
  static constexpr int kThreads = TH;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kABytes = kBM * kKc * 2;  // one A slice of a stage
  static constexpr int kBBytes = NT * kKc * 2;   // one B slice of a stage
  static constexpr int kStageBytes = kSlices * (kABytes + kBBytes);
  static constexpr int kStages = 2;
  static constexpr int kSmem = kStages * kStageBytes + 1024;
  static constexpr uint32_t kTmemCols = kSlices * NT;
  static constexpr int kCtasPerSm = 512 / (kSlices * NT);
  static_assert(2 * kBM * NT * 4 <= kStages * kStageBytes, "the staged tile fits the stages");
  static_assert(kSmem <= 227 * 1024, "shared memory");
  static_assert(kTmemCols <= 512, "TMEM columns");
};

// One product of a plan in dense form (see upload_plans): distinct input
// slots in[], and for every output t: out_t = alpha_t P + gamma_t I
// + sum_q beta[t][q] in_q + delta[t] out_0, each coefficient a double-float
// pair; scale[t] multiplies alpha_t by 4^-s (1) or 2^-s (2).  (The schemes
// of Sec. 2.1 read at most four earlier matrices per product and chain
// outputs only to the first output of the same product.)
constexpr int kMaxIn = 4;
struct DStep {
  int X, Y, nout, nin;
  int out[EPI_MAX_OUT];
  int in[kMaxIn];
  int scale[EPI_MAX_OUT];
  float2 alpha[EPI_MAX_OUT];
  float2 gamma[EPI_MAX_OUT];
  float2 beta[EPI_MAX_OUT][kMaxIn];
  float2 delta[EPI_MAX_OUT];
};
struct DPlan {
  int nsteps;
  DStep step[8];
};

__constant__ DPlan c_plans[4];

struct Desc {
  const float* A;
  float* C;
  float* S;
  int64_t n;
};

// ------------------------------------------------------------ double-float --
// Pairs (hi, lo) with |lo| <= ulp(hi) / 2: Knuth's TwoSum, the fast two-sum
// (|a| >= |b|) and an FMA-based product, as in Dekker's double-length
// arithmetic.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
__device__ __forceinline__ dfl df_mul(float2 c, dfl x) {
  const float p = c.x * x.hi;
  float e = fmaf(c.x, x.hi, -p);
  e = fmaf(c.x, x.lo, e);
  e = fmaf(c.y, x.hi, e);
  return fast_two_sum(p, e);
}
// Accumulation without renormalising after every term: acc.hi carries the
// leading sum, acc.lo the exact errors of the leading additions plus the low
// parts (renormalised once at the end with fast_two_sum).
__device__ __forceinline__ dfl df_mul_raw(float2 c, dfl x) {
  const float p = c.x * x.hi;
  float e = fmaf(c.x, x.hi, -p);
  e = fmaf(c.x, x.lo, e);
  return {p, fmaf(c.y, x.hi, e)};
}
__device__ __forceinline__ void df_acc(dfl& acc, dfl t) {
  const dfl s = two_sum(acc.hi, t.hi);
  acc.hi = s.hi;
  acc.lo += s.lo + t.lo;
}

// ------------------------------------------------------------------ operands --
// An operand matrix: rows [0, split) from (hi, lo), rows [split, ...) from
// (hi2, lo2) (the stacked [C; S]); lo null for FP32 values.  Leading dimension n.
struct Opnd {
  const float* hi;
  const float* lo;
  const float* hi2;
  const float* lo2;
  int split;
};
__device__ __forceinline__ dfl opnd_get(const Opnd& o, int r, int k, int n) {
  const float* h = o.hi;
  const float* l = o.lo;
  if (r >= o.split) {
    h = o.hi2;
    l = o.lo2;
    r -= o.split;
  }
  const int idx = r * n + k;  // n <= 256
  return {h[idx], l ? l[idx] : 0.f};
}

// Scale factors of a row / column whose largest |hi| has the bit pattern
// `bits`: |x| < 2^e, slicing scale 2^(7-e), product scale 2^(e-7).  e is kept
// >= -100 (a larger e is still valid, with fewer digits), so both are normal.
__device__ __forceinline__ void scales_of(unsigned bits, float* slice_sc, float* prod_sc) {
  const float m = __uint_as_float(bits);
  int e = 0;
  if (m > 0.f && isfinite(m)) frexpf(m, &e);
  e = max(e, -100);
  *slice_sc = ldexpf(1.f, 7 - e);
  *prod_sc = ldexpf(1.f, e - 7);
}

// The four digits of x = hi + lo in units of the slicing scale sc.
__device__ __forceinline__ void digits(dfl x, float sc, float d[kSlices]) {
  const float s = x.hi * sc;  // |s| < 128, exact
  d[0] = rintf(s);
  float r = (s - d[0]) + x.lo * sc;  // s - d[0] is exact, |r| <= 1/2 (+ lo)
  r *= 128.f;
  d[1] = rintf(r);
  r = (r - d[1]) * 128.f;
  d[2] = rintf(r);
  r = (r - d[2]) * 128.f;
  d[3] = rintf(r);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // integers |x| <= 128: exact
  return *reinterpret_cast<const uint32_t*>(&v);
}

// Byte offset of the 4-byte word holding k, k + 1 (k even, k < 32) of row r in
// a K-major tile with 64-byte rows and the 64-byte swizzle (16-byte chunk c of
// row r stored at c ^ ((r >> 1) & 3); 512-byte atoms of 8 rows).
__device__ __forceinline__ uint32_t swz64(int r, int k) {
  return (uint32_t)(r * 64 + ((((k >> 3) ^ (r >> 1)) & 3) << 4) + ((k & 7) >> 1) * 4);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------------ shared --
struct Shared {
  float sx[kMaxM], px[kMaxM];          // row scales of X (slicing, product)
  float sy[kMaxOrder], py[kMaxOrder];  // column scales of Y
  float2 dx[kMaxM];                    // X[r][r mod K] (double-float), left out of the slices of X
  unsigned colmax[kMaxOrder];
  double red[kMaxWarps * 32];
  uint64_t mma_bar[2];
  uint32_t tmem;
  int item;
  int abort_flag;
};

// Per-CTA progress of the two-stage pipeline: chunks issued so far.
struct Pipe {
  int chunks;
};

// Block-wide ||A||_1 of an FP32 matrix: FP64 column sums (warp w of W adds
// rows w, w + W, ... of 32 columns, the W partial sums are added in a fixed
// order), maximum by warp shuffles; NaN propagates.
template <int kWarps>
__device__ double block_norm1(const float* __restrict__ A, int n, Shared& sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double qnan = __longlong_as_double(0x7ff8000000000000ULL);
  double best = 0.0;
  bool nan = false;
  for (int c0 = 0; c0 < n; c0 += 32) {
    const int c = c0 + lane;
    double part = 0.0;
    if (c < n)
      for (int r = warp; r < n; r += kWarps) part += fabs((double)A[(int64_t)r * n + c]);
    sh.red[warp * 32 + lane] = part;
    __syncthreads();
    if (warp == 0 && c < n) {
      double col = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) col += sh.red[w * 32 + lane];
      if (isnan(col)) nan = true;
      best = fmax(best, col);
    }
    __syncthreads();
  }
  if (warp == 0) {
    if (nan) best = qnan;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double o = __shfl_xor_sync(0xffffffffu, best, off);
      best = (isnan(best) || isnan(o)) ? qnan : fmax(best, o);
    }
    if (lane == 0) sh.red[0] = best;
  }
  __syncthreads();
  const double r = sh.red[0];
  __syncthreads();
  return r;
}

// Row scales of X (M x K, each row without its entry X[r][r mod K], which
// is kept apart) and column scales of Y (K x N) into shared memory.  Warps
// take four rows (or a lane four k of its column) per round so that the
// loads are in flight together.
template <int kWarps>
__device__ void prepass(const Opnd& X, const Opnd& Y, int M, int N, int K, int n, Shared& sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kR = 4;
  for (int r0 = warp * kR; r0 < M; r0 += kWarps * kR) {
    unsigned mx[kR];
#pragma unroll
    for (int i = 0; i < kR; ++i) mx[i] = 0u;
    for (int k0 = 0; k0 < K; k0 += 32) {
      const int k = k0 + lane;
      dfl v[kR];
#pragma unroll
      for (int i = 0; i < kR; ++i) v[i] = (r0 + i < M && k < K) ? opnd_get(X, r0 + i, k, n) : dfl{0.f, 0.f};
#pragma unroll
      for (int i = 0; i < kR; ++i) {
        if (r0 + i >= M || k >= K) continue;
        const int d = r0 + i >= K ? r0 + i - K : r0 + i;  // (r0 + i) mod K, M <= 2K
        if (k == d) sh.dx[r0 + i] = make_float2(v[i].hi, v[i].lo);
        else mx[i] = max(mx[i], __float_as_uint(fabsf(v[i].hi)));
      }
    }
#pragma unroll
    for (int i = 0; i < kR; ++i) {
      const unsigned m = __reduce_max_sync(0xffffffffu, mx[i]);
      if (lane == 0 && r0 + i < M) scales_of(m, &sh.sx[r0 + i], &sh.px[r0 + i]);
    }
  }
  for (int c = threadIdx.x; c < N; c += kWarps * 32) sh.colmax[c] = 0u;
  __syncthreads();
  for (int c0 = 0; c0 < N; c0 += 32) {
    const int c = c0 + lane;
    unsigned mx = 0u;
    for (int k0 = warp; k0 < K; k0 += kWarps * kR) {
      float v[kR];
#pragma unroll
      for (int i = 0; i < kR; ++i) {
        const int k = k0 + i * kWarps;
        v[i] = (c < N && k < K) ? Y.hi[(int64_t)k * n + c] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < kR; ++i) mx = max(mx, __float_as_uint(fabsf(v[i])));
    }
    if (c < N) atomicMax(&sh.colmax[c], mx);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < N; c += kWarps * 32) scales_of(sh.colmax[c], &sh.sy[c], &sh.py[c]);
  __syncthreads();
}

// Slices of X rows [m0, m0 + 128) (without X[r][r mod K]) and Y columns
// [n0, n0 + n16) for k in [k0, k0 + 32) into one stage.  Each
// warp covers 8 x 8 blocks, a word (two k) per lane: the 32 words of a block
// and slice fall on distinct banks.  A warp loads every element of its
// blocks before it converts any, so the loads are in flight together.
template <int NT, int TH>
__device__ void slice_chunk(const Opnd& X, const Opnd& Y, int m0, int n0, int M, int N, int n16, int K, int k0,
                            int n, const Shared& sh, uint8_t* stA, uint8_t* stB) {
  using C = Cfg<NT, TH>;
  constexpr int kWarps = C::kWarps;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int kAB = (kBM / 8) * 4 / kWarps;  // A blocks per warp
  {
    dfl v[kAB][2];
#pragma unroll
    for (int i = 0; i < kAB; ++i) {
      const int b = warp + i * kWarps;
      const int r = m0 + (b >> 2) * 8 + (lane >> 2), k = k0 + (b & 3) * 8 + 2 * (lane & 3);
      v[i][0] = v[i][1] = dfl{0.f, 0.f};
      if (r < M) {
        const int d = r >= K ? r - K : r;  // r mod K (M <= 2K)
        if (k < K && k != d) v[i][0] = opnd_get(X, r, k, n);
        if (k + 1 < K && k + 1 != d) v[i][1] = opnd_get(X, r, k + 1, n);
      }
    }
#pragma unroll
    for (int i = 0; i < kAB; ++i) {
      const int b = warp + i * kWarps;
      const int rl = (b >> 2) * 8 + (lane >> 2), kk = (b & 3) * 8 + 2 * (lane & 3);
      const float sc = m0 + rl < M ? sh.sx[m0 + rl] : 0.f;
      float d0[kSlices], d1[kSlices];
      digits(v[i][0], sc, d0);
      digits(v[i][1], sc, d1);
      const uint32_t off = swz64(rl, kk);
#pragma unroll
      for (int p = 0; p < kSlices; ++p)
        *reinterpret_cast<uint32_t*>(stA + p * C::kABytes + off) = pack_bf16(d0[p], d1[p]);
    }
  }
  const int nb = (n16 / 8) * 4;
  for (int b0 = 0; b0 < nb; b0 += 4 * kWarps) {
    dfl v[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int b = b0 + warp + i * kWarps;
      const int c = n0 + (b >> 2) * 8 + (lane & 7), k = k0 + (b & 3) * 8 + 2 * (lane >> 3);
      v[i][0] = v[i][1] = dfl{0.f, 0.f};
      if (b < nb && c < N) {
        if (k < K) v[i][0] = opnd_get(Y, k, c, n);
        if (k + 1 < K) v[i][1] = opnd_get(Y, k + 1, c, n);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int b = b0 + warp + i * kWarps;
      if (b >= nb) break;
      const int cl = (b >> 2) * 8 + (lane & 7), kk = (b & 3) * 8 + 2 * (lane >> 3);
      const float sc = n0 + cl < N ? sh.sy[n0 + cl] : 0.f;
      float d0[kSlices], d1[kSlices];
      digits(v[i][0], sc, d0);
      digits(v[i][1], sc, d1);
      const uint32_t off = swz64(cl, kk);
#pragma unroll
      for (int q = 0; q < kSlices; ++q)
        *reinterpret_cast<uint32_t*>(stB + q * C::kBBytes + off) = pack_bf16(d0[q], d1[q]);
    }
  }
}

// The per-matrix state the epilogues need.
struct Mat {
  const float* A;
  float* C;  // caller's outputs (FP32)
  float* S;
  float* ws;  // the CTA's workspace slice
  int n, s;
  int64_t n2;
  float a2, as;  // 4^-s, 2^-s
};

// Double-float slot k (W0..W7 = 0..7, C = 8, S = 9) of the workspace.
__device__ __forceinline__ int df_index(int slot) { return slot == SL_C ? 8 : slot == SL_S ? 9 : slot - W(0); }
__device__ __forceinline__ float* df_hi(const Mat& m, int slot) { return m.ws + 2 * (int64_t)df_index(slot) * m.n2; }

// Which epilogue a product runs.
struct Epi {
  int f, k;      // chain step k of family f, or k < 0: double-angle step
  float* outC;   // double-angle: rows < n -> 2P - I here, rows >= n -> 2P to outS
  float* outS;
};

constexpr int kEpiBatch = 4;  // entries a thread finishes at once

// Finishes kEpiBatch entries (r[i], c[i]) of a product: the left-out
// diagonal term X[r][d] Y[d][c] (d = r mod n) is added to the slice product,
// then the step's epilogue runs (terms whose coefficient is zero are
// skipped; the branches are uniform).  Every load is issued before the
// arithmetic that uses it.
__device__ __forceinline__ void finish(const Opnd& Y, const Mat& m, const Epi& ep, const Shared& sh,
                                       const int (&r)[kEpiBatch], const int (&c)[kEpiBatch], dfl (&P)[kEpiBatch],
                                       const bool (&ok)[kEpiBatch]) {
  const int n = m.n;
  const bool chain = ep.k >= 0;
  const DStep& st = c_plans[chain ? ep.f : 0].step[chain ? ep.k : 0];
  const int nin = chain ? st.nin : 0;
  dfl ydc[kEpiBatch], in[kEpiBatch][kMaxIn];
#pragma unroll
  for (int i = 0; i < kEpiBatch; ++i) {
    ydc[i] = dfl{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < kMaxIn; ++q) in[i][q] = dfl{0.f, 0.f};
    if (!ok[i]) continue;
    const int d = r[i] >= n ? r[i] - n : r[i];
    ydc[i] = opnd_get(Y, d, c[i], n);
    const int idx = r[i] * n + c[i];
#pragma unroll
    for (int q = 0; q < kMaxIn; ++q) {
      if (q < nin) {
        const float* h = df_hi(m, st.in[q]);
        in[i][q] = dfl{h[idx], h[idx + m.n2]};
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kEpiBatch; ++i) {
    if (!ok[i]) continue;
    dfl p = P[i];
    df_acc(p, df_mul_raw(sh.dx[r[i]], ydc[i]));
    p = fast_two_sum(p.hi, p.lo);
    const int idx = r[i] * n + c[i];
    if (!chain) {
      const float v = 2.f * (p.hi + p.lo);
      if (r[i] < n) ep.outC[idx] = v - (r[i] == c[i] ? 1.f : 0.f);
      else ep.outS[idx - (int)m.n2] = v;
      continue;
    }
    dfl o0 = dfl{0.f, 0.f};
#pragma unroll
    for (int t = 0; t < EPI_MAX_OUT; ++t) {
      if (t < st.nout) {
        float2 al = st.alpha[t];
        const float sc = st.scale[t] == 1 ? m.a2 : st.scale[t] == 2 ? m.as : 1.f;
        al.x *= sc;
        al.y *= sc;
        dfl v = df_mul_raw(al, p);
        if (r[i] == c[i] && st.gamma[t].x != 0.f) df_acc(v, dfl{st.gamma[t].x, st.gamma[t].y});
#pragma unroll
        for (int q = 0; q < kMaxIn; ++q)
          if (q < nin && st.beta[t][q].x != 0.f) df_acc(v, df_mul_raw(st.beta[t][q], in[i][q]));
        if (t > 0 && st.delta[t].x != 0.f) df_acc(v, df_mul_raw(st.delta[t], o0));
        v = fast_two_sum(v.hi, v.lo);
        if (t == 0) o0 = v;
        const int slot = st.out[t];
        float* h = df_hi(m, slot);
        h[idx] = v.hi;
        h[idx + m.n2] = v.lo;
        if (m.s == 0 && (slot == SL_C || slot == SL_S)) (slot == SL_C ? m.C : m.S)[idx] = v.hi + v.lo;
      }
    }
  }
}

// One product P = X Y (M x N, inner K = n) of matrix m with its epilogue.
template <int NT, int TH>
__device__ bool product(const Opnd& X, const Opnd& Y, int M, int N, int K, const Mat& m, const Epi& ep,
                        Shared& sh, uint8_t* smem, Pipe& pipe) {
  using C = Cfg<NT, TH>;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = m.n;
  prepass<C::kWarps>(X, Y, M, N, K, n, sh);
  const int nchunks = (K + kKc - 1) / kKc;
  for (int m0 = 0; m0 < M; m0 += kBM) {
    for (int n0 = 0; n0 < N; n0 += NT) {
      const int ntile = min(NT, N - n0);
      const int n16 = (ntile + 15) & ~15;
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n16 >> 3) << 17) |
                             ((uint32_t)(kBM >> 4) << 24);
      for (int kc = 0; kc < nchunks; ++kc) {
        const int g = pipe.chunks;
        const int st = g & 1;
        // The stage was last read by chunk g - 2: every thread waits for that
        // commit itself, so the threads slice chunk g while thread 0 may
        // still be issuing chunk g - 1's MMAs.
        if (g >= 2 && !mbar_wait(&sh.mma_bar[st], ((g - 2) >> 1) & 1, (volatile int*)&sh.abort_flag))
          sh.abort_flag = 1;
        uint8_t* stA = smem + st * C::kStageBytes;
        uint8_t* stB = stA + kSlices * C::kABytes;
        slice_chunk<NT, TH>(X, Y, m0, n0, M, N, n16, K, kc * kKc, n, sh, stA, stB);
        fence_async_smem();
        __syncthreads();
        if (sh.abort_flag) return false;
        if (threadIdx.x == 0) {
          tc_fence_after();
          // descriptors: start address >> 4, LBO 1 (unused), SBO 512 bytes
          // (8 rows of 64 bytes), version 1, 64-byte swizzle
          constexpr uint32_t kDescHi = (512u >> 4) | (1u << 14) | (4u << 29);
          const uint32_t a_lo = ((smem_u32(stA) & 0x3FFFFu) >> 4) | (1u << 16);
          const uint32_t b_lo = ((smem_u32(stB) & 0x3FFFFu) >> 4) | (1u << 16);
#pragma unroll
          for (int j = 0; j < kKc / 16; ++j) {
            if (kc * kKc + 16 * j >= K) break;
            const bool first = kc == 0 && j == 0;
#pragma unroll
            for (int p = 0; p < kSlices; ++p) {
              const uint64_t ad = ((uint64_t)kDescHi << 32) | (uint64_t)(a_lo + (uint32_t)((p * C::kABytes + 32 * j) >> 4));
#pragma unroll
              for (int q = 0; p + q < kSlices; ++q) {
                const uint64_t bd =
                    ((uint64_t)kDescHi << 32) | (uint64_t)(b_lo + (uint32_t)((q * C::kBBytes + 32 * j) >> 4));
                // p = 0 reaches every level first: it restarts the accumulators
                mma_bf16(sh.tmem + (uint32_t)((p + q) * NT), ad, bd, idesc, (first && p == 0) ? 0u : 1u);
              }
            }
          }
          mma_commit(&sh.mma_bar[st]);
        }
        pipe.chunks = g + 1;
      }
      // every MMA of the tile has completed once the last chunk's commit has;
      // the stages are then free, and the epilogue stages through them
      {
        const int g = pipe.chunks - 1;
        if (!mbar_wait(&sh.mma_bar[g & 1], (g >> 1) & 1, (volatile int*)&sh.abort_flag)) sh.abort_flag = 1;
        __syncthreads();
        if (sh.abort_flag) return false;
        tc_fence_after();
      }
      // Epilogue.  Warp w drains TMEM lanes 32 (w & 3).. and its span of
      // columns in groups of 16, combines the levels and stages the
      // tile's P (hi and lo planes of 128 x NT floats, column index XOR-ed
      // with the row's low 5 bits, so that both the drain, lane = row, and
      // the walk, thread = column, are conflict-free) in the idle stages;
      // then every thread finishes entries of the tile, row by row.
      {
        constexpr int kSpan = NT / (C::kWarps / 4);  // columns per warp
        const int quarter = warp & 3;
        const int cbase = (warp >> 2) * kSpan;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        float* t_hi = reinterpret_cast<float*>(smem);
        float* t_lo = t_hi + kBM * NT;
        const int rl = quarter * 32 + lane;
        const float pr = m0 + rl < M ? sh.px[m0 + rl] : 0.f;
        for (int g16 = 0; g16 < kSpan; g16 += 16) {
          const int cl0 = cbase + g16;
          if (cl0 >= ntile) break;  // uniform over the warp
          uint32_t v[kSlices][16];
#pragma unroll
          for (int L = 0; L < kSlices; ++L) tmem_ld16(sh.tmem + lane_off + (uint32_t)(L * NT + cl0), v[L]);
          tmem_ld_wait();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = n0 + cl0 + j;
            const float sc = pr * (c < N ? sh.py[c] : 0.f);
            const float l0 = __uint_as_float(v[0][j]), l1 = __uint_as_float(v[1][j]);
            const float l2 = __uint_as_float(v[2][j]), l3 = __uint_as_float(v[3][j]);
            dfl P = two_sum(l0, l1 * 0x1p-7f);
            P = fast_two_sum(P.hi, P.lo + (l2 * 0x1p-14f + l3 * 0x1p-21f));
            const int a = rl * NT + ((cl0 + j) ^ (rl & 31));
            t_hi[a] = P.hi * sc;
            t_lo[a] = P.lo * sc;
          }
        }
        tc_fence_before();
        __syncthreads();
        // rows of the tile round-robin over the warps, lanes along columns:
        // kEpiBatch entries per thread, NT / 32 columns x kRows rows
        const int mrows = min(kBM, M - m0);
        constexpr int kCols = NT / 32, kRows = kEpiBatch / kCols;
        for (int rt0 = warp * kRows; rt0 < mrows; rt0 += C::kWarps * kRows) {
          int r[kEpiBatch], c[kEpiBatch];
          bool ok[kEpiBatch];
          dfl P[kEpiBatch];
#pragma unroll
          for (int i = 0; i < kEpiBatch; ++i) {
            const int rt = rt0 + i / kCols, ct = lane + 32 * (i % kCols);
            ok[i] = rt < mrows && ct < ntile;
            r[i] = m0 + rt;
            c[i] = n0 + ct;
            const int a = (rt & (kBM - 1)) * NT + (ct ^ (rt & 31));
            P[i] = ok[i] ? dfl{t_hi[a], t_lo[a]} : dfl{0.f, 0.f};
          }
          finish(Y, m, ep, sh, r, c, P, ok);
        }
      }
      // the next tile's slices overwrite the staged tile, and the next
      // product reads what this one wrote
      tc_fence_before();
      __syncthreads();
    }
  }
  return true;
}

template <int NT, int TH>
__global__ void __launch_bounds__(TH, Cfg<NT, TH>::kCtasPerSm)
    batched_kernel(const Desc* __restrict__ desc, const int* __restrict__ order, int count, int* queue,
                   float* ws_all, int64_t ws_per_cta, cs_info* infos, int32_t* status, int* err) {
  using C = Cfg<NT, TH>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ Shared sh;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    mbar_init(&sh.mma_bar[0], 1);
    mbar_init(&sh.mma_bar[1], 1);
    sh.abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(&sh.tmem, C::kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  Pipe pipe{0};
  float* ws = ws_all + (int64_t)blockIdx.x * ws_per_cta;
  for (;;) {
    if (threadIdx.x == 0) sh.item = atomicAdd(queue, 1);
    __syncthreads();
    const int i = sh.item;
    __syncthreads();
    if (i >= count || sh.abort_flag) break;
    const int j = order[i];
    const Desc d = desc[j];
    const int n = (int)d.n;
    if (n <= 0) {
      if (threadIdx.x == 0) {
        if (status) status[j] = CS_OK;
        if (infos) infos[j] = cs_info{0.0, 4, 0, 0, 1, 0.0};
      }
      continue;
    }
    const double nrm = block_norm1<C::kWarps>(d.A, n, sh);
    int f = 0, s = 0;
    const int sel = select_family(nrm, 1, &f, &s);
    if (threadIdx.x == 0) {
      if (status) status[j] = sel == 0 ? CS_OK : (sel == 3 ? CS_ENONFINITE : CS_ERANGE);
      if (infos) {
        const int prods = sel == 0 ? family_products(f) + 2 * s : 0;
        infos[j] = cs_info{nrm, sel == 0 ? family_order(f) : 0, sel == 0 ? s : 0, prods, 1,
                           2.0 * (double)n * n * n * prods};
      }
    }
    if (sel != 0) {
      const float qnan = __int_as_float(0x7fc00000);
      for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        d.C[e] = qnan;
        d.S[e] = qnan;
      }
      __syncthreads();
      continue;
    }
    Mat m;
    m.A = d.A;
    m.C = d.C;
    m.S = d.S;
    m.ws = ws;
    m.n = n;
    m.s = s;
    m.n2 = (int64_t)n * n;
    m.a2 = ldexpf(1.f, -2 * s);
    m.as = ldexpf(1.f, -s);
    auto slot_opnd = [&](int slot) {
      if (slot == SL_A) return Opnd{d.A, nullptr, nullptr, nullptr, n};
      const float* h = df_hi(m, slot);
      return Opnd{h, h + m.n2, nullptr, nullptr, n};
    };
    bool ok = true;
    const DPlan& P = c_plans[f];
    for (int k = 0; k < P.nsteps && ok; ++k) {
      const Opnd X = slot_opnd(P.step[k].X), Y = slot_opnd(P.step[k].Y);
      ok = product<NT, TH>(X, Y, n, n, n, m, Epi{f, k, nullptr, nullptr}, sh, smem, pipe);
    }
    // double-angle steps: the first reads the chain's double-float C and S,
    // the others the FP32 stacked buffers ping[0], ping[1]
    float* ping0 = ws + (int64_t)2 * kDfSlots * m.n2;
    float* ping1 = ping0 + 2 * m.n2;
    for (int q = 0; q < s && ok; ++q) {
      Opnd X, Y;
      if (q == 0) {
        const float* ch = df_hi(m, SL_C);
        const float* sh_ = df_hi(m, SL_S);
        X = Opnd{ch, ch + m.n2, sh_, sh_ + m.n2, n};
        Y = Opnd{ch, ch + m.n2, nullptr, nullptr, n};
      } else {
        const float* cur = (q & 1) ? ping0 : ping1;
        X = Opnd{cur, nullptr, cur + m.n2, nullptr, n};
        Y = Opnd{cur, nullptr, nullptr, nullptr, n};
      }
      float* nxt = (q & 1) ? ping1 : ping0;
      const bool last = q == s - 1;
      ok = product<NT, TH>(X, Y, 2 * n, n, n, m, Epi{0, -1, last ? d.C : nxt, last ? d.S : nxt + m.n2}, sh, smem, pipe);
    }
    if (!ok) break;
  }
  // Teardown: after an expired wait, wait (bounded) for the MMAs this CTA
  // issued before freeing TMEM, and raise the error word.
  __syncthreads();
  if (sh.abort_flag && threadIdx.x == 0) {
    if (pipe.chunks > 0) {
      volatile int never = 0;
      const int g = pipe.chunks - 1;
      mbar_wait(&sh.mma_bar[g & 1], (g >> 1) & 1, &never);
    }
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(sh.tmem, C::kTmemCols);
  }
}

// ------------------------------------------------------------------- host ---
struct Variant {
  int tile;  // output tile columns (N of each MMA, at most)
  int ctas_per_sm;
  int threads;
};
// Tiles of 128 x 128 (four level accumulators fill TMEM's 512 columns, one
// CTA of 512 threads per SM) or 128 x 64 (half of TMEM, two CTAs per SM, of
// 256 or 512 threads; orders above 64 take twice the tiles): the autotuner
// keeps whichever is fastest on the batch.
const Variant kVariants[] = {{128, 1, 512}, {64, 2, 256}, {64, 2, 512}};

std::mutex g_mu;
bool g_plans_uploaded[64] = {};
std::map<std::string, int> g_tuned;  // batch signature -> variant index

// A coefficient as a double-float pair (hi, lo), hi + lo = c to about 2^-48.
float2 df_pair(double c) {
  const float h = (float)c;
  return make_float2(h, (float)(c - (double)h));
}

cs_status upload_plans() {
  int dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev >= 0 && dev < 64 && g_plans_uploaded[dev]) return CS_OK;
  DPlan host[4];
  for (int f = 0; f < 4; ++f) {
    const int m = family_order(f);
    std::vector<Step> steps = chain_plan(m, 0);
    DPlan& P = host[f];
    P = DPlan{};
    P.nsteps = (int)steps.size();
    for (size_t k = 0; k < steps.size(); ++k) {
      DStep& D = P.step[k];
      D = DStep{};
      D.X = steps[k].X;
      D.Y = steps[k].Y;
      D.nout = (int)steps[k].outs.size();
      for (int t = 0; t < D.nout; ++t) {
        const OutSpec& o = steps[k].outs[t];
        D.out[t] = o.slot;
        D.alpha[t] = df_pair(o.alpha);
        D.gamma[t] = df_pair(o.gamma);
        D.scale[t] = (k == 0) ? 1 : (o.slot == SL_S ? 2 : 0);
        for (auto& b : o.beta) {
          if (b.first == SL_A) return fail(CS_EINVAL, "batched plans read A only as a product operand");
          int q = -1;
          for (int z = 0; z < D.nin; ++z)
            if (D.in[z] == b.first) q = z;
          if (q < 0) {
            if (D.nin == kMaxIn) return fail(CS_EINVAL, "batched plans read at most four matrices per product");
            q = D.nin++;
            D.in[q] = b.first;
          }
          D.beta[t][q] = df_pair(b.second);
        }
        for (auto& d : o.delta) {
          if (d.first != 0 || t == 0) return fail(CS_EINVAL, "batched plans chain outputs only to the first output");
          D.delta[t] = df_pair(d.second);
        }
      }
    }
  }
  CS_CUDA_CHECK(cudaMemcpyToSymbol(c_plans, host, sizeof(host)));
  if (dev >= 0 && dev < 64) g_plans_uploaded[dev] = true;
  return CS_OK;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  return sms;
}

struct BLayout {
  size_t desc = 0, order = 0, queue = 0, scratch = 0, total = 0;
  int64_t per_cta = 0;
  int max_ctas = 0;
};

BLayout make_blayout(int64_t count, int64_t nmax) {
  BLayout L;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  L.desc = off;
  off += al(sizeof(Desc) * (size_t)std::max<int64_t>(count, 1));
  L.order = off;
  off += al(sizeof(int) * (size_t)std::max<int64_t>(count, 1));
  L.queue = off;
  off += 256;
  L.per_cta = kFloatsPerN2 * nmax * nmax;
  L.max_ctas = sm_count() * 2;
  L.scratch = off;
  off += al(sizeof(float) * (size_t)L.per_cta * L.max_ctas);
  L.total = off;
  return L;
}

template <int NT, int TH>
cs_status launch_tile(int grid, const BLayout& L, char* ws, int count, cs_info* infos, int32_t* status, int* err,
                      cudaStream_t stream) {
  static std::atomic<unsigned long long> smem_set{0};
  CS_CHECK(smem_limit_once(batched_kernel<NT, TH>, Cfg<NT, TH>::kSmem, smem_set));
  batched_kernel<NT, TH><<<grid, TH, Cfg<NT, TH>::kSmem, stream>>>(
      (const Desc*)(ws + L.desc), (const int*)(ws + L.order), count, (int*)(ws + L.queue),
      (float*)(ws + L.scratch), L.per_cta, infos, status, err);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

cs_status launch_variant(int v, const BLayout& L, char* ws, int count, cs_info* infos, int32_t* status,
                         cudaStream_t stream) {
  const Variant& V = kVariants[v];
  const int grid = std::min(L.max_ctas, sm_count() * V.ctas_per_sm);
  int* err = tc_error_word();
  if (!err) return fail(CS_ECUDA, "cannot resolve the device error word");
  CS_CUDA_CHECK(cudaMemsetAsync(ws + L.queue, 0, sizeof(int), stream));
  if (V.tile == 128) return launch_tile<128, 512>(grid, L, ws, count, infos, status, err, stream);
  if (V.threads == 512) return launch_tile<64, 512>(grid, L, ws, count, infos, status, err, stream);
  return launch_tile<64, 256>(grid, L, ws, count, infos, status, err, stream);
}

}  // namespace bt

struct BatchedPlan {
  int64_t count = 0;
  bt::BLayout L;
  char* ws = nullptr;
  cs_info* infos = nullptr;
  int32_t* status = nullptr;
  int variant = 0;
  double flops_estimate = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

cs_status validate_batch(int64_t count, const int64_t* n, int64_t* nmax) {
  if (count < 0) return fail(CS_EINVAL, "count must be >= 0");
  if (count > (1 << 30)) return fail(CS_EINVAL, "count too large");
  if (count > 0 && !n) return fail(CS_EINVAL, "n is null");
  int64_t mx = 1;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 0 || n[i] > bt::kMaxOrder)
      return fail(CS_EINVAL, "batched orders must be in [0, 256] (use cossin for larger matrices)");
    mx = std::max(mx, n[i]);
  }
  *nmax = mx;
  return CS_OK;
}

}  // namespace
}  // namespace cs

extern "C" {

cs_status cossin_batched_workspace_size(int64_t count, const int64_t* n, size_t* bytes) {
  if (!bytes) return cs::fail(CS_EINVAL, "bytes is null");
  int64_t nmax = 1;
  CS_CHECK(cs::validate_batch(count, n, &nmax));
  *bytes = cs::bt::make_blayout(count, nmax).total;
  return CS_OK;
}

cs_status cossin_batched_plan_create(int64_t count, const int64_t* n, const float* const* A, float* const* C,
                                     float* const* S, void* ws_dev, size_t ws_bytes, cs_info* infos_dev,
                                     int32_t* status_dev, int32_t autotune, cossin_stream_t stream,
                                     cossin_batched_plan* plan_out) {
  using namespace cs;
  if (!plan_out) return fail(CS_EINVAL, "plan is null");
  *plan_out = nullptr;
  int64_t nmax = 1;
  CS_CHECK(validate_batch(count, n, &nmax));
  if (count > 0 && (!A || !C || !S)) return fail(CS_EINVAL, "null pointer array");
  const bt::BLayout L = bt::make_blayout(count, nmax);
  if (!ws_dev || ws_bytes < L.total) return fail(CS_EINVAL, "workspace missing or too small");
  if (((uintptr_t)ws_dev & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
  std::vector<bt::Desc> desc((size_t)count);
  double flops_est = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] > 0 && (!A[i] || !C[i] || !S[i])) return fail(CS_EINVAL, "null matrix pointer in batch");
    desc[i] = bt::Desc{A[i], C[i], S[i], n[i]};
    flops_est += 2.0 * (double)n[i] * n[i] * n[i];
  }
  std::vector<int> order((size_t)count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(bt::upload_plans());
  char* ws = (char*)ws_dev;
  if (count > 0) {
    CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.desc, desc.data(), sizeof(bt::Desc) * count, cudaMemcpyHostToDevice, st));
    CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
    CS_CUDA_CHECK(cudaStreamSynchronize(st));
  }
  BatchedPlan* P = new BatchedPlan;
  P->count = count;
  P->L = L;
  P->ws = ws;
  P->infos = infos_dev;
  P->status = status_dev;
  P->flops_estimate = flops_est;
  // Autotuner: time every variant on this batch, keep the fastest; the
  // choice is remembered per (device, count, largest order) in this process.
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string key = std::to_string(dev) + ":" + std::to_string(count) + ":" + std::to_string(nmax);
  int chosen = -1;
  {
    std::lock_guard<std::mutex> lk(bt::g_mu);
    auto it = bt::g_tuned.find(key);
    if (it != bt::g_tuned.end()) chosen = it->second;
  }
  const int nvar = (int)(sizeof(bt::kVariants) / sizeof(bt::kVariants[0]));
  if (chosen < 0 && autotune && count > 0) {
    cudaEvent_t e0, e1;
    CS_CUDA_CHECK(cudaEventCreate(&e0));
    CS_CUDA_CHECK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int v = 0; v < nvar; ++v) {
      cs_status rc = bt::launch_variant(v, L, ws, (int)count, infos_dev, status_dev, st);  // warm-up
      if (rc == CS_OK) {
        cudaEventRecord(e0, st);
        rc = bt::launch_variant(v, L, ws, (int)count, infos_dev, status_dev, st);
        cudaEventRecord(e1, st);
      }
      float ms = 0.f;
      if (rc != CS_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        delete P;
        return rc != CS_OK ? rc : cuda_fail(cudaGetLastError(), "batched autotune");
      }
      if (ms < best) {
        best = ms;
        chosen = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(bt::g_mu);
    bt::g_tuned[key] = chosen;
  }
  if (chosen < 0) chosen = 0;
  P->variant = chosen;
  // Capture the queue reset and the persistent launch once.
  cudaStream_t cap;
  CS_CUDA_CHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cs_status rc = CS_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "cudaStreamBeginCapture");
  } else {
    rc = count > 0 ? bt::launch_variant(chosen, L, ws, (int)count, infos_dev, status_dev, cap) : CS_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (rc == CS_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
    if (rc == CS_OK) {
      e = cudaGraphInstantiate(&P->exec, g, 0);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    }
    P->graph = g;
  }
  cudaStreamDestroy(cap);
  if (rc != CS_OK) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P;
    return rc;
  }
  *plan_out = (cossin_batched_plan)P;
  return CS_OK;
}

cs_status cossin_batched_plan_launch(cossin_batched_plan plan, cossin_stream_t stream) {
  using namespace cs;
  if (!plan) return fail(CS_EINVAL, "plan is null");
  BatchedPlan* P = (BatchedPlan*)plan;
  if (P->count == 0) return CS_OK;
  ProfScope prof(CS_KERNEL_BATCHED, P->flops_estimate, (cudaStream_t)stream);
  CS_CUDA_CHECK(cudaGraphLaunch(P->exec, (cudaStream_t)stream));
  return CS_OK;
}

cs_status cossin_batched_plan_info(cossin_batched_plan plan, int32_t* variant_tile, int32_t* variant_ctas_per_sm) {
  if (!plan) return cs::fail(CS_EINVAL, "plan is null");
  cs::BatchedPlan* P = (cs::BatchedPlan*)plan;
  if (variant_tile) *variant_tile = cs::bt::kVariants[P->variant].tile;
  if (variant_ctas_per_sm) *variant_ctas_per_sm = cs::bt::kVariants[P->variant].ctas_per_sm;
  return CS_OK;
}

cs_status cossin_batched_plan_destroy(cossin_batched_plan plan) {
  if (!plan) return CS_OK;
  cs::BatchedPlan* P = (cs::BatchedPlan*)plan;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  delete P;
  return CS_OK;
}

cs_status cossin_batched(int64_t count, const int64_t* n, const float* const* A, float* const* C, float* const* S,
                         void* ws_dev, size_t ws_bytes, cs_info* infos_dev, int32_t* status_dev,
                         cossin_stream_t stream) {
  using namespace cs;
  int64_t nmax = 1;
  CS_CHECK(validate_batch(count, n, &nmax));
  if (count == 0) return CS_OK;
  if (!A || !C || !S) return fail(CS_EINVAL, "null pointer array");
  const bt::BLayout L = bt::make_blayout(count, nmax);
  if (!ws_dev || ws_bytes < L.total) return fail(CS_EINVAL, "workspace missing or too small");
  if (((uintptr_t)ws_dev & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
  std::vector<bt::Desc> desc((size_t)count);
  double flops_est = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] > 0 && (!A[i] || !C[i] || !S[i])) return fail(CS_EINVAL, "null matrix pointer in batch");
    desc[i] = bt::Desc{A[i], C[i], S[i], n[i]};
    flops_est += 2.0 * (double)n[i] * n[i] * n[i];
  }
  std::vector<int> order((size_t)count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(bt::upload_plans());
  char* ws = (char*)ws_dev;
  CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.desc, desc.data(), sizeof(bt::Desc) * count, cudaMemcpyHostToDevice, st));
  CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  int variant = 0, dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(bt::g_mu);
    auto it = bt::g_tuned.find(std::to_string(dev) + ":" + std::to_string(count) + ":" + std::to_string(nmax));
    if (it != bt::g_tuned.end()) variant = it->second;
  }
  ProfScope prof(CS_KERNEL_BATCHED, flops_est, st);
  CS_CHECK(bt::launch_variant(variant, L, ws, (int)count, infos_dev, status_dev, st));
  // the host staging vectors must outlive the copies
  CS_CUDA_CHECK(cudaStreamSynchronize(st));
  return CS_OK;
}

}  // extern "C"
