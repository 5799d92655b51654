// gemm_ozaki.cu -- FP64 products emulated on the BF16 tensor cores.
//
// GB300 runs FP64 at 2 FMA/clk/SM, about 1/1700 of its BF16 tensor rate.  A
// product of FP64 matrices is carried to the tensor cores with integer slices
// in the manner of Ozaki's error-free splitting (Ozaki, Ogita, Oishi and Rump,
// Numer. Algorithms 2012; Mukunoki, Ozaki, Ogita and Imamura, ICCS 2020):
//
//   * each row i of X is scaled by 2^-e_i (|x| < 1 after scaling) and cut into
//     S slices of 7 bits: X_i = 2^(e_i - 7) sum_p a_p 2^(-7p), where a_0 is an
//     integer in [-128, 128] and a_p (p >= 1) an integer in [-64, 64]; slice p
//     is stored as the BF16 value a_p 2^(-7p), which is exact (8 significant
//     bits, power-of-two scale).  Columns of Y likewise with 2^-f_j.
//   * X Y = 2^(e_i + f_j - 14) sum_{p, q} (A_p B_q).  The pair products with
//     p + q <= S - 1 are formed on the tensor cores (BF16 in, FP32 out).  With
//     S = 8 the slices leave a residual of at most 2^-56 max|X_i.| per entry
//     (and likewise for Y), and the dropped pairs add at most 7 2^-56
//     max|X_i.| max|Y_.j| per k: in all at most 2^-52 K max|X_i.| max|Y_.j|
//     per entry in the worst case (random-sign errors grow like sqrt(K)).  With
//     S = 7 (50 bits) the error of one product of N(0,1) matrices measured
//     3.4e-15, too coarse for the double-angle steps at ||A||_1 = 64.
//   * Fixed-point slices lose the small entries of a row whose maximum is a
//     single large entry, and the method's matrices are often I + E (the
//     cosine near the identity, I - A_2/2 + ...).  So the entry X[r][r mod K]
//     of each row and Y[c][c] of each column are left out of the slices and
//     added exactly in the FP64 epilogue:
//       X Y = X_off Y_off + X[r][d] Y[d][c] + (c != d ? X[r][c] Y[c][c] : 0),
//     d = r mod K, so the slices only carry the off-diagonal scales.
//   * Exactness: all terms of one level L = p + q are integer multiples of
//     2^(-7L), at most (L + 3) 2^12 of them per k.  Each level has its own
//     FP32 TMEM accumulator, restarted every 512 k, so levels 0..5 are summed
//     exactly (at most 2^24 quanta); levels 6 and 7 round far below FP64
//     precision.  After every 512 k the epilogue converts each level to an
//     integer number of 2^-35 quanta (exactly for levels 0..5) and adds it
//     into int64 register sums on the integer pipes, so the sum over K is
//     exact but for levels 6, 7 (K <= 8192 keeps it below 2^63).  At the end
//     it converts once to FP64, applies 2^(e_i + f_j - 49) and the method's
//     fused linear combinations, and writes FP64.
//
// The result has FP64-class accuracy (slices carry 57 bits of each row or
// column maximum; the integer sums round once per 512 k) at a cost of
// S (S + 1) / 2 = 36 BF16 products.  Exact for operands whose entries need
// at most 57 bits below their row / column maximum (small integers, say).
//
// The same kernel with S = 4 is the BF16 multi-term product of the
// split-precision form: 29 bits of each row / column maximum, 10 slice
// products (levels 0..3, all summed exactly), at most 2^-25 K max|X_i.|
// max|Y_.j| per entry; its stages hold 64-wide k-blocks, and its level
// accumulators take 256 TMEM columns, so two sets alternate between chunks
// and the MMAs of one chunk overlap the epilogue's reading of the previous
// one.
//
// One CTA computes a 128 x 64 tile (S = 8):
//   warp 0     TMA producer: all S slices of A (128 x BK) and of B^T
//              (64 x BK) for one k-block per stage, 2 stages of 96 KB (BK = 32
//              with 64-byte swizzle for S = 8, BK = 64 with 128-byte swizzle
//              for S = 4);
//   warp 1     allocates 512 TMEM columns (8 level accumulators of 64
//              columns; two sets of 4 for S = 4) and issues the MMAs
//              (cta_group::1, M = 128, K = 16):
//              per slice p of A, N = 256, 128 and 64 instructions that take
//              4, 2 or 1 adjacent slices q, q + 1, ... of B into the
//              accumulators of levels p + q, p + q + 1, ... (14 per k-step
//              for S = 8, 5 for S = 4), the p = 0 instructions restarting
//              every accumulator at a chunk start once the epilogue has read
//              it;
//   warps 2-9  two per TMEM lane quarter, 32 columns each: after each chunk,
//              read every accumulator (freeing it at once), add it into the
//              int64 sums; at the end of a tile write the sums (as FP64) to
//              one of two scratch slots of the CTA in global memory (L2) and
//              go on with the next tile's chunks;
//   warps 10-17 the FP64 epilogue of each tile from its scratch slot, row
//              by row with coalesced loads and stores, while the next tile's
//              MMAs and drains run (done by the draining warps, it held the
//              MMAs up at the next tile's first chunk boundaries: a quarter
//              of the eight-slice kernel's time, two fifths of the
//              four-slice one's; four warps still held up the four-slice
//              kernel, as the epilogue's FP64 operations are long-latency
//              on GB300).
// Last round: a persistent grid of G CTAs over T tiles runs ceil(T / G)
// rounds, the last one partial (2048 tiles of an n = 4096 product are 13.5
// rounds of 152).  Those T mod G tiles run as two K halves each (split at a
// 512-k chunk boundary) on different CTAs; each draining warp writes its
// 32 x 32 region's int64 half to the workspace and counts the region, and
// the warp that counts it second adds the other half (the sum stays exact)
// and hands the region on, while the first hands on nothing.  No CTA waits
// for another.
// Every mbarrier wait is bounded; on expiry the CTA stops issuing, waits
// (bounded) for what it issued, frees TMEM and raises *err.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "internal.cuh"
#include "ozaki.h"
#include "sm100_ptx.cuh"

namespace cs {
namespace {

using namespace ptx;

constexpr int BM = 128;
constexpr int BN = 64;
// k per pipeline stage (BK bf16 = one swizzle row of 2 BK bytes): 32 for
// eight slices (64-byte swizzle, 2 stages of 96 KB; a 16-wide stage with
// 4 stages measured 5 % slower), 64 for four slices (128-byte swizzle,
// 2 stages of 96 KB).
__host__ __device__ constexpr int stage_k(int S) { return S == kOzakiSlicesSplit ? 64 : 32; }
constexpr int kEpiWarps = 8;  // drain TMEM into the int64 sums
constexpr int kFinWarps = 8;  // FP64 epilogue
constexpr int kThreads = 64 + 32 * (kEpiWarps + kFinWarps);
constexpr int kCols = BN / 2;          // columns per epilogue warp
constexpr int kGroupM = 8;             // M tiles per raster group
// TMA boxes of 256 rows: a tile's slices lie next to each other in global
// memory (and in a stage), so one box carries two A slices (2 x 128 rows) or
// four B slices (4 x 64 rows): 6 loads per stage instead of 16 for S = 8.
constexpr int kBoxRows = 256;
// Per slice count S: all S slices of A and B^T of one k-block form a stage,
// 192 KB of stages are in flight, and the S level accumulators of BN columns
// fill S BN TMEM columns.
__host__ __device__ constexpr int a_slice_bytes(int S) { return BM * stage_k(S) * 2; }  // one A slice of a stage
__host__ __device__ constexpr int b_slice_bytes(int S) { return BN * stage_k(S) * 2; }  // one B slice of a stage
__host__ __device__ constexpr int stage_bytes(int S) { return S * (a_slice_bytes(S) + b_slice_bytes(S)); }
__host__ __device__ constexpr int num_stages(int S) { return (192 * 1024) / stage_bytes(S); }
__host__ __device__ constexpr int smem_bytes(int S) {
  return num_stages(S) * stage_bytes(S) + 1024;
}
static_assert(smem_bytes(kOzakiSlices) <= 227 * 1024 && smem_bytes(kOzakiSlicesSplit) <= 227 * 1024,
              "shared memory");
static_assert(kOzakiSlices * BN == 512 && kOzakiSlicesSplit * BN == 256, "TMEM columns: a power of two <= 512");
// Instruction descriptors, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
// An N = w BN instruction reads the B slices q .. q + w - 1, which lie next
// to each other along N in shared memory, and writes the accumulators of
// levels p + q .. p + q + w - 1, which lie next to each other in TMEM: w
// slice pairs per instruction (a 128 x 64 x 16 MMA runs at 2/3 of the tensor
// peak on GB300, 128 x 128 x 16 at the peak), and A is read once per w pairs.
constexpr uint32_t kIdesc1 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t kIdesc2 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * BN) >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t kIdesc4 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((4 * BN) >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
// The slice products of A slice p with the B slices q in [qb, qe), in runs
// of 4, 2 and 1 adjacent slices (run grp starts at run_start, spans
// run_width, 0 past the last), one instruction each; a wider instruction
// reads the A operand from shared memory once for more slice pairs.
__host__ __device__ constexpr int run_of(int left) { return left >= 4 ? 4 : left >= 2 ? 2 : left >= 1 ? 1 : 0; }
__host__ __device__ constexpr int run_start(int qb, int qe, int grp) {
  int q = qb;
  for (int i = 0; i < grp; ++i) q += run_of(qe - q);
  return q;
}
__host__ __device__ constexpr int run_width(int qb, int qe, int grp) { return run_of(qe - run_start(qb, qe, grp)); }
// The B slices of A slice p in phase ph: all of them with one phase, else the
// levels p + q below S / 2 (ph = 0) or from S / 2 on (ph = 1).
__host__ __device__ constexpr int phase_q_begin(int S, int phases, int ph, int p) {
  return phases == 1 || ph == 0 ? 0 : (S / 2 - p > 0 ? S / 2 - p : 0);
}
__host__ __device__ constexpr int phase_q_end(int S, int phases, int ph, int p) {
  return phases == 1 || ph == 1 ? S - p : (S / 2 - p > 0 ? S / 2 - p : 0);
}
static_assert(run_width(0, 7, 0) == 4 && run_width(0, 7, 1) == 2 && run_width(0, 7, 2) == 1 &&
                  run_start(0, 7, 2) == 6 && run_width(0, 8, 2) == 0 && run_width(3, 7, 0) == 4 &&
                  phase_q_begin(8, 2, 1, 1) == 3 && phase_q_end(8, 2, 0, 1) == 3 && phase_q_end(8, 2, 0, 5) == 0,
              "slice runs");

// Shared-memory descriptors (built in the MMA loop): K-major, 64-byte
// swizzle, rows of 64 bytes, 8-row (512-byte) atoms stacked along M/N
// (stride byte offset 512), version 1, base offset 0 (tiles 1024-aligned).

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}


// ------------------------------------------------------------- slicing ---
// Exponent e with |x| * 2^-e < 1 for every x of the line: frexp of the max.
__device__ __forceinline__ int line_exponent(double mx) {
  int e = 0;
  if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
  return e;
}

// S slices of x relative to the line exponent e (|x| < 2^e), by integer
// arithmetic on the FP64 bit pattern (FP64 arithmetic is slow on GB300):
// x 2^-e is rounded to the 57-bit fixed-point integer R = x 2^(56 - e)
// (|R| < 2^56), then cut from the top into balanced base-2^7 digits
// a_p = round(R_p / 2^(49 - 7p)), R_{p+1} = R_p - a_p 2^(49 - 7p), the last
// digit taking the exact remainder: |a_0| <= 128, |a_p| <= 64.  Slice p is
// stored as the BF16 value a_p 2^(-7p) (exact).
template <int S>
__device__ __forceinline__ void cut(double x, int e, __nv_bfloat16 (&q)[S]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)((bits >> 52) & 0x7FF);
  const unsigned long long frac = bits & ((1ULL << 52) - 1);
  const long long mant = (long long)(eb ? (frac | (1ULL << 52)) : frac);  // x = mant 2^(max(eb,1) - 1075)
  const int sh = (eb ? eb : 1) - 1075 - e + 7 * S;  // R = mant 2^sh
  long long R;
  if (sh >= 0)
    R = mant << sh;  // below 2^(7S) since |x| < 2^e
  else if (sh > -63)
    R = (mant + (1LL << (-sh - 1))) >> (-sh);
  else
    R = 0;
  if (bits >> 63) R = -R;
#pragma unroll
  for (int p = 0; p < S; ++p) {
    const int pos = 7 * (S - 1 - p);
    long long a;
    if (p < S - 1) {
      a = (R + (1LL << (pos - 1))) >> pos;  // arithmetic shift: round half up
      R -= a << pos;
    } else {
      a = R;
    }
    q[p] = __float2bfloat16_rn((float)(int)a * __int_as_float((127 - 7 * p) << 23));  // a 2^(-7p)
  }
}

// Row maxima of |X| (rows x cols, leading dimension ld) without the entry
// X[r][r mod cols], which goes to xd[r]: one warp per row.
__global__ void __launch_bounds__(256) row_exp_kernel(const double* __restrict__ X, int64_t rows, int64_t cols,
                                                      int64_t ld, int* __restrict__ ex, double* __restrict__ xd,
                                                      int64_t bsx, int64_t rows_pad) {
  const int64_t row = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= rows) return;
  X += (int64_t)blockIdx.y * bsx;  // matrix blockIdx.y of a batch
  ex += (int64_t)blockIdx.y * rows_pad;
  xd += (int64_t)blockIdx.y * rows_pad;
  const int64_t d = row % cols;
  double mx = 0.0;
  for (int64_t c = lane; c < cols; c += 32)
    if (c != d) mx = fmax(mx, fabs(X[row * ld + c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    ex[row] = line_exponent(mx);
    xd[row] = X[row * ld + d];
  }
}

// Column maxima of |Y| as ordered bit patterns (non-negative doubles compare
// like their bits): atomicMax into colmax[cols], which starts at zero.
// (Y is square here: the entry Y[c][c] is left out and goes to yd[c].)
__global__ void __launch_bounds__(256) col_max_kernel(const double* __restrict__ Y, int64_t rows, int64_t cols,
                                                      int64_t ld, unsigned long long* __restrict__ colmax,
                                                      int64_t bsy, int64_t cols_pad) {
  const int64_t c = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (c >= cols) return;
  Y += (int64_t)blockIdx.z * bsy;
  colmax += (int64_t)blockIdx.z * cols_pad;
  const int64_t r0 = (int64_t)blockIdx.y * 256;
  const int64_t r1 = std::min<int64_t>(rows, r0 + 256);
  double mx = 0.0;
  for (int64_t r = r0; r < r1; ++r)
    if (r != c) mx = fmax(mx, fabs(Y[r * ld + c]));
  atomicMax(colmax + c, (unsigned long long)__double_as_longlong(mx));
}

__global__ void col_exp_kernel(const double* __restrict__ Y, int64_t ld, const unsigned long long* __restrict__ colmax,
                               int64_t cols, int* __restrict__ ex, double* __restrict__ yd, int64_t bsy,
                               int64_t cols_pad, int* __restrict__ zero, int64_t nzero) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.y == 0)  // the product kernel's piece counters start at zero
    for (int64_t i = c; i < nzero; i += (int64_t)gridDim.x * blockDim.x) zero[i] = 0;
  Y += (int64_t)blockIdx.y * bsy;
  colmax += (int64_t)blockIdx.y * cols_pad;
  ex += (int64_t)blockIdx.y * cols_pad;
  yd += (int64_t)blockIdx.y * cols_pad;
  if (c < cols) {
    ex[c] = line_exponent(__longlong_as_double((long long)colmax[c]));
    yd[c] = Y[c * ld + c];
  }
}

// Left operand: out[b][t][s][i][k] for row r = t BM + i < rows_pad (tile t
// of BM rows, its S slices next to each other so that one TMA box carries
// several), k < ldk (K contiguous), matrix b = blockIdx.y of a batch; rows
// >= rows and k >= cols are zero.
template <int S>
__global__ void __launch_bounds__(256) slice_rows_kernel(const double* __restrict__ X, int64_t rows, int64_t cols,
                                                         int64_t ld, const int* __restrict__ ex,
                                                         __nv_bfloat16* __restrict__ out, int64_t rows_pad,
                                                         int64_t ldk, int64_t bsx) {
  const int64_t plane = rows_pad * ldk;
  X += (int64_t)blockIdx.y * bsx;
  ex += (int64_t)blockIdx.y * rows_pad;
  out += (int64_t)blockIdx.y * S * plane;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < plane; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / ldk, k = i - r * ldk;
    __nv_bfloat16 q[S];
    const double x = (r < rows && k < cols && k != r % cols) ? X[r * ld + k] : 0.0;
    cut(x, r < rows ? ex[r] : 0, q);
    const int64_t t = r / BM, ri = r - t * BM;
    __nv_bfloat16* o = out + ((t * S) * BM + ri) * ldk + k;
#pragma unroll
    for (int s = 0; s < S; ++s) o[(int64_t)s * BM * ldk] = q[s];
  }
}

// Right operand Y (rows = K, cols = N, row-major): out[t][s][j][k] for column
// c = t BN + j < cols_pad, the transposed slices (K contiguous, the S slices
// of a BN-column tile next to each other), k < ldk, through a 32 x 32
// shared-memory tile per slice.
template <int S>
__global__ void __launch_bounds__(256) slice_cols_kernel(const double* __restrict__ Y, int64_t rows, int64_t cols,
                                                         int64_t ld, const int* __restrict__ ex,
                                                         __nv_bfloat16* __restrict__ out, int64_t cols_pad,
                                                         int64_t ldk, int64_t bsy) {
  __shared__ __nv_bfloat16 tile[S][32][34];
  Y += (int64_t)blockIdx.z * bsy;
  ex += (int64_t)blockIdx.z * cols_pad;
  out += (int64_t)blockIdx.z * S * cols_pad * ldk;
  const int64_t k0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  for (int j = ty; j < 32; j += 8) {
    const int64_t k = k0 + j, c = c0 + tx;
    const double y = (k < rows && c < cols && k != c) ? Y[k * ld + c] : 0.0;
    __nv_bfloat16 q[S];
    cut(y, c < cols ? ex[c] : 0, q);
#pragma unroll
    for (int s = 0; s < S; ++s) tile[s][j][tx] = q[s];
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t c = c0 + j, k = k0 + tx;
    if (c >= cols_pad || k >= ldk) continue;
    const int64_t t = c / BN, ci = c - t * BN;
    __nv_bfloat16* o = out + ((t * S) * BN + ci) * ldk + k;
#pragma unroll
    for (int s = 0; s < S; ++s) o[(int64_t)s * BN * ldk] = tile[s][tx][j];
  }
}

// ---------------------------------------------------------------- product ---
__device__ __forceinline__ double pow2(int e) {
  if (e > -1023 && e < 1024) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

// Persistent: CTA i takes the tiles i, i + gridDim.x, ... of the batch's
// (matrix, tile) list.  Pipeline stages and chunks are counted across tiles,
// so the producer and the MMA warp run on into the next tile while the
// epilogue warps finish the previous one (its accumulators are released
// before the FP64 epilogue, which stages through its own shared memory).
template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_kernel(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, int M, int N, int K,
                 int Mpad, int Npad, const int* __restrict__ ex_all, const int* __restrict__ fx_all,
                 const double* __restrict__ X_all, int64_t ldx, const double* __restrict__ Y_all, int64_t ldy,
                 const double* __restrict__ xd_all, const double* __restrict__ yd_all, int64_t ldo,
                 const __grid_constant__ Epilogue<double> epi, int* err, int64_t bsx, int64_t bsy, int64_t bse,
                 int batch, double* __restrict__ hand, long long* __restrict__ pieces, int* __restrict__ piece_cnt) {
  constexpr int kAcc = S;  // one accumulator of BN columns per level p + q < S
  constexpr int BK = stage_k(S);
  constexpr int kSwizzleBytes = BK * 2;  // one swizzle row = one stage row
  constexpr int kChunkKb = 512 / BK;     // k-blocks per 512-k accumulator chunk
  constexpr int kABytes = a_slice_bytes(S);
  constexpr int kBBytes = b_slice_bytes(S);
  constexpr int kBoxBytes = kBoxRows * BK * 2;
  constexpr int kStageBytes = stage_bytes(S);
  constexpr int kStages = num_stages(S);
  // Two sets of level accumulators when they fit in the 512 TMEM columns
  // (S = 4): the MMAs of chunk c + 1 run while the epilogue drains chunk c.
  constexpr int kBufs = 2 * S * BN <= 512 ? 2 : 1;
  constexpr uint32_t kTmemCols = (uint32_t)(S * BN * kBufs);
  constexpr int kPhases = kBufs == 1 ? 2 : 1;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t chunk_bar[kBufs];
  __shared__ __align__(8) uint64_t free_bar[kBufs][kAcc];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ __align__(8) uint64_t hand_full[2];  // a tile's sums are in scratch slot t % 2
  __shared__ __align__(8) uint64_t hand_free[2];  // the FP64 epilogue is done with the slot
  __shared__ int hand_skip[2];  // per slot: bit w = region of draining warp w finished elsewhere
  __shared__ int kb_consumed;
  __shared__ int chunks_committed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nM = Mpad / BM, nN = Npad / BN;
  const int tiles_per_matrix = nM * nN;
  const int total = tiles_per_matrix * batch;
  const int num_kb = (K + BK - 1) / BK;
  const int num_chunks = (num_kb + kChunkKb - 1) / kChunkKb;
  // Tile t of a matrix: groups of kGroupM rows of M tiles, N fastest within a
  // group, so that the CTAs resident at once share their slices in L2.
  auto tile_of = [&](int u, int& bat, int& m0, int& n0) {
    bat = u / tiles_per_matrix;
    const int t = u - bat * tiles_per_matrix;
    const int group = t / (kGroupM * nN);
    const int rows = min(kGroupM, nM - group * kGroupM);
    const int within = t - group * kGroupM * nN;
    m0 = (group * kGroupM + within % rows) * BM;
    n0 = (within / rows) * BN;
  };
  // Work items: the whole tiles, then (with `pieces`) the tiles of the last,
  // partial round of the persistent grid as two K halves each (split at a
  // chunk boundary), so that the last round spreads over every CTA.  Each
  // draining warp writes its region of a half to `pieces`; of the two CTAs
  // that hold a region's halves, the second to count it in piece_cnt adds
  // the other half and hands the region on, the first hands on nothing.
  const int tail = (pieces != nullptr && num_chunks >= 2 && total > (int)gridDim.x) ? total % (int)gridDim.x : 0;
  const int whole = total - tail;
  const int items = whole + 2 * tail;
  const int half_kb = (num_chunks / 2) * kChunkKb;
  auto item_of = [&](int v, int& u, int& kb0, int& kb1, int& piece) {
    if (v < whole) {
      u = v;
      kb0 = 0;
      kb1 = num_kb;
      piece = -1;
    } else {
      const int w = v - whole;
      u = whole + (w >> 1);
      piece = w & 1;
      kb0 = piece ? half_kb : 0;
      kb1 = piece ? num_kb : half_kb;
    }
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&chunk_bar[b], 1);
      for (int a = 0; a < kAcc; ++a) mbar_init(&free_bar[b][a], kEpiWarps);
    }
    abort_flag = 0;
    for (int h = 0; h < 2; ++h) {
      mbar_init(&hand_full[h], kEpiWarps);
      mbar_init(&hand_free[h], kFinWarps);
      hand_skip[h] = 0;
    }
    kb_consumed = 0;
    chunks_committed = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(&tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int kb_issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      tma_prefetch(&mA);
      tma_prefetch(&mB);
      int g = 0;  // k-blocks issued so far, over all tiles
      for (int v = blockIdx.x; v < items && !abort_flag; v += gridDim.x) {
        int u, kb0, kb1, piece;
        item_of(v, u, kb0, kb1, piece);
        int bat, m0, n0;
        tile_of(u, bat, m0, n0);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int st = g % kStages;
          if (g >= kStages && !mbar_wait(&empty_bar[st], ((g / kStages) & 1) ^ 1, &abort_flag)) {
            abort_flag = 1;
            break;
          }
          uint8_t* base = smem + st * kStageBytes;
          mbar_arrive_expect_tx(&full_bar[st], kStageBytes);
          // the S slices of tile (m0, n0): rows a_row0 .. + S BM of the A
          // slices, b_row0 .. + S BN of the B slices
          const int a_row0 = (bat * nM + m0 / BM) * S * BM, b_row0 = (bat * nN + n0 / BN) * S * BN;
#pragma unroll
          for (int h = 0; h < S * BM / kBoxRows; ++h)
            tma_load_2d(base + h * kBoxBytes, &mA, &full_bar[st], kb * BK, a_row0 + h * kBoxRows);
#pragma unroll
          for (int h = 0; h < S * BN / kBoxRows; ++h)
            tma_load_2d(base + S * kABytes + h * kBoxBytes, &mB, &full_bar[st], kb * BK, b_row0 + h * kBoxRows);
          kb_issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // Descriptor words: the low word carries the start address (>> 4) and
      // LBO = 1, the high word SBO = 8 rows x swizzle bytes, version 1 and
      // the swizzle mode (6 = 32-byte, 4 = 64-byte); every operand of a stage
      // is at a compile-time offset from the stage base, so each MMA costs
      // two integer adds to issue.
      constexpr uint32_t kDescHi =
          ((uint32_t)(8 * kSwizzleBytes) >> 4) | (1u << 14) |
          ((kSwizzleBytes == 32 ? 6u : kSwizzleBytes == 64 ? 4u : 2u) << 29);
      int g = 0;   // k-blocks consumed so far, over all tiles
      int cg = 0;  // chunks committed so far, over all tiles
      for (int v = blockIdx.x; v < items && !abort_flag; v += gridDim.x) {
        int u, kb0, kb1, piece;
        item_of(v, u, kb0, kb1, piece);
        int kb = kb0;
        for (int c = kb0 / kChunkKb; c * kChunkKb < kb1 && !abort_flag; ++c, ++cg) {
          for (int kk = 0; kk < kChunkKb && kb < kb1; ++kk, ++kb, ++g) {
            const int st = g % kStages;
            if (!mbar_wait(&full_bar[st], (g / kStages) & 1, &abort_flag)) {
              abort_flag = 1;
              break;
            }
            tc_fence_after();
            const uint32_t a_lo = ((smem_u32(smem + st * kStageBytes) & 0x3FFFFu) >> 4) | (1u << 16);
            const uint32_t b_lo = a_lo + (uint32_t)((S * kABytes) >> 4);
            const bool chunk_start = kk == 0;
            // chunk cg accumulates into set cg % kBufs, which chunk
            // cg - kBufs used before; the epilogue must have read that one
            const int buf = cg % kBufs;
            const uint32_t acc0 = tmem + (uint32_t)(buf * S * BN);
            const bool wait_free = kk == 0 && cg >= kBufs;
            const uint32_t free_par = (uint32_t)((cg / kBufs - 1) & 1);
            bool stop = false;
            // With one set of accumulators (S = 8) a stage's MMAs run in two
            // phases, levels below S / 2 for every k-step, then the rest: at
            // a chunk start the first phase needs only the lower levels back
            // from the draining warps, which free them first.
#pragma unroll
            for (int ph = 0; ph < kPhases; ++ph) {
#pragma unroll
              for (int j = 0; j < BK / 16; ++j) {  // K = 16 bf16 (32 bytes) per instruction
#pragma unroll
                for (int p = 0; p < S; ++p) {
                  const int qb = phase_q_begin(S, kPhases, ph, p), qe = phase_q_end(S, kPhases, ph, p);
                  if (qb >= qe) continue;
                  const uint64_t ad =
                      ((uint64_t)kDescHi << 32) | (uint64_t)(a_lo + (uint32_t)((p * kABytes + 32 * j) >> 4));
                  // B slices q .. q + w - 1 in one N = w BN instruction into
                  // the accumulators of levels p + q .. p + q + w - 1 < S
#pragma unroll
                  for (int grp = 0; grp < 3; ++grp) {
                    const int w = run_width(qb, qe, grp);
                    if (w == 0) break;
                    const int q = run_start(qb, qe, grp);
                    const uint64_t bd =
                        ((uint64_t)kDescHi << 32) | (uint64_t)(b_lo + (uint32_t)((q * kBBytes + 32 * j) >> 4));
                    // p = 0 touches each level of a phase first: there a chunk
                    // restarts its accumulators, after the epilogue has read them
                    const bool restart = chunk_start && j == 0 && p == 0;
                    if (restart && wait_free) {
                      bool freed = true;
#pragma unroll
                      for (int l = 0; l < 4; ++l)
                        if (l < w) freed = freed && mbar_wait(&free_bar[buf][q + l], free_par, &abort_flag);
                      if (!freed) {
                        abort_flag = 1;
                        stop = true;
                        break;
                      }
                      tc_fence_after();
                    }
                    mma_bf16(acc0 + (uint32_t)((p + q) * BN), ad, bd, w == 4 ? kIdesc4 : w == 2 ? kIdesc2 : kIdesc1,
                             restart ? 0u : 1u);
                  }
                  if (stop) break;
                }
                if (stop) break;
              }
              if (stop) break;
            }
            if (stop) break;
            mma_commit(&empty_bar[st]);
            kb_consumed = g + 1;
          }
          mma_commit(&chunk_bar[cg % kBufs]);  // also tracks the MMAs of an aborted chunk
          chunks_committed = cg + 1;
        }
      }
    }
  } else if (warp < 2 + kEpiWarps) {
    const int quarter = warp & 3;                // TMEM lanes 32*quarter .. +31
    const int col0 = ((warp - 2) >> 2) * kCols;  // this warp's 32 columns
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int region = quarter + 4 * ((warp - 2) >> 2);  // rows 32 quarter.., columns col0..
    int cg = 0;  // chunks drained so far, over all items
    int t = 0;   // items handed over so far
    for (int v = blockIdx.x; v < items; v += gridDim.x, ++t) {
      int u, kb0, kb1, piece;
      item_of(v, u, kb0, kb1, piece);
      // Fixed-point sums with quantum 2^-35 of the slice products: each
      // chunk's level-L value (L <= 5) is an integer multiple of 2^(-7L) below
      // 2^24 quanta and converts exactly; levels 6, 7 are rounded to 2^-35.
      // For K <= 8192 the sum stays below 2^63.
      long long acc[kCols];
#pragma unroll
      for (int j = 0; j < kCols; ++j) acc[j] = 0;
      bool ok = true;
      for (int c = kb0 / kChunkKb; c * kChunkKb < kb1; ++c, ++cg) {
        int w = 1;
        if (lane == 0) {
          w = mbar_wait(&chunk_bar[cg % kBufs], (cg / kBufs) & 1, &abort_flag) && !abort_flag;
          if (!w) abort_flag = 1;
        }
        w = __shfl_sync(0xffffffffu, w, 0);
        if (!w) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll 1
        for (int a = 0; a < kAcc; ++a) {
          uint32_t v0[16], v1[16];
          const uint32_t tq = tmem + lane_off + (uint32_t)((cg % kBufs) * S * BN + a * BN + col0);
          tmem_ld16(tq, v0);
          tmem_ld16(tq + 16u, v1);
          tmem_ld_wait();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&free_bar[cg % kBufs][a]);
          const int e = 7 * a < 35 ? 7 * a : 35;  // value * 2^e is an integer (rounded for levels > 5)
          const float sc = __int_as_float((127 + e) << 23);
          const long long unit = 1LL << (35 - e);
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            acc[j] += (long long)__float2int_rn(__uint_as_float(v0[j]) * sc) * unit;
            acc[16 + j] += (long long)__float2int_rn(__uint_as_float(v1[j]) * sc) * unit;
          }
        }
      }
      // A K half of a split tile: write this region's half; the warp that
      // counts the region second adds the other half and hands it on.
      bool mine = true;
      if (ok && piece >= 0) {
        const int q = u - whole;
        long long* __restrict__ own = pieces + (((int64_t)q * 2 + piece) * BM + quarter * 32 + lane) * BN + col0;
#pragma unroll
        for (int j = 0; j < kCols; j += 2) *reinterpret_cast<longlong2*>(own + j) = make_longlong2(acc[j], acc[j + 1]);
        __threadfence();
        __syncwarp();
        int second = 0;
        if (lane == 0) second = atomicAdd(&piece_cnt[q * kEpiWarps + region], 1);
        mine = __shfl_sync(0xffffffffu, second, 0) != 0;
        if (mine) {
          __threadfence();
          const long long* other = pieces + (((int64_t)q * 2 + (1 - piece)) * BM + quarter * 32 + lane) * BN + col0;
#pragma unroll
          for (int j = 0; j < kCols; j += 2) {
            const longlong2 o = __ldcg(reinterpret_cast<const longlong2*>(other + j));
            acc[j] += o.x;
            acc[j + 1] += o.y;
          }
        }
      }
      // Hand the sums to the finishing warps through this CTA's scratch slot
      // t % 2, once they are done with item t - 2 there, and go on to the
      // next item's chunks (a region handed on by the other CTA is marked
      // in hand_skip).
      if (ok && t >= 2) {
        int w = 1;
        if (lane == 0) {
          w = mbar_wait(&hand_free[t & 1], ((t >> 1) - 1) & 1, &abort_flag) && !abort_flag;
          if (!w) abort_flag = 1;
        }
        ok = __shfl_sync(0xffffffffu, w, 0) != 0;
      }
      if (!ok) break;
      if (mine) {
        double* __restrict__ hrow = hand + ((int64_t)(blockIdx.x * 2 + (t & 1)) * BM + quarter * 32 + lane) * BN + col0;
#pragma unroll
        for (int j = 0; j < kCols; j += 2)
          *reinterpret_cast<double2*>(hrow + j) = make_double2((double)acc[j], (double)acc[j + 1]);
        __threadfence();  // the sums reach L2, where the finishing warps read them
      }
      __syncwarp();
      if (lane == 0) {
        if (mine) atomicAnd(&hand_skip[t & 1], ~(1 << region));
        else atomicOr(&hand_skip[t & 1], 1 << region);
        mbar_arrive(&hand_full[t & 1]);
      }
    }
  } else {
    // FP64 epilogue of each tile from its scratch slot: warp fw walks rows
    // fw, fw + kFinWarps, ... with coalesced loads and stores.
    const int fw = warp - 2 - kEpiWarps;
    int t = 0;
    for (int v = blockIdx.x; v < items; v += gridDim.x, ++t) {
      int u, kb0, kb1, piece;
      item_of(v, u, kb0, kb1, piece);
      int w = 1;
      if (lane == 0) {
        w = mbar_wait(&hand_full[t & 1], (t >> 1) & 1, &abort_flag) && !abort_flag;
        if (!w) abort_flag = 1;
      }
      if (!__shfl_sync(0xffffffffu, w, 0)) break;
      // regions (row quarter, column half) that the other CTA finishes
      const int skip = *(volatile int*)&hand_skip[t & 1];
      int bat, m0, n0;
      tile_of(u, bat, m0, n0);
      const int* __restrict__ ex = ex_all + (int64_t)bat * Mpad;
      const int* __restrict__ fx = fx_all + (int64_t)bat * Npad;
      const double* __restrict__ xd = xd_all + (int64_t)bat * Mpad;
      const double* __restrict__ yd = yd_all + (int64_t)bat * Npad;
      const double* __restrict__ X = X_all + (int64_t)bat * bsx;
      const double* __restrict__ Y = Y_all + (int64_t)bat * bsy;
      const double* __restrict__ hslot = hand + (int64_t)(blockIdx.x * 2 + (t & 1)) * BM * BN;
      const int64_t eoff = (int64_t)bat * bse;
      // a plain product (one output, P itself) skips the linear combination
      const bool plain = epi.split_row < 0 && epi.n_out == 1 && epi.n_in == 0 && epi.alpha[0] == 1.0 &&
                         epi.gamma[0] == 0.0;
#pragma unroll 1
      for (int rl = fw; rl < BM; rl += kFinWarps) {
        const int r = m0 + rl;
        if (r >= M) break;
        const int er = ex[r] - 14 - 35;
        const int d = r % K;
        const double xdr = xd[r];
        const double* __restrict__ yrow = Y + (int64_t)d * ldy;
        const double* __restrict__ xrow = X + (int64_t)r * ldx;
#pragma unroll
        for (int h = 0; h < BN / 32; ++h) {
          const int cl = 32 * h + lane;
          const int cc = n0 + cl;
          if (cc >= N || ((skip >> ((rl >> 5) + 4 * h)) & 1)) continue;
          // P = X_off Y_off (slices) + X[r][d] Y[d][c] + X[r][c] Y[c][c] (c != d)
          const double dterm = cc != d ? xrow[cc] * yd[cc] : 0.0;
          const double p = fma(__ldcg(hslot + rl * BN + cl), pow2(er + fx[cc]), fma(xdr, yrow[cc], dterm));
          if (plain) {
            epi.out[0][eoff + (int64_t)r * ldo + cc] = p;
          } else if (epi.split_row >= 0) {
            const bool top = r < epi.split_row;
            const int64_t rr = top ? r : r - epi.split_row;
            const int o = top ? 0 : 1;
            epi.out[o][eoff + rr * ldo + cc] = fma(epi.alpha[o], p, rr == cc ? epi.gamma[o] : 0.0);
          } else {
            const int64_t idx = eoff + (int64_t)r * ldo + cc;
            double in[EPI_MAX_IN], o[EPI_MAX_OUT];
#pragma unroll
            for (int q = 0; q < EPI_MAX_IN; ++q) in[q] = q < epi.n_in ? epi.in[q][idx] : 0.0;
#pragma unroll
            for (int t2 = 0; t2 < EPI_MAX_OUT; ++t2) {
              if (t2 >= epi.n_out) break;
              double v = fma(epi.alpha[t2], p, r == cc ? epi.gamma[t2] : 0.0);
#pragma unroll
              for (int q = 0; q < EPI_MAX_IN; ++q)
                if (q < epi.n_in) v += epi.beta[t2][q] * in[q];
#pragma unroll
              for (int uu = 0; uu < EPI_MAX_OUT; ++uu)
                if (uu < t2) v += epi.delta[t2][uu] * o[uu];
              o[t2] = v;
            }
#pragma unroll
            for (int t2 = 0; t2 < EPI_MAX_OUT; ++t2) {
              if (t2 >= epi.n_out) break;
              epi.out[t2][idx] = o[t2];
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&hand_free[t & 1]);
    }
  }

  // Teardown: if a wait expired, wait (bounded) for the copies and MMAs this
  // CTA issued before freeing TMEM.
  __syncthreads();
  if (abort_flag) {
    if (warp == 0 && lane == 0) {
      volatile int never = 0;
      for (int g = kb_consumed; g < kb_issued; ++g) mbar_wait(&full_bar[g % kStages], (g / kStages) & 1, &never);
    }
    if (warp == 1 && lane == 0 && chunks_committed > 0) {
      volatile int never = 0;
      const int c = chunks_committed - 1;
      mbar_wait(&chunk_bar[c % kBufs], (c / kBufs) & 1, &never);
    }
    if (threadIdx.x == 0) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ------------------------------------------------------------ tensor maps ---
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Row-major BF16 matrix [rows][cols] (leading dimension ld elements), box of
// box_k columns x box_rows rows, swizzle of 2 box_k bytes (64 or 128).
cs_status make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_k,
                   int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(CS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (((uintptr_t)base & 15) || (ld * 2) % 16) return fail(CS_EINVAL, "TMA operand not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, box_k == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(CS_ECUDA, "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
  return CS_OK;
}

int grid_for(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 152 * 16); }

}  // namespace

OzakiDims ozaki_dims(int64_t M, int64_t N, int64_t K, int64_t batch, int slices) {
  OzakiDims d;
  d.Mpad = (M + BM - 1) / BM * BM;
  d.Npad = (N + BN - 1) / BN * BN;
  d.ldk = (K + 31) / 32 * 32;  // the slicing kernels work in 32 x 32 tiles
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t nb = (size_t)(batch > 0 ? batch : 1);
  const size_t S = (size_t)(slices > 0 ? slices : kOzakiSlices);
  d.a_bytes = al(nb * S * d.Mpad * d.ldk * 2);
  d.b_bytes = al(nb * S * d.Npad * d.ldk * 2);
  d.ex_bytes = al(nb * sizeof(int) * (size_t)d.Mpad);
  d.fx_bytes = al(nb * sizeof(int) * (size_t)d.Npad);
  d.colmax_bytes = al(nb * sizeof(unsigned long long) * (size_t)d.Npad);
  d.xd_bytes = al(nb * sizeof(double) * (size_t)d.Mpad);
  d.yd_bytes = al(nb * sizeof(double) * (size_t)d.Npad);
  // two tiles of sums per persistent CTA (at most one CTA per SM)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    sms = 256;
  const int64_t tiles = (int64_t)nb * (d.Mpad / BM) * (d.Npad / BN);
  d.hand_ctas = (int)std::min<int64_t>(tiles, sms);
  d.hand_bytes = al((size_t)d.hand_ctas * 2 * BM * BN * sizeof(double));
  // the K halves of the last round's tiles (fewer than one per CTA) and a
  // counter per region of each, when a tile has at least two 512-k chunks
  if (tiles > d.hand_ctas && K > 512) {
    d.split_tiles = d.hand_ctas - 1;
    d.piece_bytes = al((size_t)d.split_tiles * 2 * BM * BN * sizeof(long long));
    d.cnt_bytes = al((size_t)d.split_tiles * kEpiWarps * sizeof(int));
  }
  d.total = d.a_bytes + d.b_bytes + d.ex_bytes + d.fx_bytes + d.colmax_bytes + d.xd_bytes + d.yd_bytes + d.hand_bytes +
            d.piece_bytes + d.cnt_bytes;
  return d;
}

namespace {

// Slicing kernels and the product kernel for S slices (arguments checked by
// the caller).
template <int S>
cs_status launch_emu(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx, int64_t ldy,
                     const Epilogue<double>& epi, int64_t ldo, int64_t batch, int64_t bsx, int64_t bsy, int64_t bse,
                     const OzakiDims& d, char* w, int* err, cudaStream_t stream) {
  constexpr int kSmem = smem_bytes(S);
  __nv_bfloat16* a_sl = (__nv_bfloat16*)w;
  __nv_bfloat16* b_sl = (__nv_bfloat16*)(w + d.a_bytes);
  int* ex = (int*)(w + d.a_bytes + d.b_bytes);
  int* fx = (int*)(w + d.a_bytes + d.b_bytes + d.ex_bytes);
  unsigned long long* colmax = (unsigned long long*)(w + d.a_bytes + d.b_bytes + d.ex_bytes + d.fx_bytes);
  double* xd = (double*)((char*)colmax + d.colmax_bytes);
  double* yd = (double*)((char*)xd + d.xd_bytes);
  double* hand = (double*)((char*)yd + d.yd_bytes);
  long long* pieces = (long long*)((char*)hand + d.hand_bytes);
  int* piece_cnt = (int*)((char*)pieces + d.piece_bytes);
  const unsigned nb = (unsigned)batch;
  {
    ProfScope prof(CS_KERNEL_OTHER, (double)batch * (double)(M * K + K * N) * (8.0 + 2.0 * S), stream);
    row_exp_kernel<<<dim3((unsigned)((M + 7) / 8), nb), 256, 0, stream>>>(X, M, K, ldx, ex, xd, bsx, d.Mpad);
    CS_CUDA_CHECK(cudaMemsetAsync(colmax, 0, d.colmax_bytes, stream));
    col_max_kernel<<<dim3((unsigned)((N + 255) / 256), (unsigned)((K + 255) / 256), nb), 256, 0, stream>>>(
        Y, K, N, ldy, colmax, bsy, d.Npad);
    col_exp_kernel<<<dim3((unsigned)((N + 255) / 256), nb), 256, 0, stream>>>(
        Y, ldy, colmax, N, fx, yd, bsy, d.Npad, piece_cnt, (int64_t)(d.cnt_bytes / sizeof(int)));
    const unsigned sgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(grid_for(d.Mpad * d.ldk), 152 * 16 / batch + 1));
    slice_rows_kernel<S><<<dim3(sgrid, nb), 256, 0, stream>>>(X, M, K, ldx, ex, a_sl, d.Mpad, d.ldk, bsx);
    slice_cols_kernel<S><<<dim3((unsigned)(d.Npad / 32), (unsigned)(d.ldk / 32), nb), 256, 0, stream>>>(
        Y, K, N, ldy, fx, b_sl, d.Npad, d.ldk, bsy);
    CS_CUDA_CHECK(cudaGetLastError());
  }
  ProfScope prof(CS_KERNEL_GEMM_EMU, 2.0 * (double)batch * (double)M * (double)N * (double)K, stream);
  CUtensorMap mA, mB;
  static_assert(S * BM % kBoxRows == 0 && S * BN % kBoxRows == 0, "whole boxes of slices");
  CS_CHECK(make_map(&mA, a_sl, batch * S * d.Mpad, d.ldk, d.ldk, stage_k(S), kBoxRows));
  CS_CHECK(make_map(&mB, b_sl, batch * S * d.Npad, d.ldk, d.ldk, stage_k(S), kBoxRows));
  static std::atomic<unsigned long long> smem_set{0};
  CS_CHECK(smem_limit_once(ozaki_kernel<S>, kSmem, smem_set));
  const int64_t tiles = (d.Npad / BN) * (d.Mpad / BM) * batch;
  if (tiles > INT32_MAX) return fail(CS_EINVAL, "gemm_f64_emu: grid too large");
  int sms = 0, dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  CS_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)std::min<int64_t>(std::min<int64_t>(tiles, sms > 0 ? sms : 1), d.hand_ctas);
  // the last round's tiles split in K halves (the kernel takes tiles % grid
  // of them; col_exp_kernel zeroed their counters)
  const bool split = d.split_tiles > 0 && tiles > (int64_t)grid && tiles % grid != 0 &&
                     (int64_t)(tiles % grid) <= d.split_tiles;
  ozaki_kernel<S><<<grid, kThreads, kSmem, stream>>>(mA, mB, (int)M, (int)N, (int)K, (int)d.Mpad, (int)d.Npad, ex,
                                                     fx, X, ldx, Y, ldy, xd, yd, ldo, epi, err, bsx, bsy, bse,
                                                     (int)batch, hand, split ? pieces : nullptr,
                                                     split ? piece_cnt : nullptr);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace

cs_status gemm_f64_emu_batched(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx,
                               int64_t ldy, const Epilogue<double>& epi, int64_t ldo, int64_t batch, int64_t bsx,
                               int64_t bsy, int64_t bse, void* work, size_t work_bytes, int* err,
                               cudaStream_t stream, int slices) {
  if (slices != kOzakiSlices && slices != kOzakiSlicesSplit) return fail(CS_EINVAL, "gemm_f64_emu: slices must be 8 or 4");
  if (M <= 0 || N <= 0 || batch <= 0) return CS_OK;
  if (M > (1 << 20) || N > (1 << 20) || K > (1 << 20)) return fail(CS_EINVAL, "gemm_f64_emu: size too large");
  if (K <= 0 || N != K) return fail(CS_EINVAL, "gemm_f64_emu: the right operand must be square");
  if (K > kOzakiMaxK) return fail(CS_EINVAL, "gemm_f64_emu: K above 8192 (the int64 sums would overflow)");
  if (batch > 65535) return fail(CS_EINVAL, "gemm_f64_emu: batch above 65535");
  const OzakiDims d = ozaki_dims(M, N, K, batch, slices);
  if (!work || work_bytes < d.total || ((uintptr_t)work & 255)) return fail(CS_EINVAL, "gemm_f64_emu: workspace");
  if (!err) return fail(CS_ECUDA, "gemm_f64_emu: no device error word");
  if (batch * slices * d.Mpad > INT32_MAX || batch * slices * d.Npad > INT32_MAX)
    return fail(CS_EINVAL, "gemm_f64_emu: too large");
  if (slices == kOzakiSlicesSplit)
    return launch_emu<kOzakiSlicesSplit>(X, Y, M, N, K, ldx, ldy, epi, ldo, batch, bsx, bsy, bse, d, (char*)work, err,
                                         stream);
  return launch_emu<kOzakiSlices>(X, Y, M, N, K, ldx, ldy, epi, ldo, batch, bsx, bsy, bse, d, (char*)work, err,
                                  stream);
}

cs_status gemm_f64_emu(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx, int64_t ldy,
                       const Epilogue<double>& epi, int64_t ldo, void* work, size_t work_bytes, int* err,
                       cudaStream_t stream, int slices) {
  return gemm_f64_emu_batched(X, Y, M, N, K, ldx, ldy, epi, ldo, 1, 0, 0, 0, work, work_bytes, err, stream, slices);
}

namespace {
__global__ void __launch_bounds__(256) transpose_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                        int64_t n, int64_t bs) {
  __shared__ double tile[32][33];
  src += (int64_t)blockIdx.z * bs;
  dst += (int64_t)blockIdx.z * bs;
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int j = ty; j < 32; j += 8)
    if (r0 + j < n && c0 + tx < n) tile[j][tx] = src[(r0 + j) * n + c0 + tx];
  __syncthreads();
  for (int j = ty; j < 32; j += 8)
    if (c0 + j < n && r0 + tx < n) dst[(c0 + j) * n + r0 + tx] = tile[tx][j];
}
}  // namespace

cs_status transpose_f64_batched(const double* src, double* dst, int64_t n, int64_t batch, int64_t bs,
                                cudaStream_t stream) {
  if (n <= 0 || batch <= 0) return CS_OK;
  if (batch > 65535) return fail(CS_EINVAL, "transpose: batch above 65535");
  ProfScope prof(CS_KERNEL_OTHER, 16.0 * (double)batch * (double)n * (double)n, stream);
  const unsigned g = (unsigned)((n + 31) / 32);
  transpose_kernel<<<dim3(g, g, (unsigned)batch), 256, 0, stream>>>(src, dst, n, bs);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace cs
