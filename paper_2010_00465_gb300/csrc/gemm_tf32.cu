// gemm_tf32.cu -- four-pass TF32 tensor-core product on tcgen05/TMEM with
// TMA-fed operands and the method's linear combinations fused in the epilogue.
//
// FP32 accuracy from TF32 tensor cores: every matrix is held as a pair
// (hi, lo) of TF32 values, hi = tf32(x) and lo = tf32(x - hi) (22 significant
// bits together), and the product is
//   X Y = X_hi Y_hi + (X_lo Y_hi + X_hi Y_lo + X_lo Y_lo)
// with FP32 accumulation.  The epilogue that produces a matrix also writes its
// (hi, lo) split and, for matrices later used as a right operand, the
// transposed split, so both operands are always fed K-major.
//
// Tensor-core FP32 accumulation is not IEEE: every MMA adds into the TMEM
// accumulator with truncation, so the error of a long accumulation grows
// linearly with K and is biased toward zero (measured on GB300: 4e-5 relative
// at K = 4096, against 1e-6 for an FP32 FFMA product).  The kernel therefore
//   * accumulates X_hi Y_hi and the correction passes in separate TMEM
//     accumulators, so the small terms are not truncated against the large
//     sum; the corrections (2^-11 of the main term) accumulate over the whole
//     K, where their own truncation stays far below FP32 rounding of the sum;
//   * starts a fresh main accumulator every kGroup k-blocks (128 k) and
//     promotes it into Kahan-compensated FP32 register sums (two TMEM buffers
//     ping-pong, so the tensor pipe keeps running while one is drained).
//     Promoting every 32 k kept the error at 1.4e-7 (K = 4096) but the MMAs
//     then waited for the drains: 1.09 ms per n = 4096 product against
//     0.95 ms every 64 k (2.0e-7), 0.84 ms every 128 k (3.4e-7) and 0.78 ms
//     every 256 k (6.4e-7, not taken: the error nearly doubles for 6 %).
//
// One CTA computes a 128 x 128 tile:
//   warp 0     TMA producer: X_hi, X_lo (128 x 32) and Y^T_hi, Y^T_lo
//              (128 x 32) per stage into 128-byte-swizzled shared memory;
//   warp 1     allocates 512 TMEM columns (main x 2 buffers, corrections); one lane
//              issues the MMAs (cta_group::1, M = N = 128, K = 8 per
//              instruction) and commits stages and accumulator buffers;
//   warps 2-9  two per TMEM lane quarter, 64 columns each: drain each main
//              accumulator buffer into Kahan-compensated FP32 register sums
//              (compensation terms in TMEM), then run the epilogue: linear
//              combinations, (hi, lo) split, row-major and transposed stores.
// Measured on GB300 (N(0,1) operands): relative Frobenius error of one
// product 3.4e-7 at K = 4096 (1.3e-7 at K = 256, where one group covers all
// of K), against 1.2e-6 and 2.9e-7 for cuBLAS FP32 (FFMA).
// Every mbarrier wait is bounded; on expiry the CTA stops issuing work, waits
// (bounded) for what it already issued, frees TMEM and raises *err.
#include <cuda.h>

#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "tc_gemm.h"

namespace cs {
namespace {

using namespace ptx;

constexpr int BM = 128;
constexpr int BN = 128;
constexpr int BK = 32;  // 32 floats = 128 bytes = one swizzle row
#ifndef COSSIN_TC_EPI_WARPS
#define COSSIN_TC_EPI_WARPS 8
#endif
// Epilogue warps: kEpiWarps / 4 per TMEM lane quarter, kHalf columns each.
constexpr int kEpiWarps = COSSIN_TC_EPI_WARPS;
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr int kHalf = BN / (kEpiWarps / 4);
constexpr int kABytes = BM * BK * 4;
constexpr int kBBytes = BN * BK * 4;
constexpr int kStageBytes = 2 * (kABytes + kBBytes);
constexpr int kStages = 3;
constexpr int kSmem = kStages * kStageBytes + 1024;
static_assert(3 * BM * BN * 4 <= kStages * kStageBytes, "epilogue tiles fit the stages");
#ifndef COSSIN_TC_GROUP
#define COSSIN_TC_GROUP 4
#endif
constexpr int kGroup = COSSIN_TC_GROUP;  // k-blocks per accumulator buffer before promotion
constexpr uint32_t kTmemCols = 512;    // main buffer b at 128 b, corrections at 256, compensation at 384
// Instruction descriptor: D = F32 (bits 4-5), A = B = TF32 (bits 7-9, 10-12),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kIdesc =
    (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void split_store(float v, float* hi, float* lo, int64_t idx) {
  if (lo) {
    const float h = tf32_rna(v);
    hi[idx] = h;
    lo[idx] = COSSIN_LO(v - h);
  } else {
    hi[idx] = v;
  }
}

// The register file is split over 4 sub-partitions: with 10 warps (3 on two
// of them) a thread gets at most 168 registers, with 18 warps 96.
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tf32_kernel(const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
                     const __grid_constant__ CUtensorMap mYh, const __grid_constant__ CUtensorMap mYl, int M, int N,
                     int K, int ldo, const __grid_constant__ TcEpilogue epi, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[kStages];
  __shared__ __align__(8) uint64_t empty_bar[kStages];
  __shared__ __align__(8) uint64_t tfull_bar[2];
  __shared__ __align__(8) uint64_t tempty_bar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ int kb_consumed;
  __shared__ int groups_committed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int num_kb = (K + BK - 1) / BK;
  const int num_groups = (num_kb + kGroup - 1) / kGroup;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull_bar[b], 1);
      mbar_init(&tempty_bar[b], kEpiWarps);
    }
    abort_flag = 0;
    kb_consumed = 0;
    groups_committed = 0;
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
      tma_prefetch(&mXh);
      tma_prefetch(&mXl);
      tma_prefetch(&mYh);
      tma_prefetch(&mYl);
      for (int kb = 0; kb < num_kb; ++kb) {
        const int st = kb % kStages;
        if (kb >= kStages && !mbar_wait(&empty_bar[st], ((kb / kStages) & 1) ^ 1, &abort_flag)) {
          abort_flag = 1;
          break;
        }
        uint8_t* base = smem + st * kStageBytes;
        mbar_arrive_expect_tx(&full_bar[st], kStageBytes);
        tma_load_2d(base, &mXh, &full_bar[st], kb * BK, m0);
        tma_load_2d(base + kABytes, &mXl, &full_bar[st], kb * BK, m0);
        tma_load_2d(base + 2 * kABytes, &mYh, &full_bar[st], kb * BK, n0);
        tma_load_2d(base + 2 * kABytes + kBBytes, &mYl, &full_bar[st], kb * BK, n0);
        kb_issued = kb + 1;
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int kb = 0;
      for (int g = 0; g < num_groups && !abort_flag; ++g) {
        const int b = g & 1;
        if (g >= 2 && !mbar_wait(&tempty_bar[b], ((g >> 1) & 1) ^ 1, &abort_flag)) {
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d_main = tmem + 128u * b, d_corr = tmem + 256u;
        for (int kk = 0; kk < kGroup && kb < num_kb; ++kk, ++kb) {
          const int st = kb % kStages;
          if (!mbar_wait(&full_bar[st], (kb / kStages) & 1, &abort_flag)) {
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          // Descriptor words of desc_kmajor_sw128: the low word carries the
          // start address (>> 4) and LBO = 1; every operand of the stage is at
          // a compile-time offset from the stage base, so the per-MMA cost is
          // one integer add (the issuing thread is otherwise the bottleneck).
          constexpr uint32_t kDescHi = (1024u >> 4) | (1u << 14) | (2u << 29);
          const uint32_t base = ((smem_u32(smem + st * kStageBytes) & 0x3FFFFu) >> 4) | (1u << 16);
          auto desc = [&](uint32_t byte_off) { return ((uint64_t)kDescHi << 32) | (uint64_t)(base + (byte_off >> 4)); };
          const uint32_t fresh_main = kk != 0, fresh_corr = kb != 0;
#pragma unroll
          for (int j = 0; j < BK / 8; ++j) {  // K = 8 tf32 (32 bytes) per instruction
            const uint32_t off = 32u * j;
            const uint64_t ah = desc(off), al = desc(kABytes + off);
            const uint64_t bh = desc(2 * kABytes + off), bl = desc(2 * kABytes + kBBytes + off);
            mma_tf32(d_main, ah, bh, kIdesc, j ? 1u : fresh_main);  // fresh every group
            mma_tf32(d_corr, al, bh, kIdesc, j ? 1u : fresh_corr);  // whole K
            mma_tf32(d_corr, ah, bl, kIdesc, 1);
            mma_tf32(d_corr, al, bl, kIdesc, 1);
          }
          mma_commit(&empty_bar[st]);
          kb_consumed = kb + 1;
        }
        mma_commit(&tfull_bar[b]);  // also tracks the MMAs of an aborted group
        groups_committed = g + 1;
      }
    }
  } else {
    const int quarter = warp & 3;              // TMEM lanes 32*quarter .. +31
    const int col0 = ((warp - 2) >> 2) * kHalf;  // this warp's kHalf columns
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    // Kahan-compensated running sums of the promoted main partials: the
    // running sums stay in registers, their compensation terms in TMEM
    // columns 384..511 (read and rewritten every group), so the sum over K
    // adds essentially no FP32 rounding of its own.
    float acc_hi[kHalf];
#pragma unroll
    for (int c = 0; c < kHalf; ++c) acc_hi[c] = 0.f;
    const uint32_t t_comp = tmem + lane_off + 384u + (uint32_t)col0;
    bool ok = true;
    for (int g = 0; g < num_groups; ++g) {
      const int b = g & 1;
      // lane 0 waits and the warp follows its outcome, so the warp-collective
      // TMEM loads below are never reached by part of a warp
      int w = 1;
      if (lane == 0) {
        w = mbar_wait(&tfull_bar[b], (g >> 1) & 1, &abort_flag) && !abort_flag;
        if (!w) abort_flag = 1;
      }
      w = __shfl_sync(0xffffffffu, w, 0);
      if (!w) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t t_main = tmem + lane_off + 128u * b + (uint32_t)col0;
      // Read the whole main buffer first and release it to the MMA warp at
      // once; the compensated sums (TMEM columns 384..511, touched by the
      // epilogue only) are updated afterwards, off the MMA warp's path.
      uint32_t vm[kHalf / 8][8];
#pragma unroll
      for (int i = 0; i < kHalf / 8; ++i) tmem_ld8(t_main + (uint32_t)(8 * i), vm[i]);
      tmem_ld_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty_bar[b]);
#pragma unroll
      for (int i = 0; i < kHalf / 8; ++i) {
        uint32_t vc[8];
        if (g > 0) {
          tmem_ld8(t_comp + (uint32_t)(8 * i), vc);
          tmem_ld_wait();
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = 8 * i + j;
          const float lo = g > 0 ? __uint_as_float(vc[j]) : 0.f;
          const float y = __uint_as_float(vm[i][j]) - lo;
          const float t = acc_hi[c] + y;
          vc[j] = __float_as_uint((t - acc_hi[c]) - y);
          acc_hi[c] = t;
        }
        tmem_st8(t_comp + (uint32_t)(8 * i), vc);
      }
      tmem_st_wait();
    }
    // The epilogue runs through shared memory (the pipeline stages are idle
    // now): the tile P is staged row-per-thread, then walked row by row with
    // coalesced input reads and row-major stores, while outputs that are
    // also wanted transposed are staged again and written column by column.
    // (The thread-per-row epilogue took up to 44 % of a CTA's time in the
    // method's multi-output steps: its row-major accesses are uncoalesced.)
    // Tiles are 128 x 128 floats with an XOR swizzle (column ^ (row & 31)),
    // conflict-free for both access directions; tile 0 holds P and is reused
    // by the first transposed output, tiles 1 and 2 take the next two.
    float* tiles = (float*)smem;
    auto sw = [](int rl, int cl) { return rl * BN + (cl ^ (rl & 31)); };
    if (ok) {
      // sum = main (compensated) + corrections (accumulated over the whole
      // K in TMEM columns 256..383, complete since the last group's commit)
      const uint32_t t_corr = tmem + lane_off + 256u + (uint32_t)col0;
      const int rl = quarter * 32 + lane;
#pragma unroll
      for (int c0 = 0; c0 < kHalf; c0 += 8) {
        uint32_t vc[8], vk[8];
        tmem_ld8(t_corr + (uint32_t)c0, vc);
        tmem_ld8(t_comp + (uint32_t)c0, vk);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 8; ++j)
          tiles[sw(rl, col0 + c0 + j)] = acc_hi[c0 + j] + (__uint_as_float(vc[j]) - __uint_as_float(vk[j]));
      }
    }
    // transposed outputs staged in tiles 0..2 (more would be written directly)
    int tslot[EPI_MAX_OUT];
    int n_staged = 0;
#pragma unroll
    for (int t = 0; t < EPI_MAX_OUT; ++t) tslot[t] = (t < epi.n_out && epi.outT_hi[t] && n_staged < 3) ? n_staged++ : -1;
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
    const int we = warp - 2;
    if (!abort_flag) {
#pragma unroll 1
      for (int rl = we; rl < BM; rl += kEpiWarps) {
        const int r = m0 + rl;
        if (r >= M) break;
#pragma unroll 1
        for (int g = 0; g < BN / 32; ++g) {
          const int cl = 32 * g + lane;
          const int c = n0 + cl;
          if (c >= N) continue;
          const float p = tiles[sw(rl, cl)];
          if (epi.split_row >= 0) {
            const bool top = r < epi.split_row;
            const int rr = top ? r : r - (int)epi.split_row;
            const int t = top ? 0 : 1;
            const float val = epi.alpha[t] * p + (rr == c ? epi.gamma[t] : 0.f);
            split_store(val, epi.out_hi[t], epi.out_lo[t], (int64_t)rr * ldo + c);
            if (epi.outT_hi[t]) {
              if (tslot[t] >= 0)
                tiles[tslot[t] * BM * BN + sw(rl, cl)] = val;
              else
                split_store(val, epi.outT_hi[t], epi.outT_lo[t], (int64_t)c * ldo + rr);
            }
          } else {
            const int64_t idx = (int64_t)r * ldo + c;
            float in[EPI_MAX_IN], o[EPI_MAX_OUT];
#pragma unroll
            for (int q = 0; q < EPI_MAX_IN; ++q) {
              in[q] = 0.f;
              if (q < epi.n_in) {
                in[q] = epi.in_hi[q][idx];
                if (epi.in_lo[q]) in[q] += epi.in_lo[q][idx];
              }
            }
#pragma unroll
            for (int t = 0; t < EPI_MAX_OUT; ++t) {
              if (t >= epi.n_out) break;
              float val = epi.alpha[t] * p + (r == c ? epi.gamma[t] : 0.f);
#pragma unroll
              for (int q = 0; q < EPI_MAX_IN; ++q)
                if (q < epi.n_in) val = fmaf(epi.beta[t][q], in[q], val);
#pragma unroll
              for (int u = 0; u < EPI_MAX_OUT; ++u)
                if (u < t) val = fmaf(epi.delta[t][u], o[u], val);
              o[t] = val;
            }
#pragma unroll
            for (int t = 0; t < EPI_MAX_OUT; ++t) {
              if (t >= epi.n_out) break;
              split_store(o[t], epi.out_hi[t], epi.out_lo[t], idx);
              if (epi.outT_hi[t]) {
                if (tslot[t] >= 0)
                  tiles[tslot[t] * BM * BN + sw(rl, cl)] = o[t];
                else
                  split_store(o[t], epi.outT_hi[t], epi.outT_lo[t], (int64_t)c * ldo + r);
              }
            }
          }
        }
      }
    }
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
    if (!abort_flag) {
#pragma unroll 1
      for (int t = 0; t < EPI_MAX_OUT; ++t) {
        if (t >= epi.n_out || tslot[t] < 0) continue;
        const float* tile = tiles + tslot[t] * BM * BN;
#pragma unroll 1
        for (int cl = we; cl < BN; cl += kEpiWarps) {
          const int c = n0 + cl;
          if (c >= N) break;
#pragma unroll
          for (int g = 0; g < BM / 32; ++g) {
            const int rl = 32 * g + lane;
            const int r = m0 + rl;
            if (r >= M) continue;
            // stacked mode: only output 0 (rows below split_row) is transposed
            if (epi.split_row >= 0 && r >= epi.split_row) continue;
            split_store(tile[sw(rl, cl)], epi.outT_hi[t], epi.outT_lo[t], (int64_t)c * ldo + r);
          }
        }
      }
    }
  }

  // Teardown: if a wait expired, wait (bounded) for the copies and MMAs this
  // CTA issued before freeing TMEM.
  __syncthreads();
  if (abort_flag) {
    if (warp == 0 && lane == 0) {
      volatile int never = 0;
      for (int kb = kb_consumed; kb < kb_issued; ++kb)
        mbar_wait(&full_bar[kb % kStages], (kb / kStages) & 1, &never);
    }
    if (warp == 1 && lane == 0 && groups_committed > 0) {
      volatile int never = 0;
      const int g = groups_committed - 1;
      mbar_wait(&tfull_bar[g & 1], (g >> 1) & 1, &never);
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

// Row-major FP32 matrix [rows][cols] with leading dimension ld (floats), box of
// 32 columns x box_rows rows, 128-byte swizzle, zero fill outside.
cs_status make_map(CUtensorMap* m, const float* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(CS_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (((uintptr_t)base & 15) || (ld * 4) % 16) return fail(CS_EINVAL, "TMA operand not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 4)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(CS_ECUDA, "cuTensorMapEncodeTiled failed with CUresult " + std::to_string((int)r));
  return CS_OK;
}

cs_status launch(const TcOperand& X, const TcOperand& YT, int M, int N, int K, int ldo, const TcEpilogue& epi,
                 int* err, cudaStream_t stream) {
  CUtensorMap mXh, mXl, mYh, mYl;
  CS_CHECK(make_map(&mXh, X.hi, M, K, X.ld, BM));
  CS_CHECK(make_map(&mXl, X.lo, M, K, X.ld, BM));
  CS_CHECK(make_map(&mYh, YT.hi, N, K, YT.ld, BN));
  CS_CHECK(make_map(&mYl, YT.lo, N, K, YT.ld, BN));
  static std::atomic<unsigned long long> smem_set{0};
  CS_CHECK(smem_limit_once(gemm_tf32_kernel, kSmem, smem_set));
  dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
  gemm_tf32_kernel<<<grid, kThreads, kSmem, stream>>>(mXh, mXl, mYh, mYl, M, N, K, ldo, epi, err);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace

cs_status gemm_tf32(const TcOperand& X, const TcOperand& YT, int64_t M, int64_t N, int64_t K, int64_t ldo,
                    const TcEpilogue& epi, int* err, cudaStream_t stream) {
  if (M <= 0 || N <= 0) return CS_OK;
  if (M > (1 << 30) || N > (1 << 30) || K > (1 << 30)) return fail(CS_EINVAL, "gemm_tf32: size too large");
  ProfScope prof(CS_KERNEL_GEMM_TF32, 2.0 * (double)M * (double)N * (double)K, stream);
  return launch(X, YT, (int)M, (int)N, (int)K, (int)ldo, epi, err, stream);
}

}  // namespace cs
