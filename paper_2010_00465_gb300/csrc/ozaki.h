// ozaki.h -- FP64 products emulated on the BF16 tensor cores (gemm_ozaki.cu).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "internal.cuh"

namespace cs {

// 7-bit slices per operand.  8 slices carry 57 bits of each row / column
// maximum (FP64-class products, one 64-column TMEM accumulator per level, so
// at most 8); 4 slices carry 29 bits (FP32-class products for the Taylor
// chain of the split-precision form).
constexpr int kOzakiSlices = 8;
constexpr int kOzakiSlicesSplit = 4;

constexpr int64_t kOzakiMaxK = 8192;  // inner dimension limit of the int64 sums

// Scratch of one emulated product: the BF16 slices of both operands, their
// row / column exponents, the column maxima, two tiles of sums per CTA of the
// product kernel (at most one per SM of the current device), and the K
// halves of the tiles of its last round.
struct OzakiDims {
  int64_t Mpad = 0, Npad = 0, ldk = 0;
  size_t a_bytes = 0, b_bytes = 0, ex_bytes = 0, fx_bytes = 0, colmax_bytes = 0, xd_bytes = 0, yd_bytes = 0;
  size_t hand_bytes = 0;
  int hand_ctas = 0;
  int64_t split_tiles = 0;  // at most this many last-round tiles split in K halves
  size_t piece_bytes = 0, cnt_bytes = 0;
  size_t total = 0;
};
OzakiDims ozaki_dims(int64_t M, int64_t N, int64_t K, int64_t batch = 1, int slices = kOzakiSlices);

// P = X Y (X: M x K, Y: K x K, row-major FP64; M = K or the stacked 2K) with
// the fused FP64 epilogue of gemm_f64 (stacked mode included); the entries
// X[r][r mod K] and Y[c][c] are added exactly in FP64, the rest is emulated.
// `work` holds ozaki_dims(M, N, K, 1, slices).total bytes (256-byte
// aligned); `slices` is kOzakiSlices or kOzakiSlicesSplit.  A bounded wait
// that expires raises *err.
cs_status gemm_f64_emu(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx, int64_t ldy,
                       const Epilogue<double>& epi, int64_t ldo, void* work, size_t work_bytes, int* err,
                       cudaStream_t stream, int slices = kOzakiSlices);

// The same over `batch` independent products: operand b at X + b bsx and
// Y + b bsy, every epilogue matrix at + b bse; `work` holds
// ozaki_dims(M, N, K, batch, slices).total bytes.
cs_status gemm_f64_emu_batched(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx,
                               int64_t ldy, const Epilogue<double>& epi, int64_t ldo, int64_t batch, int64_t bsx,
                               int64_t bsy, int64_t bse, void* work, size_t work_bytes, int* err,
                               cudaStream_t stream, int slices = kOzakiSlices);

// dst_b = src_b^T for `batch` n x n row-major FP64 matrices at stride bs (dst
// must not overlap src).
cs_status transpose_f64_batched(const double* src, double* dst, int64_t n, int64_t batch, int64_t bs,
                                cudaStream_t stream);

}  // namespace cs
