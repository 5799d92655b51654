// tc_gemm.h -- the four-pass TF32 tensor-core product and its helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace cs {

// A matrix held as (hi, lo) = (tf32(x), tf32(x - tf32(x))), row-major, leading
// dimension ld floats (a multiple of 4 so that rows start 16-byte aligned).
struct TcOperand {
  const float* hi;
  const float* lo;
  int64_t ld;
};

// FP32 epilogue of the tensor-core product (same algebra as Epilogue<T>):
//   out_t = alpha_t P + gamma_t I + sum_q beta_tq in_q + sum_{u<t} delta_tu out_u
// Inputs are in_hi[q] (+ in_lo[q] if non-null).  Each output is written as a
// (hi, lo) split, or as the plain value if out_lo[t] is null; outT_* (if
// non-null) receive the transposed split.  Stacked mode (split_row >= 0):
// rows < split_row go to output 0, the others to output 1 at row - split_row.
struct TcEpilogue {
  int32_t n_in = 0;
  int32_t n_out = 0;
  int64_t split_row = -1;
  const float* in_hi[EPI_MAX_IN] = {};
  const float* in_lo[EPI_MAX_IN] = {};
  float* out_hi[EPI_MAX_OUT] = {};
  float* out_lo[EPI_MAX_OUT] = {};
  float* outT_hi[EPI_MAX_OUT] = {};
  float* outT_lo[EPI_MAX_OUT] = {};
  float alpha[EPI_MAX_OUT] = {};
  float gamma[EPI_MAX_OUT] = {};
  float beta[EPI_MAX_OUT][EPI_MAX_IN] = {};
  float delta[EPI_MAX_OUT][EPI_MAX_OUT] = {};
};

// P = X (M x K) times Y (K x N), Y given transposed (YT: N x K), both K-major.
// ldo: leading dimension of every epilogue matrix (128 x 128 output tiles).
// *err (device int) is set to 1 if a bounded wait expired.
cs_status gemm_tf32(const TcOperand& X, const TcOperand& YT, int64_t M, int64_t N, int64_t K, int64_t ldo,
                    const TcEpilogue& epi, int* err, cudaStream_t stream);

// (hi, lo) split of scale * (an n x n row-major matrix, FP32 or FP64 source,
// leading dimension n) into padded (ld) hi/lo and, if hiT is non-null, the
// transposed split.  The scaled value is rounded to FP32 once.  With
// zero_diag the diagonal of the splits is 0 (the chain products add the
// diagonal terms exactly in FP64).
cs_status split_f32(const float* src, int64_t n, int64_t ld, float* hi, float* lo, float* hiT, float* loT,
                    cudaStream_t stream, double scale = 1.0, bool zero_diag = false);
cs_status split_f64(const double* src, int64_t n, int64_t ld, float* hi, float* lo, float* hiT, float* loT,
                    cudaStream_t stream, double scale = 1.0, bool zero_diag = false);

// dst (n x n, leading dimension n) = hi + lo (padded ld), as FP32 or FP64.
cs_status combine_f32(const float* hi, const float* lo, int64_t n, int64_t ld, float* dst, cudaStream_t stream);
cs_status combine_f64(const float* hi, const float* lo, int64_t n, int64_t ld, double* dst, cudaStream_t stream);

// Device word raised by a tensor-core kernel whose bounded wait expired.
int* tc_error_word();

// Launch one bounded wait that cannot be satisfied (limit in SM clocks); it
// raises the device error word, which the next API call reports.
cs_status wait_selftest(long long limit_cycles, cudaStream_t stream);

}  // namespace cs
