// internal.cuh -- shared declarations of the cos/sin library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "cossin.h"

namespace cs {

// ---------------------------------------------------------------- errors ---
void set_error(const std::string& msg);
cs_status fail(cs_status st, const std::string& msg);
cs_status cuda_fail(cudaError_t e, const char* what);

#define CS_CUDA_CHECK(expr)                                   \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return ::cs::cuda_fail(e_, #expr); \
  } while (0)

// Stream-ordered device allocation of the library's own buffers; a failure
// (or one injected by cossin_selftest_fail_next_alloc) returns CS_ENOMEM.
cs_status dev_alloc(void** p, size_t bytes, cudaStream_t stream, const char* what);

#define CS_CHECK(expr)                       \
  do {                                       \
    cs_status st_ = (expr);                  \
    if (st_ != CS_OK) return st_;            \
  } while (0)

// Raises `kernel`'s dynamic shared-memory limit to `bytes` once per device
// (the attribute belongs to the device's context); `done` holds one bit per
// device ordinal below 64, others are set on every call.
template <typename Kernel>
inline cs_status smem_limit_once(Kernel* kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ULL << dev : 0ULL;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return CS_OK;
  CS_CUDA_CHECK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done.fetch_or(bit, std::memory_order_acq_rel);
  return CS_OK;
}

// --------------------------------------------------------------- epilogue ---
// Every product P = X Y of the method is followed by linear combinations of P,
// the identity and matrices already computed (Sec. 2.1).  The epilogue applies
// them where P leaves the accumulators:
//   out_t[r][c] = alpha_t * P[r][c] + gamma_t * (r == c) + sum_j beta_tj * in_j[r][c]
//                 + sum_{u < t} delta_tu * out_u[r][c]
// In "stacked" mode (double-angle step, [C; S] * C) rows r < split_row go to
// out_0 and rows r >= split_row go to out_1 at row r - split_row, each with its
// own alpha and gamma, and no inputs are read.
// out_t may equal in_j: each element is read before it is written, by the
// same thread.
constexpr int EPI_MAX_IN = 6;
constexpr int EPI_MAX_OUT = 6;

template <typename T>
struct Epilogue {
  int32_t n_in = 0;
  int32_t n_out = 0;
  int64_t split_row = -1;  // >= 0 selects stacked mode
  const T* in[EPI_MAX_IN] = {};
  T* out[EPI_MAX_OUT] = {};
  // TF32 path: a matrix is held as a pair (hi, lo) with hi = tf32(x) and
  // lo = x - hi exactly.  If out_lo[t] is non-null, out[t] receives hi and
  // out_lo[t] receives lo; if in_lo[j] is non-null the input is in[j] + in_lo[j].
  T* out_lo[EPI_MAX_OUT] = {};
  const T* in_lo[EPI_MAX_IN] = {};
  double alpha[EPI_MAX_OUT] = {};
  double gamma[EPI_MAX_OUT] = {};
  double beta[EPI_MAX_OUT][EPI_MAX_IN] = {};
  double delta[EPI_MAX_OUT][EPI_MAX_OUT] = {};
};

template <typename T>
struct EpiBuilder {
  Epilogue<T> e;
  int add_in(const T* p, const T* lo = nullptr) {
    e.in[e.n_in] = p;
    e.in_lo[e.n_in] = lo;
    return e.n_in++;
  }
  int add_out(T* p, double alpha, double gamma, T* lo = nullptr) {
    e.out[e.n_out] = p;
    e.out_lo[e.n_out] = lo;
    e.alpha[e.n_out] = alpha;
    e.gamma[e.n_out] = gamma;
    return e.n_out++;
  }
  void beta(int out, int in, double b) { e.beta[out][in] = b; }
  void delta(int out, int prev_out, double d) { e.delta[out][prev_out] = d; }
};

// ------------------------------------------------------------- profiling ---
struct ProfScope {
  int kind;
  double work;
  cudaStream_t stream;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ProfScope(int kind, double work, cudaStream_t stream);
  ~ProfScope();
};

// ---------------------------------------------------------------- kernels ---
// FP64 product with fused epilogue: P = op(X) op(Y), op = identity or
// transpose, M x N result, inner dimension K.  Batched over `batch` matrices
// with element strides bsx, bsy (operands) and bse (every epilogue matrix).
// ldo is the leading dimension of the epilogue matrices.
cs_status gemm_f64(const double* X, const double* Y, int64_t M, int64_t N, int64_t K,
                   int64_t ldx, int64_t ldy, bool transX, bool transY, const Epilogue<double>& epi,
                   int64_t ldo, int64_t batch, int64_t bsx, int64_t bsy, int64_t bse,
                   cudaStream_t stream, void* split_ws = nullptr, size_t split_bytes = 0);
// Scratch that lets gemm_f64 split the tiles of its last, partial wave over K
// (one product, batch 1; 0 when it would not split); given at least this
// many bytes, gemm_f64 does.
size_t gemm_f64_split_bytes(int64_t M, int64_t N, int64_t K);

// ||A||_1 for an FP64 or FP32 matrix into a device double (*out_dev).
// partial_dev: scratch of norm1_scratch_elems(n) doubles (column partial sums,
// pass-2 block maxima and a ticket word).
int64_t norm1_scratch_elems(int64_t n);
cs_status norm1_f64(const double* A, int64_t n, double* partial_dev, double* out_dev,
                    cudaStream_t stream);
cs_status norm1_f32(const float* A, int64_t n, double* partial_dev, double* out_dev,
                    cudaStream_t stream);

// ||A_b||_1 for `count` contiguous FP64 matrices of order n, one block each.
cs_status norm1_batched_f64(const double* A, int64_t n, int64_t count, double* out, cudaStream_t stream);

// dst[i] = scale * src[i], i < count (FP64).
cs_status scale_f64(const double* src, double* dst, int64_t count, double scale, cudaStream_t stream);
// Element-wise FP32 -> FP64 (exact) and FP64 -> FP32 (rounded to nearest).
cs_status convert_f32_f64(const float* src, double* dst, int64_t count, cudaStream_t stream);
cs_status convert_f64_f32(const double* src, float* dst, int64_t count, cudaStream_t stream);

// The executors behind the ABI (cossin_api.cu, adjoint.cu): cos/sin and the
// adjoint of scale * A.
cs_status cossin_impl(const void* A, int64_t n, cs_prec prec, void* C, void* S, void* ws, size_t ws_bytes,
                      int32_t force_m, int32_t force_s, cs_info* info, cudaStream_t stream, double scale);
// backward_impl: with ws null the library allocates its buffers
// stream-ordered; else it takes them from ws (ws_bytes, 256-byte aligned) and
// allocates nothing.
cs_status backward_impl(int64_t count, int64_t n, double scale, const double* A, const double* G_C,
                        const double* G_S, double* dA, double* C, double* S, int32_t force_m, int32_t force_s,
                        cs_info* infos_host, cudaStream_t stream, bool emu = false, void* ws = nullptr,
                        size_t ws_bytes = 0);
size_t backward_workspace_bytes(int64_t count, int64_t n, int max_s, bool emu);
cs_status check_prec(cs_prec prec);
// One small FP64 matrix (n <= 128) in a single cooperative launch (small_f64.cu).
struct Layout;
bool small_f64_eligible(cs_prec prec, int64_t n);
cs_status small_f64(const double* A, int64_t n, double* C, double* S, char* ws, const Layout& L, int32_t force_m,
                    int32_t force_s, cs_info* info, cudaStream_t stream, double scale);
// Every precision keeps FP64 intermediates.  uses_emu: some products are
// sliced BF16 tensor-core products (CS_FP64_EMU, CS_SPLIT_EMU, CS_SPLIT_BF16,
// CS_FP32); f64_operands: every product takes FP64 operands (all but the TF32
// split forms, whose chain products take (hi, lo) TF32 splits).
bool uses_emu(cs_prec p);
bool f64_operands(cs_prec p);
// Slices of the emulated double-angle products of a precision (four for
// CS_FP32, eight for the FP64-class ones).
int square_slices(cs_prec p);
size_t elem_size(cs_prec p);
bool overlaps(const void* a, size_t na, const void* b, size_t nb);

// Host selection (step 2).
cs_status select_ms(double norm1, int table, int* m, int* s);
int products_of(int m);

}  // namespace cs
