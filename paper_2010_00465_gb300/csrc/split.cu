// split.cu -- (hi, lo) TF32 splits of a matrix (with an optional transposed
// copy, through a 32 x 32 shared-memory tile so both stores coalesce), the
// recombination hi + lo into the caller's FP32 or FP64 matrix, and the device
// error word of the tensor-core kernels.
#include <algorithm>

#include "internal.cuh"
#include "sm100_ptx.cuh"
#include "tc_gemm.h"

namespace cs {
namespace {

__device__ int g_tc_error;

template <typename T>
__global__ void __launch_bounds__(256) split_kernel(const T* __restrict__ src, int64_t n, int64_t ld,
                                                    float* __restrict__ hi, float* __restrict__ lo,
                                                    float* __restrict__ hiT, float* __restrict__ loT, double scale,
                                                    bool zero_diag) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < n && c < n && !(zero_diag && r == c)) {
      v = scale == 1.0 ? (float)src[r * n + c] : (float)((double)src[r * n + c] * scale);
    }
    if (r < n && c < n) {
      const float h = ptx::tf32_rna(v);
      hi[r * ld + c] = h;
      lo[r * ld + c] = COSSIN_LO(v - h);
    }
    tile[i][threadIdx.x] = v;
  }
  if (hiT == nullptr) return;  // uniform over the block
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = c0 + i, c = r0 + threadIdx.x;  // row of the transpose = column of src
    if (r < n && c < n) {
      const float v = tile[threadIdx.x][i];
      const float h = ptx::tf32_rna(v);
      hiT[r * ld + c] = h;
      loT[r * ld + c] = COSSIN_LO(v - h);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) combine_kernel(const float* __restrict__ hi, const float* __restrict__ lo,
                                                      int64_t n, int64_t ld, T* __restrict__ dst) {
  const int64_t total = n * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / n, c = i - r * n;
    dst[i] = (T)hi[r * ld + c] + (T)lo[r * ld + c];
  }
}

template <typename T>
cs_status split_impl(const T* src, int64_t n, int64_t ld, float* hi, float* lo, float* hiT, float* loT,
                     double scale, bool zero_diag, cudaStream_t stream) {
  if (n <= 0) return CS_OK;
  ProfScope prof(CS_KERNEL_OTHER, (double)n * n * (sizeof(T) + (hiT ? 16.0 : 8.0)), stream);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  split_kernel<T><<<grid, block, 0, stream>>>(src, n, ld, hi, lo, hiT, loT, scale, zero_diag);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

template <typename T>
cs_status combine_impl(const float* hi, const float* lo, int64_t n, int64_t ld, T* dst, cudaStream_t stream) {
  if (n <= 0) return CS_OK;
  ProfScope prof(CS_KERNEL_OTHER, (double)n * n * (8.0 + sizeof(T)), stream);
  const int64_t total = n * n;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
  combine_kernel<T><<<blocks, 256, 0, stream>>>(hi, lo, n, ld, dst);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace

cs_status split_f32(const float* src, int64_t n, int64_t ld, float* hi, float* lo, float* hiT, float* loT,
                    cudaStream_t stream, double scale, bool zero_diag) {
  return split_impl<float>(src, n, ld, hi, lo, hiT, loT, scale, zero_diag, stream);
}
cs_status split_f64(const double* src, int64_t n, int64_t ld, float* hi, float* lo, float* hiT, float* loT,
                    cudaStream_t stream, double scale, bool zero_diag) {
  return split_impl<double>(src, n, ld, hi, lo, hiT, loT, scale, zero_diag, stream);
}

namespace {
__global__ void __launch_bounds__(256) scale_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                                    int64_t count, double scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = scale * src[i];
}

template <typename S, typename D>
__global__ void __launch_bounds__(256) convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

template <typename S, typename D>
cs_status convert(const S* src, D* dst, int64_t count, cudaStream_t stream) {
  if (count <= 0) return CS_OK;
  ProfScope prof(CS_KERNEL_OTHER, (double)(sizeof(S) + sizeof(D)) * (double)count, stream);
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
  convert_kernel<S, D><<<blocks, 256, 0, stream>>>(src, dst, count);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}
}  // namespace

cs_status convert_f32_f64(const float* src, double* dst, int64_t count, cudaStream_t stream) {
  return convert<float, double>(src, dst, count, stream);
}
cs_status convert_f64_f32(const double* src, float* dst, int64_t count, cudaStream_t stream) {
  return convert<double, float>(src, dst, count, stream);
}

cs_status scale_f64(const double* src, double* dst, int64_t count, double scale, cudaStream_t stream) {
  if (count <= 0) return CS_OK;
  ProfScope prof(CS_KERNEL_OTHER, 16.0 * (double)count, stream);
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 152 * 16);
  scale_kernel<<<blocks, 256, 0, stream>>>(src, dst, count, scale);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}
cs_status combine_f32(const float* hi, const float* lo, int64_t n, int64_t ld, float* dst, cudaStream_t stream) {
  return combine_impl<float>(hi, lo, n, ld, dst, stream);
}
cs_status combine_f64(const float* hi, const float* lo, int64_t n, int64_t ld, double* dst, cudaStream_t stream) {
  return combine_impl<double>(hi, lo, n, ld, dst, stream);
}

namespace {
// The failure path of every bounded wait, exercised on purpose: an mbarrier
// that nothing arrives at, waited on with a short limit; on expiry the kernel
// raises the error word the tensor-core kernels raise and returns.
__global__ void wait_selftest_kernel(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x != 0) return;
  abort_flag = 0;
  ptx::mbar_init(&bar, 1);
  ptx::fence_mbar_init();
  if (!ptx::mbar_wait_limit(&bar, 0, &abort_flag, limit)) atomicExch(err, 1);
}
}  // namespace

cs_status wait_selftest(long long limit_cycles, cudaStream_t stream) {
  int* err = tc_error_word();
  if (!err) return fail(CS_ECUDA, "cannot resolve the device error word");
  wait_selftest_kernel<<<1, 32, 0, stream>>>(err, limit_cycles);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

int* tc_error_word() {
  int* p = nullptr;
  if (cudaGetSymbolAddress((void**)&p, g_tc_error) != cudaSuccess) return nullptr;
  return p;
}

}  // namespace cs
