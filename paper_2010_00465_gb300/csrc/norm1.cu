// norm1.cu -- step 1 of the method: theta = ||A||_1 = max_j sum_i |a_ij|
// (Sec. 4: the algorithm is driven by the matrix 1-norm).
//
// Row-major A, so a column sum walks down a stride-n column.  Pass 1 gives
// each thread one column and a chunk of ROWS rows: a warp reads 32 adjacent
// columns of one row per step (coalesced), and every block writes its column
// partial sums for its row chunk.  Pass 2 adds the partials of each column in
// a fixed order (deterministic), then takes the maximum with warp shuffles and
// one shared-memory round.  Accumulation is FP64 for both input types.  A NaN
// anywhere makes the result NaN; Inf stays Inf.
#include <math.h>

#include "internal.cuh"

namespace cs {
namespace {

constexpr int kCols = 256;  // threads (= columns) per block in pass 1
constexpr int kRows = 64;   // rows per chunk in pass 1

template <typename T>
__global__ void __launch_bounds__(kCols) colsum_partial(const T* __restrict__ A, int64_t n,
                                                        double* __restrict__ partial) {
  const int64_t col = (int64_t)blockIdx.x * kCols + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * kRows;
  if (col >= n) return;
  const int64_t r1 = min(r0 + (int64_t)kRows, n);
  const T* p = A + r0 * n + col;
  double acc = 0.0;
  int64_t r = r0;
  // eight independent loads in flight per thread
  for (; r + 8 <= r1; r += 8, p += 8 * n) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = fabs((double)__ldg(p + u * n));
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u];
  }
  for (; r < r1; ++r, p += n) acc += fabs((double)__ldg(p));
  partial[(int64_t)blockIdx.y * n + col] = acc;
}

__device__ __forceinline__ double max_nan(double a, double b) {
  return (isnan(a) || isnan(b)) ? __longlong_as_double(0x7ff8000000000000ULL) : fmax(a, b);
}

__global__ void __launch_bounds__(1024) colsum_finish(const double* __restrict__ partial,
                                                      int64_t n, int64_t chunks,
                                                      double* __restrict__ out) {
  double best = 0.0;
  for (int64_t c = threadIdx.x; c < n; c += blockDim.x) {
    double s = 0.0;
    for (int64_t k = 0; k < chunks; ++k) s += partial[k * n + c];
    best = max_nan(best, s);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = max_nan(best, __shfl_xor_sync(0xffffffffu, best, off));
  __shared__ double warp_best[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_best[warp] = best;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    best = lane < nw ? warp_best[lane] : 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = max_nan(best, __shfl_xor_sync(0xffffffffu, best, off));
    if (lane == 0) *out = best;
  }
}

template <typename T>
cs_status norm1_impl(const T* A, int64_t n, double* partial, double* out, cudaStream_t stream) {
  if (n <= 0) {
    CS_CUDA_CHECK(cudaMemsetAsync(out, 0, sizeof(double), stream));
    return CS_OK;
  }
  const int64_t chunks = (n + kRows - 1) / kRows;
  ProfScope prof(CS_KERNEL_NORM1, (double)n * (double)n * sizeof(T), stream);
  dim3 grid((unsigned)((n + kCols - 1) / kCols), (unsigned)chunks);
  colsum_partial<T><<<grid, kCols, 0, stream>>>(A, n, partial);
  colsum_finish<<<1, 1024, 0, stream>>>(partial, n, chunks, out);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace

int64_t norm1_scratch_elems(int64_t n) { return n <= 0 ? 1 : ((n + kRows - 1) / kRows) * n; }

cs_status norm1_f64(const double* A, int64_t n, double* partial, double* out, cudaStream_t stream) {
  return norm1_impl<double>(A, n, partial, out, stream);
}

cs_status norm1_f32(const float* A, int64_t n, double* partial, double* out, cudaStream_t stream) {
  return norm1_impl<float>(A, n, partial, out, stream);
}

}  // namespace cs
