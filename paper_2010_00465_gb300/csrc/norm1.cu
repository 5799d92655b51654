// norm1.cu -- step 1 of the method: theta = ||A||_1 = max_j sum_i |a_ij|
// (Sec. 4: the algorithm is driven by the matrix 1-norm).
//
// Row-major A, so a column sum walks down a stride-n column.  Pass 1 gives
// each thread one column and a chunk of kRows rows: a warp reads 32 adjacent
// columns of one row per step (coalesced), and every block writes its column
// partial sums for its row chunk.  Pass 2 adds the partials of each column in
// a fixed order (deterministic), then takes the maximum with warp shuffles and
// one shared-memory round per block, the last block reducing the block maxima.
//
// GB300 adds FP64 at 2 per clock per SM, which would cap pass 1 below the HBM
// rate (one add per element), so pass 1 sums on the integer pipes: each
// |a| = m 2^(e - bias) (integer significand m, biased exponent e) is aligned
// to the largest exponent E seen so far in the chunk with g guard bits
// (g = 3 for FP64, 32 for FP32, so that m 2^g < 2^56), m 2^(g - (E - e))
// truncated to an integer, and added into an int64 sum (below 2^62 for 64
// rows); the sum is shifted when E grows.  Each term and
// each shift drops less than 2^-55 of the chunk's largest element, so the
// chunk sum is within 2^-48 relative of the exact one before its single
// conversion to FP64.  A chunk holding an Inf or NaN is summed again in FP64
// (a NaN anywhere makes the result NaN; Inf stays Inf).  Pass 2 and the
// maxima are FP64.
#include <math.h>

#include <mutex>

#include "internal.cuh"

namespace cs {
namespace {

constexpr int kCols = 256;  // threads (= columns) per block in pass 1
constexpr int kRows = 64;   // rows per chunk in pass 1
static_assert(kRows <= 64, "the int64 chunk sums hold at most 64 terms below 2^56");

// Bit layout of the element type: significand bits (without the implicit
// one), exponent field width and bias.
template <typename T>
struct Layout754;
template <>
struct Layout754<double> {
  using U = unsigned long long;
  static constexpr int kMant = 52, kExpMax = 0x7FF, kBias = 1075;  // |x| = m 2^(e - 1075)
  static constexpr int kGuard = 3;                                  // m 2^kGuard < 2^56
  __device__ static U bits(const double* p) { return (U)__double_as_longlong(__ldg(p)); }
};
template <>
struct Layout754<float> {
  using U = unsigned int;
  static constexpr int kMant = 23, kExpMax = 0xFF, kBias = 150;  // |x| = m 2^(e - 150)
  static constexpr int kGuard = 32;                               // m 2^kGuard < 2^56
  __device__ static U bits(const float* p) { return (U)__float_as_uint(__ldg(p)); }
};

__device__ __forceinline__ unsigned long long shr(unsigned long long x, int k) { return k > 63 ? 0ULL : x >> k; }

template <typename T>
__global__ void __launch_bounds__(kCols) colsum_partial(const T* __restrict__ A, int64_t n,
                                                        double* __restrict__ partial, unsigned int* __restrict__ ticket) {
  using L = Layout754<T>;
  // pass 2 counts its blocks on this word; pass 1 runs first on the stream
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *ticket = 0u;
  const int64_t col = (int64_t)blockIdx.x * kCols + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * kRows;
  if (col >= n) return;
  const int64_t r1 = min(r0 + (int64_t)kRows, n);
  const T* p = A + r0 * n + col;
  unsigned long long sum = 0;  // sum of m 2^(3 - (E - e))
  int E = 1;                   // alignment exponent (the smallest biased exponent of a finite value)
  bool special = false;        // an Inf or NaN in the chunk
  // one element: significand with the implicit one, effective exponent
  auto unpack = [](typename L::U b, unsigned long long& m, int& e) {
    const int eb = (int)((b >> L::kMant) & (typename L::U)L::kExpMax);
    m = (unsigned long long)(b & (((typename L::U)1 << L::kMant) - 1));
    if (eb) m |= 1ULL << L::kMant;
    e = eb ? eb : 1;
  };
  int64_t r = r0;
  // eight independent loads in flight per thread
  for (; r + 8 <= r1; r += 8, p += 8 * n) {
    typename L::U v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = L::bits(p + u * n);
    unsigned long long m[8];
    int e[8];
    int emax = E;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      unpack(v[u], m[u], e[u]);
      special |= e[u] == L::kExpMax;
      emax = max(emax, e[u]);
    }
    sum = shr(sum, emax - E);
    E = emax;
#pragma unroll
    for (int u = 0; u < 8; ++u) sum += shr(m[u] << L::kGuard, E - e[u]);
  }
  for (; r < r1; ++r, p += n) {
    unsigned long long m;
    int e;
    unpack(L::bits(p), m, e);
    special |= e == L::kExpMax;
    if (e > E) {
      sum = shr(sum, e - E);
      E = e;
    }
    sum += shr(m << L::kGuard, E - e);
  }
  double acc;
  if (!special) {
    acc = ldexp((double)sum, E - L::kBias - L::kGuard);
  } else {
    acc = 0.0;
    for (int64_t rr = r0; rr < r1; ++rr) acc += fabs((double)__ldg(A + rr * n + col));
  }
  partial[(int64_t)blockIdx.y * n + col] = acc;
}

__device__ __forceinline__ double max_nan(double a, double b) {
  return (isnan(a) || isnan(b)) ? __longlong_as_double(0x7ff8000000000000ULL) : fmax(a, b);
}

// Pass 2: a block takes 32 columns; its 8 warps each add every eighth chunk
// partial of those columns (warp g: chunks g, g + 8, ..., in order), the 8
// sums of a column are added in a fixed tree order (deterministic), each
// block reduces its columns to a maximum, and the last block to finish
// reduces the block maxima into *out.
constexpr int kFinCols = 32, kFinGroups = 8;
__global__ void __launch_bounds__(kFinCols * kFinGroups) colsum_finish(const double* __restrict__ partial, int64_t n,
                                                                       int64_t chunks, double* __restrict__ block_max,
                                                                       unsigned int* __restrict__ ticket,
                                                                       double* __restrict__ out) {
  __shared__ double part[kFinGroups][kFinCols];
  __shared__ double warp_best[kFinGroups];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t col = (int64_t)blockIdx.x * kFinCols + lane;
  double acc = 0.0;
  if (col < n) {
    int64_t k = warp;
    // four loads in flight per thread
    for (; k + 3 * kFinGroups < chunks; k += 4 * kFinGroups) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = partial[(k + u * kFinGroups) * n + col];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += v[u];
    }
    for (; k < chunks; k += kFinGroups) acc += partial[k * n + col];
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    double best = ((part[0][lane] + part[1][lane]) + (part[2][lane] + part[3][lane])) +
                  ((part[4][lane] + part[5][lane]) + (part[6][lane] + part[7][lane]));
    if (col >= n) best = 0.0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) best = max_nan(best, __shfl_xor_sync(0xffffffffu, best, off));
    if (lane == 0) {
      block_max[blockIdx.x] = best;
      __threadfence();
      last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double b = 0.0;
  for (int64_t i = threadIdx.x; i < gridDim.x; i += blockDim.x) b = max_nan(b, ((volatile double*)block_max)[i]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) b = max_nan(b, __shfl_xor_sync(0xffffffffu, b, off));
  if (lane == 0) warp_best[warp] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = warp_best[0];
    for (int w = 1; w < kFinGroups; ++w) r = max_nan(r, warp_best[w]);
    *out = r;
    *ticket = 0u;  // ready for the next call
  }
}

// ||A_b||_1 of `count` matrices of order n (contiguous, stride n^2), one
// block per matrix: each thread sums whole columns, then a block maximum.
__global__ void __launch_bounds__(kCols) norm1_batched_kernel(const double* __restrict__ A, int64_t n,
                                                              double* __restrict__ out) {
  const double* M = A + (int64_t)blockIdx.x * n * n;
  double best = 0.0;
  for (int64_t c = threadIdx.x; c < n; c += kCols) {
    double sum = 0.0;
    for (int64_t r = 0; r < n; ++r) sum += fabs(M[r * n + c]);
    best = max_nan(best, sum);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = max_nan(best, __shfl_xor_sync(0xffffffffu, best, off));
  __shared__ double warp_best[kCols / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_best[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = warp_best[0];
    for (int w = 1; w < kCols / 32; ++w) b = max_nan(b, warp_best[w]);
    out[blockIdx.x] = b;
  }
}

template <typename T>
cs_status norm1_impl(const T* A, int64_t n, double* partial, double* out, cudaStream_t stream) {
  if (n <= 0) {
    CS_CUDA_CHECK(cudaMemsetAsync(out, 0, sizeof(double), stream));
    return CS_OK;
  }
  const int64_t chunks = (n + kRows - 1) / kRows;
  const int64_t col_blocks = (n + kCols - 1) / kCols;
  const int64_t fin_blocks = (n + kFinCols - 1) / kFinCols;
  double* block_max = partial + chunks * n;
  unsigned int* ticket = (unsigned int*)(block_max + fin_blocks);
  ProfScope prof(CS_KERNEL_NORM1, (double)n * (double)n * sizeof(T), stream);
  dim3 grid((unsigned)col_blocks, (unsigned)chunks);
  colsum_partial<T><<<grid, kCols, 0, stream>>>(A, n, partial, ticket);
  colsum_finish<<<(unsigned)fin_blocks, kFinCols * kFinGroups, 0, stream>>>(partial, n, chunks, block_max, ticket,
                                                                           out);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace

// partial sums (chunks x n), block maxima (one per pass-2 block) and a ticket word
int64_t norm1_scratch_elems(int64_t n) {
  if (n <= 0) return 2;
  return ((n + kRows - 1) / kRows) * n + (n + kFinCols - 1) / kFinCols + 1;
}

cs_status norm1_f64(const double* A, int64_t n, double* partial, double* out, cudaStream_t stream) {
  return norm1_impl<double>(A, n, partial, out, stream);
}

cs_status norm1_f32(const float* A, int64_t n, double* partial, double* out, cudaStream_t stream) {
  return norm1_impl<float>(A, n, partial, out, stream);
}

cs_status norm1_batched_f64(const double* A, int64_t n, int64_t count, double* out, cudaStream_t stream) {
  if (count <= 0) return CS_OK;
  if (count > 2147483647LL) return fail(CS_EINVAL, "norm1_batched: count too large");
  ProfScope prof(CS_KERNEL_NORM1, (double)n * (double)n * sizeof(double) * (double)count, stream);
  norm1_batched_kernel<<<(unsigned)count, kCols, 0, stream>>>(A, n, out);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

// ------------------------------------------------- allocation-free variant ---
// Scratch for callers that cannot allocate device memory: the partial sums,
// block maxima and ticket word of the two passes above for n <= kStaticMaxN,
// about 2 MB, held by every GPU that loads the library until the process ends.
constexpr int64_t kStaticMaxN = 4096;
constexpr int64_t kStaticElems = ((kStaticMaxN + kRows - 1) / kRows) * kStaticMaxN +
                                 (kStaticMaxN + kFinCols - 1) / kFinCols + 1;
static __device__ __align__(256) double g_static_scratch[kStaticElems];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
double* g_static_addr[kMaxDevices] = {};

// The array's name in host code is only a host-side stand-in; its device
// address is looked up once per device, with that device current.
cs_status static_scratch(double** out) {
  int dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(CS_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_addr[dev]) {
    double* p = nullptr;
    CS_CUDA_CHECK(cudaGetSymbolAddress((void**)&p, g_static_scratch));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return CS_OK;
}
}  // namespace

}  // namespace cs

extern "C" cs_status cossin_norm1_noalloc(const void* A, int64_t n, cs_prec prec, double* norm1_dev,
                                          cossin_stream_t stream) {
  if (cs::check_prec(prec) != CS_OK) return CS_EINVAL;
  if (n < 0) return cs::fail(CS_EINVAL, "n must be >= 0");
  if (n > cs::kStaticMaxN)
    return cs::fail(CS_EINVAL, "cossin_norm1_noalloc: n = " + std::to_string(n) +
                                   " exceeds the static scratch limit of 4096; use cossin_norm1");
  if (!norm1_dev) return cs::fail(CS_EINVAL, "norm1_dev is null");
  if (n > 0 && !A) return cs::fail(CS_EINVAL, "null matrix pointer");
  double* scratch = nullptr;
  CS_CHECK(cs::static_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  if (prec == CS_FP32) return cs::norm1_f32((const float*)A, n, scratch, norm1_dev, st);
  return cs::norm1_f64((const double*)A, n, scratch, norm1_dev, st);
}
