// unitary.cu -- the propagator e^{-itA} = cos(tA) - i sin(tA) of Sec. 1 (the
// Schroedinger case, real A), and its adjoint for real-parameter gradients.
//
// The scheme runs at t A with t folded into the plans' first and last
// coefficients (no scaled copy of A); C and S land in the workspace and one
// elementwise kernel writes U as interleaved (re, im) pairs.  For the
// adjoint the real loss Re <G, U> = <Re G, C> + <-Im G, S> is the cos/sin
// loss with cotangents (Re G, -Im G), so the FP64 reverse pass of the cos/sin
// schemes at t A gives dL/dA directly.
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"
#include "plan.h"

namespace cs {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) interleave_kernel(const T* __restrict__ C, const T* __restrict__ S,
                                                         T* __restrict__ U, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    U[2 * i] = C[i];
    U[2 * i + 1] = -S[i];
  }
}

__global__ void __launch_bounds__(256) deinterleave_kernel(const double* __restrict__ G, double* __restrict__ GC,
                                                           double* __restrict__ GS, int64_t count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    GC[i] = G[2 * i];
    GS[i] = -G[2 * i + 1];
  }
}

int grid_for(int64_t count) { return (int)std::min<int64_t>((count + 255) / 256, 152 * 8); }

template <typename T>
cs_status interleave(const T* C, const T* S, T* U, int64_t count, cudaStream_t stream) {
  if (count <= 0) return CS_OK;
  ProfScope prof(CS_KERNEL_OTHER, 4.0 * sizeof(T) * (double)count, stream);
  interleave_kernel<T><<<grid_for(count), 256, 0, stream>>>(C, S, U, count);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace
}  // namespace cs

extern "C" cs_status cossin_unitary_workspace_size(int64_t n, cs_prec prec, size_t* bytes) {
  CS_CHECK(cs::check_prec(prec));
  if (n < 0 || n > cs::kMaxN) return cs::fail(CS_EINVAL, "n out of range [0, 65536]");
  if (!bytes) return cs::fail(CS_EINVAL, "null output pointer");
  *bytes = cs::make_layout(n, prec, true).total;
  return CS_OK;
}

extern "C" cs_status cossin_unitary(const void* A, int64_t n, double t, cs_prec prec, void* U, void* ws,
                                    size_t ws_bytes, int32_t force_m, int32_t force_s, cs_info* info,
                                    cossin_stream_t stream) {
  using namespace cs;
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(check_prec(prec));
  if (n < 0 || n > kMaxN) return fail(CS_EINVAL, "n out of range [0, 65536]");
  if (!isfinite(t)) return fail(CS_EINVAL, "t must be finite");
  if (n == 0) return cossin_impl(A, 0, prec, nullptr, nullptr, nullptr, 0, force_m, force_s, info, st, t);
  if (!A || !U) return fail(CS_EINVAL, "null matrix pointer");
  const size_t el = elem_size(prec);
  const size_t n2 = (size_t)n * (size_t)n;
  if (overlaps(A, n2 * el, U, 2 * n2 * el)) return fail(CS_EINVAL, "A and U must not overlap");
  const Layout L = make_layout(n, prec, true);
  void* buf = nullptr;
  if (!ws) {
    CS_CHECK(dev_alloc(&buf, L.total, st, "cossin_unitary workspace"));
    ws = buf;
    ws_bytes = L.total;
  }
  cs_status rc = CS_OK;
  if (ws_bytes < L.total) rc = fail(CS_EINVAL, "workspace missing or too small (cossin_unitary_workspace_size)");
  else if (((uintptr_t)ws & 255) != 0) rc = fail(CS_EINVAL, "workspace must be 256-byte aligned");
  if (rc == CS_OK) {
    char* w = (char*)ws;
    void* C = w + L.out_c;
    void* S = w + L.out_s;
    // The cos/sin executors use the leading L.out_c bytes, which hold the
    // layout of make_layout(n, prec) unchanged.
    rc = cossin_impl(A, n, prec, C, S, ws, L.out_c, force_m, force_s, info, st, t);
    if (rc == CS_OK) {
      if (prec == CS_FP32)
        rc = interleave<float>((const float*)C, (const float*)S, (float*)U, (int64_t)n2, st);
      else
        rc = interleave<double>((const double*)C, (const double*)S, (double*)U, (int64_t)n2, st);
    }
  }
  if (buf) cudaFreeAsync(buf, st);
  return rc;
}

extern "C" cs_status cossin_unitary_backward(int64_t count, int64_t n, double t, const double* A, const double* G,
                                             double* dA, double* U, int32_t force_m, int32_t force_s,
                                             cs_info* infos_host, cossin_stream_t stream) {
  using namespace cs;
  cudaStream_t st = (cudaStream_t)stream;
  if (count < 0 || n < 0 || n > kMaxN) return fail(CS_EINVAL, "count or n out of range");
  if (n > 0 && count > (int64_t(1) << 46) / (n * n)) return fail(CS_EINVAL, "count * n^2 above 2^46 elements");
  if (!isfinite(t)) return fail(CS_EINVAL, "t must be finite");
  if (count == 0 || n == 0) return backward_impl(count, n, t, A, nullptr, nullptr, dA, nullptr, nullptr, force_m,
                                                 force_s, infos_host, st);
  if (!A || !G || !dA) return fail(CS_EINVAL, "null matrix pointer");
  const int64_t total = count * n * n;
  const size_t real_bytes = sizeof(double) * (size_t)total;
  if (overlaps(dA, real_bytes, A, real_bytes) || overlaps(dA, real_bytes, G, 2 * real_bytes) ||
      (U && (overlaps(U, 2 * real_bytes, A, real_bytes) || overlaps(U, 2 * real_bytes, G, 2 * real_bytes) ||
             overlaps(U, 2 * real_bytes, dA, real_bytes))))
    return fail(CS_EINVAL, "outputs must not overlap inputs or each other");
  char* buf = nullptr;
  const size_t need = (U ? 4 : 2) * real_bytes;
  CS_CHECK(dev_alloc((void**)&buf, need, st, "cossin_unitary_backward scratch"));
  double* GC = (double*)buf;
  double* GS = (double*)(buf + real_bytes);
  double* C = U ? (double*)(buf + 2 * real_bytes) : nullptr;
  double* S = U ? (double*)(buf + 3 * real_bytes) : nullptr;
  cs_status rc = CS_OK;
  deinterleave_kernel<<<grid_for(total), 256, 0, st>>>(G, GC, GS, total);
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) rc = cuda_fail(ce, "deinterleave");
  if (rc == CS_OK)
    rc = backward_impl(count, n, t, A, GC, GS, dA, C, S, force_m, force_s, infos_host, st);
  if (rc == CS_OK && U) rc = interleave<double>(C, S, U, total, st);
  cudaFreeAsync(buf, st);
  return rc;
}
