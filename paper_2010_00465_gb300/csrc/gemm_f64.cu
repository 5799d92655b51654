// gemm_f64.cu -- FP64 matrix product with the method's linear combinations
// fused into the epilogue.
//
// Every step of the method that costs anything is a product of two n x n
// matrices followed by a few linear combinations (Sec. 2.1: each scheme
// "uses the results from all previous" stages; Sec. 1: double-angle steps).
// On GB300 the tensor-core generation (tcgen05) has no FP64 kind, and the
// chip's FP64 rate is about 1.25 TFLOP/s, roughly two FP64 FMAs per clock
// per SM.  That rate, not memory, bounds this kernel: a 128 x 128 block tile
// with an 8 x 8 register tile per thread gives 64 FMAs per 16 shared-memory
// loads, far more reuse than the FP64 pipe can consume, so the kernel keeps
// the FP64 pipe busy with a simple single-buffered main loop.
//
// Operands may be transposed (op(X) = X^T reads X column-wise): the adjoint
// needs X^T G and G Y^T.  A batch of equally sized problems runs on grid.z.
#include "internal.cuh"

namespace cs {
namespace {

constexpr int BK = 8, THREADS = 256;

// TILE x TILE block tile (TILE = 128 or 64); thread (ty, tx) of 16 x 16 owns
// rows {h*64 + ty*4 + i} and columns {h*64 + tx*4 + j}, h < TILE/64, i, j < 4.
template <int TILE, bool TX, bool TY>
__global__ void __launch_bounds__(THREADS)
gemm_f64_kernel(const double* __restrict__ X, const double* __restrict__ Y, int64_t M, int64_t N,
                int64_t K, int64_t ldx, int64_t ldy, int64_t ldo, int64_t bsx, int64_t bsy,
                int64_t bse, const Epilogue<double> epi) {
  constexpr int BM = TILE, BN = TILE, R = TILE / 16;
  __shared__ double Xs[BK][BM];
  __shared__ double Ys[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int64_t b = blockIdx.z;
  X += b * bsx;
  Y += b * bsy;

  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    // op(X) tile: rows m0..m0+127, columns k0..k0+7, stored k-major.
#pragma unroll
    for (int t = 0; t < (BM * BK) / THREADS; ++t) {
      const int i = tid + t * THREADS;
      int mm, kk;
      if (TX) {  // element (m, k) = X[k][m]: consecutive threads walk m
        kk = i / BM;
        mm = i % BM;
      } else {   // element (m, k) = X[m][k]: consecutive threads walk k
        mm = i / BK;
        kk = i % BK;
      }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = TX ? X[gk * ldx + gm] : X[gm * ldx + gk];
      Xs[kk][mm] = v;
    }
    // op(Y) tile: rows k0..k0+7, columns n0..n0+127.
#pragma unroll
    for (int t = 0; t < (BN * BK) / THREADS; ++t) {
      const int i = tid + t * THREADS;
      int kk, nn;
      if (TY) {  // element (k, n) = Y[n][k]
        nn = i / BK;
        kk = i % BK;
      } else {   // element (k, n) = Y[k][n]
        kk = i / BN;
        nn = i % BN;
      }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      double v = 0.0;
      if (gk < K && gn < N) v = TY ? Y[gn * ldy + gk] : Y[gk * ldy + gn];
      Ys[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[R], c[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        a[i] = Xs[kk][(i / 4) * 64 + ty * 4 + (i % 4)];
        c[i] = Ys[kk][(i / 4) * 64 + tx * 4 + (i % 4)];
      }
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], c[j], acc[i][j]);
    }
    __syncthreads();
  }

  // Epilogue over this thread's rows and columns of the block tile.
  const int64_t eoff = b * bse;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t r = m0 + (i / 4) * 64 + ty * 4 + (i % 4);
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int64_t c = n0 + (j / 4) * 64 + tx * 4 + (j % 4);
      if (c >= N) continue;
      const double p = acc[i][j];
      if (epi.split_row >= 0) {
        const bool top = r < epi.split_row;
        const int64_t rr = top ? r : r - epi.split_row;
        const int t = top ? 0 : 1;
        epi.out[t][eoff + rr * ldo + c] = epi.alpha[t] * p + (rr == c ? epi.gamma[t] : 0.0);
      } else {
        const int64_t idx = eoff + r * ldo + c;
        double in[EPI_MAX_IN], o[EPI_MAX_OUT];
#pragma unroll
        for (int q = 0; q < EPI_MAX_IN; ++q) in[q] = q < epi.n_in ? epi.in[q][idx] : 0.0;
#pragma unroll
        for (int t = 0; t < EPI_MAX_OUT; ++t) {
          if (t >= epi.n_out) break;
          double v = epi.alpha[t] * p + (r == c ? epi.gamma[t] : 0.0);
#pragma unroll
          for (int q = 0; q < EPI_MAX_IN; ++q)
            if (q < epi.n_in) v += epi.beta[t][q] * in[q];
#pragma unroll
          for (int u = 0; u < t; ++u) v += epi.delta[t][u] * o[u];
          o[t] = v;
        }
#pragma unroll
        for (int t = 0; t < EPI_MAX_OUT; ++t) {
          if (t >= epi.n_out) break;
          epi.out[t][idx] = o[t];
        }
      }
    }
  }
}

}  // namespace

cs_status gemm_f64(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx,
                   int64_t ldy, bool transX, bool transY, const Epilogue<double>& epi, int64_t ldo,
                   int64_t batch, int64_t bsx, int64_t bsy, int64_t bse, cudaStream_t stream) {
  if (M <= 0 || N <= 0 || batch <= 0) return CS_OK;
  // 128-wide tiles unless that leaves fewer than two waves of CTAs (small
  // batched products), where 64-wide tiles balance the SMs better.
  const int64_t ctas128 = ((M + 127) / 128) * ((N + 127) / 128) * batch;
  const int tile = ctas128 < 2 * 152 ? 64 : 128;
  if ((M + tile - 1) / tile > 65535 || batch > 65535) return fail(CS_EINVAL, "gemm_f64: grid too large");
  dim3 grid((unsigned)((N + tile - 1) / tile), (unsigned)((M + tile - 1) / tile), (unsigned)batch);
  ProfScope prof(CS_KERNEL_GEMM_F64, 2.0 * (double)M * (double)N * (double)K * (double)batch, stream);
#define CS_F64_LAUNCH(T)                                                                                           \
  if (!transX && !transY)                                                                                          \
    gemm_f64_kernel<T, false, false><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi); \
  else if (transX && !transY)                                                                                      \
    gemm_f64_kernel<T, true, false><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi);  \
  else if (!transX && transY)                                                                                      \
    gemm_f64_kernel<T, false, true><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi);  \
  else                                                                                                             \
    gemm_f64_kernel<T, true, true><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi);
  if (tile == 64) {
    CS_F64_LAUNCH(64)
  } else {
    CS_F64_LAUNCH(128)
  }
#undef CS_F64_LAUNCH
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace cs
