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

// The fused epilogue for entry (r, c) of a product with value p.
__device__ __forceinline__ void epilogue_store(const Epilogue<double>& epi, int64_t eoff, int64_t r, int64_t c,
                                               int64_t ldo, double p) {
  if (epi.split_row >= 0) {
    const bool top = r < epi.split_row;
    const int64_t rr = top ? r : r - epi.split_row;
    const int t = top ? 0 : 1;
    epi.out[t][eoff + rr * ldo + c] = epi.alpha[t] * p + (rr == c ? epi.gamma[t] : 0.0);
    return;
  }
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

// Split of the last, partial wave of tiles over K (one product, batch 1):
// the grid is one-dimensional over the tiles in row-major order; tiles from
// `first` on are cut into `parts` k-ranges of `kchunk`, whose partial sums go
// to ws (one TILE x TILE block per piece, in each thread's register order)
// and are added, in piece order, by gemm_f64_split_finish, which then runs
// the epilogue.  parts == 0: the plain three-dimensional grid.
struct SplitK {
  int64_t first = 0;
  int64_t kchunk = 0;
  int parts = 0;
  int ntn = 0;  // tile columns
  double* ws = nullptr;
};

// TILE x TILE block tile (TILE = 128 or 64); thread (ty, tx) of 16 x 16 owns
// rows {h*64 + ty*4 + i} and columns {h*64 + tx*4 + j}, h < TILE/64, i, j < 4.
template <int TILE, bool TX, bool TY>
__global__ void __launch_bounds__(THREADS)
gemm_f64_kernel(const double* __restrict__ X, const double* __restrict__ Y, int64_t M, int64_t N,
                int64_t K, int64_t ldx, int64_t ldy, int64_t ldo, int64_t bsx, int64_t bsy,
                int64_t bse, const Epilogue<double> epi, const SplitK sk) {
  constexpr int BM = TILE, BN = TILE, R = TILE / 16;
  __shared__ double Xs[BK][BM];
  __shared__ double Ys[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  int64_t m0, n0, b = 0, kbeg = 0, kend = K;
  double* part = nullptr;  // this piece's partial sums (split tiles only)
  if (sk.parts == 0) {
    m0 = (int64_t)blockIdx.y * BM;
    n0 = (int64_t)blockIdx.x * BN;
    b = blockIdx.z;
  } else {
    int64_t t = blockIdx.x;
    if (t >= sk.first) {
      const int64_t piece = t - sk.first;
      t = sk.first + piece / sk.parts;
      kbeg = (piece % sk.parts) * sk.kchunk;
      kend = min(K, kbeg + sk.kchunk);
      part = sk.ws + piece * (int64_t)(BM * BN);
    }
    m0 = (t / sk.ntn) * BM;
    n0 = (t % sk.ntn) * BN;
  }
  X += b * bsx;
  Y += b * bsy;

  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
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

  if (part) {  // a piece of a split tile: its partial sums, for the finishing kernel
    double2* dst = reinterpret_cast<double2*>(part + (int64_t)tid * R * R);
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; j += 2) dst[(i * R + j) / 2] = make_double2(acc[i][j], acc[i][j + 1]);
    return;
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
      epilogue_store(epi, eoff, r, c, ldo, acc[i][j]);
    }
  }
}

// The split tiles: tile first + blockIdx.x adds its pieces' partial sums in
// piece order and runs the epilogue, with the main kernel's thread layout.
template <int TILE>
__global__ void __launch_bounds__(THREADS)
gemm_f64_split_finish(int64_t M, int64_t N, int64_t ldo, const Epilogue<double> epi, const SplitK sk) {
  constexpr int R = TILE / 16;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t t = sk.first + blockIdx.x;
  const int64_t m0 = (t / sk.ntn) * TILE, n0 = (t % sk.ntn) * TILE;
  const double* base = sk.ws + (int64_t)blockIdx.x * sk.parts * (TILE * TILE) + (int64_t)tid * R * R;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = base[i * R + j];
  for (int p = 1; p < sk.parts; ++p) {
    const double* src = base + (int64_t)p * (TILE * TILE);
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[i][j] += src[i * R + j];
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t r = m0 + (i / 4) * 64 + ty * 4 + (i % 4);
    if (r >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int64_t c = n0 + (j / 4) * 64 + tx * 4 + (j % 4);
      if (c >= N) continue;
      epilogue_store(epi, 0, r, c, ldo, acc[i][j]);
    }
  }
}

// Small products (a single matrix of order up to a few hundred has too few
// 64-wide tiles to occupy the SMs, and each SM retires only two FP64 FMAs a
// clock): TS x TS outputs per CTA, one per thread, k-slices of TS staged in
// shared memory.
template <int TS, bool TX, bool TY>
__global__ void __launch_bounds__(TS * TS)
gemm_f64_small_kernel(const double* __restrict__ X, const double* __restrict__ Y, int64_t M, int64_t N,
                      int64_t K, int64_t ldx, int64_t ldy, int64_t ldo, int64_t bsx, int64_t bsy,
                      int64_t bse, const Epilogue<double> epi) {
  __shared__ double Xs[TS][TS + 1];  // [m][k]
  __shared__ double Ys[TS][TS + 1];  // [k][n]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t m0 = (int64_t)blockIdx.y * TS, n0 = (int64_t)blockIdx.x * TS;
  const int64_t b = blockIdx.z;
  X += b * bsx;
  Y += b * bsy;
  double acc = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += TS) {
    {  // thread (ty, tx) loads op(X)[m0 + ty][k0 + tx] and op(Y)[k0 + ty][n0 + tx]
      const int64_t gm = m0 + ty, gk = k0 + tx;
      Xs[ty][tx] = (gm < M && gk < K) ? (TX ? X[gk * ldx + gm] : X[gm * ldx + gk]) : 0.0;
      const int64_t gk2 = k0 + ty, gn = n0 + tx;
      Ys[ty][tx] = (gk2 < K && gn < N) ? (TY ? Y[gn * ldy + gk2] : Y[gk2 * ldy + gn]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TS; ++kk) acc = fma(Xs[ty][kk], Ys[kk][tx], acc);
    __syncthreads();
  }
  const int64_t r = m0 + ty, c = n0 + tx;
  if (r < M && c < N) epilogue_store(epi, b * bse, r, c, ldo, acc);
}

// How to split the last wave of 128-wide tiles of one M x N x K product
// over K: the tiles that do not fill a last wave of the SMs' resident CTAs
// (W per wave) run as `parts` pieces each, so that the pieces spread over all
// the SMs (a partial wave of tail tiles takes a whole tile time; tail x parts
// pieces take ceil(tail parts / W) / parts of one).  parts = 0: no split.
struct SplitPlan {
  int64_t tiles = 0, tail = 0, kchunk = 0;
  int parts = 0, ntn = 0;
  size_t bytes = 0;
};

// One 128-wide CTA per SM: 256 threads of about 200 registers each (the
// plan only needs the count to balance the pieces, not to be correct, and the
// workspace query that sizes their scratch must not create a context).
int resident_ctas_128(int sms) { return sms; }

SplitPlan split_plan(int64_t M, int64_t N, int64_t K, int sms) {
  SplitPlan sp;
  const int64_t ntm = (M + 127) / 128;
  sp.ntn = (int)((N + 127) / 128);
  sp.tiles = ntm * sp.ntn;
  if (sms <= 0 || sp.tiles < 2 * (int64_t)sms) return sp;  // the 128-wide kernel runs from two waves on
  const int64_t W = resident_ctas_128(sms);
  sp.tail = sp.tiles % W;
  if (sp.tail == 0) return sp;
  double best = 1.0;
  int parts = 1;
  for (int q = 2; q <= 4; ++q) {
    if (K / q < 512) break;  // pieces of at least 512 k
    const double cost = (double)((sp.tail * q + W - 1) / W) / q;
    if (cost < best - 0.05) {
      best = cost;
      parts = q;
    }
  }
  if (parts == 1) return sp;
  sp.kchunk = ((K + parts - 1) / parts + BK - 1) / BK * BK;
  sp.parts = (int)((K + sp.kchunk - 1) / sp.kchunk);
  sp.bytes = (size_t)sp.tail * sp.parts * 128 * 128 * sizeof(double);
  return sp;
}

int current_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return sms;
}

}  // namespace

size_t gemm_f64_split_bytes(int64_t M, int64_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  return split_plan(M, N, K, current_sms()).bytes;
}

cs_status gemm_f64(const double* X, const double* Y, int64_t M, int64_t N, int64_t K, int64_t ldx,
                   int64_t ldy, bool transX, bool transY, const Epilogue<double>& epi, int64_t ldo,
                   int64_t batch, int64_t bsx, int64_t bsy, int64_t bse, cudaStream_t stream, void* split_ws,
                   size_t split_bytes) {
  if (M <= 0 || N <= 0 || batch <= 0) return CS_OK;
  // 128-wide tiles unless that leaves fewer than two waves of CTAs (small
  // batched products), where 64-wide tiles balance the SMs better.
  int dev = 0, sms = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  CS_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // 128-wide tiles; 64-wide ones if that leaves fewer than two waves of
  // CTAs; 16- or 8-wide single-output-per-thread tiles when even 64-wide
  // tiles would leave most SMs idle (single matrices of small order).
  auto ctas = [&](int t) { return ((M + t - 1) / t) * ((N + t - 1) / t) * batch; };
  int tile = ctas(128) < 2 * (int64_t)sms ? 64 : 128;
  if (tile == 64 && ctas(64) < sms / 2) tile = ctas(16) >= sms / 2 ? 16 : 8;
  // Batches of small products (a 128-wide tile or a few per matrix, as the
  // adjoint's 512 products of order 128): 64-wide tiles, four times the
  // CTAs, fill the last wave better and hide the short K loop's latency
  // (512 x n = 128 adjoint: 117 -> 104 ms).
  if (batch > 1 && tile == 128 && ((M + 127) / 128) * ((N + 127) / 128) <= 4) tile = 64;
  if ((M + tile - 1) / tile > 65535 || batch > 65535) return fail(CS_EINVAL, "gemm_f64: grid too large");
  dim3 grid((unsigned)((N + tile - 1) / tile), (unsigned)((M + tile - 1) / tile), (unsigned)batch);
  ProfScope prof(CS_KERNEL_GEMM_F64, 2.0 * (double)M * (double)N * (double)K * (double)batch, stream);
  if (tile <= 16) {
#define CS_F64_SMALL(TS)                                                                                            \
  {                                                                                                                 \
    const dim3 blk(TS, TS);                                                                                         \
    if (!transX && !transY)                                                                                         \
      gemm_f64_small_kernel<TS, false, false><<<grid, blk, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi); \
    else if (transX && !transY)                                                                                     \
      gemm_f64_small_kernel<TS, true, false><<<grid, blk, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi);  \
    else if (!transX && transY)                                                                                     \
      gemm_f64_small_kernel<TS, false, true><<<grid, blk, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi);  \
    else                                                                                                            \
      gemm_f64_small_kernel<TS, true, true><<<grid, blk, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi);   \
  }
    if (tile == 16) CS_F64_SMALL(16) else CS_F64_SMALL(8)
#undef CS_F64_SMALL
    CS_CUDA_CHECK(cudaGetLastError());
    return CS_OK;
  }
  SplitK sk;
  if (tile == 128 && batch == 1 && split_ws) {
    const SplitPlan sp = split_plan(M, N, K, sms);
    if (sp.parts > 1 && sp.bytes <= split_bytes) {
      sk.first = sp.tiles - sp.tail;
      sk.kchunk = sp.kchunk;
      sk.parts = sp.parts;
      sk.ntn = sp.ntn;
      sk.ws = (double*)split_ws;
      const int64_t ctas = sk.first + sp.tail * sp.parts;
      if (ctas > INT32_MAX) return fail(CS_EINVAL, "gemm_f64: grid too large");
      grid = dim3((unsigned)ctas, 1, 1);
    }
  }
#define CS_F64_LAUNCH(T)                                                                                           \
  if (!transX && !transY)                                                                                          \
    gemm_f64_kernel<T, false, false><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi, sk); \
  else if (transX && !transY)                                                                                      \
    gemm_f64_kernel<T, true, false><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi, sk);  \
  else if (!transX && transY)                                                                                      \
    gemm_f64_kernel<T, false, true><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi, sk);  \
  else                                                                                                             \
    gemm_f64_kernel<T, true, true><<<grid, THREADS, 0, stream>>>(X, Y, M, N, K, ldx, ldy, ldo, bsx, bsy, bse, epi, sk);
  if (tile == 64) {
    CS_F64_LAUNCH(64)
  } else {
    CS_F64_LAUNCH(128)
  }
#undef CS_F64_LAUNCH
  if (sk.parts > 1) {
    CS_CUDA_CHECK(cudaGetLastError());
    gemm_f64_split_finish<128><<<(unsigned)(grid.x - sk.first) / (unsigned)sk.parts, THREADS, 0, stream>>>(M, N, ldo, epi, sk);
  }
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

namespace {

// Register-only FP64 FMA throughput: every thread runs CH independent
// dependency chains, so the FP64 pipes rather than latency set the rate.  The
// multiplier and addend come in as arguments, so every FMA takes register
// operands as the product kernels' do.
template <int CH>
__global__ void fma_rate_kernel(double* out, long long rounds, double b, double c) {
  double a[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) a[i] = 1.0 + 1e-3 * i + 1e-9 * threadIdx.x;
  for (long long r = 0; r < rounds; ++r) {
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = fma(a[i], b, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < CH; ++i) sum += a[i];
  if (sum == 12345.678) out[blockIdx.x] = sum;  // never true; keeps the chains live
}

}  // namespace

}  // namespace cs

extern "C" cs_status cossin_fp64_product_launches(int64_t M, int64_t N, int64_t K, int32_t* launches) {
  using namespace cs;
  if (!launches || M < 0 || N < 0 || K < 0) return fail(CS_EINVAL, "cossin_fp64_product_launches: bad arguments");
  *launches = (M == 0 || N == 0) ? 0 : (gemm_f64_split_bytes(M, N, K) > 0 ? 2 : 1);
  return CS_OK;
}

extern "C" cs_status cossin_fp64_fma_rate(int64_t rounds, double* tflops, cossin_stream_t stream) {
  using namespace cs;
  if (!tflops) return fail(CS_EINVAL, "tflops is null");
  if (rounds <= 0 || rounds > (int64_t(1) << 30)) return fail(CS_EINVAL, "rounds must be in [1, 2^30]");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  CS_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * 4;
  double* out = nullptr;
  CS_CHECK(dev_alloc((void**)&out, sizeof(double) * grid, st, "cossin_fp64_fma_rate scratch"));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cs_status rc = CS_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = fail(CS_ECUDA, "cudaEventCreate");
  if (rc == CS_OK) {
    fma_rate_kernel<16><<<grid, 256, 0, st>>>(out, rounds / 8 + 1, 0.9999999, 1e-9);  // warm-up
    cudaEventRecord(e0, st);
    fma_rate_kernel<16><<<grid, 256, 0, st>>>(out, rounds, 0.9999999, 1e-9);
    cudaEventRecord(e1, st);
    const cudaError_t ce = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (ce != cudaSuccess) rc = cuda_fail(ce, "fma_rate_kernel");
    else if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) rc = fail(CS_ECUDA, "event timing failed");
    else *tflops = 2.0 * 16.0 * (double)rounds * 256.0 * grid / (ms * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  return rc;
}
