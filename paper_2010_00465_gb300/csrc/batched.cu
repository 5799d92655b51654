// batched.cu -- cos/sin of many FP32 matrices of uneven order and norm, each
// with its own (2m, s), in one persistent launch.
//
// Every CTA takes matrices from a device work queue (longest first: the host
// orders the batch by n^3), computes ||A||_1 (FP64 accumulation), chooses
// (2m, s) from Table 2 on the device, and runs the same product plan as the
// single-matrix path: Pi_2m products with the scheme's linear combinations
// fused into each product's epilogue, then s double-angle products
// [C; S] C.  Orders are at most kMaxOrder = 256, so the products are CTA-level
// FP32 FMA tiles (IEEE accumulation; intermediates stay in the CTA's own
// workspace slice, hot in L2).  Tile shapes (64 or 128 rows/columns per CTA
// tile for orders above 64) and occupancies are timed by the plan's autotuner.
//
// Graph capture: the plan records the queue reset and the persistent launch
// in a CUDA graph once; each replay is one graph launch.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "internal.cuh"
#include "plan.h"
#include "theta_table.cuh"

namespace cs {
namespace bt {

constexpr int kThreads = 256;
constexpr int kMaxOrder = 256;
constexpr int kBK = 16;
constexpr int kSlots = 8 + 4;  // W0..W7 and two stacked [C; S] buffers (2 each)

// One product of a plan in dense form: distinct input slots in[], and for
// every output t: out_t = alpha_t P + gamma_t I + sum_q beta[t][q] in_q
// + sum_{u<t} delta[t][u] out_u; scale[t] multiplies alpha_t by 4^-s (1) or
// 2^-s (2).
struct DStep {
  int X, Y, nout, nin;
  int out[EPI_MAX_OUT];
  int in[EPI_MAX_IN];
  int scale[EPI_MAX_OUT];
  float alpha[EPI_MAX_OUT];
  float gamma[EPI_MAX_OUT];
  float beta[EPI_MAX_OUT][EPI_MAX_IN];
  float delta[EPI_MAX_OUT][EPI_MAX_OUT];
};
struct DPlan {
  int nsteps;
  DStep step[8];
};

__constant__ DPlan c_plans[4];

struct Desc {
  const float* A;
  float* C;
  float* S;
  int64_t n;
};

struct Slots {
  float* p[SL_COUNT];
};

// Block-wide ||A||_1 with FP64 accumulation: one thread per column.
__device__ double block_norm1(const float* __restrict__ A, int n, double* red) {
  double best = 0.0;
  bool nan = false;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double sum = 0.0;
    for (int r = 0; r < n; ++r) sum += fabs((double)A[(int64_t)r * n + c]);
    if (isnan(sum)) nan = true;
    best = fmax(best, sum);
  }
  if (nan) best = __longlong_as_double(0x7ff8000000000000ULL);
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, best, off);
    best = (isnan(best) || isnan(o)) ? __longlong_as_double(0x7ff8000000000000ULL) : fmax(best, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  double r = red[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
    r = (isnan(r) || isnan(red[w])) ? __longlong_as_double(0x7ff8000000000000ULL) : fmax(r, red[w]);
  __syncthreads();
  return r;
}

// One CTA product P = X Y (M x N, inner K, leading dimension ld for every
// matrix) in tiles of T x T; the epilogue is either a plan step (st != null)
// or the stacked double-angle form (rows < split to outC as 2X - I, the rest
// to outS as 2X).
//
// 256 threads as 16 x 16; thread (ty, tx) owns rows {ty*H + i, T/2 + ty*H + i}
// and columns {tx*H + j, T/2 + tx*H + j}, H = T/32, so that its operands are
// read from shared memory as float4 without bank conflicts.  The k-panels
// (kBK deep) are double-buffered: the next panel is fetched from global
// memory into registers while the current one is multiplied.
template <int T>
__device__ void cta_product(const float* __restrict__ X, const float* __restrict__ Y, int M, int N, int K, int ld,
                            const DStep* st, const Slots& sl, float a2, float as, int split, float* outC,
                            float* outS, float* smem) {
  constexpr int H = T / 32;      // half micro-tile edge: 4 (T = 128) or 2 (T = 64)
  constexpr int R = 2 * H;       // micro-tile edge
  constexpr int LD = T + 4;      // shared-memory row pitch (floats)
  constexpr int PER = (T * kBK) / kThreads;  // panel elements per thread per operand
  float (*Xs)[kBK][LD] = reinterpret_cast<float (*)[kBK][LD]>(smem);           // [2][kBK][LD]
  float (*Ys)[kBK][LD] = reinterpret_cast<float (*)[kBK][LD]>(smem + 2 * kBK * LD);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* inp[EPI_MAX_IN];
  float* outp[EPI_MAX_OUT];
  float alph[EPI_MAX_OUT];
  int nin = 0, nout = 0;
  if (st) {
    nin = st->nin;
    nout = st->nout;
#pragma unroll
    for (int q = 0; q < EPI_MAX_IN; ++q) inp[q] = q < nin ? sl.p[st->in[q]] : nullptr;
#pragma unroll
    for (int t = 0; t < EPI_MAX_OUT; ++t) {
      outp[t] = t < nout ? sl.p[st->out[t]] : nullptr;
      alph[t] = st->scale[t] == 1 ? st->alpha[t] * a2 : st->scale[t] == 2 ? st->alpha[t] * as : st->alpha[t];
    }
  }
  for (int m0 = 0; m0 < M; m0 += T) {
    for (int n0 = 0; n0 < N; n0 += T) {
      float acc[R][R];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = 0.f;
      float xr[PER], yr[PER];
#define CS_BT_FETCH(k0_)                                                     \
  _Pragma("unroll") for (int t = 0; t < PER; ++t) {                          \
    const int e = tid + t * kThreads;                                        \
    const int mm = e / kBK, kk = e % kBK;                                    \
    const int gm = m0 + mm, gk = (k0_) + kk;                                 \
    xr[t] = (gm < M && gk < K) ? X[(int64_t)gm * ld + gk] : 0.f;             \
    const int kk2 = e / T, nn = e % T;                                       \
    const int gk2 = (k0_) + kk2, gn = n0 + nn;                               \
    yr[t] = (gk2 < K && gn < N) ? Y[(int64_t)gk2 * ld + gn] : 0.f;           \
  }
#define CS_BT_STASH(buf_)                                                    \
  _Pragma("unroll") for (int t = 0; t < PER; ++t) {                          \
    const int e = tid + t * kThreads;                                        \
    Xs[(buf_)][e % kBK][e / kBK] = xr[t];                                    \
    Ys[(buf_)][e / T][e % T] = yr[t];                                        \
  }
      CS_BT_FETCH(0)
      CS_BT_STASH(0)
      __syncthreads();
      int buf = 0;
      for (int k0 = 0; k0 < K; k0 += kBK) {
        const bool more = k0 + kBK < K;
        if (more) {
          CS_BT_FETCH(k0 + kBK)
        }
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
          float a[R], b[R];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int q = 0; q < H; q += 4 > H ? H : 4) {
              if (H >= 4) {
                const float4 va = *reinterpret_cast<const float4*>(&Xs[buf][kk][h * (T / 2) + ty * H + q]);
                const float4 vb = *reinterpret_cast<const float4*>(&Ys[buf][kk][h * (T / 2) + tx * H + q]);
                a[h * H + q] = va.x; a[h * H + q + 1] = va.y; a[h * H + q + 2] = va.z; a[h * H + q + 3] = va.w;
                b[h * H + q] = vb.x; b[h * H + q + 1] = vb.y; b[h * H + q + 2] = vb.z; b[h * H + q + 3] = vb.w;
              } else {
                const float2 va = *reinterpret_cast<const float2*>(&Xs[buf][kk][h * (T / 2) + ty * H]);
                const float2 vb = *reinterpret_cast<const float2*>(&Ys[buf][kk][h * (T / 2) + tx * H]);
                a[h * H] = va.x; a[h * H + 1] = va.y;
                b[h * H] = vb.x; b[h * H + 1] = vb.y;
              }
            }
          }
#pragma unroll
          for (int i = 0; i < R; ++i)
#pragma unroll
            for (int j = 0; j < R; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
          CS_BT_STASH(buf ^ 1)
          __syncthreads();
          buf ^= 1;
        }
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {  // unrolled: acc[i][j] stays in registers
        const int r = m0 + (i < H ? ty * H + i : T / 2 + ty * H + (i - H));
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int c = n0 + (j < H ? tx * H + j : T / 2 + tx * H + (j - H));
          if (c >= N) continue;
          const float p = acc[i][j];
          if (!st) {
            if (r < split) outC[(int64_t)r * ld + c] = 2.f * p - (r == c ? 1.f : 0.f);
            else outS[(int64_t)(r - split) * ld + c] = 2.f * p;
            continue;
          }
          const int64_t idx = (int64_t)r * ld + c;
          float in[EPI_MAX_IN], o[EPI_MAX_OUT];
#pragma unroll
          for (int q = 0; q < EPI_MAX_IN; ++q) in[q] = q < nin ? inp[q][idx] : 0.f;
#pragma unroll
          for (int t = 0; t < EPI_MAX_OUT; ++t) {
            if (t >= nout) break;
            float v = alph[t] * p + (r == c ? st->gamma[t] : 0.f);
#pragma unroll
            for (int q = 0; q < EPI_MAX_IN; ++q)
              if (q < nin) v = fmaf(st->beta[t][q], in[q], v);
#pragma unroll
            for (int u = 0; u < t; ++u) v = fmaf(st->delta[t][u], o[u], v);
            o[t] = v;
          }
#pragma unroll
          for (int t = 0; t < EPI_MAX_OUT; ++t)
            if (t < nout) outp[t][idx] = o[t];
        }
      }
      __syncthreads();  // the next tile overwrites both panel buffers
    }
  }
#undef CS_BT_FETCH
#undef CS_BT_STASH
}

// T is the tile edge for orders above 64; orders <= 64 always use 64-wide tiles.
template <int T, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) batched_kernel(const Desc* __restrict__ desc, const int* __restrict__ order,
                                                           int count, int* queue, float* ws_all, int64_t ws_per_cta,
                                                           cs_info* infos, int32_t* status) {
  __shared__ __align__(16) float panels[4 * kBK * (T + 4)];
  __shared__ double red[kThreads / 32];
  __shared__ int item;
  float* ws = ws_all + (int64_t)blockIdx.x * ws_per_cta;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(queue, 1);
    __syncthreads();
    const int i = item;
    __syncthreads();
    if (i >= count) break;
    const int j = order[i];
    const Desc d = desc[j];
    const int n = (int)d.n;
    if (n <= 0) {
      if (threadIdx.x == 0) {
        if (status) status[j] = CS_OK;
        if (infos) infos[j] = cs_info{0.0, 4, 0, 0, 1, 0.0};
      }
      continue;
    }
    const double nrm = block_norm1(d.A, n, red);
    int f = 0, s = 0;
    const int sel = select_family(nrm, 1, &f, &s);
    if (threadIdx.x == 0) {
      if (status) status[j] = sel == 0 ? CS_OK : (sel == 3 ? CS_ENONFINITE : CS_ERANGE);
      if (infos) {
        const int prods = sel == 0 ? family_products(f) + 2 * s : 0;
        infos[j] = cs_info{nrm, sel == 0 ? family_order(f) : 0, sel == 0 ? s : 0, prods, 1,
                           2.0 * (double)n * n * n * prods};
      }
    }
    if (sel != 0) {
      const float qnan = __int_as_float(0x7fc00000);
      for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
        d.C[e] = qnan;
        d.S[e] = qnan;
      }
      __syncthreads();
      continue;
    }
    const int64_t n2 = (int64_t)n * n;
    float* ping0 = ws + 8 * n2;
    float* ping1 = ws + 10 * n2;
    Slots sl;
    sl.p[SL_A] = const_cast<float*>(d.A);
    sl.p[SL_C] = s == 0 ? d.C : ping0;
    sl.p[SL_S] = s == 0 ? d.S : ping0 + n2;
    for (int w = 0; w < kWorkSlots; ++w) sl.p[W(w)] = ws + w * n2;
    const float a2 = ldexpf(1.f, -2 * s), as = ldexpf(1.f, -s);
    const DPlan& P = c_plans[f];
    for (int k = 0; k < P.nsteps; ++k) {
      const DStep* st = &P.step[k];
      if (T == 128 && n > 64)
        cta_product<128>(sl.p[st->X], sl.p[st->Y], n, n, n, n, st, sl, a2, as, 0, nullptr, nullptr, panels);
      else
        cta_product<64>(sl.p[st->X], sl.p[st->Y], n, n, n, n, st, sl, a2, as, 0, nullptr, nullptr, panels);
    }
    for (int q = 0; q < s; ++q) {
      float* cur = (q & 1) ? ping1 : ping0;
      float* nxt = (q & 1) ? ping0 : ping1;
      const bool last = q == s - 1;
      if (T == 128 && n > 64)
        cta_product<128>(cur, cur, 2 * n, n, n, n, nullptr, sl, 0.f, 0.f, n, last ? d.C : nxt,
                         last ? d.S : nxt + n2, panels);
      else
        cta_product<64>(cur, cur, 2 * n, n, n, n, nullptr, sl, 0.f, 0.f, n, last ? d.C : nxt,
                        last ? d.S : nxt + n2, panels);
    }
  }
}

// ------------------------------------------------------------------- host ---
struct Variant {
  int tile;
  int ctas_per_sm;
};
// {64, 4} compiles with 64 registers per thread to fit 32 warps per SM; the
// autotuner keeps whichever variant is fastest on the batch.  (A 128-wide
// tile at 2 CTAs per SM would spill 3 KB per thread.)
const Variant kVariants[] = {{128, 1}, {64, 2}, {64, 1}, {64, 4}};

std::mutex g_mu;
bool g_plans_uploaded[64] = {};
std::map<std::string, int> g_tuned;  // batch signature -> variant index

cs_status upload_plans() {
  int dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev >= 0 && dev < 64 && g_plans_uploaded[dev]) return CS_OK;
  DPlan host[4];
  for (int f = 0; f < 4; ++f) {
    const int m = family_order(f);
    std::vector<Step> steps = chain_plan(m, 0);
    DPlan& P = host[f];
    P = DPlan{};
    P.nsteps = (int)steps.size();
    for (size_t k = 0; k < steps.size(); ++k) {
      DStep& D = P.step[k];
      D = DStep{};
      D.X = steps[k].X;
      D.Y = steps[k].Y;
      D.nout = (int)steps[k].outs.size();
      for (int t = 0; t < D.nout; ++t) {
        const OutSpec& o = steps[k].outs[t];
        D.out[t] = o.slot;
        D.alpha[t] = (float)o.alpha;
        D.gamma[t] = (float)o.gamma;
        D.scale[t] = (k == 0) ? 1 : (o.slot == SL_S ? 2 : 0);
        for (auto& b : o.beta) {
          int q = -1;
          for (int z = 0; z < D.nin; ++z)
            if (D.in[z] == b.first) q = z;
          if (q < 0) {
            q = D.nin++;
            D.in[q] = b.first;
          }
          D.beta[t][q] = (float)b.second;
        }
        for (auto& d : o.delta) D.delta[t][d.first] = (float)d.second;
      }
    }
  }
  CS_CUDA_CHECK(cudaMemcpyToSymbol(c_plans, host, sizeof(host)));
  if (dev >= 0 && dev < 64) g_plans_uploaded[dev] = true;
  return CS_OK;
}

int sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 152;
  return sms;
}

struct BLayout {
  size_t desc = 0, order = 0, queue = 0, scratch = 0, total = 0;
  int64_t per_cta = 0;
  int max_ctas = 0;
};

BLayout make_blayout(int64_t count, int64_t nmax) {
  BLayout L;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t off = 0;
  L.desc = off;
  off += al(sizeof(Desc) * (size_t)std::max<int64_t>(count, 1));
  L.order = off;
  off += al(sizeof(int) * (size_t)std::max<int64_t>(count, 1));
  L.queue = off;
  off += 256;
  L.per_cta = kSlots * nmax * nmax;
  L.max_ctas = sm_count() * 4;
  L.scratch = off;
  off += al(sizeof(float) * (size_t)L.per_cta * L.max_ctas);
  L.total = off;
  return L;
}

cs_status launch_variant(int v, const BLayout& L, char* ws, int count, cs_info* infos, int32_t* status,
                         cudaStream_t stream) {
  const Variant& V = kVariants[v];
  const int grid = std::min(L.max_ctas, sm_count() * V.ctas_per_sm);
  int* queue = (int*)(ws + L.queue);
  CS_CUDA_CHECK(cudaMemsetAsync(queue, 0, sizeof(int), stream));
  const Desc* desc = (const Desc*)(ws + L.desc);
  const int* order = (const int*)(ws + L.order);
  float* scratch = (float*)(ws + L.scratch);
  if (V.tile == 128)
    batched_kernel<128, 1><<<grid, kThreads, 0, stream>>>(desc, order, count, queue, scratch, L.per_cta, infos, status);
  else if (V.ctas_per_sm >= 4)
    batched_kernel<64, 4><<<grid, kThreads, 0, stream>>>(desc, order, count, queue, scratch, L.per_cta, infos, status);
  else
    batched_kernel<64, 2><<<grid, kThreads, 0, stream>>>(desc, order, count, queue, scratch, L.per_cta, infos, status);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

}  // namespace bt

struct BatchedPlan {
  int64_t count = 0;
  bt::BLayout L;
  char* ws = nullptr;
  cs_info* infos = nullptr;
  int32_t* status = nullptr;
  int variant = 0;
  double flops_estimate = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

cs_status validate_batch(int64_t count, const int64_t* n, int64_t* nmax) {
  if (count < 0) return fail(CS_EINVAL, "count must be >= 0");
  if (count > (1 << 30)) return fail(CS_EINVAL, "count too large");
  if (count > 0 && !n) return fail(CS_EINVAL, "n is null");
  int64_t mx = 1;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] < 0 || n[i] > bt::kMaxOrder)
      return fail(CS_EINVAL, "batched orders must be in [0, 256] (use cossin for larger matrices)");
    mx = std::max(mx, n[i]);
  }
  *nmax = mx;
  return CS_OK;
}

}  // namespace
}  // namespace cs

extern "C" {

cs_status cossin_batched_workspace_size(int64_t count, const int64_t* n, size_t* bytes) {
  if (!bytes) return cs::fail(CS_EINVAL, "bytes is null");
  int64_t nmax = 1;
  CS_CHECK(cs::validate_batch(count, n, &nmax));
  *bytes = cs::bt::make_blayout(count, nmax).total;
  return CS_OK;
}

cs_status cossin_batched_plan_create(int64_t count, const int64_t* n, const float* const* A, float* const* C,
                                     float* const* S, void* ws_dev, size_t ws_bytes, cs_info* infos_dev,
                                     int32_t* status_dev, int32_t autotune, cossin_stream_t stream,
                                     cossin_batched_plan* plan_out) {
  using namespace cs;
  if (!plan_out) return fail(CS_EINVAL, "plan is null");
  *plan_out = nullptr;
  int64_t nmax = 1;
  CS_CHECK(validate_batch(count, n, &nmax));
  if (count > 0 && (!A || !C || !S)) return fail(CS_EINVAL, "null pointer array");
  const bt::BLayout L = bt::make_blayout(count, nmax);
  if (!ws_dev || ws_bytes < L.total) return fail(CS_EINVAL, "workspace missing or too small");
  if (((uintptr_t)ws_dev & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
  std::vector<bt::Desc> desc((size_t)count);
  double flops_est = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] > 0 && (!A[i] || !C[i] || !S[i])) return fail(CS_EINVAL, "null matrix pointer in batch");
    desc[i] = bt::Desc{A[i], C[i], S[i], n[i]};
    flops_est += 2.0 * (double)n[i] * n[i] * n[i];
  }
  std::vector<int> order((size_t)count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(bt::upload_plans());
  char* ws = (char*)ws_dev;
  if (count > 0) {
    CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.desc, desc.data(), sizeof(bt::Desc) * count, cudaMemcpyHostToDevice, st));
    CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
    CS_CUDA_CHECK(cudaStreamSynchronize(st));
  }
  BatchedPlan* P = new BatchedPlan;
  P->count = count;
  P->L = L;
  P->ws = ws;
  P->infos = infos_dev;
  P->status = status_dev;
  P->flops_estimate = flops_est;
  // Autotuner: time every variant on this batch, keep the fastest; the
  // choice is remembered per (device, count, largest order) in this process.
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string key = std::to_string(dev) + ":" + std::to_string(count) + ":" + std::to_string(nmax);
  int chosen = -1;
  {
    std::lock_guard<std::mutex> lk(bt::g_mu);
    auto it = bt::g_tuned.find(key);
    if (it != bt::g_tuned.end()) chosen = it->second;
  }
  const int nvar = (int)(sizeof(bt::kVariants) / sizeof(bt::kVariants[0]));
  if (chosen < 0 && autotune && count > 0) {
    cudaEvent_t e0, e1;
    CS_CUDA_CHECK(cudaEventCreate(&e0));
    CS_CUDA_CHECK(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int v = 0; v < nvar; ++v) {
      cs_status rc = bt::launch_variant(v, L, ws, (int)count, infos_dev, status_dev, st);  // warm-up
      if (rc == CS_OK) {
        cudaEventRecord(e0, st);
        rc = bt::launch_variant(v, L, ws, (int)count, infos_dev, status_dev, st);
        cudaEventRecord(e1, st);
      }
      float ms = 0.f;
      if (rc != CS_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        delete P;
        return rc != CS_OK ? rc : cuda_fail(cudaGetLastError(), "batched autotune");
      }
      if (ms < best) {
        best = ms;
        chosen = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lk(bt::g_mu);
    bt::g_tuned[key] = chosen;
  }
  if (chosen < 0) chosen = 0;
  P->variant = chosen;
  // Capture the queue reset and the persistent launch once.
  cudaStream_t cap;
  CS_CUDA_CHECK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cs_status rc = CS_OK;
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    rc = cuda_fail(cudaGetLastError(), "cudaStreamBeginCapture");
  } else {
    rc = count > 0 ? bt::launch_variant(chosen, L, ws, (int)count, infos_dev, status_dev, cap) : CS_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (rc == CS_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamEndCapture");
    if (rc == CS_OK) {
      e = cudaGraphInstantiate(&P->exec, g, 0);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
    }
    P->graph = g;
  }
  cudaStreamDestroy(cap);
  if (rc != CS_OK) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P;
    return rc;
  }
  *plan_out = (cossin_batched_plan)P;
  return CS_OK;
}

cs_status cossin_batched_plan_launch(cossin_batched_plan plan, cossin_stream_t stream) {
  using namespace cs;
  if (!plan) return fail(CS_EINVAL, "plan is null");
  BatchedPlan* P = (BatchedPlan*)plan;
  if (P->count == 0) return CS_OK;
  ProfScope prof(CS_KERNEL_BATCHED, P->flops_estimate, (cudaStream_t)stream);
  CS_CUDA_CHECK(cudaGraphLaunch(P->exec, (cudaStream_t)stream));
  return CS_OK;
}

cs_status cossin_batched_plan_info(cossin_batched_plan plan, int32_t* variant_tile, int32_t* variant_ctas_per_sm) {
  if (!plan) return cs::fail(CS_EINVAL, "plan is null");
  cs::BatchedPlan* P = (cs::BatchedPlan*)plan;
  if (variant_tile) *variant_tile = cs::bt::kVariants[P->variant].tile;
  if (variant_ctas_per_sm) *variant_ctas_per_sm = cs::bt::kVariants[P->variant].ctas_per_sm;
  return CS_OK;
}

cs_status cossin_batched_plan_destroy(cossin_batched_plan plan) {
  if (!plan) return CS_OK;
  cs::BatchedPlan* P = (cs::BatchedPlan*)plan;
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  delete P;
  return CS_OK;
}

cs_status cossin_batched(int64_t count, const int64_t* n, const float* const* A, float* const* C, float* const* S,
                         void* ws_dev, size_t ws_bytes, cs_info* infos_dev, int32_t* status_dev,
                         cossin_stream_t stream) {
  using namespace cs;
  int64_t nmax = 1;
  CS_CHECK(validate_batch(count, n, &nmax));
  if (count == 0) return CS_OK;
  if (!A || !C || !S) return fail(CS_EINVAL, "null pointer array");
  const bt::BLayout L = bt::make_blayout(count, nmax);
  if (!ws_dev || ws_bytes < L.total) return fail(CS_EINVAL, "workspace missing or too small");
  if (((uintptr_t)ws_dev & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
  std::vector<bt::Desc> desc((size_t)count);
  double flops_est = 0;
  for (int64_t i = 0; i < count; ++i) {
    if (n[i] > 0 && (!A[i] || !C[i] || !S[i])) return fail(CS_EINVAL, "null matrix pointer in batch");
    desc[i] = bt::Desc{A[i], C[i], S[i], n[i]};
    flops_est += 2.0 * (double)n[i] * n[i] * n[i];
  }
  std::vector<int> order((size_t)count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(bt::upload_plans());
  char* ws = (char*)ws_dev;
  CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.desc, desc.data(), sizeof(bt::Desc) * count, cudaMemcpyHostToDevice, st));
  CS_CUDA_CHECK(cudaMemcpyAsync(ws + L.order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st));
  int variant = 0, dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(bt::g_mu);
    auto it = bt::g_tuned.find(std::to_string(dev) + ":" + std::to_string(count) + ":" + std::to_string(nmax));
    if (it != bt::g_tuned.end()) variant = it->second;
  }
  ProfScope prof(CS_KERNEL_BATCHED, flops_est, st);
  CS_CHECK(bt::launch_variant(variant, L, ws, (int)count, infos_dev, status_dev, st));
  // the host staging vectors must outlive the copies
  CS_CUDA_CHECK(cudaStreamSynchronize(st));
  return CS_OK;
}

}  // extern "C"
