// small_f64.cu -- cos/sin of one small FP64 matrix (n <= 128) in a single
// cooperative launch.
//
// For a single small matrix the separate steps cost more than their work:
// the 1-norm's host round trip (the (2m, s) choice needs it) and one launch
// per product, each product a handful of tiles.  Here one kernel does all of
// it: every CTA adds FP64 column sums of |A| for its columns, a grid barrier,
// every CTA takes the maximum and chooses (2m, s) from Table 1 itself (the
// same rule and table as the host), then the scheme's products and the
// double-angle steps run with 8 x 8 output tiles spread over the CTAs and a
// grid barrier after each product, the fused linear combinations in FP64.
// The kernel is launched cooperatively, so every CTA is resident and the
// barriers (bounded spins on a global generation word) always complete; a
// spin that runs out sets the error word and the CTAs return.
#include <cooperative_groups.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "plan.h"
#include "tc_gemm.h"
#include "theta_table.cuh"

namespace cs {
namespace sm {

constexpr int kTS = 8;                // output tile edge (one entry per thread)
constexpr int kThreads = kTS * kTS;
constexpr int64_t kMaxOrder = 128;
constexpr long long kSpinLimit = 1LL << 26;  // polls of the barrier word (far beyond any wait here)

// The plans of the five families (2m = 4, 8, 16, 24 and the T9 sine variant)
// in dense form with FP64 coefficients; scale[t] = 1 multiplies alpha_t by
// (scale 2^-s)^2, 2 by scale 2^-s.
struct Step64 {
  int X, Y, nout, nin;
  int out[EPI_MAX_OUT];
  int in[EPI_MAX_IN];
  int scale[EPI_MAX_OUT];
  double alpha[EPI_MAX_OUT];
  double gamma[EPI_MAX_OUT];
  double beta[EPI_MAX_OUT][EPI_MAX_IN];
  double delta[EPI_MAX_OUT][EPI_MAX_OUT];
};
struct Plan64 {
  int m, nsteps;
  Step64 step[8];
};
constexpr int kPlans = 5;
__constant__ Plan64 c_plan64[kPlans];

// Where the kernel keeps its barrier words, the column sums and the record
// of the call (in the caller's workspace).
struct Ctl {
  unsigned count, gen;
  int status, m, s;
  double norm1;
};

// Grid barrier: a release fetch-add on the arrival count; the last arrival
// resets it and bumps the generation word with a release add; the others
// poll the generation with acquire loads (bounded).
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ bool grid_barrier(Ctl* ctl, unsigned nblocks, int* err) {
  __syncthreads();
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned g = ld_acquire(&ctl->gen);
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], 1;" : "=r"(old) : "l"(&ctl->count) : "memory");
    if (old == nblocks - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&ctl->count) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&ctl->gen) : "memory");
    } else {
      long long polls = 0;
      while (ld_acquire(&ctl->gen) == g) {
        if (++polls > kSpinLimit) {
          ok = 0;
          atomicExch(err, 1);
          break;
        }
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

struct Slots {
  double* p[SL_COUNT];
};

// P = X Y (M x n, inner n) in kTS x kTS tiles over the grid, with the step's
// epilogue (st != null) or the double-angle epilogue (rows < n -> 2P - I to
// outC, rows >= n -> 2P to outS).  Matrices written earlier in this launch
// (by other SMs) are read through L2 only (ld.global.cg): an SM's L1 is not
// kept coherent with other SMs' stores.
__device__ void product(const double* X, const double* Y, int M, int n, const Step64* st, const Slots& sl,
                        double a2, double as, double* outC, double* outS) {
  // the tile's whole k range at once (n <= 128): one round trip to L2 per tile
  __shared__ double Xs[kTS][kMaxOrder + 1];  // rows r0.. of X
  __shared__ double Ys[kMaxOrder][kTS + 1];  // columns c0.. of Y
  const int tx = threadIdx.x % kTS, ty = threadIdx.x / kTS;
  const int tm = (M + kTS - 1) / kTS, tn = (n + kTS - 1) / kTS;
  for (int t = blockIdx.x; t < tm * tn; t += gridDim.x) {
    const int r0 = (t / tn) * kTS, c0 = (t % tn) * kTS;
    const int r = r0 + ty, c = c0 + tx;
    const bool mine = r < M && c < n;
    const int64_t idx = (int64_t)r * n + c;
    // this entry's epilogue inputs are loaded together with the panels
    double in[EPI_MAX_IN];
#pragma unroll
    for (int q = 0; q < EPI_MAX_IN; ++q) in[q] = (st && mine && q < st->nin) ? __ldcg(sl.p[st->in[q]] + idx) : 0.0;
    // every load of the two panels is issued before any is stored: X rows
    // r0.. (thread t takes k = t, t + 64 of all kTS rows) and Y columns c0..
    // (thread t takes column t % kTS of rows t / kTS + 8 q)
    constexpr int kXk = kMaxOrder / kThreads, kYq = kMaxOrder * kTS / kThreads;
    double xv[kTS][kXk], yv[kYq];
#pragma unroll
    for (int i = 0; i < kTS; ++i)
#pragma unroll
      for (int h = 0; h < kXk; ++h) {
        const int k = threadIdx.x + h * kThreads;
        xv[i][h] = (r0 + i < M && k < n) ? __ldcg(X + (int64_t)(r0 + i) * n + k) : 0.0;
      }
    const int yj = threadIdx.x % kTS, yk0 = threadIdx.x / kTS;
#pragma unroll
    for (int q = 0; q < kYq; ++q) {
      const int k = yk0 + q * (kThreads / kTS);
      yv[q] = (k < n && c0 + yj < n) ? __ldcg(Y + (int64_t)k * n + c0 + yj) : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kTS; ++i)
#pragma unroll
      for (int h = 0; h < kXk; ++h) Xs[i][threadIdx.x + h * kThreads] = xv[i][h];
#pragma unroll
    for (int q = 0; q < kYq; ++q) Ys[yk0 + q * (kThreads / kTS)][yj] = yv[q];
    __syncthreads();
    double acc = 0.0;
    for (int k = 0; k < n; ++k) acc = fma(Xs[ty][k], Ys[k][tx], acc);
    __syncthreads();
    if (!mine) continue;
    if (!st) {
      if (r < n) outC[(int64_t)r * n + c] = 2.0 * acc - (r == c ? 1.0 : 0.0);
      else outS[(int64_t)(r - n) * n + c] = 2.0 * acc;
      continue;
    }
    double o[EPI_MAX_OUT];
#pragma unroll
    for (int u = 0; u < EPI_MAX_OUT; ++u) {
      if (u >= st->nout) break;
      const double al = st->alpha[u] * (st->scale[u] == 1 ? a2 : st->scale[u] == 2 ? as : 1.0);
      double v = al * acc + (r == c ? st->gamma[u] : 0.0);
#pragma unroll
      for (int q = 0; q < EPI_MAX_IN; ++q)
        if (q < st->nin) v = fma(st->beta[u][q], in[q], v);
#pragma unroll
      for (int w = 0; w < EPI_MAX_OUT; ++w)
        if (w < u) v = fma(st->delta[u][w], o[w], v);
      o[u] = v;
    }
#pragma unroll
    for (int u = 0; u < EPI_MAX_OUT; ++u)
      if (u < st->nout) sl.p[st->out[u]][idx] = o[u];
  }
}

struct Args {
  const double* A;
  double* C;
  double* S;
  double* w[kWorkSlots];
  double* ping[2];
  double* colsum;  // n doubles
  Ctl* ctl;
  int* err;
  int n;
  int force_m, force_s;
  double scale;
};

__global__ void __launch_bounds__(kThreads) small_cossin_kernel(const __grid_constant__ Args a) {
  const int n = a.n;
  const unsigned nb = gridDim.x;
  // 1. ||A||_1: CTA b sums columns b, b + G, ... (FP64; threads take rows,
  // the two warps' sums combined by shuffles and one shared word)
  __shared__ double part[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    double sum = 0.0;
    for (int r = threadIdx.x; r < n; r += kThreads) sum += fabs(a.A[(int64_t)r * n + c]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) part[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < kThreads / 32; ++i) t += part[i];
      a.colsum[c] = t;
    }
    __syncthreads();
  }
  if (!grid_barrier(a.ctl, nb, a.err)) return;
  // 2. every CTA takes the maximum (threads load the column sums together,
  // NaN propagates) and chooses (2m, s) the same way
  __shared__ double wmax[kThreads / 32];
  double nrm = 0.0;
  bool nan = false;
  for (int c = threadIdx.x; c < n; c += kThreads) {
    const double v = __ldcg(a.colsum + c);
    if (isnan(v)) nan = true;
    nrm = fmax(nrm, v);
  }
  const double qnan = __longlong_as_double(0x7ff8000000000000ULL);
  if (nan) nrm = qnan;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double o = __shfl_xor_sync(0xffffffffu, nrm, off);
    nrm = (isnan(nrm) || isnan(o)) ? qnan : fmax(nrm, o);
  }
  if (lane == 0) wmax[warp] = nrm;
  __syncthreads();
  nrm = wmax[0];
  for (int i = 1; i < kThreads / 32; ++i) nrm = (isnan(nrm) || isnan(wmax[i])) ? qnan : fmax(nrm, wmax[i]);
  nrm *= fabs(a.scale);
  // the choice runs on one thread (FP64 on GB300 is slow enough that 64
  // redundant copies of the loop cost microseconds) and is broadcast
  __shared__ int sel[3];
  if (threadIdx.x == 0) {
    int m = a.force_m, s = a.force_s, status = CS_OK;
    if (!isfinite(nrm)) {
      status = CS_ENONFINITE;
    } else if (m < 0) {
      int f = 0;
      if (select_family(nrm, 0, &f, &s) != 0) status = CS_ERANGE;
      else m = family_order(f);
    }
    sel[0] = status;
    sel[1] = m;
    sel[2] = s;
    if (blockIdx.x == 0) {
      a.ctl->status = status;
      a.ctl->m = m;
      a.ctl->s = s;
      a.ctl->norm1 = nrm;
    }
  }
  __syncthreads();
  const int status = sel[0], m = sel[1], s = sel[2];
  if (status != CS_OK) return;
  // plans in the order 4, 8, 9, 16, 24
  const int pi = m == 4 ? 0 : m == 8 ? 1 : m == 9 ? 2 : m == 16 ? 3 : 4;
  const Plan64& P = c_plan64[pi];
  // 3. the scheme's products, then the double-angle steps (ping-pong over
  // the stacked [C; S] buffers; the last step writes C and S)
  const int64_t n2 = (int64_t)n * n;
  Slots sl;
  sl.p[SL_A] = const_cast<double*>(a.A);
  sl.p[SL_C] = s == 0 ? a.C : a.ping[0];
  sl.p[SL_S] = s == 0 ? a.S : a.ping[0] + n2;
  for (int i = 0; i < kWorkSlots; ++i) sl.p[W(i)] = a.w[i];
  const double a2 = a.scale * a.scale * ldexp(1.0, -2 * s), as = a.scale * ldexp(1.0, -s);
  for (int k = 0; k < P.nsteps; ++k) {
    const Step64* st = &P.step[k];
    product(sl.p[st->X], sl.p[st->Y], n, n, st, sl, a2, as, nullptr, nullptr);
    if (!grid_barrier(a.ctl, nb, a.err)) return;
  }
  for (int j = 0; j < s; ++j) {
    const double* cur = a.ping[j & 1];
    const bool last = j == s - 1;
    double* nc = last ? a.C : a.ping[(j + 1) & 1];
    double* ns = last ? a.S : a.ping[(j + 1) & 1] + n2;
    product(cur, cur, 2 * n, n, nullptr, sl, 0.0, 0.0, nc, ns);
    if (!last && !grid_barrier(a.ctl, nb, a.err)) return;
  }
}

std::mutex g_mu;
unsigned long long g_uploaded = 0;  // one bit per device ordinal below 64

cs_status upload_plans() {
  int dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ULL << dev : 0ULL;
  std::lock_guard<std::mutex> lk(g_mu);
  if (bit && (g_uploaded & bit)) return CS_OK;
  Plan64 host[kPlans];
  const int ms[kPlans] = {4, 8, 9, 16, 24};
  for (int p = 0; p < kPlans; ++p) {
    const std::vector<Step> steps = chain_plan(ms[p], 0, 1.0);
    Plan64& P = host[p];
    P = Plan64{};
    P.m = ms[p];
    P.nsteps = (int)steps.size();
    if (P.nsteps > 8) return fail(CS_EINVAL, "plan longer than the small kernel holds");
    for (size_t k = 0; k < steps.size(); ++k) {
      Step64& D = P.step[k];
      D.X = steps[k].X;
      D.Y = steps[k].Y;
      D.nout = (int)steps[k].outs.size();
      for (int t = 0; t < D.nout; ++t) {
        const OutSpec& o = steps[k].outs[t];
        D.out[t] = o.slot;
        D.alpha[t] = o.alpha;
        D.gamma[t] = o.gamma;
        D.scale[t] = (k == 0) ? 1 : (o.slot == SL_S ? 2 : 0);
        for (auto& b : o.beta) {
          int q = -1;
          for (int z = 0; z < D.nin; ++z)
            if (D.in[z] == b.first) q = z;
          if (q < 0) {
            if (D.nin == EPI_MAX_IN) return fail(CS_EINVAL, "plan step reads too many matrices");
            q = D.nin++;
            D.in[q] = b.first;
          }
          D.beta[t][q] = b.second;
        }
        for (auto& d : o.delta) D.delta[t][d.first] = d.second;
      }
    }
  }
  CS_CUDA_CHECK(cudaMemcpyToSymbol(c_plan64, host, sizeof(host)));
  g_uploaded |= bit;
  return CS_OK;
}

}  // namespace sm

bool small_f64_eligible(cs_prec prec, int64_t n) { return prec == CS_FP64 && n >= 1 && n <= sm::kMaxOrder; }

// cos/sin of scale * A for one FP64 matrix of order n <= 128 (see the file
// comment).  The workspace is make_layout(n, CS_FP64); the call synchronises
// `stream` once at the end to report the status and fill `info`.
cs_status small_f64(const double* A, int64_t n, double* C, double* S, char* ws, const Layout& L, int32_t force_m,
                    int32_t force_s, cs_info* info, cudaStream_t stream, double scale) {
  using namespace sm;
  CS_CHECK(upload_plans());
  int dev = 0;
  CS_CUDA_CHECK(cudaGetDevice(&dev));
  // per-device constants of the launch, looked up once
  struct DevInfo {
    int* err = nullptr;
    int sms = 0, per_sm = 0;
  };
  static DevInfo g_dev[64];
  static std::mutex g_dev_mu;
  DevInfo di;
  {
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (dev >= 0 && dev < 64) di = g_dev[dev];
  }
  if (!di.err) {
    di.err = tc_error_word();
    if (!di.err) return fail(CS_ECUDA, "cannot resolve the device error word");
    CS_CUDA_CHECK(cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev));
    CS_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&di.per_sm, small_cossin_kernel, kThreads, 0));
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (dev >= 0 && dev < 64) g_dev[dev] = di;
  }
  int* err = di.err;
  Args a{};
  a.A = A;
  a.C = C;
  a.S = S;
  for (int i = 0; i < kWorkSlots; ++i) a.w[i] = (double*)(ws + L.w[i]);
  a.ping[0] = (double*)(ws + L.ping64[0]);
  a.ping[1] = (double*)(ws + L.ping64[1]);
  // the norm scratch of the layout holds the column sums and the control words
  a.colsum = (double*)(ws + L.norm_partial);
  a.ctl = (Ctl*)(ws + L.norm_out);
  a.err = err;
  a.n = (int)n;
  a.force_m = force_m;
  a.force_s = force_s;
  a.scale = scale;
  // as many CTAs as the largest product has tiles, at most one wave
  const int tiles = (int)(((2 * n + kTS - 1) / kTS) * ((n + kTS - 1) / kTS));
  const int grid = std::max(1, std::min(tiles, di.sms * std::max(di.per_sm, 1)));
  CS_CUDA_CHECK(cudaMemsetAsync(a.ctl, 0, sizeof(Ctl), stream));
  {
    ProfScope prof(CS_KERNEL_OTHER, 0.0, stream);
    void* params[] = {(void*)&a};
    CS_CUDA_CHECK(cudaLaunchCooperativeKernel((const void*)small_cossin_kernel, grid, kThreads, params, 0, stream));
  }
  // one synchronisation: the record of the call and the error word
  static thread_local Ctl* h_ctl = nullptr;
  static thread_local int* h_err = nullptr;
  if (!h_ctl) CS_CUDA_CHECK(cudaMallocHost((void**)&h_ctl, sizeof(Ctl)));
  if (!h_err) CS_CUDA_CHECK(cudaMallocHost((void**)&h_err, sizeof(int)));
  CS_CUDA_CHECK(cudaMemcpyAsync(h_ctl, a.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
  CS_CUDA_CHECK(cudaMemcpyAsync(h_err, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CS_CUDA_CHECK(cudaStreamSynchronize(stream));
  if (*h_err) {
    CS_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), stream));
    return fail(CS_ETIMEOUT, "a bounded wait gave up (in this or an earlier call)");
  }
  if (h_ctl->status == CS_ENONFINITE) return fail(CS_ENONFINITE, "||A||_1 is not finite");
  if (h_ctl->status == CS_ERANGE) return fail(CS_ERANGE, "select: ||A||_1 needs more than 64 double-angle steps");
  if (info) {
    const int prods = products_of(h_ctl->m) + 2 * h_ctl->s;
    *info = cs_info{h_ctl->norm1, h_ctl->m, h_ctl->s, prods, 0, 2.0 * (double)n * n * n * prods};
  }
  return CS_OK;
}

}  // namespace cs
