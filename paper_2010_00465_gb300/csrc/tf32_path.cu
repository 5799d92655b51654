// tf32_path.cu -- executor of the product plans for the split-precision forms
// whose Taylor chain runs on the four-pass TF32 tensor-core kernel
// (CS_SPLIT_TF32, CS_SPLIT_EMU); their double-angle steps run in FP64
// (native, or emulated on the BF16 tensor cores).
//
// Every intermediate is kept in FP64 ("master" copies).  A chain product
// P = X Y runs on the zero-diagonal (hi, lo) TF32 splits of X and Y, which
// the epilogue that produced them wrote beside the masters, and its raw FP32
// result goes to a scratch matrix; an FP64 element-wise epilogue then adds the
// diagonal terms exactly,
//   X Y = X_off Y_off + X[r][r] Y[r][c] + (r != c) X[r][c] Y[c][c],
// applies the scheme's linear combinations to the FP64 masters and writes
// the outputs' masters and, for outputs read later as product operands, their
// splits (row-major for a left operand, transposed for a right one).
// Intermediates rounded to FP32 (or to the 22 bits of a split) each step
// would be amplified by the double-angle recurrence well past 2e-5 at
// ||A||_1 near 64.
#include <stdlib.h>

#include <vector>

#include "internal.cuh"
#include "plan.h"
#include "sm100_ptx.cuh"
#include "tc_gemm.h"

namespace cs {
namespace {

struct TcSlot {
  float* hi = nullptr;
  float* lo = nullptr;
  float* hiT = nullptr;
  float* loT = nullptr;
};

// The FP64 epilogue of one chain step.
struct SplitEpi {
  Epilogue<double> e;      // linear combinations on FP64 masters (in[], out[])
  const float* P;          // raw product of the zero-diagonal splits, n x ld
  const double* X;         // masters of the operands (n x n, leading dimension n)
  const double* Y;
  float* hi[EPI_MAX_OUT];  // splits of the outputs (null: not needed)
  float* lo[EPI_MAX_OUT];
  float* hiT[EPI_MAX_OUT];
  float* loT[EPI_MAX_OUT];
  int64_t ld;
};

__device__ __forceinline__ void split_to(float v, float* hi, float* lo, int64_t idx) {
  const float h = ptx::tf32_rna(v);
  hi[idx] = h;
  lo[idx] = COSSIN_LO(v - h);
}

// 32 x 32 tiles, 32 x 8 threads (four rows each); transposed splits go
// through a shared-memory tile so both stores coalesce.
__global__ void __launch_bounds__(256) split_epilogue_kernel(const __grid_constant__ SplitEpi ep, int64_t n) {
  __shared__ float tile[32][33];
  const Epilogue<double>& e = ep.e;
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  double o[4][EPI_MAX_OUT];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t r = r0 + ty + 8 * i, c = c0 + tx;
#pragma unroll
    for (int t = 0; t < EPI_MAX_OUT; ++t) o[i][t] = 0.0;
    if (r >= n || c >= n) continue;
    const int64_t idx = r * n + c;
    double p = (double)ep.P[r * ep.ld + c] + ep.X[r * n + r] * ep.Y[idx];
    if (r != c) p += ep.X[idx] * ep.Y[c * n + c];
    double in[EPI_MAX_IN];
#pragma unroll
    for (int q = 0; q < EPI_MAX_IN; ++q) in[q] = q < e.n_in ? e.in[q][idx] : 0.0;
#pragma unroll
    for (int t = 0; t < EPI_MAX_OUT; ++t) {
      if (t < e.n_out) {
        double v = e.alpha[t] * p + (r == c ? e.gamma[t] : 0.0);
#pragma unroll
        for (int q = 0; q < EPI_MAX_IN; ++q)
          if (q < e.n_in) v = fma(e.beta[t][q], in[q], v);
#pragma unroll
        for (int u = 0; u < EPI_MAX_OUT; ++u)
          if (u < t) v = fma(e.delta[t][u], o[i][u], v);
        o[i][t] = v;
      }
    }
#pragma unroll
    for (int t = 0; t < EPI_MAX_OUT; ++t) {
      if (t < e.n_out) {
        e.out[t][idx] = o[i][t];
        if (ep.hi[t]) split_to(r == c ? 0.f : (float)o[i][t], ep.hi[t], ep.lo[t], r * ep.ld + c);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < EPI_MAX_OUT; ++t) {
    if (t >= e.n_out || !ep.hiT[t]) continue;  // uniform over the block
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) tile[ty + 8 * i][tx] = (float)o[i][t];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t rr = c0 + ty + 8 * i, cc = r0 + tx;  // row of the transpose = column of the tile
      if (rr < n && cc < n) split_to(rr == cc ? 0.f : tile[tx][ty + 8 * i], ep.hiT[t], ep.loT[t], rr * ep.ld + cc);
    }
  }
}

cs_status split_epilogue(const SplitEpi& ep, int64_t n, cudaStream_t stream) {
  ProfScope prof(CS_KERNEL_OTHER, (double)n * n * (4.0 + 16.0 + 8.0 * (ep.e.n_in + ep.e.n_out)), stream);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
  split_epilogue_kernel<<<grid, block, 0, stream>>>(ep, n);
  CS_CUDA_CHECK(cudaGetLastError());
  return CS_OK;
}

// How the matrix written into `slot` by step i is read by the later steps
// before it is overwritten: as a left operand (row-major split) and/or as a
// right operand (transposed split).
void operand_uses(const std::vector<Step>& plan, size_t i, int slot, bool* as_x, bool* as_y) {
  *as_x = *as_y = false;
  for (size_t j = i + 1; j < plan.size(); ++j) {
    if (plan[j].X == slot) *as_x = true;
    if (plan[j].Y == slot) *as_y = true;
    for (const OutSpec& o : plan[j].outs)
      if (o.slot == slot) return;
  }
}

}  // namespace

cs_status run_tf32(const double* A, int64_t n, cs_prec prec, double* C, double* S, char* ws, const Layout& L,
                   const PlanSpec& spec, cudaStream_t stream) {
  const int s = spec.s;
  const int64_t ld = L.ld32;
  const size_t n2 = (size_t)n * (size_t)n;
  auto F = [&](size_t off) { return (float*)(ws + off); };
  double* ping[2] = {(double*)(ws + L.ping64[0]), (double*)(ws + L.ping64[1])};
  double* master[SL_COUNT] = {};
  TcSlot split[SL_COUNT];
  master[SL_A] = const_cast<double*>(A);
  master[SL_C] = s == 0 ? C : ping[0];
  master[SL_S] = s == 0 ? S : ping[0] + n2;
  split[SL_A] = {F(L.a4[0]), F(L.a4[1]), F(L.a4[2]), F(L.a4[3])};
  split[SL_C] = {F(L.c4[0]), F(L.c4[1]), F(L.c4[2]), F(L.c4[3])};
  for (int w = 0; w < kWorkSlots; ++w) {
    master[W(w)] = (double*)(ws + L.w[w]);
    split[W(w)] = {F(L.w4[w][0]), F(L.w4[w][1]), F(L.w4[w][2]), F(L.w4[w][3])};
  }
  int* err = tc_error_word();
  if (!err) return fail(CS_ECUDA, "cannot resolve the device error word");

  // The input goes to SL_A, or scaled to W0 for the c(t^2 A), s(t, A) variant.
  const int in_slot = spec.scale_into_w0 ? W(0) : SL_A;
  if (spec.scale_into_w0) CS_CHECK(scale_f64(A, master[W(0)], (int64_t)n2, spec.input_scale, stream));
  {
    const TcSlot& t = split[in_slot];
    CS_CHECK(split_f64(master[in_slot], n, ld, t.hi, t.lo, t.hiT, t.loT, stream, 1.0, true));
  }

  float* p32 = F(L.p32);
  const std::vector<Step>& plan = spec.steps;
  for (size_t i = 0; i < plan.size(); ++i) {
    const Step& st = plan[i];
    // raw product of the splits into p32
    TcEpilogue raw;
    raw.n_out = 1;
    raw.out_hi[0] = p32;
    raw.alpha[0] = 1.f;
    const TcOperand X{split[st.X].hi, split[st.X].lo, ld};
    const TcOperand YT{split[st.Y].hiT, split[st.Y].loT, ld};
    CS_CHECK(gemm_tf32(X, YT, n, n, n, ld, raw, err, stream));
    // FP64 epilogue on the masters
    SplitEpi ep{};
    ep.P = p32;
    ep.X = master[st.X];
    ep.Y = master[st.Y];
    ep.ld = ld;
    EpiBuilder<double> b;
    std::vector<int> in_slots;
    auto in_index = [&](int sl) {
      for (size_t q = 0; q < in_slots.size(); ++q)
        if (in_slots[q] == sl) return (int)q;
      in_slots.push_back(sl);
      return b.add_in(master[sl]);
    };
    for (const OutSpec& o : st.outs) {
      if (o.slot == st.X || o.slot == st.Y) return fail(CS_EINVAL, "plan step overwrites its own operand");
      const int t = b.add_out(master[o.slot], o.alpha, o.gamma);
      for (auto& bc : o.beta) b.beta(t, in_index(bc.first), bc.second);
      for (auto& dc : o.delta) b.delta(t, dc.first, dc.second);
      bool as_x, as_y;
      operand_uses(plan, i, o.slot, &as_x, &as_y);
      if ((as_x || as_y) && !split[o.slot].hi) return fail(CS_EINVAL, "plan reads S as a product operand");
      if (as_x) {
        ep.hi[t] = split[o.slot].hi;
        ep.lo[t] = split[o.slot].lo;
      }
      if (as_y) {
        ep.hiT[t] = split[o.slot].hiT;
        ep.loT[t] = split[o.slot].loT;
      }
    }
    ep.e = b.e;
    CS_CHECK(split_epilogue(ep, n, stream));
  }
  // The chain's C and S are FP64 already; the double-angle steps run in FP64.
  if (s == 0) return CS_OK;
  return square_f64(ping, n, s, C, S, stream, f64_product(prec, ws, L));
}

// One plain product on the tensor-core kernel (used by cossin_matmul).
cs_status matmul_tf32(const void* X, const void* Y, int64_t n, bool f64_io, void* P, cudaStream_t stream) {
  const int64_t ld = (n + 31) / 32 * 32;
  const size_t sz = sizeof(float) * (size_t)n * (size_t)ld;
  char* ws = nullptr;
  CS_CHECK(dev_alloc((void**)&ws, 8 * sz, stream, "cossin_matmul scratch"));
  float* b[8];
  for (int k = 0; k < 8; ++k) b[k] = (float*)(ws + k * sz);
  cs_status rc;
  if (f64_io) {
    rc = split_f64((const double*)X, n, ld, b[0], b[1], nullptr, nullptr, stream);
    if (rc == CS_OK) rc = split_f64((const double*)Y, n, ld, b[2], b[3], b[4], b[5], stream);
  } else {
    rc = split_f32((const float*)X, n, ld, b[0], b[1], nullptr, nullptr, stream);
    if (rc == CS_OK) rc = split_f32((const float*)Y, n, ld, b[2], b[3], b[4], b[5], stream);
  }
  if (rc == CS_OK) {
    TcEpilogue e;
    e.n_out = 1;
    e.out_hi[0] = b[6];
    e.out_lo[0] = b[7];
    e.alpha[0] = 1.f;
    int* err = tc_error_word();
    rc = err ? gemm_tf32(TcOperand{b[0], b[1], ld}, TcOperand{b[4], b[5], ld}, n, n, n, ld, e, err, stream)
             : fail(CS_ECUDA, "cannot resolve the device error word");
  }
  if (rc == CS_OK)
    rc = f64_io ? combine_f64(b[6], b[7], n, ld, (double*)P, stream) : combine_f32(b[6], b[7], n, ld, (float*)P, stream);
  cudaFreeAsync(ws, stream);
  return rc;
}

}  // namespace cs
