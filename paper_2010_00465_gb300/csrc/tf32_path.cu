// tf32_path.cu -- executor of the product plans on the four-pass TF32
// tensor-core kernel: the FP32 path (everything on tensor cores) and the
// split-precision path (Taylor chain on tensor cores, double-angle steps in FP64).
#include <stdlib.h>

#include <vector>

#include "internal.cuh"
#include "plan.h"
#include "tc_gemm.h"

namespace cs {
namespace {

struct TcSlot {
  float* hi = nullptr;
  float* lo = nullptr;
  float* hiT = nullptr;
  float* loT = nullptr;
};

// Is the matrix written into `slot` by step i read as a right operand later
// (before it is overwritten)?  Right operands are fed transposed.
bool needs_transpose(const std::vector<Step>& plan, size_t i, int slot, bool squaring_follows) {
  for (size_t j = i + 1; j < plan.size(); ++j) {
    if (plan[j].Y == slot) return true;
    for (const OutSpec& o : plan[j].outs)
      if (o.slot == slot) return false;
  }
  return slot == SL_C && squaring_follows;
}

}  // namespace

cs_status run_tf32(const void* A, int64_t n, cs_prec prec, void* C, void* S, char* ws, const Layout& L,
                   const PlanSpec& spec, cudaStream_t stream) {
  const int s = spec.s;
  const int64_t ld = L.ld32;
  auto F = [&](size_t off) { return (float*)(ws + off); };
  TcSlot slot[SL_COUNT];
  slot[SL_A] = {F(L.a4[0]), F(L.a4[1]), F(L.a4[2]), F(L.a4[3])};
  for (int w = 0; w < kWorkSlots; ++w) slot[W(w)] = {F(L.w4[w][0]), F(L.w4[w][1]), F(L.w4[w][2]), F(L.w4[w][3])};
  TcSlot ping[2];
  for (int p = 0; p < 2; ++p) ping[p] = {F(L.ping4[p][0]), F(L.ping4[p][1]), F(L.ping4[p][2]), F(L.ping4[p][3])};
  slot[SL_C] = ping[0];
  slot[SL_S] = {ping[0].hi + n * ld, ping[0].lo + n * ld, nullptr, nullptr};
  int* err = tc_error_word();
  if (!err) return fail(CS_ECUDA, "cannot resolve the device error word");

  // The input goes to SL_A, or scaled to W0 for the c(t^2 A), s(t, A) variant.
  const TcSlot& in = spec.scale_into_w0 ? slot[W(0)] : slot[SL_A];
  if (prec == CS_FP32)
    CS_CHECK(split_f32((const float*)A, n, ld, in.hi, in.lo, in.hiT, in.loT, stream, spec.input_scale));
  else
    CS_CHECK(split_f64((const double*)A, n, ld, in.hi, in.lo, in.hiT, in.loT, stream, spec.input_scale));

  const bool tc_squaring = (prec == CS_FP32) && s > 0;
  const std::vector<Step>& plan = spec.steps;
  for (size_t i = 0; i < plan.size(); ++i) {
    const Step& st = plan[i];
    TcEpilogue e;
    std::vector<int> in_slots;
    auto in_index = [&](int sl) {
      for (size_t q = 0; q < in_slots.size(); ++q)
        if (in_slots[q] == sl) return (int)q;
      in_slots.push_back(sl);
      e.in_hi[e.n_in] = slot[sl].hi;
      e.in_lo[e.n_in] = slot[sl].lo;
      return e.n_in++;
    };
    for (const OutSpec& o : st.outs) {
      const int t = e.n_out++;
      e.out_hi[t] = slot[o.slot].hi;
      e.out_lo[t] = slot[o.slot].lo;
      if (needs_transpose(plan, i, o.slot, tc_squaring)) {
        e.outT_hi[t] = slot[o.slot].hiT;
        e.outT_lo[t] = slot[o.slot].loT;
      }
      e.alpha[t] = (float)o.alpha;
      e.gamma[t] = (float)o.gamma;
      for (auto& b : o.beta) e.beta[t][in_index(b.first)] = (float)b.second;
      for (auto& d : o.delta) e.delta[t][d.first] = (float)d.second;
    }
    const TcOperand X{slot[st.X].hi, slot[st.X].lo, ld};
    const TcOperand YT{slot[st.Y].hiT, slot[st.Y].loT, ld};
    CS_CHECK(gemm_tf32(X, YT, n, n, n, ld, e, err, stream));
  }

  if (prec == CS_FP32) {
    // Double-angle steps on tensor cores: [C'; S'] = [C; S] C (Sec. 1).
    for (int j = 0; j < s; ++j) {
      const TcSlot& cur = ping[j & 1];
      const TcSlot& nxt = ping[(j + 1) & 1];
      TcEpilogue e;
      e.split_row = n;
      e.n_out = 2;
      e.out_hi[0] = nxt.hi;
      e.out_lo[0] = nxt.lo;
      e.outT_hi[0] = j == s - 1 ? nullptr : nxt.hiT;
      e.outT_lo[0] = j == s - 1 ? nullptr : nxt.loT;
      e.out_hi[1] = nxt.hi + n * ld;
      e.out_lo[1] = nxt.lo + n * ld;
      e.alpha[0] = e.alpha[1] = 2.f;
      e.gamma[0] = -1.f;
      e.gamma[1] = 0.f;
      const TcOperand X{cur.hi, cur.lo, ld};
      const TcOperand YT{cur.hiT, cur.loT, ld};
      CS_CHECK(gemm_tf32(X, YT, 2 * n, n, n, ld, e, err, stream));
    }
    const TcSlot& fin = ping[s & 1];
    CS_CHECK(combine_f32(fin.hi, fin.lo, n, ld, (float*)C, stream));
    CS_CHECK(combine_f32(fin.hi + n * ld, fin.lo + n * ld, n, ld, (float*)S, stream));
    return CS_OK;
  }
  // Split precision: the chain's C and S go to FP64, the double-angle steps run in FP64.
  if (s == 0) {
    CS_CHECK(combine_f64(ping[0].hi, ping[0].lo, n, ld, (double*)C, stream));
    CS_CHECK(combine_f64(ping[0].hi + n * ld, ping[0].lo + n * ld, n, ld, (double*)S, stream));
    return CS_OK;
  }
  double* p64[2] = {(double*)(ws + L.ping64[0]), (double*)(ws + L.ping64[1])};
  CS_CHECK(combine_f64(ping[0].hi, ping[0].lo, n, ld, p64[0], stream));
  CS_CHECK(combine_f64(ping[0].hi + n * ld, ping[0].lo + n * ld, n, ld, p64[0] + n * n, stream));
  return square_f64(p64, n, s, (double*)C, (double*)S, stream, f64_product(prec, ws, L));
}

// One plain product on the tensor-core kernel (used by cossin_matmul).
cs_status matmul_tf32(const void* X, const void* Y, int64_t n, bool f64_io, void* P, cudaStream_t stream) {
  const int64_t ld = (n + 31) / 32 * 32;
  const size_t sz = sizeof(float) * (size_t)n * (size_t)ld;
  char* ws = nullptr;
  CS_CUDA_CHECK(cudaMallocAsync((void**)&ws, 8 * sz, stream));
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
