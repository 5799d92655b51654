// plan.h -- the product plans of the factorised Taylor schemes and the
// workspace layout (host side, shared by the FP64 and TF32 executors).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <utility>

#include "internal.cuh"
#include "ozaki.h"
#include <vector>

namespace cs {

constexpr int kMaxS = 64;          // largest number of double-angle steps accepted
constexpr int64_t kMaxN = 65536;   // largest matrix order accepted
constexpr int kWorkSlots = 8;      // intermediates of the longest scheme (2m = 24)

enum Slot { SL_A = 0, SL_C = 1, SL_S = 2, SL_W0 = 3, SL_COUNT = SL_W0 + kWorkSlots };
constexpr int W(int i) { return SL_W0 + i; }

// out = alpha * P + gamma * I + sum beta_j * slot_j + sum delta_u * (earlier output u of the step)
struct OutSpec {
  int slot;
  double alpha;
  double gamma;
  std::vector<std::pair<int, double>> beta;   // (slot, coefficient)
  std::vector<std::pair<int, double>> delta;  // (index of an earlier output, coefficient)
};

struct Step {
  int X, Y;  // P = slot X * slot Y
  std::vector<OutSpec> outs;
};

// `scale` evaluates the scheme at scale * A (the unitary e^{-itA} takes t):
// the first product folds scale^2 4^-s and the last scale 2^-s.
std::vector<Step> chain_plan(int m, int s, double scale = 1.0);

// What an executor runs: the product steps, then s double-angle steps.  With
// scale_into_w0 the input is first copied into W0 scaled by input_scale (the
// c(t^2 A), s(t, A) variant starts from B = (t / 2^s)^2 A there).
struct PlanSpec {
  std::vector<Step> steps;
  int s = 0;
  bool scale_into_w0 = false;
  double input_scale = 1.0;
};

PlanSpec cossin_spec(int m, int s, double scale = 1.0);
// family 0: k = 3 with P_{3,4}^s, 1: k = 3 with P_4^s, 2: k = 4, 3: k = 5 (Sec. 2.2)
PlanSpec cs_spec(int family, int sigma, double t);
int cs_products(int family);

// Byte offsets into the caller's workspace.  Every precision: w[8] (n x n
// doubles), ping64[2] (stacked [C; S], 2n x n doubles).  CS_FP32 adds a64
// (its input in FP64).  The TF32 split forms add the (hi, lo) TF32 operand
// splits {hi, lo, hi^T, lo^T} (n x ld32 floats each) of A (a4), W0..W7 (w4)
// and C (c4), and p32, the raw product of one chain step.  The emulated
// precisions add the scratch of one emulated product.
struct Layout {
  size_t norm_partial = 0, norm_out = 0;
  size_t w[kWorkSlots] = {};
  size_t ping64[2] = {};
  size_t a64 = 0;
  int64_t ld32 = 0;
  size_t a4[4] = {};
  size_t w4[kWorkSlots][4] = {};
  size_t c4[4] = {};
  size_t p32 = 0;
  size_t ozaki = 0, ozaki_bytes = 0;  // scratch of one emulated product
  size_t splitk = 0, splitk_bytes = 0;  // native FP64 products: last-wave pieces split over K
  size_t out_c = 0, out_s = 0;  // n x n C and S of the precision's type (with_outputs)
  size_t total = 0;
};

Layout make_layout(int64_t n, int prec, bool with_outputs = false);

// How the FP64 executors form a product P = X Y (row-major, X: M x K, Y: K x N)
// with its epilogue: natively (gemm_f64) or, with emu_work set, on the BF16
// tensor cores (gemm_f64_emu) with `slices` slices, using that scratch.
struct F64Product {
  void* emu_work = nullptr;
  size_t emu_bytes = 0;
  void* split_work = nullptr;  // native FP64: scratch for splitting the last wave over K
  size_t split_bytes = 0;
  int* err = nullptr;
  int slices = kOzakiSlices;
  cs_status operator()(const double* X, const double* Y, int64_t M, int64_t N, int64_t K,
                       const Epilogue<double>& e, cudaStream_t stream) const;
};
// The product of the double-angle steps for `prec`, and that of the Taylor
// chain (four slices for CS_SPLIT_BF16 and CS_FP32).
F64Product f64_product(cs_prec prec, char* ws, const Layout& L);
F64Product chain_product(cs_prec prec, char* ws, const Layout& L);

// Double-angle steps in FP64 on the stacked buffers ping[2] (each 2n x n):
// starts from [C; S] in ping[0]; the last step writes C and S.
cs_status square_f64(double* const ping[2], int64_t n, int s, double* C, double* S, cudaStream_t stream,
                     const F64Product& prod = F64Product{});

}  // namespace cs
