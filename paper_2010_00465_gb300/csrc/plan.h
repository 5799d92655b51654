// plan.h -- the product plans of the factorised Taylor schemes and the
// workspace layout (host side, shared by the FP64 and TF32 executors).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include <utility>
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

std::vector<Step> chain_plan(int m, int s);

// Byte offsets into the caller's workspace.
struct Layout {
  size_t norm_partial = 0, norm_out = 0;
  size_t w[kWorkSlots] = {}, w_lo[kWorkSlots] = {};
  size_t a_hi = 0, a_lo = 0;
  size_t ping64[2] = {}, ping32[2] = {}, ping32_lo[2] = {};
  size_t total = 0;
};

Layout make_layout(int64_t n, int prec);

}  // namespace cs
