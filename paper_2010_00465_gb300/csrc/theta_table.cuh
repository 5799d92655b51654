// theta_table.cuh -- admissible norms theta_2m and the (2m, s) choice, shared
// by the host (single-matrix calls) and the device (batched kernel).
//
// Table 1 (double, u = 2^-53) and Table 2 (single, u = 2^-24) of the paper,
// families 2m = 4, 8, 16, 24 with Pi_2m = 3, 4, 6, 7 products.  Table 1's k = 7
// sine entry reads 1.97, but the printed k = 7 sine coefficients match the
// series only through A^21; the Sec. 3 error series (150 terms) with them
// reaches 2^-53 at 1.8555, the value used here.
#pragma once

#include <math.h>

namespace cs {

constexpr int kSelMaxS = 64;

__host__ __device__ inline double theta_of(int table, int f, bool sine) {
  if (table == 0) {
    if (!sine) return f == 0 ? 6.5633e-3 : f == 1 ? 1.1495e-1 : f == 2 ? 9.8108e-1 : 2.5675;
    return f == 0 ? 1.777e-2 : f == 1 ? 8.0438e-2 : f == 2 ? 1.1184 : 1.8555;
  }
  if (!sine) return f == 0 ? 1.8709e-1 : f == 1 ? 8.5756e-1 : f == 2 ? 2.9935 : 5.5555;
  return f == 0 ? 3.1386e-1 : f == 1 ? 7.492e-1 : f == 2 ? 3.2152 : 4.3819;
}

__host__ __device__ inline int family_order(int f) { return f == 0 ? 4 : f == 1 ? 8 : f == 2 ? 16 : 24; }
__host__ __device__ inline int family_products(int f) { return f == 0 ? 3 : f == 1 ? 4 : f == 2 ? 6 : 7; }

// Minimal Pi_2m + 2s over the four families with norm / 2^s <= min(theta^c, theta^s);
// ties go to the smaller s.  Returns 0, 3 (non-finite norm) or 4 (s > 64).
__host__ __device__ inline int select_family(double norm, int table, int* f_out, int* s_out) {
  if (!isfinite(norm)) return 3;
  int best = -1, best_s = 0, best_cost = 1 << 30;
  for (int f = 0; f < 4; ++f) {
    const double th = fmin(theta_of(table, f, false), theta_of(table, f, true));
    int sf = 0;
    while (sf <= kSelMaxS && ldexp(norm, -sf) > th) ++sf;
    if (sf > kSelMaxS) continue;
    const int cost = family_products(f) + 2 * sf;
    if (cost < best_cost || (cost == best_cost && sf < best_s)) {
      best = f;
      best_s = sf;
      best_cost = cost;
    }
  }
  if (best < 0) return 4;
  *f_out = best;
  *s_out = best_s;
  return 0;
}

}  // namespace cs
