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

// Sec. 2.2 schemes on B = t^2 A (families: k = 3 with P_{3,4}^s, k = 3 with
// P_4^s, k = 4, k = 5; 2, 3, 4, 5 products).  The paper prints no admissible
// norms for them; these are the largest ||B||_1 at which the Sec. 3 error
// series (150 terms) of the cosine part, and of the sine part divided by t,
// stay <= u (the cosine values are theta_2m^2 of Tables 1-2).
__host__ __device__ inline double theta_cs(int table, int f) {
  if (table == 0) return f == 0 ? 3.44587e-3 : f == 1 ? 1.32137e-2 : f == 2 ? 9.62511e-1 : 3.64043;
  return f == 0 ? 5.22375e-1 : f == 1 ? 7.35401e-1 : f == 2 ? 8.96121 : 21.8484;
}
__host__ __device__ inline int cs_family_products(int f) { return f + 2; }

// Minimal Pi + 2 sigma with ||B||_1 / 4^sigma <= theta_cs; 0, 3 or 4 as select_family.
__host__ __device__ inline int select_cs_family(double normB, int table, int* f_out, int* s_out) {
  if (!isfinite(normB)) return 3;
  int best = -1, best_s = 0, best_cost = 1 << 30;
  for (int f = 0; f < 4; ++f) {
    int sg = 0;
    while (sg <= kSelMaxS && ldexp(normB, -2 * sg) > theta_cs(table, f)) ++sg;
    if (sg > kSelMaxS) continue;
    const int cost = cs_family_products(f) + 2 * sg;
    if (cost < best_cost || (cost == best_cost && sg < best_s)) {
      best = f;
      best_s = sg;
      best_cost = cost;
    }
  }
  if (best < 0) return 4;
  *f_out = best;
  *s_out = best_s;
  return 0;
}

}  // namespace cs
