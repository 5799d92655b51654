/*
 * cossin_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, deliberately unoptimised FP64 CPU restatement of the method
 * of Seydaoglu, Bader, Blanes and Casas, "Computing the matrix sine and
 * cosine simultaneously with a reduced number of products" (arXiv:2010.00465).
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may call it.  It shares no code, header, table or constant with the CUDA
 * library: every coefficient below is typed from the paper.
 *
 * Steps, in the paper's order and notation:
 *   1. theta = ||A||_1, the exact matrix 1-norm (Sec. 4: "the matrix 1-norm
 *      has been used").
 *   2. Choice of the family 2m in {4, 8, 16, 24} and of the scaling s from the
 *      admissible norms theta_2m of Tables 1 and 2 (Sec. 3).  The paper gives
 *      no explicit rule; this oracle takes, over the four families, the one
 *      that minimises Pi_2m + 2 s with s = max(0, ceil(log2(theta/theta_m))),
 *      theta_m = min(theta^c_2m, theta^s_2m); ties go to the smaller s.
 *   3. A_s = 2^-s A and A_2 = A_s * A_s.
 *   4. The factorised Taylor schemes of Sec. 2.1 (eqs. Algorithm3cA/3sA,
 *      Algorithm4cA/4sA, Algorithm6cA/6sA with eq:cosm8 and the z list,
 *      Algorithm7cA/7sA with Coefs7cA/Coefs7sA), written out literally.
 *   5. s double-angle steps (Sec. 1): cos 2X = 2 cos^2 X - I and
 *      sin 2X = 2 sin X cos X.
 *
 * Matrices are dense, row-major, n x n, FP64.  Every product is the textbook
 * triple loop Z_ij = sum_k X_ik Y_kj with k ascending; rows are shared out
 * over OpenMP threads, which changes no arithmetic.  Build with
 * -ffp-contract=off so that x86 and Arm hosts give identical results.
 *
 * Parity status: every function here is pinned by tests that do not rely on
 * this file (Taylor coefficients read off a nilpotent shift matrix, closed
 * forms, identities, high-precision brute force, recomputed theta tables).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Status codes returned by the oracle (independent of the library's). */
#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ENOMEM 2
#define ORC_ENONFINITE 3
#define ORC_ERANGE 4

#define ORC_MAX_S 64

/* Admissible norms theta_2m for the new Taylor schemes, Table 1 (double,
 * u = 2^-53) and Table 2 (single, u = 2^-24), columns 2m = 4, 8, 16, 24.
 * One deliberate deviation: Table 1 prints 1.97 for the k = 7 sine, but the
 * printed Coefs7sA coefficients reproduce the sine series only through A^21
 * (z5 and z6 both multiply T24, leaving 11 free coefficients for the 12 odd
 * powers A^1..A^23), and the error series of Sec. 3 summed to 150 terms with
 * those coefficients reaches u = 2^-53 at 1.8555.  The oracle uses 1.8555. */
static const double THETA_COS[2][4] = {
    {6.5633e-3, 1.1495e-1, 9.8108e-1, 2.5675},
    {1.8709e-1, 8.5756e-1, 2.9935, 5.5555},
};
static const double THETA_SIN[2][4] = {
    {1.777e-2, 8.0438e-2, 1.1184, 1.8555},
    {3.1386e-1, 7.492e-1, 3.2152, 4.3819},
};
/* Pi_2m: matrix products for cos and sin together (Tables 1-2, last row). */
static const int PI_2M[4] = {3, 4, 6, 7};
static const int ORDER_2M[4] = {4, 8, 16, 24};

typedef struct {
  double norm1;
  int m;        /* 2m of the family used: 4, 8, 16 or 24 */
  int s;        /* number of double-angle steps */
  int products; /* Pi_2m + 2 s */
} oracle_info;

static int g_threads = 0;

void oracle_set_threads(int t) { g_threads = t; }

int oracle_get_threads(void) {
#ifdef _OPENMP
  return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
  return 1;
#endif
}

/* Step 1: ||A||_1 = max_j sum_i |a_ij|. */
double oracle_norm1(const double* A, long n) {
  double best = 0.0;
  int nan_seen = 0;
  for (long j = 0; j < n; ++j) {
    double col = 0.0;
    for (long i = 0; i < n; ++i) col += fabs(A[i * n + j]);
    if (isnan(col)) nan_seen = 1;
    else if (col > best) best = col;
  }
  return nan_seen ? NAN : best;
}

double oracle_theta(int prec, int family_index, int which_sine) {
  if (prec < 0 || prec > 1 || family_index < 0 || family_index > 3) return -1.0;
  return which_sine ? THETA_SIN[prec][family_index] : THETA_COS[prec][family_index];
}

/* Step 2.  prec: 0 = double table, 1 = single table. */
int oracle_select(double norm, int prec, int* m_out, int* s_out) {
  if (prec < 0 || prec > 1) return ORC_EINVAL;
  if (!isfinite(norm)) return ORC_ENONFINITE;
  int best_m = -1, best_s = 0, best_cost = 1 << 30;
  for (int f = 0; f < 4; ++f) {
    double th = fmin(THETA_COS[prec][f], THETA_SIN[prec][f]);
    int s = 0;
    while (ldexp(norm, -s) > th) ++s;
    if (s > ORC_MAX_S) continue;
    int cost = PI_2M[f] + 2 * s;
    if (cost < best_cost || (cost == best_cost && s < best_s)) {
      best_cost = cost;
      best_m = ORDER_2M[f];
      best_s = s;
    }
  }
  if (best_m < 0) return ORC_ERANGE;
  *m_out = best_m;
  *s_out = best_s;
  return ORC_OK;
}

/* Z = X * Y, textbook definition. Z must not alias X or Y. */
static void matmul(const double* X, const double* Y, double* Z, long n) {
#pragma omp parallel for schedule(static) num_threads(oracle_get_threads())
  for (long i = 0; i < n; ++i) {
    for (long j = 0; j < n; ++j) {
      double acc = 0.0;
      for (long k = 0; k < n; ++k) acc += X[i * n + k] * Y[k * n + j];
      Z[i * n + j] = acc;
    }
  }
}

/* out = cI * I + sum_t c[t] * M[t]; out may alias any M[t]. */
static void lincomb(double* out, long n, double cI, int nt, const double* c,
                    const double* const* M) {
  for (long i = 0; i < n; ++i)
    for (long j = 0; j < n; ++j) {
      double v = (i == j) ? cI : 0.0;
      for (int t = 0; t < nt; ++t) v += c[t] * M[t][i * n + j];
      out[i * n + j] = v;
    }
}

static void scale(double* out, const double* X, double a, long n) {
  for (long i = 0; i < n * n; ++i) out[i] = a * X[i];
}

#define NEWMAT(p)                                           \
  do {                                                      \
    p = (double*)malloc((size_t)n * (size_t)n * sizeof(double)); \
    if (!p) { rc = ORC_ENOMEM; goto done; }                 \
  } while (0)

/* k = 3 products: eqs. Algorithm3cA (T4c) and Algorithm3sA (T5s). */
static int chain_m4(const double* As, const double* A2, long n, double* C, double* S) {
  int rc = ORC_OK;
  double *A4 = NULL, *Q = NULL;
  NEWMAT(A4); NEWMAT(Q);
  matmul(A2, A2, A4, n);                                   /* A4 = A2^2 */
  {
    const double c[2] = {-1.0 / 2.0, 1.0 / 24.0};          /* 1/2!, 1/4! */
    const double* M[2] = {A2, A4};
    lincomb(C, n, 1.0, 2, c, M);                           /* T4c */
  }
  {
    const double c[2] = {-1.0 / 6.0, 1.0 / 120.0};         /* 1/3!, 1/5! */
    const double* M[2] = {A2, A4};
    lincomb(Q, n, 1.0, 2, c, M);
  }
  matmul(As, Q, S, n);                                     /* T5s = A (...) */
done:
  free(A4); free(Q);
  return rc;
}

/* k = 4 products: eqs. Algorithm4cA (T8c) and Algorithm4sA (T_{7,9}s). */
static int chain_m8(const double* As, const double* A2, long n, double* C, double* S) {
  int rc = ORC_OK;
  double *A4 = NULL, *R = NULL, *A8 = NULL, *Q = NULL;
  NEWMAT(A4); NEWMAT(R); NEWMAT(A8); NEWMAT(Q);
  matmul(A2, A2, A4, n);                                   /* A4 = A2^2 */
  {
    const double c[2] = {-1.0 / 720.0, 1.0 / 40320.0};     /* -1/6!, 1/8! */
    const double* M[2] = {A2, A4};
    lincomb(R, n, 0.0, 2, c, M);
  }
  matmul(A4, R, A8, n);                                    /* A8 = A4 (...) */
  {
    const double c[3] = {-1.0 / 2.0, 1.0 / 24.0, 1.0};
    const double* M[3] = {A2, A4, A8};
    lincomb(C, n, 1.0, 3, c, M);                           /* T8c */
  }
  {
    const double c[3] = {-1.0 / 6.0, 1.0 / 120.0, 720.0 / 5040.0}; /* 6!/7! */
    const double* M[3] = {A2, A4, A8};
    lincomb(Q, n, 1.0, 3, c, M);
  }
  matmul(As, Q, S, n);                                     /* T_{7,9}s */
done:
  free(A4); free(R); free(A8); free(Q);
  return rc;
}

/* The k = 4 alternative with a five-product sine: T8c of eq. Algorithm4cA and
 * T9s of eq. Algorithm5sA, whose A8' = A4 (-A2/7! + A4/9!) costs one more
 * product than the (6!/7!) A8 reuse of T_{7,9}s but matches sin through A^9.
 * Not used in Tables 1-2; reached only by forcing 2m = 9. */
static int chain_m9(const double* As, const double* A2, long n, double* C, double* S) {
  int rc = ORC_OK;
  double *A4 = NULL, *R = NULL, *A8 = NULL, *Q = NULL;
  NEWMAT(A4); NEWMAT(R); NEWMAT(A8); NEWMAT(Q);
  matmul(A2, A2, A4, n);                                   /* A4 = A2^2 */
  {
    const double c[2] = {-1.0 / 720.0, 1.0 / 40320.0};     /* -1/6!, 1/8! */
    const double* M[2] = {A2, A4};
    lincomb(R, n, 0.0, 2, c, M);
  }
  matmul(A4, R, A8, n);                                    /* A8 = A4 (...) */
  {
    const double c[3] = {-1.0 / 2.0, 1.0 / 24.0, 1.0};
    const double* M[3] = {A2, A4, A8};
    lincomb(C, n, 1.0, 3, c, M);                           /* T8c */
  }
  {
    const double c[2] = {-1.0 / 5040.0, 1.0 / 362880.0};   /* -1/7!, 1/9! */
    const double* M[2] = {A2, A4};
    lincomb(R, n, 0.0, 2, c, M);
  }
  matmul(A4, R, Q, n);                                     /* A8' = A4 (...) */
  {
    const double c[3] = {-1.0 / 6.0, 1.0 / 120.0, 1.0};
    const double* M[3] = {A2, A4, Q};
    lincomb(R, n, 1.0, 3, c, M);
  }
  matmul(As, R, S, n);                                     /* T9s = A (...) */
done:
  free(A4); free(R); free(A8); free(Q);
  return rc;
}

/* k = 6 products: eq. Algorithm6cA with coefficients eq:cosm8 (T16c) and
 * eq. Algorithm6sA with the z list printed after it (T_{17,25}s). */
static int chain_m16(const double* As, const double* A2, long n, double* C, double* S) {
  int rc = ORC_OK;
  double *A4 = NULL, *R = NULL, *A8 = NULL, *L = NULL, *A16 = NULL, *W = NULL,
         *C24 = NULL, *Q = NULL;
  const double r = sqrt(36681.0);
  const double x1 = 7.0 / 500.0;
  const double x2 = -7.0 / 60000.0;
  const double x3 = (-1533.0 + 7.0 * r) / 2500.0;
  const double x4 = -5.0 * (124581.0 + 391.0 * r) / 10594584.0;
  const double x5 = 9775.0 / 10594584.0;
  const double x6 = -5.0 * (1001.0 + r) / 508540032.0;
  const double x7 = 3125.0 / 889945056.0;
  const double x8 = (1549211.0 + 3246.0 * r) / 63063000.0;
  const double z0 = 8887.0 / 4794.0;
  const double z1 = -1897.0 / 3196.0;
  const double z2 = 25259.0 / 575280.0;
  const double z3 = -965093875.0 / 9674368704.0;
  const double z4 = -4093.0 / 4794.0;
  const double z5 = 25698275.0 / 29023106112.0;
  const double z6 = -3907675.0 / 348277273344.0;
  const double z7 = 11865625.0 / 3656911370112.0;
  const double z8 = 25.0 / 308756448.0;
  NEWMAT(A4); NEWMAT(R); NEWMAT(A8); NEWMAT(L); NEWMAT(A16); NEWMAT(W);
  NEWMAT(C24); NEWMAT(Q);
  matmul(A2, A2, A4, n);                                   /* A4 = A2^2 */
  {
    const double c[2] = {x1, x2};
    const double* M[2] = {A2, A4};
    lincomb(R, n, 0.0, 2, c, M);
  }
  matmul(A4, R, A8, n);                                    /* A8 = A4(x1 A2 + x2 A4) */
  {
    const double c[2] = {x3, 1.0};
    const double* M[2] = {A4, A8};
    lincomb(L, n, 0.0, 2, c, M);                           /* x3 A4 + A8 */
  }
  {
    const double c[3] = {x5, x6, x7};
    const double* M[3] = {A2, A4, A8};
    lincomb(W, n, x4, 3, c, M);                            /* x4 I + x5 A2 + x6 A4 + x7 A8 */
  }
  matmul(L, W, A16, n);                                    /* A16 */
  {
    const double c[3] = {-0.5, x8, 1.0};
    const double* M[3] = {A2, A4, A16};
    lincomb(C, n, 1.0, 3, c, M);                           /* T16c */
  }
  {
    /* the scheme prints z5 in front of both I and A2 */
    const double c[4] = {z5, z6, z7, z8};
    const double* M[4] = {A2, A4, A8, C};
    lincomb(W, n, z5, 4, c, M);
  }
  matmul(W, A8, C24, n);                                   /* C24 */
  {
    const double c[5] = {z1, z2, z3, z4, 1.0};
    const double* M[5] = {A2, A4, A8, C, C24};
    lincomb(Q, n, z0, 5, c, M);
  }
  matmul(As, Q, S, n);                                     /* T_{17,25}s */
done:
  free(A4); free(R); free(A8); free(L); free(A16); free(W); free(C24); free(Q);
  return rc;
}

/* k = 7 products: eq. Algorithm7cA with Coefs7cA (T24c) and eq. Algorithm7sA
 * with Coefs7sA (T_{23,49}s). */
static int chain_m24(const double* As, const double* A2, long n, double* C, double* S) {
  int rc = ORC_OK;
  /* a[i][j-1] multiplies A_{2i} in C_j (A_0 = I). */
  static const double a[4][4] = {
      {0.0, 0.55751443809990408029, 0.75936877868464999248, 0.0},
      {0.0, -0.61577924683458386455, -0.01560333979813817129,
       -0.039649968743474473091},
      {0.02264979811206039519, 0.00747198841446687051, 0.00010936989591908396,
       0.000155490073503821463},
      {-0.00013110924142135755, -0.00003362444420476012,
       -1.03893360877457159499e-6, -1.126739663071170022488e-6},
  };
  static const double z[12] = {
      0.10090808375109885598,  -0.07668753546445299316,
      0.00084924846993243257,  -0.00001220406904464391,
      0.98499703159318860027,  -0.84925233648155398756,
      1.0,                     0.00095544138280925799,
      4.56337109377154270633e-6, 2.73461259403000427141e-8,
      0.00048550288474842477,  -4.15891109384923342531e-7,
  };
  double *A4 = NULL, *A6 = NULL, *Cj[4] = {NULL, NULL, NULL, NULL}, *A12 = NULL,
         *L = NULL, *A24 = NULL, *W = NULL, *C48 = NULL, *Q = NULL;
  NEWMAT(A4); NEWMAT(A6);
  for (int j = 0; j < 4; ++j) NEWMAT(Cj[j]);
  NEWMAT(A12); NEWMAT(L); NEWMAT(A24); NEWMAT(W); NEWMAT(C48); NEWMAT(Q);
  matmul(A2, A2, A4, n);                                   /* A4 = A2^2 */
  matmul(A4, A2, A6, n);                                   /* A6 = A4 A2 */
  for (int j = 0; j < 4; ++j) {
    const double c[3] = {a[1][j], a[2][j], a[3][j]};
    const double* M[3] = {A2, A4, A6};
    lincomb(Cj[j], n, a[0][j], 3, c, M);                   /* C_1 .. C_4 */
  }
  matmul(Cj[3], Cj[3], A12, n);                            /* C4^2 */
  {
    const double c[2] = {1.0, 1.0};
    const double* M[2] = {Cj[2], A12};
    lincomb(A12, n, 0.0, 2, c, M);                         /* A12 = C3 + C4^2 */
  }
  {
    const double c[2] = {1.0, 1.0};
    const double* M[2] = {Cj[1], A12};
    lincomb(L, n, 0.0, 2, c, M);                           /* C2 + A12 */
  }
  matmul(L, A12, A24, n);                                  /* A24 */
  {
    const double c[2] = {1.0, 1.0};
    const double* M[2] = {Cj[0], A24};
    lincomb(C, n, 0.0, 2, c, M);                           /* T24c = C1 + A24 */
  }
  {
    const double c[5] = {z[7], z[8], z[9], z[10], z[11]};
    const double* M[5] = {A2, A4, A6, A12, C};
    lincomb(W, n, z[6], 5, c, M);
  }
  matmul(W, C, C48, n);                                    /* C48 */
  {
    const double c[6] = {z[1], z[2], z[3], z[4], z[5], 1.0};
    const double* M[6] = {A2, A4, A6, A12, C, C48};
    lincomb(Q, n, z[0], 6, c, M);
  }
  matmul(As, Q, S, n);                                     /* T_{23,49}s */
done:
  free(A4); free(A6);
  for (int j = 0; j < 4; ++j) free(Cj[j]);
  free(A12); free(L); free(A24); free(W); free(C48); free(Q);
  return rc;
}

/*
 * cos(A) and sin(A) of a dense row-major n x n FP64 matrix.
 *   prec      0 = double table (u = 2^-53), 1 = single table (u = 2^-24)
 *   force_m   -1 for the automatic choice, else 4, 8, 16 or 24, or 9 for
 *             T8c with the five-product sine T9s (eq. Algorithm5sA)
 *   force_s   -1 for the automatic choice, else 0 .. 64
 * C, S: caller-owned n x n outputs.  info may be NULL.
 */
int oracle_cossin(const double* A, long n, int prec, int force_m, int force_s,
                  double* C, double* S, oracle_info* info) {
  if (n < 0 || prec < 0 || prec > 1) return ORC_EINVAL;
  if (force_m != -1 && force_m != 4 && force_m != 8 && force_m != 9 && force_m != 16 && force_m != 24)
    return ORC_EINVAL;
  if (force_s < -1 || force_s > ORC_MAX_S) return ORC_EINVAL;
  if ((force_m == -1) != (force_s == -1)) return ORC_EINVAL;
  double nrm = oracle_norm1(A, n);
  int m, s, rc = ORC_OK;
  if (!isfinite(nrm)) return ORC_ENONFINITE;
  if (force_m == -1) {
    rc = oracle_select(nrm, prec, &m, &s);
    if (rc != ORC_OK) return rc;
  } else {
    m = force_m;
    s = force_s;
  }
  int f = (m == 4) ? 0 : (m == 8 || m == 9) ? 1 : (m == 16) ? 2 : 3;
  if (info) {
    info->norm1 = nrm;
    info->m = m;
    info->s = s;
    info->products = PI_2M[f] + (m == 9) + 2 * s;  /* T9s: one product more */
  }
  if (n == 0) return ORC_OK;

  double *As = NULL, *A2 = NULL, *C2 = NULL, *T = NULL;
  NEWMAT(As); NEWMAT(A2); NEWMAT(C2); NEWMAT(T);
  scale(As, A, ldexp(1.0, -s), n);                         /* A_s = 2^-s A */
  matmul(As, As, A2, n);                                   /* A_2 = A_s^2 */
  switch (m) {
    case 4: rc = chain_m4(As, A2, n, C, S); break;
    case 8: rc = chain_m8(As, A2, n, C, S); break;
    case 9: rc = chain_m9(As, A2, n, C, S); break;
    case 16: rc = chain_m16(As, A2, n, C, S); break;
    default: rc = chain_m24(As, A2, n, C, S); break;
  }
  if (rc != ORC_OK) goto done;
  /* Double-angle recovery, Sec. 1: cos 2X = 2cos^2 X - I, sin 2X = 2 sin X cos X. */
  for (int j = 0; j < s; ++j) {
    matmul(C, C, C2, n);
    matmul(S, C, T, n);
    for (long i = 0; i < n; ++i)
      for (long k = 0; k < n; ++k) {
        C[i * n + k] = 2.0 * C2[i * n + k] - ((i == k) ? 1.0 : 0.0);
        S[i * n + k] = 2.0 * T[i * n + k];
      }
  }
done:
  free(As); free(A2); free(C2); free(T);
  return rc;
}

/* ------------------------------------------------------------------------
 * Sec. 2.2: c(t^2 A) = cos(sqrt(t^2 A)) and s(t, A) = A^(-1/2) sin(sqrt(t^2 A))
 * together, evaluated on B = t^2 A directly (the schemes of Sec. 2.1 with
 * A_2 replaced by B and the last sine product replaced by the scalar t), and
 * recovered with c(4 t^2 A) = 2 c^2 - I, s(2t, A) = 2 s c (Sec. 1).
 *
 * Families (products):  0 = k=3 with P_{3,4}^s (2),  1 = k=3 with P_4^s (3),
 *                       2 = k=4 (4),                   3 = k=5 (5).
 * Reading of eq. Algorithm83eA for P_{3,4}^s: the printed "- (6!/7!) B_4"
 * has the wrong sign; B_4 already carries -1/6!, and only "+" reproduces the
 * series through B^3 (as in eq. Algorithm4sA).
 * The paper gives no admissible norms for these schemes.  THETA_CS holds the
 * largest ||B||_1 at which the Sec. 3 error series (150 terms) of the cosine
 * part, and of the sine part divided by t, stay <= u; it is the smaller of the
 * two (the cosine values are theta_2m^2 of Tables 1-2).
 * ---------------------------------------------------------------------- */
static const double THETA_CS[2][4] = {
    {3.44587e-3, 1.32137e-2, 9.62511e-1, 3.64043},
    {5.22375e-1, 7.35401e-1, 8.96121, 21.8484},
};
static const int PI_CS[4] = {2, 3, 4, 5};

double oracle_cs_theta(int prec, int family) {
  if (prec < 0 || prec > 1 || family < 0 || family > 3) return -1.0;
  return THETA_CS[prec][family];
}

/* (family, sigma) of minimal cost Pi + 2 sigma with ||B||_1 / 4^sigma <= theta. */
int oracle_cs_select(double normB, int prec, int* f_out, int* s_out) {
  if (prec < 0 || prec > 1) return ORC_EINVAL;
  if (!isfinite(normB)) return ORC_ENONFINITE;
  int best = -1, best_s = 0, best_cost = 1 << 30;
  for (int f = 0; f < 4; ++f) {
    int sg = 0;
    while (ldexp(normB, -2 * sg) > THETA_CS[prec][f]) ++sg;
    if (sg > ORC_MAX_S) continue;
    const int cost = PI_CS[f] + 2 * sg;
    if (cost < best_cost || (cost == best_cost && sg < best_s)) {
      best_cost = cost;
      best = f;
      best_s = sg;
    }
  }
  if (best < 0) return ORC_ERANGE;
  *f_out = best;
  *s_out = best_s;
  return ORC_OK;
}

/* k = 3 products: eq. Algorithm83eA (P_4^c) with P_{3,4}^s or P_4^s. */
static int cs_k3(const double* B, double t, long n, int with_p4s, double* C, double* S) {
  int rc = ORC_OK;
  double *B2 = NULL, *R = NULL, *B4 = NULL, *T = NULL;
  NEWMAT(B2); NEWMAT(R); NEWMAT(B4); NEWMAT(T);
  matmul(B, B, B2, n);                                       /* B_2 = B^2 */
  {
    const double c[2] = {-1.0 / 720.0, 1.0 / 40320.0};       /* -B/6! + B_2/8! */
    const double* M[2] = {B, B2};
    lincomb(R, n, 0.0, 2, c, M);
  }
  matmul(B2, R, B4, n);                                      /* B_4 */
  {
    const double c[3] = {-1.0 / 2.0, 1.0 / 24.0, 1.0};
    const double* M[3] = {B, B2, B4};
    lincomb(C, n, 1.0, 3, c, M);                             /* P_4^c */
  }
  if (!with_p4s) {
    const double c[3] = {-t / 6.0, t / 120.0, t * 720.0 / 5040.0};
    const double* M[3] = {B, B2, B4};
    lincomb(S, n, t, 3, c, M);                               /* P_{3,4}^s, "+" (6!/7!) B_4 */
  } else {
    const double c[2] = {-1.0 / 5040.0, 1.0 / 362880.0};     /* -B/7! + B_2/9! */
    const double* M[2] = {B, B2};
    lincomb(R, n, 0.0, 2, c, M);
    matmul(B2, R, T, n);
    const double c2[3] = {-t / 6.0, t / 120.0, t};
    const double* M2[3] = {B, B2, T};
    lincomb(S, n, t, 3, c2, M2);                             /* P_4^s */
  }
done:
  free(B2); free(R); free(B4); free(T);
  return rc;
}

/* k = 4 products: P_8^c with the coefficients of eq. cosm8 (y0 = 1,
 * y1 = -1/2, y2 = x8) and P_{8,12}^s with the z list of Sec. 2.1, k = 6. */
static int cs_k4(const double* B, double t, long n, double* C, double* S) {
  int rc = ORC_OK;
  double *B2 = NULL, *R = NULL, *B4 = NULL, *L = NULL, *Wm = NULL, *B8 = NULL, *C12 = NULL;
  const double r = sqrt(36681.0);
  const double x1 = 7.0 / 500.0, x2 = -7.0 / 60000.0, x3 = (-1533.0 + 7.0 * r) / 2500.0;
  const double x4 = -5.0 * (124581.0 + 391.0 * r) / 10594584.0, x5 = 9775.0 / 10594584.0;
  const double x6 = -5.0 * (1001.0 + r) / 508540032.0, x7 = 3125.0 / 889945056.0;
  const double x8 = (1549211.0 + 3246.0 * r) / 63063000.0;
  const double z0 = 8887.0 / 4794.0, z1 = -1897.0 / 3196.0, z2 = 25259.0 / 575280.0;
  const double z3 = -965093875.0 / 9674368704.0, z4 = -4093.0 / 4794.0;
  const double z5 = 25698275.0 / 29023106112.0, z6 = -3907675.0 / 348277273344.0;
  const double z7 = 11865625.0 / 3656911370112.0, z8 = 25.0 / 308756448.0;
  NEWMAT(B2); NEWMAT(R); NEWMAT(B4); NEWMAT(L); NEWMAT(Wm); NEWMAT(B8); NEWMAT(C12);
  matmul(B, B, B2, n);
  {
    const double c[2] = {x1, x2};
    const double* M[2] = {B, B2};
    lincomb(R, n, 0.0, 2, c, M);
  }
  matmul(B2, R, B4, n);                                      /* B_4 = B_2 (x1 B + x2 B_2) */
  {
    const double c[2] = {x3, 1.0};
    const double* M[2] = {B2, B4};
    lincomb(L, n, 0.0, 2, c, M);
  }
  {
    const double c[3] = {x5, x6, x7};
    const double* M[3] = {B, B2, B4};
    lincomb(Wm, n, x4, 3, c, M);
  }
  matmul(L, Wm, B8, n);                                      /* B_8 */
  {
    const double c[3] = {-0.5, x8, 1.0};
    const double* M[3] = {B, B2, B8};
    lincomb(C, n, 1.0, 3, c, M);                             /* P_8^c */
  }
  {
    const double c[4] = {z5, z6, z7, z8};
    const double* M[4] = {B, B2, B4, C};
    lincomb(Wm, n, z5, 4, c, M);
  }
  matmul(Wm, B4, C12, n);                                    /* C_12 */
  {
    const double c[5] = {t * z1, t * z2, t * z3, t * z4, t};
    const double* M[5] = {B, B2, B4, C, C12};
    lincomb(S, n, t * z0, 5, c, M);                          /* P_{8,12}^s */
  }
done:
  free(B2); free(R); free(B4); free(L); free(Wm); free(B8); free(C12);
  return rc;
}

/* k = 5 products: eq. poly12 (P_12^c) with Coefs7cA and P_{11,24}^s with
 * Coefs7sA (its P_12^c(A) read as P_12^c(B)). */
static int cs_k5(const double* B, double t, long n, double* C, double* S) {
  int rc = ORC_OK;
  static const double a[4][4] = {
      {0.0, 0.55751443809990408029, 0.75936877868464999248, 0.0},
      {0.0, -0.61577924683458386455, -0.01560333979813817129, -0.039649968743474473091},
      {0.02264979811206039519, 0.00747198841446687051, 0.00010936989591908396,
       0.000155490073503821463},
      {-0.00013110924142135755, -0.00003362444420476012, -1.03893360877457159499e-6,
       -1.126739663071170022488e-6},
  };
  static const double z[12] = {
      0.10090808375109885598,  -0.07668753546445299316, 0.00084924846993243257,
      -0.00001220406904464391, 0.98499703159318860027,  -0.84925233648155398756,
      1.0,                     0.00095544138280925799,  4.56337109377154270633e-6,
      2.73461259403000427141e-8, 0.00048550288474842477, -4.15891109384923342531e-7,
  };
  double *B2 = NULL, *B3 = NULL, *D[4] = {NULL, NULL, NULL, NULL}, *B6 = NULL, *L = NULL, *P = NULL,
         *Wm = NULL, *C24 = NULL;
  NEWMAT(B2); NEWMAT(B3);
  for (int j = 0; j < 4; ++j) NEWMAT(D[j]);
  NEWMAT(B6); NEWMAT(L); NEWMAT(P); NEWMAT(Wm); NEWMAT(C24);
  matmul(B, B, B2, n);
  matmul(B2, B, B3, n);
  for (int j = 0; j < 4; ++j) {
    const double c[3] = {a[1][j], a[2][j], a[3][j]};
    const double* M[3] = {B, B2, B3};
    lincomb(D[j], n, a[0][j], 3, c, M);                      /* D_1 .. D_4 */
  }
  matmul(D[3], D[3], B6, n);
  {
    const double c[2] = {1.0, 1.0};
    const double* M[2] = {D[2], B6};
    lincomb(B6, n, 0.0, 2, c, M);                            /* B_6 = D_3 + D_4^2 */
  }
  {
    const double c[2] = {1.0, 1.0};
    const double* M[2] = {D[1], B6};
    lincomb(L, n, 0.0, 2, c, M);
  }
  matmul(L, B6, P, n);
  {
    const double c[2] = {1.0, 1.0};
    const double* M[2] = {D[0], P};
    lincomb(C, n, 0.0, 2, c, M);                             /* P_12^c */
  }
  {
    const double c[5] = {z[7], z[8], z[9], z[10], z[11]};
    const double* M[5] = {B, B2, B3, B6, C};
    lincomb(Wm, n, z[6], 5, c, M);
  }
  matmul(Wm, C, C24, n);                                     /* C_24 */
  {
    const double c[6] = {t * z[1], t * z[2], t * z[3], t * z[4], t * z[5], t};
    const double* M[6] = {B, B2, B3, B6, C, C24};
    lincomb(S, n, t * z[0], 6, c, M);                        /* P_{11,24}^s */
  }
done:
  free(B2); free(B3);
  for (int j = 0; j < 4; ++j) free(D[j]);
  free(B6); free(L); free(P); free(Wm); free(C24);
  return rc;
}

/* C = c(t^2 A), S = s(t, A).  force_family / force_sigma as force_m / force_s. */
int oracle_cs(const double* A, long n, double t, int prec, int force_family, int force_sigma, double* C,
              double* S, oracle_info* info) {
  if (n < 0 || prec < 0 || prec > 1 || !isfinite(t)) return ORC_EINVAL;
  if (force_family < -1 || force_family > 3) return ORC_EINVAL;
  if (force_sigma < -1 || force_sigma > ORC_MAX_S) return ORC_EINVAL;
  if ((force_family == -1) != (force_sigma == -1)) return ORC_EINVAL;
  const double normB = t * t * oracle_norm1(A, n);
  int f, sg, rc = ORC_OK;
  if (!isfinite(normB)) return ORC_ENONFINITE;
  if (force_family == -1) {
    rc = oracle_cs_select(normB, prec, &f, &sg);
    if (rc != ORC_OK) return rc;
  } else {
    f = force_family;
    sg = force_sigma;
  }
  if (info) {
    info->norm1 = normB;
    info->m = f;
    info->s = sg;
    info->products = PI_CS[f] + 2 * sg;
  }
  if (n == 0) return ORC_OK;
  const double ts = ldexp(t, -sg);                           /* t / 2^sigma */
  double *Bs = NULL, *C2 = NULL, *T = NULL;
  NEWMAT(Bs); NEWMAT(C2); NEWMAT(T);
  scale(Bs, A, ts * ts, n);                                  /* B = (t/2^sigma)^2 A */
  switch (f) {
    case 0: rc = cs_k3(Bs, ts, n, 0, C, S); break;
    case 1: rc = cs_k3(Bs, ts, n, 1, C, S); break;
    case 2: rc = cs_k4(Bs, ts, n, C, S); break;
    default: rc = cs_k5(Bs, ts, n, C, S); break;
  }
  if (rc != ORC_OK) goto done;
  for (int j = 0; j < sg; ++j) {                             /* c(4t^2A) = 2c^2 - I, s(2t,A) = 2sc */
    matmul(C, C, C2, n);
    matmul(S, C, T, n);
    for (long i = 0; i < n; ++i)
      for (long k = 0; k < n; ++k) {
        C[i * n + k] = 2.0 * C2[i * n + k] - ((i == k) ? 1.0 : 0.0);
        S[i * n + k] = 2.0 * T[i * n + k];
      }
  }
done:
  free(Bs); free(C2); free(T);
  return rc;
}

/* Plain matrix product, exposed so that tests can assemble identities. */
void oracle_matmul(const double* X, const double* Y, double* Z, long n) { matmul(X, Y, Z, n); }
