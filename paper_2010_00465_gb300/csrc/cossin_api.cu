// cossin_api.cu -- host side of the library: argument checks, the choice of
// (m, s), the product plans of the factorised Taylor schemes, the double-angle
// recovery, workspace layout, error reporting and kernel timing hooks.
#include <math.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"
#include "ozaki.h"
#include "plan.h"
#include "tc_gemm.h"
#include "theta_table.cuh"

namespace cs {

// ---------------------------------------------------------------- errors ---
static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

cs_status fail(cs_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

cs_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return CS_ECUDA;
}

// ------------------------------------------------------------ allocation ---
static std::atomic<int> g_fail_allocs{0};

cs_status dev_alloc(void** p, size_t bytes, cudaStream_t stream, const char* what) {
  *p = nullptr;
  int left = g_fail_allocs.load();
  while (left > 0 && !g_fail_allocs.compare_exchange_weak(left, left - 1)) {
  }
  if (left > 0) return fail(CS_ENOMEM, std::string(what) + ": allocation failed (injected)");
  const cudaError_t e = cudaMallocAsync(p, bytes, stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(CS_ENOMEM, std::string(what) + ": allocation of " + std::to_string(bytes) +
                               " bytes failed: " + cudaGetErrorString(e));
  }
  return CS_OK;
}

// ------------------------------------------------------------- profiling ---
namespace {
struct ProfRecord {
  int kind;
  double work;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRecord> g_prof_pending;
double g_prof_ms[CS_KERNEL_KINDS] = {};
int64_t g_prof_n[CS_KERNEL_KINDS] = {};
double g_prof_work[CS_KERNEL_KINDS] = {};
}  // namespace

ProfScope::ProfScope(int kind_, double work_, cudaStream_t stream_)
    : kind(kind_), work(work_), stream(stream_) {
  bool on;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    on = g_prof_on;
  }
  if (!on) return;
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    ev[0] = ev[1] = nullptr;
    return;
  }
  cudaEventRecord(ev[0], stream);
}

ProfScope::~ProfScope() {
  if (!ev[0]) return;
  cudaEventRecord(ev[1], stream);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_pending.push_back({kind, work, ev[0], ev[1]});
}

static void prof_drain() {
  std::vector<ProfRecord> pend;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    pend.swap(g_prof_pending);
  }
  for (auto& r : pend) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_prof_mu);
      g_prof_ms[r.kind] += ms;
      g_prof_n[r.kind] += 1;
      g_prof_work[r.kind] += r.work;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
}

// -------------------------------------------------------------- selection ---
int products_of(int m) {
  if (m == 9) return 5;  // T8c with the five-product sine T9s (eq. Algorithm5sA)
  for (int f = 0; f < 4; ++f)
    if (family_order(f) == m) return family_products(f);
  return -1;
}

cs_status select_ms(double norm1, int table, int* m, int* s) {
  if (table < 0 || table > 1) return fail(CS_EINVAL, "select: table must be 0 (double) or 1 (single)");
  if (!isfinite(norm1)) return fail(CS_ENONFINITE, "select: ||A||_1 is not finite");
  if (norm1 < 0) return fail(CS_EINVAL, "select: negative norm");
  int f = 0, sf = 0;
  if (select_family(norm1, table, &f, &sf) != 0)
    return fail(CS_ERANGE, "select: ||A||_1 needs more than 64 double-angle steps");
  *m = family_order(f);
  *s = sf;
  return CS_OK;
}

// ------------------------------------------------------------- workspace ---
static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout make_layout(int64_t n, int prec, bool with_outputs) {
  Layout L;
  const size_t n2 = (size_t)n * (size_t)n;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  L.norm_partial = take(sizeof(double) * (size_t)norm1_scratch_elems(n));
  L.norm_out = take(sizeof(double));
  // Every precision keeps its intermediates in FP64: the double-angle
  // recurrence amplifies the rounding of stored intermediates far beyond
  // FP32 level at ||A||_1 near 64 (an FP32-stored evaluation with exactly
  // rounded products is 1.3e-5 from the FP64 result on a 1 x 1 matrix).
  for (int w = 0; w < kWorkSlots; ++w) L.w[w] = take(sizeof(double) * n2);
  L.ping64[0] = take(sizeof(double) * 2 * n2);
  L.ping64[1] = take(sizeof(double) * 2 * n2);
  if (prec == CS_FP32) L.a64 = take(sizeof(double) * n2);  // the FP32 input in FP64
  if (prec == CS_SPLIT_TF32 || prec == CS_SPLIT_EMU) {
    // operand splits of the four-pass TF32 chain products and their raw product
    L.ld32 = (n + 31) / 32 * 32;
    const size_t sz = sizeof(float) * (size_t)n * (size_t)L.ld32;
    for (int k = 0; k < 4; ++k) L.a4[k] = take(sz);
    for (int w = 0; w < kWorkSlots; ++w)
      for (int k = 0; k < 4; ++k) L.w4[w][k] = take(sz);
    for (int k = 0; k < 4; ++k) L.c4[k] = take(sz);
    L.p32 = take(sz);
  }
  if (!uses_emu((cs_prec)prec)) {
    // native FP64 products: the pieces of the tiles split over K
    L.splitk_bytes = std::max(gemm_f64_split_bytes(n, n, n), gemm_f64_split_bytes(2 * n, n, n));
    if (L.splitk_bytes) L.splitk = take(L.splitk_bytes);
  }
  if (uses_emu((cs_prec)prec)) {
    // the stacked double-angle product is the largest emulated one
    L.ozaki_bytes = ozaki_dims(2 * n, n, n, 1, square_slices((cs_prec)prec)).total;
    L.ozaki = take(L.ozaki_bytes);
  }
  if (with_outputs) {
    const size_t el = prec == CS_FP32 ? sizeof(float) : sizeof(double);
    L.out_c = take(el * n2);
    L.out_s = take(el * n2);
  }
  L.total = off;
  return L;
}

// ------------------------------------------------------------------ plans ---
// Products of the factorised schemes of Sec. 2.1, written as data.  Slot SL_A
// is A itself, SL_C and SL_S receive T^c_2m(A_s) and the sine approximant,
// W0..W7 hold intermediates.  Every step is P = X Y followed by its epilogue;
// the first product folds the scaling (A_s)^2 = 4^-s A A and the last folds
// A_s = 2^-s A into alpha (times scale^2 and scale for a scaled argument).
std::vector<Step> chain_plan(int m, int s, double scale) {
  const double a2 = scale * scale * ldexp(1.0, -2 * s), as = scale * ldexp(1.0, -s);
  std::vector<Step> P;
  auto out = [](int slot, double alpha, double gamma, std::vector<std::pair<int, double>> beta = {},
                std::vector<std::pair<int, double>> delta = {}) {
    return OutSpec{slot, alpha, gamma, std::move(beta), std::move(delta)};
  };
  P.push_back(Step{SL_A, SL_A, {out(W(0), a2, 0.0)}});  // A2 = (2^-s A)^2
  if (m == 4) {
    // eqs. Algorithm3cA, Algorithm3sA: T4c = I - A2/2! + A4/4!, T5s = A(I - A2/3! + A4/5!)
    P.push_back(Step{W(0), W(0), {out(SL_C, 1.0 / 24, 1.0, {{W(0), -0.5}}),
                                  out(W(1), 1.0 / 120, 1.0, {{W(0), -1.0 / 6}})}});
    P.push_back(Step{SL_A, W(1), {out(SL_S, as, 0.0)}});
  } else if (m == 8) {
    // eqs. Algorithm4cA, Algorithm4sA: A8 = A4(-A2/6! + A4/8!),
    // T8c = I - A2/2 + A4/24 + A8, T79s = A(I - A2/3! + A4/5! + (6!/7!) A8)
    P.push_back(Step{W(0), W(0), {out(W(1), 1.0, 0.0),                                 // A4
                                  out(W(2), 1.0 / 40320, 0.0, {{W(0), -1.0 / 720}}),   // -A2/6! + A4/8!
                                  out(W(3), 1.0 / 24, 1.0, {{W(0), -0.5}}),            // I - A2/2 + A4/24
                                  out(W(4), 1.0 / 120, 1.0, {{W(0), -1.0 / 6}})}});    // I - A2/6 + A4/120
    P.push_back(Step{W(1), W(2), {out(SL_C, 1.0, 0.0, {{W(3), 1.0}}),
                                  out(W(4), 720.0 / 5040.0, 0.0, {{W(4), 1.0}})}});
    P.push_back(Step{SL_A, W(4), {out(SL_S, as, 0.0)}});
  } else if (m == 9) {
    // eq. Algorithm4cA for the cosine and eq. Algorithm5sA for the sine:
    // A8' = A4(-A2/7! + A4/9!), T9s = A(I - A2/3! + A4/5! + A8') (one product more)
    P.push_back(Step{W(0), W(0), {out(W(1), 1.0, 0.0),                                   // A4
                                  out(W(2), 1.0 / 40320, 0.0, {{W(0), -1.0 / 720}}),     // -A2/6! + A4/8!
                                  out(W(3), 1.0 / 24, 1.0, {{W(0), -0.5}}),              // I - A2/2 + A4/24
                                  out(W(4), 1.0 / 120, 1.0, {{W(0), -1.0 / 6}}),         // I - A2/6 + A4/120
                                  out(W(5), 1.0 / 362880, 0.0, {{W(0), -1.0 / 5040}})}}); // -A2/7! + A4/9!
    P.push_back(Step{W(1), W(2), {out(SL_C, 1.0, 0.0, {{W(3), 1.0}})}});
    P.push_back(Step{W(1), W(5), {out(W(4), 1.0, 0.0, {{W(4), 1.0}})}});
    P.push_back(Step{SL_A, W(4), {out(SL_S, as, 0.0)}});
  } else if (m == 16) {
    // eq. Algorithm6cA with eq. cosm8, eq. Algorithm6sA with its z list.
    const double r = sqrt(36681.0);
    const double x1 = 7.0 / 500.0, x2 = -7.0 / 60000.0, x3 = (-1533.0 + 7.0 * r) / 2500.0;
    const double x4 = -5.0 * (124581.0 + 391.0 * r) / 10594584.0, x5 = 9775.0 / 10594584.0;
    const double x6 = -5.0 * (1001.0 + r) / 508540032.0, x7 = 3125.0 / 889945056.0;
    const double x8 = (1549211.0 + 3246.0 * r) / 63063000.0;
    const double z0 = 8887.0 / 4794.0, z1 = -1897.0 / 3196.0, z2 = 25259.0 / 575280.0;
    const double z3 = -965093875.0 / 9674368704.0, z4 = -4093.0 / 4794.0;
    const double z5 = 25698275.0 / 29023106112.0, z6 = -3907675.0 / 348277273344.0;
    const double z7 = 11865625.0 / 3656911370112.0, z8 = 25.0 / 308756448.0;
    P.push_back(Step{W(0), W(0), {out(W(1), 1.0, 0.0),                       // A4
                                  out(W(2), x2, 0.0, {{W(0), x1}})}});       // x1 A2 + x2 A4
    P.push_back(Step{W(1), W(2), {out(W(3), 1.0, 0.0),                                     // A8
                                  out(W(4), 1.0, 0.0, {{W(1), x3}}),                       // x3 A4 + A8
                                  out(W(5), x7, x4, {{W(0), x5}, {W(1), x6}}),             // x4 I + x5 A2 + x6 A4 + x7 A8
                                  out(W(6), z3, z0, {{W(0), z1}, {W(1), z2}}),             // z0 I + z1 A2 + z2 A4 + z3 A8
                                  out(W(7), z7, z5, {{W(0), z5}, {W(1), z6}})}});          // z5 I + z5 A2 + z6 A4 + z7 A8
    P.push_back(Step{W(4), W(5), {out(SL_C, 1.0, 1.0, {{W(0), -0.5}, {W(1), x8}}),          // T16 = I - A2/2 + x8 A4 + A16
                                  out(W(6), 0.0, 0.0, {{W(6), 1.0}}, {{0, z4}}),           // ... + z4 T16
                                  out(W(7), 0.0, 0.0, {{W(7), 1.0}}, {{0, z8}})}});        // ... + z8 T16
    P.push_back(Step{W(7), W(3), {out(W(2), 1.0, 0.0, {{W(6), 1.0}})}});                    // C24 = (...) A8; sum
    P.push_back(Step{SL_A, W(2), {out(SL_S, as, 0.0)}});
  } else {
    // eq. Algorithm7cA with Coefs7cA, eq. Algorithm7sA with Coefs7sA.
    // a[i][j-1] multiplies A_{2i} in C_j (A_0 = I).
    static const double a[4][4] = {
        {0.0, 0.55751443809990408029, 0.75936877868464999248, 0.0},
        {0.0, -0.61577924683458386455, -0.01560333979813817129, -0.039649968743474473091},
        {0.02264979811206039519, 0.00747198841446687051, 0.00010936989591908396,
         0.000155490073503821463},
        {-0.00013110924142135755, -0.00003362444420476012, -1.03893360877457159499e-6,
         -1.126739663071170022488e-6}};
    static const double z[12] = {0.10090808375109885598,   -0.07668753546445299316,
                                 0.00084924846993243257,   -0.00001220406904464391,
                                 0.98499703159318860027,   -0.84925233648155398756,
                                 1.0,                      0.00095544138280925799,
                                 4.56337109377154270633e-6, 2.73461259403000427141e-8,
                                 0.00048550288474842477,   -4.15891109384923342531e-7};
    P.push_back(Step{W(0), W(0), {out(W(1), 1.0, 0.0)}});  // A4
    std::vector<OutSpec> o;
    for (int j = 0; j < 4; ++j)  // C_{j+1} = a0 I + a1 A2 + a2 A4 + a3 A6 -> W2..W5
      o.push_back(out(W(2 + j), a[3][j], a[0][j], {{W(0), a[1][j]}, {W(1), a[2][j]}}));
    o.push_back(out(W(6), z[3], z[0], {{W(0), z[1]}, {W(1), z[2]}}));  // sine sum, first terms
    o.push_back(out(W(7), z[9], z[6], {{W(0), z[7]}, {W(1), z[8]}}));  // left factor of C48
    P.push_back(Step{W(1), W(0), o});                                  // A6 = A4 A2
    P.push_back(Step{W(5), W(5), {out(W(4), 1.0, 0.0, {{W(4), 1.0}}),               // A12 = C3 + C4^2
                                  out(W(3), 0.0, 0.0, {{W(3), 1.0}}, {{0, 1.0}}),    // C2 + A12
                                  out(W(6), 0.0, 0.0, {{W(6), 1.0}}, {{0, z[4]}}),
                                  out(W(7), 0.0, 0.0, {{W(7), 1.0}}, {{0, z[10]}})}});
    P.push_back(Step{W(3), W(4), {out(SL_C, 1.0, 0.0, {{W(2), 1.0}}),               // T24 = C1 + A24
                                  out(W(6), 0.0, 0.0, {{W(6), 1.0}}, {{0, z[5]}}),
                                  out(W(7), 0.0, 0.0, {{W(7), 1.0}}, {{0, z[11]}})}});
    P.push_back(Step{W(7), SL_C, {out(W(0), 1.0, 0.0, {{W(6), 1.0}})}});             // C48; sum
    P.push_back(Step{SL_A, W(0), {out(SL_S, as, 0.0)}});
  }
  return P;
}

// ------------------------------------------------------------------ specs ---
PlanSpec cossin_spec(int m, int s, double scale) {
  PlanSpec P;
  P.steps = chain_plan(m, s, scale);
  P.s = s;
  return P;
}

int cs_products(int family) { return cs_family_products(family); }

// Sec. 2.2: the schemes of Sec. 2.1 evaluated on B = t^2 A directly.  B takes
// the place of A_2 (slot W0, written scaled before the steps, so the first
// product A A disappears) and the sine's last product A (...) becomes the
// scalar t: the output that fed it is written to S scaled by t / 2^sigma.
// Family 0 is the k = 4 chain (P_4^c with P_{3,4}^s, whose printed minus
// sign in front of (6!/7!) B_4 is read as plus); family 1 adds the product
// B_2 (-B/7! + B_2/9!) for P_4^s; families 2 and 3 are the k = 6 and k = 7
// chains (P_8^c, P_{8,12}^s and P_12^c, P_{11,24}^s).
PlanSpec cs_spec(int family, int sigma, double t) {
  const double ts = ldexp(t, -sigma);
  PlanSpec P;
  P.s = sigma;
  P.scale_into_w0 = true;
  P.input_scale = ts * ts;
  if (family == 1) {
    auto out = [](int slot, double alpha, double gamma, std::vector<std::pair<int, double>> beta = {}) {
      return OutSpec{slot, alpha, gamma, std::move(beta), {}};
    };
    P.steps.push_back(Step{W(0), W(0), {out(W(1), 1.0, 0.0),                                   // B_2
                                        out(W(2), 1.0 / 40320, 0.0, {{W(0), -1.0 / 720}}),     // -B/6! + B_2/8!
                                        out(W(3), 1.0 / 24, 1.0, {{W(0), -0.5}}),              // I - B/2! + B_2/4!
                                        out(W(4), 1.0 / 362880, 0.0, {{W(0), -1.0 / 5040}}),   // -B/7! + B_2/9!
                                        out(W(5), 1.0 / 120, 1.0, {{W(0), -1.0 / 6}})}});      // I - B/3! + B_2/5!
    P.steps.push_back(Step{W(1), W(2), {out(SL_C, 1.0, 0.0, {{W(3), 1.0}})}});                 // P_4^c
    P.steps.push_back(Step{W(1), W(4), {out(SL_S, ts, 0.0, {{W(5), ts}})}});                   // P_4^s
    return P;
  }
  const int m = family == 0 ? 8 : family == 2 ? 16 : 24;
  std::vector<Step> full = chain_plan(m, 0);
  // drop A_2 = A A (W0 holds B) and the final S = A (...)
  const Step last = full.back();
  P.steps.assign(full.begin() + 1, full.end() - 1);
  const int q = last.Y;  // the sine's right factor
  for (auto it = P.steps.rbegin(); it != P.steps.rend(); ++it) {
    bool found = false;
    for (OutSpec& o : it->outs) {
      if (o.slot != q) continue;
      o.slot = SL_S;
      o.alpha *= ts;
      o.gamma *= ts;
      for (auto& b : o.beta) b.second *= ts;
      for (auto& d : o.delta) d.second *= ts;
      found = true;
    }
    if (found) break;
  }
  return P;
}

// -------------------------------------------------------------- execution ---
namespace {

struct F64Slots {
  const double* p[SL_COUNT] = {};
};

template <typename T>
Epilogue<T> build_epilogue(const Step& st, T* const* hi, T* const* lo) {
  EpiBuilder<T> b;
  std::vector<int> in_slots;
  auto in_index = [&](int slot) {
    for (size_t i = 0; i < in_slots.size(); ++i)
      if (in_slots[i] == slot) return (int)i;
    in_slots.push_back(slot);
    return b.add_in(hi[slot], lo ? lo[slot] : nullptr);
  };
  for (const OutSpec& o : st.outs) {
    const int t = b.add_out(hi[o.slot], o.alpha, o.gamma, lo ? lo[o.slot] : nullptr);
    for (auto& bc : o.beta) b.beta(t, in_index(bc.first), bc.second);
    for (auto& dc : o.delta) b.delta(t, dc.first, dc.second);
  }
  return b.e;
}

cs_status run_f64(const double* A, int64_t n, double* C, double* S, char* ws, const Layout& L, const PlanSpec& P,
                  const F64Product& chain, const F64Product& prod, cudaStream_t stream) {
  double* slot[SL_COUNT] = {};
  double* ping[2] = {(double*)(ws + L.ping64[0]), (double*)(ws + L.ping64[1])};
  const size_t n2 = (size_t)n * (size_t)n;
  const int s = P.s;
  slot[SL_A] = const_cast<double*>(A);
  slot[SL_C] = s == 0 ? C : ping[0];
  slot[SL_S] = s == 0 ? S : ping[0] + n2;
  for (int w = 0; w < kWorkSlots; ++w) slot[W(w)] = (double*)(ws + L.w[w]);
  if (P.scale_into_w0) CS_CHECK(scale_f64(A, slot[W(0)], (int64_t)n2, P.input_scale, stream));
  for (const Step& st : P.steps) {
    Epilogue<double> e = build_epilogue<double>(st, slot, nullptr);
    CS_CHECK(chain(slot[st.X], slot[st.Y], n, n, n, e, stream));
  }
  return square_f64(ping, n, s, C, S, stream, prod);
}

}  // namespace

// The FP64 executor for every precision whose products take FP64 operands
// (all but the TF32 split forms).  CS_FP32 converts its input to FP64 once,
// runs the plan with four-slice products and FP64 intermediates, and rounds
// C and S to FP32 once at the end (the FP64 result of the last step lands in
// ping[s & 1], which the last double-angle step does not read).
cs_status run_plan_f64(const void* A, int64_t n, cs_prec prec, void* C, void* S, char* w, const Layout& L,
                       const PlanSpec& spec, cudaStream_t stream) {
  if (prec != CS_FP32)
    return run_f64((const double*)A, n, (double*)C, (double*)S, w, L, spec, chain_product(prec, w, L),
                   f64_product(prec, w, L), stream);
  const int64_t n2 = n * n;
  double* a64 = (double*)(w + L.a64);
  CS_CHECK(convert_f32_f64((const float*)A, a64, n2, stream));
  double* fin = (double*)(w + L.ping64[spec.s & 1]);
  CS_CHECK(run_f64(a64, n, fin, fin + n2, w, L, spec, chain_product(prec, w, L), f64_product(prec, w, L), stream));
  CS_CHECK(convert_f64_f32(fin, (float*)C, n2, stream));
  return convert_f64_f32(fin + n2, (float*)S, n2, stream);
}

// Double-angle steps (Sec. 1): [C'; S'] = [C; S] C with C' = 2X - I, S' = 2X,
// one stacked 2n x n x n product per step, ping-ponging between the buffers.
cs_status F64Product::operator()(const double* X, const double* Y, int64_t M, int64_t N, int64_t K,
                                 const Epilogue<double>& e, cudaStream_t stream) const {
  if (emu_work) return gemm_f64_emu(X, Y, M, N, K, K, N, e, N, emu_work, emu_bytes, err, stream, slices);
  return gemm_f64(X, Y, M, N, K, K, N, false, false, e, N, 1, 0, 0, 0, stream, split_work, split_bytes);
}

int square_slices(cs_prec prec) { return prec == CS_FP32 ? kOzakiSlicesSplit : kOzakiSlices; }

F64Product f64_product(cs_prec prec, char* ws, const Layout& L) {
  F64Product p;
  if (uses_emu(prec)) {
    p.emu_work = ws + L.ozaki;
    p.emu_bytes = L.ozaki_bytes;
    p.err = tc_error_word();
    p.slices = square_slices(prec);
  } else if (L.splitk_bytes) {
    p.split_work = ws + L.splitk;
    p.split_bytes = L.splitk_bytes;
  }
  return p;
}

F64Product chain_product(cs_prec prec, char* ws, const Layout& L) {
  F64Product p = f64_product(prec, ws, L);
  if (prec == CS_SPLIT_BF16 || prec == CS_FP32) p.slices = kOzakiSlicesSplit;
  return p;
}

cs_status square_f64(double* const ping[2], int64_t n, int s, double* C, double* S, cudaStream_t stream,
                     const F64Product& prod) {
  const size_t n2 = (size_t)n * (size_t)n;
  for (int j = 0; j < s; ++j) {
    double* cur = ping[j & 1];
    const bool last = (j == s - 1);
    double* nc = last ? C : ping[(j + 1) & 1];
    double* ns = last ? S : ping[(j + 1) & 1] + n2;
    Epilogue<double> e;
    e.split_row = n;
    e.n_out = 2;
    e.out[0] = nc;
    e.out[1] = ns;
    e.alpha[0] = 2.0;
    e.alpha[1] = 2.0;
    e.gamma[0] = -1.0;
    e.gamma[1] = 0.0;
    CS_CHECK(prod(cur, cur, 2 * n, n, n, e, stream));
  }
  return CS_OK;
}

bool uses_emu(cs_prec p) {
  return p == CS_FP64_EMU || p == CS_SPLIT_EMU || p == CS_SPLIT_BF16 || p == CS_FP32;
}

bool f64_operands(cs_prec p) { return p != CS_SPLIT_TF32 && p != CS_SPLIT_EMU; }

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const char* pa = (const char*)a;
  const char* pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

size_t elem_size(cs_prec p) { return p == CS_FP32 ? sizeof(float) : sizeof(double); }

cs_status check_prec(cs_prec prec) {
  if (prec != CS_FP64 && prec != CS_FP32 && prec != CS_SPLIT_TF32 && prec != CS_FP64_EMU && prec != CS_SPLIT_EMU &&
      prec != CS_SPLIT_BF16)
    return fail(CS_EINVAL, "unknown precision");
  return CS_OK;
}

namespace {

struct PinnedWords {
  double norm;
  int err;
};
thread_local PinnedWords* t_pinned = nullptr;

}  // namespace

// Reads ||A||_1 from the device (one 8-byte copy and a stream synchronisation)
// together with the tensor-core kernels' error word, which reports a bounded
// wait that expired in an earlier call on this device.
cs_status read_norm(const double* dev, double* host, cudaStream_t stream) {
  if (!t_pinned) CS_CUDA_CHECK(cudaMallocHost((void**)&t_pinned, sizeof(PinnedWords)));
  int* errw = tc_error_word();
  if (dev) CS_CUDA_CHECK(cudaMemcpyAsync(&t_pinned->norm, dev, sizeof(double), cudaMemcpyDeviceToHost, stream));
  if (errw) CS_CUDA_CHECK(cudaMemcpyAsync(&t_pinned->err, errw, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CS_CUDA_CHECK(cudaStreamSynchronize(stream));
  if (host) *host = t_pinned->norm;
  if (errw && t_pinned->err) {
    CS_CUDA_CHECK(cudaMemsetAsync(errw, 0, sizeof(int), stream));
    return fail(CS_ETIMEOUT, "a tensor-core kernel gave up on a bounded wait in an earlier call");
  }
  return CS_OK;
}

cs_status run_tf32(const double* A, int64_t n, cs_prec prec, double* C, double* S, char* ws, const Layout& L,
                   const PlanSpec& P, cudaStream_t stream);
cs_status matmul_tf32(const void* X, const void* Y, int64_t n, bool f64_io, void* P, cudaStream_t stream);

// cos and sin of scale * A (scale = 1 for cossin / cossin_ex); the workspace
// is make_layout(n, prec).total bytes.
cs_status cossin_impl(const void* A, int64_t n, cs_prec prec, void* C, void* S, void* ws, size_t ws_bytes,
                      int32_t force_m, int32_t force_s, cs_info* info, cudaStream_t stream, double scale) {
  CS_CHECK(check_prec(prec));
  if (!isfinite(scale)) return fail(CS_EINVAL, "t must be finite");
  if (n < 0 || n > kMaxN) return fail(CS_EINVAL, "n out of range [0, 65536]");
  if (uses_emu(prec) && n > kOzakiMaxK) return fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if ((force_m == -1) != (force_s == -1)) return fail(CS_EINVAL, "force_m and force_s must both be -1 or both set");
  if (force_m != -1 && products_of(force_m) < 0) return fail(CS_EINVAL, "force_m must be 4, 8, 9, 16 or 24");
  if (force_s < -1 || force_s > kMaxS) return fail(CS_EINVAL, "force_s must be in [0, 64]");
  const int table = (prec == CS_FP64 || prec == CS_FP64_EMU) ? 0 : 1;
  if (n == 0) {
    if (info) *info = cs_info{0.0, force_m == -1 ? 4 : force_m, force_s == -1 ? 0 : force_s, 0, table, 0.0};
    return CS_OK;
  }
  if (!A || !C || !S) return fail(CS_EINVAL, "null matrix pointer");
  const size_t bytes = (size_t)n * (size_t)n * elem_size(prec);
  if (overlaps(A, bytes, C, bytes) || overlaps(A, bytes, S, bytes) || overlaps(C, bytes, S, bytes))
    return fail(CS_EINVAL, "A, C and S must not overlap");
  const Layout L = make_layout(n, prec);
  if (!ws || ws_bytes < L.total) return fail(CS_EINVAL, "workspace missing or too small");
  if (((uintptr_t)ws & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
  char* w = (char*)ws;
  // a single small FP64 matrix: one cooperative launch, (2m, s) chosen on the device
  if (small_f64_eligible(prec, n))
    return small_f64((const double*)A, n, (double*)C, (double*)S, w, L, force_m, force_s, info, stream, scale);
  double* nrm_dev = (double*)(w + L.norm_out);
  if (prec == CS_FP32)
    CS_CHECK(norm1_f32((const float*)A, n, (double*)(w + L.norm_partial), nrm_dev, stream));
  else
    CS_CHECK(norm1_f64((const double*)A, n, (double*)(w + L.norm_partial), nrm_dev, stream));
  double nrm = 0.0;
  CS_CHECK(read_norm(nrm_dev, &nrm, stream));
  if (!isfinite(nrm)) return fail(CS_ENONFINITE, "||A||_1 is not finite");
  nrm *= fabs(scale);
  if (!isfinite(nrm)) return fail(CS_ENONFINITE, "||t A||_1 is not finite");
  int m, s;
  if (force_m == -1) {
    CS_CHECK(select_ms(nrm, table, &m, &s));
  } else {
    m = force_m;
    s = force_s;
  }
  const int prods = products_of(m) + 2 * s;
  if (info) *info = cs_info{nrm, m, s, prods, table, 2.0 * (double)n * (double)n * (double)n * prods};
  const PlanSpec spec = cossin_spec(m, s, scale);
  if (f64_operands(prec)) return run_plan_f64(A, n, prec, C, S, w, L, spec, stream);
  return run_tf32((const double*)A, n, prec, (double*)C, (double*)S, w, L, spec, stream);
}

cs_status cs_check_args(int64_t n, double t, cs_prec prec, int32_t force_f, int32_t force_s) {
  CS_CHECK(check_prec(prec));
  if (n < 0 || n > kMaxN) return fail(CS_EINVAL, "n out of range [0, 65536]");
  if (uses_emu(prec) && n > kOzakiMaxK) return fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if (!isfinite(t)) return fail(CS_EINVAL, "t must be finite");
  if ((force_f == -1) != (force_s == -1)) return fail(CS_EINVAL, "force_family and force_sigma must both be -1 or both set");
  if (force_f < -1 || force_f > 3) return fail(CS_EINVAL, "force_family must be in [0, 3]");
  if (force_s < -1 || force_s > kMaxS) return fail(CS_EINVAL, "force_sigma must be in [0, 64]");
  return CS_OK;
}

// c(t^2 A), s(t, A) of Sec. 2.2 (see cs_spec); info->m is the family index.
cs_status cs_impl(const void* A, int64_t n, double t, cs_prec prec, void* C, void* S, void* ws, size_t ws_bytes,
                  int32_t force_f, int32_t force_s, cs_info* info, cudaStream_t stream) {
  CS_CHECK(cs_check_args(n, t, prec, force_f, force_s));
  const int table = (prec == CS_FP64 || prec == CS_FP64_EMU) ? 0 : 1;
  if (n == 0) {
    if (info) *info = cs_info{0.0, force_f == -1 ? 0 : force_f, force_s == -1 ? 0 : force_s, 0, table, 0.0};
    return CS_OK;
  }
  if (!A || !C || !S) return fail(CS_EINVAL, "null matrix pointer");
  const size_t bytes = (size_t)n * (size_t)n * elem_size(prec);
  if (overlaps(A, bytes, C, bytes) || overlaps(A, bytes, S, bytes) || overlaps(C, bytes, S, bytes))
    return fail(CS_EINVAL, "A, C and S must not overlap");
  const Layout L = make_layout(n, prec);
  if (!ws || ws_bytes < L.total) return fail(CS_EINVAL, "workspace missing or too small");
  if (((uintptr_t)ws & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
  char* w = (char*)ws;
  double* nrm_dev = (double*)(w + L.norm_out);
  if (prec == CS_FP32)
    CS_CHECK(norm1_f32((const float*)A, n, (double*)(w + L.norm_partial), nrm_dev, stream));
  else
    CS_CHECK(norm1_f64((const double*)A, n, (double*)(w + L.norm_partial), nrm_dev, stream));
  double nrm = 0.0;
  CS_CHECK(read_norm(nrm_dev, &nrm, stream));
  const double normB = t * t * nrm;
  if (!isfinite(normB)) return fail(CS_ENONFINITE, "||t^2 A||_1 is not finite");
  int f, sg;
  if (force_f == -1) {
    const int rc = select_cs_family(normB, table, &f, &sg);
    if (rc == 3) return fail(CS_ENONFINITE, "||t^2 A||_1 is not finite");
    if (rc == 4) return fail(CS_ERANGE, "||t^2 A||_1 needs more than 64 double-angle steps");
  } else {
    f = force_f;
    sg = force_s;
  }
  const int prods = cs_family_products(f) + 2 * sg;
  if (info) *info = cs_info{normB, f, sg, prods, table, 2.0 * (double)n * (double)n * (double)n * prods};
  const PlanSpec spec = cs_spec(f, sg, t);
  if (f64_operands(prec)) return run_plan_f64(A, n, prec, C, S, w, L, spec, stream);
  return run_tf32((const double*)A, n, prec, (double*)C, (double*)S, w, L, spec, stream);
}

}  // namespace cs

// ====================================================================== ABI ===
extern "C" {

cs_status cossin_workspace_size(int64_t n, cs_prec prec, size_t* bytes) {
  if (!bytes) return cs::fail(CS_EINVAL, "bytes is null");
  CS_CHECK(cs::check_prec(prec));
  if (n < 0 || n > cs::kMaxN) return cs::fail(CS_EINVAL, "n out of range [0, 65536]");
  if (cs::uses_emu(prec) && n > cs::kOzakiMaxK) return cs::fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  *bytes = cs::make_layout(n, prec).total;
  return CS_OK;
}

cs_status cossin_norm1(const void* A, int64_t n, cs_prec prec, double* norm1, cossin_stream_t stream) {
  CS_CHECK(cs::check_prec(prec));
  if (!norm1) return cs::fail(CS_EINVAL, "norm1 is null");
  if (n < 0 || n > cs::kMaxN) return cs::fail(CS_EINVAL, "n out of range [0, 65536]");
  if (cs::uses_emu(prec) && n > cs::kOzakiMaxK) return cs::fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if (n == 0) {
    *norm1 = 0.0;
    return CS_OK;
  }
  if (!A) return cs::fail(CS_EINVAL, "null matrix pointer");
  const size_t part = sizeof(double) * ((size_t)cs::norm1_scratch_elems(n) + 1);
  void* buf = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(cs::dev_alloc(&buf, part, st, "cossin_norm1 scratch"));
  double* out = (double*)buf;
  double* partial = out + 1;
  cs_status rc = prec == CS_FP32 ? cs::norm1_f32((const float*)A, n, partial, out, st)
                                 : cs::norm1_f64((const double*)A, n, partial, out, st);
  if (rc == CS_OK) rc = cs::read_norm(out, norm1, st);
  cudaFreeAsync(buf, st);
  return rc;
}

cs_status cossin_select(double norm1, int32_t table, int32_t* m, int32_t* s) {
  if (!m || !s) return cs::fail(CS_EINVAL, "null output pointer");
  int mm, ss;
  CS_CHECK(cs::select_ms(norm1, table, &mm, &ss));
  *m = mm;
  *s = ss;
  return CS_OK;
}

cs_status cossin_ex(const void* A, int64_t n, cs_prec prec, void* C, void* S, void* ws, size_t ws_bytes,
                    int32_t force_m, int32_t force_s, cs_info* info, cossin_stream_t stream) {
  return cs::cossin_impl(A, n, prec, C, S, ws, ws_bytes, force_m, force_s, info, (cudaStream_t)stream, 1.0);
}

cs_status cossin(const void* A, int64_t n, cs_prec prec, void* C, void* S, cossin_stream_t stream) {
  CS_CHECK(cs::check_prec(prec));
  if (n < 0 || n > cs::kMaxN) return cs::fail(CS_EINVAL, "n out of range [0, 65536]");
  if (cs::uses_emu(prec) && n > cs::kOzakiMaxK) return cs::fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if (n == 0) return CS_OK;
  size_t bytes = cs::make_layout(n, prec).total;
  void* ws = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  CS_CHECK(cs::dev_alloc(&ws, bytes, st, "cossin workspace"));
  cs_status rc = cs::cossin_impl(A, n, prec, C, S, ws, bytes, -1, -1, nullptr, st, 1.0);
  cudaFreeAsync(ws, st);
  return rc;
}

cs_status cossin_matmul(const void* X, const void* Y, int64_t n, cs_prec prec, void* P, cossin_stream_t stream) {
  CS_CHECK(cs::check_prec(prec));
  if (n < 0 || n > cs::kMaxN) return cs::fail(CS_EINVAL, "n out of range [0, 65536]");
  if (cs::uses_emu(prec) && n > cs::kOzakiMaxK) return cs::fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if (n == 0) return CS_OK;
  if (!X || !Y || !P) return cs::fail(CS_EINVAL, "null matrix pointer");
  const size_t bytes = (size_t)n * (size_t)n * cs::elem_size(prec);
  if (cs::overlaps(P, bytes, X, bytes) || cs::overlaps(P, bytes, Y, bytes))
    return cs::fail(CS_EINVAL, "P must not overlap X or Y");
  cudaStream_t st = (cudaStream_t)stream;
  if (!cs::f64_operands(prec)) return cs::matmul_tf32(X, Y, n, true, P, st);
  cs::Epilogue<double> e;
  e.n_out = 1;
  e.alpha[0] = 1.0;
  if (prec == CS_FP64) {
    e.out[0] = (double*)P;
    const size_t split = cs::gemm_f64_split_bytes(n, n, n);
    void* sw = nullptr;
    if (split) CS_CHECK(cs::dev_alloc(&sw, split, st, "cossin_matmul split scratch"));
    const cs_status rc =
        cs::gemm_f64((const double*)X, (const double*)Y, n, n, n, n, n, false, false, e, n, 1, 0, 0, 0, st, sw, split);
    if (sw) cudaFreeAsync(sw, st);
    return rc;
  }
  // Emulated products; CS_FP32 takes FP32 operands to FP64 and rounds the
  // product to FP32 once.
  const bool f32 = prec == CS_FP32;
  const size_t n2 = (size_t)n * (size_t)n;
  cs::F64Product prod;
  prod.slices = (prec == CS_SPLIT_BF16 || f32) ? cs::kOzakiSlicesSplit : cs::kOzakiSlices;
  prod.emu_bytes = cs::ozaki_dims(n, n, n, 1, prod.slices).total;
  prod.err = cs::tc_error_word();
  if (!prod.err) return cs::fail(CS_ECUDA, "cannot resolve the device error word");
  const size_t conv = f32 ? (3 * sizeof(double) * n2 + 255) & ~(size_t)255 : 0;
  char* buf = nullptr;
  CS_CHECK(cs::dev_alloc((void**)&buf, conv + prod.emu_bytes, st, "cossin_matmul scratch"));
  prod.emu_work = buf + conv;
  const double* X64 = (const double*)X;
  const double* Y64 = (const double*)Y;
  e.out[0] = (double*)P;
  cs_status rc = CS_OK;
  if (f32) {
    double* x = (double*)buf;
    X64 = x;
    Y64 = x + n2;
    e.out[0] = x + 2 * n2;
    rc = cs::convert_f32_f64((const float*)X, x, (int64_t)n2, st);
    if (rc == CS_OK) rc = cs::convert_f32_f64((const float*)Y, x + n2, (int64_t)n2, st);
  }
  if (rc == CS_OK) rc = prod(X64, Y64, n, n, n, e, st);
  if (rc == CS_OK && f32) rc = cs::convert_f64_f32(e.out[0], (float*)P, (int64_t)n2, st);
  cudaFreeAsync(buf, st);
  return rc;
}

cs_status cossin_cs(const void* A, int64_t n, double t, cs_prec prec, void* C, void* S, void* ws, size_t ws_bytes,
                    int32_t force_family, int32_t force_sigma, cs_info* info, cossin_stream_t stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (ws) return cs::cs_impl(A, n, t, prec, C, S, ws, ws_bytes, force_family, force_sigma, info, st);
  CS_CHECK(cs::cs_check_args(n, t, prec, force_family, force_sigma));
  if (n == 0) return cs::cs_impl(A, n, t, prec, C, S, nullptr, 0, force_family, force_sigma, info, st);
  const size_t bytes = cs::make_layout(n, prec).total;
  void* buf = nullptr;
  CS_CHECK(cs::dev_alloc(&buf, bytes, st, "cossin_cs workspace"));
  cs_status rc = cs::cs_impl(A, n, t, prec, C, S, buf, bytes, force_family, force_sigma, info, st);
  cudaFreeAsync(buf, st);
  return rc;
}

cs_status cossin_cs_select(double normB, int32_t table, int32_t* family, int32_t* sigma) {
  if (table < 0 || table > 1) return cs::fail(CS_EINVAL, "cs_select: table must be 0 (double) or 1 (single)");
  if (!family || !sigma) return cs::fail(CS_EINVAL, "cs_select: null output pointer");
  if (normB < 0) return cs::fail(CS_EINVAL, "cs_select: negative norm");
  int f = 0, sg = 0;
  const int rc = cs::select_cs_family(normB, table, &f, &sg);
  if (rc == 3) return cs::fail(CS_ENONFINITE, "cs_select: ||t^2 A||_1 is not finite");
  if (rc == 4) return cs::fail(CS_ERANGE, "cs_select: more than 64 double-angle steps needed");
  *family = f;
  *sigma = sg;
  return CS_OK;
}

void cossin_selftest_fail_next_alloc(int32_t count) { cs::g_fail_allocs.store(count > 0 ? count : 0); }

cs_status cossin_selftest_wait_timeout(cossin_stream_t stream) {
  // about 1 ms at 2 GHz: the kernel gives up, raises the error word, returns
  return cs::wait_selftest(2000000LL, (cudaStream_t)stream);
}

const char* cossin_last_error(void) { return cs::g_last_error.c_str(); }

cs_status cossin_device_status(cossin_stream_t stream) {
  return cs::read_norm(nullptr, nullptr, (cudaStream_t)stream);
}

void cossin_prof_enable(int32_t on) {
  std::lock_guard<std::mutex> lk(cs::g_prof_mu);
  cs::g_prof_on = on != 0;
}

void cossin_prof_reset(void) {
  cs::prof_drain();
  std::lock_guard<std::mutex> lk(cs::g_prof_mu);
  for (int k = 0; k < CS_KERNEL_KINDS; ++k) {
    cs::g_prof_ms[k] = 0;
    cs::g_prof_n[k] = 0;
    cs::g_prof_work[k] = 0;
  }
}

cs_status cossin_prof_read(int32_t kind, double* ms, int64_t* launches, double* work) {
  if (kind < 0 || kind >= CS_KERNEL_KINDS) return cs::fail(CS_EINVAL, "unknown kernel kind");
  cs::prof_drain();
  std::lock_guard<std::mutex> lk(cs::g_prof_mu);
  if (ms) *ms = cs::g_prof_ms[kind];
  if (launches) *launches = cs::g_prof_n[kind];
  if (work) *work = cs::g_prof_work[kind];
  return CS_OK;
}

}  // extern "C"
