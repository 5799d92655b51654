// adjoint.cu -- reverse mode of the approximant at fixed (2m, s), FP64.
//
// The computed cos and sin are polynomials r_c(A), r_s(A) evaluated by the
// product plans of the factorised schemes (Sec. 2.1) and the double-angle
// steps (Sec. 1).  For a loss <G_C, r_c(A)> + <G_S, r_s(A)> the gradient is
// obtained by running the plans backwards:
//   * the forward pass is re-run in write-once form, keeping every operand of
//     every product (the tape; the s double-angle levels C_j, S_j included);
//   * each step's epilogue is linear, so its adjoint needs only the
//     coefficients: an elementwise kernel turns the adjoints of the step's
//     outputs into P^ (adjoint of the product) and adds into the adjoints of
//     the step's inputs;
//   * each product P = X Y adds P^ Y^T into X^ and X^T P^ into Y^
//     (FP64 products with transposed operands and accumulating epilogues);
//   * a double-angle step C' = 2 C C - I, S' = 2 S C adds
//     2 (C'^ C^T + C^T C'^) + 2 S^T S'^ into C^ and 2 S'^ C^T into S^.
// Matrices that share (2m, s) are gathered and processed as one batch.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "internal.cuh"
#include "ozaki.h"
#include "plan.h"
#include "tc_gemm.h"
#include "theta_table.cuh"

namespace cs {
namespace {

struct AdjStep {
  int32_t nout = 0, nin = 0;
  const double* adj_out[EPI_MAX_OUT] = {};  // null: that output's adjoint is zero
  double* adj_in[EPI_MAX_IN] = {};
  double* phat = nullptr;
  double alpha[EPI_MAX_OUT] = {};
  double beta[EPI_MAX_OUT][EPI_MAX_IN] = {};
  double delta[EPI_MAX_OUT][EPI_MAX_OUT] = {};
};

// Elementwise adjoint of one epilogue over `total` elements (all arrays share
// one layout).  Outputs are visited last to first so that adjoints reaching an
// output through a later output's delta term are complete when it is used.
__global__ void __launch_bounds__(256) epilogue_adjoint(const AdjStep a, int64_t total) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    double tot[EPI_MAX_OUT];
    double ph = 0.0;
#pragma unroll
    for (int t = EPI_MAX_OUT - 1; t >= 0; --t) {
      if (t >= a.nout) continue;
      double v = a.adj_out[t] ? a.adj_out[t][i] : 0.0;
#pragma unroll
      for (int u = EPI_MAX_OUT - 1; u > 0; --u)
        if (u > t && u < a.nout) v += a.delta[u][t] * tot[u];
      tot[t] = v;
      ph += a.alpha[t] * v;
    }
    a.phat[i] = ph;
#pragma unroll
    for (int q = 0; q < EPI_MAX_IN; ++q) {
      if (q >= a.nin) break;
      double g = 0.0;
#pragma unroll
      for (int t = 0; t < EPI_MAX_OUT; ++t)
        if (t < a.nout) g += a.beta[t][q] * tot[t];
      a.adj_in[q][i] += g;
    }
  }
}

__global__ void gather_kernel(const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ idx,
                              int64_t n2, int64_t count) {
  const int64_t total = n2 * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / n2, r = e - b * n2;
    dst[e] = src[(int64_t)idx[b] * n2 + r];
  }
}

__global__ void scatter_kernel(const double* __restrict__ src, double* __restrict__ dst, const int* __restrict__ idx,
                               int64_t n2, int64_t count) {
  const int64_t total = n2 * count;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / n2, r = e - b * n2;
    dst[(int64_t)idx[b] * n2 + r] = src[e];
  }
}

int blocks_for(int64_t total) { return (int)std::min<int64_t>((total + 255) / 256, 152 * 8); }

// The batched FP64 products of the forward and reverse passes: native, or
// emulated on the BF16 tensor cores (gemm_f64_emu_batched, which takes its
// operands untransposed: a transposed operand is materialised first).
struct AdjProd {
  bool emu = false;
  void* work = nullptr;
  size_t work_bytes = 0;
  double* tbuf[2] = {};
  int* err = nullptr;
  cs_status operator()(const double* X, bool tX, const double* Y, bool tY, const Epilogue<double>& e, int64_t n,
                       int64_t g, cudaStream_t st) const {
    const int64_t n2 = n * n;
    if (!emu) return gemm_f64(X, Y, n, n, n, n, n, tX, tY, e, n, g, n2, n2, n2, st);
    if (tX) {
      CS_CHECK(transpose_f64_batched(X, tbuf[0], n, g, n2, st));
      X = tbuf[0];
    }
    if (tY) {
      CS_CHECK(transpose_f64_batched(Y, tbuf[1], n, g, n2, st));
      Y = tbuf[1];
    }
    return gemm_f64_emu_batched(X, Y, n, n, n, n, n, e, n, g, n2, n2, n2, work, work_bytes, err, st);
  }
};

// Write-once form of a plan: value ids for every step output.
struct SsaStep {
  int X, Y;                 // value ids of the operands
  std::vector<int> out;     // value id per output
  std::vector<int> in;      // value ids of the distinct epilogue inputs
  Epilogue<double> coef;    // alpha, gamma, beta (indexed by `in`), delta
};

struct Ssa {
  int nvalues = 0;
  int A = 0, C = -1, S = -1;
  std::vector<SsaStep> steps;
};

Ssa make_ssa(int m, int s, double scale) {
  Ssa g;
  int cur[SL_COUNT];
  for (int k = 0; k < SL_COUNT; ++k) cur[k] = -1;
  g.A = g.nvalues++;
  cur[SL_A] = g.A;
  for (const Step& st : chain_plan(m, s, scale)) {
    SsaStep q;
    q.X = cur[st.X];
    q.Y = cur[st.Y];
    for (size_t t = 0; t < st.outs.size(); ++t) {
      const OutSpec& o = st.outs[t];
      q.coef.alpha[t] = o.alpha;
      q.coef.gamma[t] = o.gamma;
      for (auto& b : o.beta) {
        const int v = cur[b.first];
        int qi = -1;
        for (size_t k = 0; k < q.in.size(); ++k)
          if (q.in[k] == v) qi = (int)k;
        if (qi < 0) {
          qi = (int)q.in.size();
          q.in.push_back(v);
        }
        q.coef.beta[t][qi] = b.second;
      }
      for (auto& d : o.delta) q.coef.delta[t][d.first] = d.second;
    }
    for (size_t t = 0; t < st.outs.size(); ++t) q.out.push_back(g.nvalues++);
    for (size_t t = 0; t < st.outs.size(); ++t) cur[st.outs[t].slot] = q.out[t];
    q.coef.n_out = (int)st.outs.size();
    q.coef.n_in = (int)q.in.size();
    g.steps.push_back(q);
  }
  g.C = cur[SL_C];
  g.S = cur[SL_S];
  return g;
}

// Device memory of one backward call: bump allocation from the caller's
// workspace (mark / release per (2m, s) group), or stream-ordered
// allocations of the library's own when no workspace is given.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  cudaStream_t st = nullptr;
  std::vector<void*> owned;
  cs_status get(void** p, size_t bytes, const char* what) {
    if (!base) {
      CS_CHECK(dev_alloc(p, bytes, st, what));
      owned.push_back(*p);
      return CS_OK;
    }
    const size_t off = (used + 255) & ~(size_t)255;
    if (off + bytes > cap) return fail(CS_EINVAL, std::string("backward workspace too small at ") + what);
    *p = base + off;
    used = off + bytes;
    return CS_OK;
  }
  // frees (or returns to the bump pointer) everything taken after `mark`
  void release(size_t mark, size_t nowned) {
    while (owned.size() > nowned) {
      cudaFreeAsync(owned.back(), st);
      owned.pop_back();
    }
    used = mark;
  }
};

// Accumulating product: Acc += op(X) op(Y), batched with stride n^2.
cs_status gemm_acc(const AdjProd& prod, const double* X, bool tX, const double* Y, bool tY, double* Acc,
                   double scale, int64_t n, int64_t batch, cudaStream_t stream) {
  Epilogue<double> e;
  e.n_in = 1;
  e.in[0] = Acc;
  e.n_out = 1;
  e.out[0] = Acc;
  e.alpha[0] = scale;
  e.beta[0][0] = 1.0;
  return prod(X, tX, Y, tY, e, n, batch, stream);
}

// Values one group's forward tape keeps per matrix (chain values and the
// double-angle levels), which sizes its buffer.
int tape_values(int m, int s) { return make_ssa(m, s, 1.0).nvalues + 2 * s; }

cs_status run_group(const double* A, const double* GC, const double* GS, double* dA, double* C_out, double* S_out,
                    int64_t n, int m, int s, int64_t g, double scale, const AdjProd& prod, Arena& arena,
                    cudaStream_t stream) {
  const Ssa ssa = make_ssa(m, s, scale);
  const int64_t n2 = n * n;
  const int nlev = s + 1;
  // values: chain values, then the double-angle levels C_1..C_s, S_1..S_s
  const int nval = ssa.nvalues + 2 * s;
  auto levC = [&](int j) { return j == 0 ? ssa.C : ssa.nvalues + (j - 1); };
  auto levS = [&](int j) { return j == 0 ? ssa.S : ssa.nvalues + s + (j - 1); };
  (void)nlev;
  const size_t per = sizeof(double) * (size_t)n2 * (size_t)g;
  const size_t total = per * (size_t)(2 * nval + 1);
  char* buf = nullptr;
  const size_t mark = arena.used, nowned = arena.owned.size();
  CS_CHECK(arena.get((void**)&buf, total, "the adjoint's tape"));
  auto val = [&](int v) { return (double*)(buf + per * (size_t)v); };
  auto adj = [&](int v) { return (double*)(buf + per * (size_t)(nval + v)); };
  double* phat = (double*)(buf + per * (size_t)(2 * nval));
  cs_status rc = CS_OK;
  cudaError_t ce = cudaMemsetAsync(buf + per * (size_t)nval, 0, per * (size_t)nval, stream);
  if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemsetAsync");
  if (rc == CS_OK) ce = cudaMemcpyAsync(val(ssa.A), A, per, cudaMemcpyDeviceToDevice, stream);
  if (rc == CS_OK && ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemcpyAsync");
  // ---- forward, write-once
  for (size_t i = 0; rc == CS_OK && i < ssa.steps.size(); ++i) {
    const SsaStep& q = ssa.steps[i];
    Epilogue<double> e = q.coef;
    for (int k = 0; k < e.n_in; ++k) e.in[k] = val(q.in[k]);
    for (int t = 0; t < e.n_out; ++t) e.out[t] = val(q.out[t]);
    rc = prod(val(q.X), false, val(q.Y), false, e, n, g, stream);
  }
  for (int j = 0; rc == CS_OK && j < s; ++j) {
    Epilogue<double> ec;
    ec.n_out = 1;
    ec.out[0] = val(levC(j + 1));
    ec.alpha[0] = 2.0;
    ec.gamma[0] = -1.0;
    rc = prod(val(levC(j)), false, val(levC(j)), false, ec, n, g, stream);
    if (rc != CS_OK) break;
    Epilogue<double> es;
    es.n_out = 1;
    es.out[0] = val(levS(j + 1));
    es.alpha[0] = 2.0;
    rc = prod(val(levS(j)), false, val(levC(j)), false, es, n, g, stream);
  }
  if (rc == CS_OK && C_out) ce = cudaMemcpyAsync(C_out, val(levC(s)), per, cudaMemcpyDeviceToDevice, stream);
  if (rc == CS_OK && S_out && ce == cudaSuccess) ce = cudaMemcpyAsync(S_out, val(levS(s)), per, cudaMemcpyDeviceToDevice, stream);
  if (rc == CS_OK && ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemcpyAsync");
  // ---- reverse
  if (rc == CS_OK) ce = cudaMemcpyAsync(adj(levC(s)), GC, per, cudaMemcpyDeviceToDevice, stream);
  if (rc == CS_OK && ce == cudaSuccess) ce = cudaMemcpyAsync(adj(levS(s)), GS, per, cudaMemcpyDeviceToDevice, stream);
  if (rc == CS_OK && ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemcpyAsync");
  for (int j = s - 1; rc == CS_OK && j >= 0; --j) {
    const double* C = val(levC(j));
    const double* S = val(levS(j));
    const double* Ch = adj(levC(j + 1));
    const double* Sh = adj(levS(j + 1));
    double* Cj = adj(levC(j));
    double* Sj = adj(levS(j));
    rc = gemm_acc(prod, Ch, false, C, true, Cj, 2.0, n, g, stream);                  // 2 C'^ C^T
    if (rc == CS_OK) rc = gemm_acc(prod, C, true, Ch, false, Cj, 2.0, n, g, stream);  // 2 C^T C'^
    if (rc == CS_OK) rc = gemm_acc(prod, S, true, Sh, false, Cj, 2.0, n, g, stream);  // 2 S^T S'^
    if (rc == CS_OK) rc = gemm_acc(prod, Sh, false, C, true, Sj, 2.0, n, g, stream);  // 2 S'^ C^T
  }
  for (int i = (int)ssa.steps.size() - 1; rc == CS_OK && i >= 0; --i) {
    const SsaStep& q = ssa.steps[i];
    AdjStep a;
    a.nout = q.coef.n_out;
    a.nin = q.coef.n_in;
    for (int t = 0; t < a.nout; ++t) {
      a.adj_out[t] = adj(q.out[t]);
      a.alpha[t] = q.coef.alpha[t];
      for (int k = 0; k < a.nin; ++k) a.beta[t][k] = q.coef.beta[t][k];
      for (int u = 0; u < a.nout; ++u) a.delta[t][u] = q.coef.delta[t][u];
    }
    for (int k = 0; k < a.nin; ++k) a.adj_in[k] = adj(q.in[k]);
    a.phat = phat;
    const int64_t tot = n2 * g;
    epilogue_adjoint<<<blocks_for(tot), 256, 0, stream>>>(a, tot);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      rc = cuda_fail(ce, "epilogue_adjoint");
      break;
    }
    rc = gemm_acc(prod, phat, false, val(q.Y), true, adj(q.X), 1.0, n, g, stream);            // X^ += P^ Y^T
    if (rc == CS_OK) rc = gemm_acc(prod, val(q.X), true, phat, false, adj(q.Y), 1.0, n, g, stream);  // Y^ += X^T P^
  }
  if (rc == CS_OK) ce = cudaMemcpyAsync(dA, adj(ssa.A), per, cudaMemcpyDeviceToDevice, stream);
  if (rc == CS_OK && ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemcpyAsync");
  arena.release(mark, nowned);
  return rc;
}

}  // namespace

int64_t adjoint_products(int m, int s) { return 3 * products_of(m) + 6 * s; }

namespace {
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device bytes of one (2m, s) group of g matrices of order n: gathered
// inputs and outputs (6 n^2 g doubles and the index list), the emulated
// products' scratch and transposes, and the tape.
size_t group_bytes(int64_t n, int64_t g, int m, int s, bool emu) {
  const size_t per = sizeof(double) * (size_t)n * (size_t)n * (size_t)g;
  size_t b = al256(6 * per + sizeof(int) * (size_t)g);
  if (emu) b += al256(ozaki_dims(n, n, n, g).total + 2 * per);
  b += al256(per * (size_t)(2 * tape_values(m, s) + 1));
  return b;
}
}  // namespace

size_t backward_workspace_bytes(int64_t count, int64_t n, int max_s, bool emu) {
  int worst_m = 4;
  for (int m : {4, 8, 9, 16, 24})
    if (tape_values(m, max_s) > tape_values(worst_m, max_s)) worst_m = m;
  return al256(sizeof(double) * (size_t)count) + group_bytes(n, count, worst_m, max_s, emu);
}

// Gradient of <G_C, r_c(scale A)> + <G_S, r_s(scale A)> with respect to A; the
// scale sits in the plans' coefficients, so the reverse pass carries it.
cs_status backward_impl(int64_t count, int64_t n, double scale, const double* A, const double* G_C,
                        const double* G_S, double* dA, double* C, double* S, int32_t force_m, int32_t force_s,
                        cs_info* infos_host, cudaStream_t st, bool emu, void* ws, size_t ws_bytes) {
  if (count < 0 || n < 0 || n > kMaxN) return fail(CS_EINVAL, "count or n out of range");
  if (n > 0 && count > (int64_t(1) << 46) / (n * n)) return fail(CS_EINVAL, "count * n^2 above 2^46 elements");
  if (emu && n > kOzakiMaxK) return fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if (!isfinite(scale)) return fail(CS_EINVAL, "t must be finite");
  if ((force_m == -1) != (force_s == -1)) return fail(CS_EINVAL, "force_m and force_s must both be -1 or both set");
  if (force_m != -1 && products_of(force_m) < 0) return fail(CS_EINVAL, "force_m must be 4, 8, 9, 16 or 24");
  if (force_s < -1 || force_s > kMaxS) return fail(CS_EINVAL, "force_s must be in [0, 64]");
  if (count == 0 || n == 0) return CS_OK;
  if (!A || !G_C || !G_S || !dA) return fail(CS_EINVAL, "null matrix pointer");
  const int64_t n2 = n * n;
  const size_t bytes = sizeof(double) * (size_t)n2 * (size_t)count;
  auto ov = [&](const void* a, const void* b) {
    return a && b && (const char*)a < (const char*)b + bytes && (const char*)b < (const char*)a + bytes;
  };
  if (ov(dA, A) || ov(dA, G_C) || ov(dA, G_S) || ov(C, A) || ov(S, A) || ov(C, S) || ov(C, dA) || ov(S, dA))
    return fail(CS_EINVAL, "outputs must not overlap inputs or each other");
  Arena arena;
  arena.st = st;
  if (ws) {
    if (((uintptr_t)ws & 255) != 0) return fail(CS_EINVAL, "workspace must be 256-byte aligned");
    const size_t allw = (size_t)n * (size_t)n * (size_t)count * sizeof(double);
    if (overlaps(ws, ws_bytes, A, allw) || overlaps(ws, ws_bytes, G_C, allw) || overlaps(ws, ws_bytes, G_S, allw) ||
        overlaps(ws, ws_bytes, dA, allw) || (C && overlaps(ws, ws_bytes, C, allw)) ||
        (S && overlaps(ws, ws_bytes, S, allw)))
      return fail(CS_EINVAL, "workspace must not overlap the matrices");
    arena.base = (char*)ws;
    arena.cap = ws_bytes;
  }
  // norms of every matrix, one synchronisation
  std::vector<double> norms((size_t)count);
  {
    double* outs = nullptr;
    CS_CHECK(arena.get((void**)&outs, sizeof(double) * count, "the norms"));
    cs_status rc = norm1_batched_f64(A, n, count, outs, st);
    cudaError_t ce = rc == CS_OK ? cudaMemcpyAsync(norms.data(), outs, sizeof(double) * count, cudaMemcpyDeviceToHost, st)
                                 : cudaSuccess;
    cudaError_t ce2 = cudaStreamSynchronize(st);
    arena.release(0, 0);
    if (rc != CS_OK) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaMemcpyAsync");
    if (ce2 != cudaSuccess) return cuda_fail(ce2, "cudaStreamSynchronize");
  }
  // with the norms out of the way the groups take the whole workspace
  arena.used = 0;
  for (double& v : norms) v *= fabs(scale);
  std::map<std::pair<int, int>, std::vector<int>> groups;
  for (int64_t b = 0; b < count; ++b) {
    int m, s;
    if (force_m == -1) {
      CS_CHECK(select_ms(norms[b], 0, &m, &s));
    } else {
      if (!isfinite(norms[b])) return fail(CS_ENONFINITE, "||A||_1 is not finite");
      m = force_m;
      s = force_s;
    }
    groups[{m, s}].push_back((int)b);
    if (infos_host) {
      const int prods = (int)adjoint_products(m, s);
      infos_host[b] = cs_info{norms[b], m, s, prods, 0, 2.0 * (double)n * n * n * prods};
    }
  }
  if (ws) {
    size_t need = 0;
    for (auto& kv : groups)
      need = std::max(need, group_bytes(n, (int64_t)kv.second.size(), kv.first.first, kv.first.second, emu));
    if (need > ws_bytes)
      return fail(CS_EINVAL, "backward workspace too small: the selected (2m, s) need " + std::to_string(need) +
                                 " bytes (cossin_backward_workspace_size with the largest s)");
  }
  for (auto& kv : groups) {
    const int m = kv.first.first, s = kv.first.second;
    const std::vector<int>& idx = kv.second;
    const int64_t g = (int64_t)idx.size();
    const size_t per = sizeof(double) * (size_t)n2 * (size_t)g;
    const bool need_c = C != nullptr, need_s = S != nullptr;
    char* gb = nullptr;
    const size_t mark = arena.used, nowned = arena.owned.size();
    CS_CHECK(arena.get((void**)&gb, 6 * per + sizeof(int) * g, "the gathered matrices"));
    double* gA = (double*)gb;
    double* gGC = (double*)(gb + per);
    double* gGS = (double*)(gb + 2 * per);
    double* gdA = (double*)(gb + 3 * per);
    double* gC = (double*)(gb + 4 * per);
    double* gS = (double*)(gb + 5 * per);
    int* didx = (int*)(gb + 6 * per);
    cs_status rc = CS_OK;
    cudaError_t ce = cudaMemcpyAsync(didx, idx.data(), sizeof(int) * g, cudaMemcpyHostToDevice, st);
    if (ce != cudaSuccess) rc = cuda_fail(ce, "cudaMemcpyAsync");
    const int nb = blocks_for(n2 * g);
    if (rc == CS_OK) {
      gather_kernel<<<nb, 256, 0, st>>>(A, gA, didx, n2, g);
      gather_kernel<<<nb, 256, 0, st>>>(G_C, gGC, didx, n2, g);
      gather_kernel<<<nb, 256, 0, st>>>(G_S, gGS, didx, n2, g);
      ce = cudaGetLastError();
      if (ce != cudaSuccess) rc = cuda_fail(ce, "gather");
    }
    AdjProd prod;
    char* eb = nullptr;
    if (rc == CS_OK && emu) {
      prod.emu = true;
      prod.err = tc_error_word();
      prod.work_bytes = ozaki_dims(n, n, n, g).total;
      const size_t tb = sizeof(double) * (size_t)n2 * (size_t)g;
      rc = arena.get((void**)&eb, prod.work_bytes + 2 * tb, "the emulated products' scratch");
      if (rc == CS_OK && !prod.err) rc = fail(CS_ECUDA, "cannot resolve the device error word");
      if (rc == CS_OK) {
        prod.work = eb;
        prod.tbuf[0] = (double*)(eb + prod.work_bytes);
        prod.tbuf[1] = (double*)(eb + prod.work_bytes + tb);
      }
    }
    if (rc == CS_OK)
      rc = run_group(gA, gGC, gGS, gdA, need_c ? gC : nullptr, need_s ? gS : nullptr, n, m, s, g, scale, prod, arena,
                     st);
    if (rc == CS_OK) {
      scatter_kernel<<<nb, 256, 0, st>>>(gdA, dA, didx, n2, g);
      if (need_c) scatter_kernel<<<nb, 256, 0, st>>>(gC, C, didx, n2, g);
      if (need_s) scatter_kernel<<<nb, 256, 0, st>>>(gS, S, didx, n2, g);
      ce = cudaGetLastError();
      if (ce != cudaSuccess) rc = cuda_fail(ce, "scatter");
    }
    // the host index vector must outlive its copy
    cudaError_t ce2 = cudaStreamSynchronize(st);
    arena.release(mark, nowned);
    if (rc != CS_OK) return rc;
    if (ce2 != cudaSuccess) return cuda_fail(ce2, "cudaStreamSynchronize");
  }
  return CS_OK;
}

}  // namespace cs

extern "C" cs_status cossin_backward(int64_t count, int64_t n, const double* A, const double* G_C,
                                     const double* G_S, double* dA, double* C, double* S, int32_t force_m,
                                     int32_t force_s, cs_info* infos_host, cossin_stream_t stream) {
  return cs::backward_impl(count, n, 1.0, A, G_C, G_S, dA, C, S, force_m, force_s, infos_host,
                           (cudaStream_t)stream, false, nullptr, 0);
}

extern "C" cs_status cossin_backward_ex(int64_t count, int64_t n, const double* A, const double* G_C,
                                        const double* G_S, double* dA, double* C, double* S, int32_t force_m,
                                        int32_t force_s, cs_prec prec, cs_info* infos_host, cossin_stream_t stream) {
  if (prec != CS_FP64 && prec != CS_FP64_EMU) return cs::fail(CS_EINVAL, "the adjoint runs in CS_FP64 or CS_FP64_EMU");
  return cs::backward_impl(count, n, 1.0, A, G_C, G_S, dA, C, S, force_m, force_s, infos_host,
                           (cudaStream_t)stream, prec == CS_FP64_EMU, nullptr, 0);
}

extern "C" cs_status cossin_backward_workspace_size(int64_t count, int64_t n, cs_prec prec, int32_t max_s,
                                                    size_t* bytes) {
  if (!bytes) return cs::fail(CS_EINVAL, "bytes is null");
  if (prec != CS_FP64 && prec != CS_FP64_EMU) return cs::fail(CS_EINVAL, "the adjoint runs in CS_FP64 or CS_FP64_EMU");
  if (count < 0 || n < 0 || n > cs::kMaxN) return cs::fail(CS_EINVAL, "count or n out of range");
  if (n > 0 && count > (int64_t(1) << 46) / (n * n)) return cs::fail(CS_EINVAL, "count * n^2 above 2^46 elements");
  if (prec == CS_FP64_EMU && n > cs::kOzakiMaxK) return cs::fail(CS_EINVAL, "the emulated FP64 products support n <= 8192");
  if (max_s < 0 || max_s > cs::kMaxS) return cs::fail(CS_EINVAL, "max_s must be in [0, 64]");
  *bytes = (count == 0 || n == 0) ? 0 : cs::backward_workspace_bytes(count, n, max_s, prec == CS_FP64_EMU);
  return CS_OK;
}

extern "C" cs_status cossin_backward_ws(int64_t count, int64_t n, const double* A, const double* G_C,
                                        const double* G_S, double* dA, double* C, double* S, int32_t force_m,
                                        int32_t force_s, cs_prec prec, void* ws, size_t ws_bytes, cs_info* infos_host,
                                        cossin_stream_t stream) {
  if (prec != CS_FP64 && prec != CS_FP64_EMU) return cs::fail(CS_EINVAL, "the adjoint runs in CS_FP64 or CS_FP64_EMU");
  if (!ws && count > 0 && n > 0) return cs::fail(CS_EINVAL, "workspace is null");
  return cs::backward_impl(count, n, 1.0, A, G_C, G_S, dA, C, S, force_m, force_s, infos_host,
                           (cudaStream_t)stream, prec == CS_FP64_EMU, ws, ws_bytes);
}
