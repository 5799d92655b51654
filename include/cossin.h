/*
 * cossin.h -- C ABI of the GB300 (sm_103a) library that computes cos(A) and
 * sin(A) of a real dense n x n matrix together, by the method of Seydaoglu,
 * Bader, Blanes and Casas, "Computing the matrix sine and cosine
 * simultaneously with a reduced number of products" (arXiv:2010.00465).
 *
 * The method (paper section / equation in brackets):
 *   1. theta = ||A||_1, the exact matrix 1-norm            [Sec. 4]
 *   2. the family 2m in {4, 8, 16, 24} and the scaling s from the admissible
 *      norms theta_2m of Table 1 (double) or Table 2 (single) [Sec. 3]
 *   3. B = A_2 = (2^-s A)^2                                 [Sec. 1]
 *   4. the factorised Taylor schemes, cos as T^c_2m(A_s) and sin as
 *      A_s * p(A_2), with Pi_2m = 3, 4, 6, 7 products       [Sec. 2.1]
 *   5. s double-angle steps C <- 2C^2 - I, S <- 2SC         [Sec. 1]
 *
 * Conventions for every entry point:
 *   - Matrices are dense, row-major and contiguous (leading dimension n).
 *     Because f(A^T) = f(A)^T for cos and sin, a column-major caller gets
 *     column-major results from the same call.
 *   - Pointers named *_dev are device pointers owned by the caller; the
 *     library never frees them.  The library allocates device memory only
 *     where an entry point says so.
 *   - Every call is asynchronous on `stream` except where stated; results
 *     are ready once the stream is synchronised.  Argument errors are
 *     detected before any work is queued and return a status without side
 *     effects.  No C++ exception crosses this interface.
 *   - On a status other than CS_OK, cossin_last_error() returns a message
 *     for the calling thread.
 *   - n = 0 is a valid no-op.  A = 0 gives C = I, S = 0.
 */
#ifndef COSSIN_H
#define COSSIN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object as cudaStream_t / CUstream; NULL is the legacy default stream. */
typedef struct CUstream_st* cossin_stream_t;

typedef enum {
  CS_OK = 0,
  CS_EINVAL = 1,      /* bad argument: size, alias, precision, forced (m, s), workspace */
  CS_ENOMEM = 2,      /* a device allocation made by the library failed (no work was queued) */
  CS_ENONFINITE = 3,  /* ||A||_1 is Inf or NaN */
  CS_ERANGE = 4,      /* the scaling would need s > 64 */
  CS_ECUDA = 5,       /* a CUDA runtime call failed (message has the CUDA error) */
  CS_ETIMEOUT = 6     /* a bounded wait in a tensor-core kernel expired in an earlier call */
} cs_status;

typedef enum {
  /* FP64 in and out; double table (u = 2^-53); every product in FP64. */
  CS_FP64 = 0,
  /* FP32 in and out; single table (u = 2^-24).  The input is taken to FP64
   * once; every product, the Taylor chain's and the double-angle steps', is
   * a BF16 tensor-core product of four 7-bit slices per row / column (as
   * CS_SPLIT_BF16's chain products) with FP64 intermediates, and C and S are
   * rounded to FP32 once at the end (FP32-stored intermediates would let
   * the double-angle recurrence amplify their rounding past 2e-5 at
   * ||A||_1 near 64).  cossin_matmul with this prec forms the four-slice
   * product of FP32 operands.  n <= 8192 (CS_EINVAL above). */
  CS_FP32 = 1,
  /* FP64 in and out; single table; the Taylor chain (steps 3-4) as
   * four-pass TF32 tensor-core products of (hi, lo) splits of FP64
   * intermediates (the diagonal of the left operand added in FP64, the
   * linear combinations in FP64), while the norm, the choice of (m, s) and
   * the double-angle steps run in FP64. */
  CS_SPLIT_TF32 = 2,
  /* FP64 in and out; double table; every product emulated on the BF16
   * tensor cores: rows of the left and columns of the right operand cut into
   * eight 7-bit integer slices (57 bits of each row / column maximum), the
   * 36 slice products with p + q <= 7 summed exactly per level in FP32 and
   * promoted every 512 k into exact int64 fixed-point sums; the diagonal
   * entries X[r][r], Y[c][c] are added in FP64 (not part of the paper;
   * FP64-class accuracy: at most 2^-52 K max|X_i.| max|Y_.j| per entry of a
   * product in the worst case, below the FP64 product's rounding for N(0,1)
   * data at n = 4096).  n <= 8192 (CS_EINVAL above). */
  CS_FP64_EMU = 3,
  /* As CS_SPLIT_TF32, with the FP64 double-angle products emulated as in
   * CS_FP64_EMU (n <= 8192). */
  CS_SPLIT_EMU = 4,
  /* FP64 in and out; single table; every product on the BF16 tensor cores:
   * the Taylor chain (steps 3-4) as BF16 multi-term products of four 7-bit
   * slices per row / column (29 bits of each row / column maximum, the 10
   * slice products with p + q <= 3, FP32-class: at most 2^-25 K max|X_i.|
   * max|Y_.j| per entry), the double-angle steps as in CS_FP64_EMU; the
   * norm and the choice of (m, s) in FP64.  cossin_matmul with this prec
   * forms the four-slice product.  n <= 8192 (CS_EINVAL above). */
  CS_SPLIT_BF16 = 5
} cs_prec;

/* Status of the asynchronous part.  A call's status covers its arguments,
 * its workspace and its 1-norm (read on the host before the products are
 * queued); the products then run asynchronously, and a tensor-core product
 * whose bounded wait expired (see cossin_device_status) is reported by the
 * next call that reads the device error word, or by cossin_device_status
 * after the stream is synchronised. */

/* What one call did. */
typedef struct {
  double norm1;      /* ||A||_1 as computed on the device (FP64) */
  int32_t m;         /* 2m of the family used: 4, 8, 16 or 24 */
  int32_t s;         /* double-angle steps */
  int32_t products;  /* Pi_2m + 2 s matrix products */
  int32_t table;     /* 0 = double table (Table 1), 1 = single table (Table 2) */
  double flops;      /* algorithmic flops 2 n^3 (Pi_2m + 2 s) */
} cs_info;

/* Bytes of device workspace cossin_ex needs for one n x n matrix in `prec`.
 * Host-only: queues no work and creates no context; it reads the current
 * device's SM count (the FP64 and emulated products keep per-SM scratch). */
cs_status cossin_workspace_size(int64_t n, cs_prec prec, size_t* bytes);

/* Steps 1-2 only.  theta = ||A||_1 of the device matrix A_dev (FP32 for
 * CS_FP32, FP64 for every other prec), computed on the device with
 * FP64 accumulation; blocks until it is on the host.  Uses a small
 * library-owned device buffer (allocated on first use per device). */
cs_status cossin_norm1(const void* A_dev, int64_t n, cs_prec prec, double* norm1,
                       cossin_stream_t stream);

/* Step 1 for callers that cannot allocate device memory: code that runs while
 * a CUDA graph is being captured (an allocation there breaks the capture),
 * code inside a framework whose device memory must all come from the
 * framework's own pool, and latency-sensitive loops where cudaMalloc's
 * implicit synchronisation is not acceptable.  The paper has no counterpart;
 * this is the same computation as cossin_norm1, but it allocates nothing and
 * does not synchronise: theta = ||A||_1 is written to the device double
 * *norm1_dev on `stream`.
 *   - n must be <= 4096 (CS_EINVAL otherwise).  The scratch is a static
 *     device array of about 2 MB that every GPU loading the library holds
 *     until the process exits.
 *   - The first call on each device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *     The address is kept for the life of the process: after a
 *     cudaDeviceReset of that device the kept address is stale, so do not
 *     call this entry point on that device again in the same process.
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents (the words that must start at zero are cleared on
 *     `stream` by each call).  Calls that overlap on the GPU (concurrent
 *     streams, or concurrent host threads on one device) race: serialise them. */
cs_status cossin_norm1_noalloc(const void* A_dev, int64_t n, cs_prec prec, double* norm1_dev,
                               cossin_stream_t stream);

/* Step 2 on the host: the (2m, s) of minimal cost Pi_2m + 2 s over the four
 * families with ||A_s||_1 = theta / 2^s <= min(theta^c_2m, theta^s_2m)
 * (Tables 1-2; ties go to the smaller s).  table: 0 double, 1 single. */
cs_status cossin_select(double norm1, int32_t table, int32_t* m, int32_t* s);

/* cos(A) and sin(A).  A_dev, C_dev, S_dev: n x n device matrices of the
 * precision's element type (C and S must not overlap A or each other).
 * Allocates its workspace with cudaMallocAsync on `stream` and frees it on
 * the same stream; synchronises the stream once to read ||A||_1. */
cs_status cossin(const void* A_dev, int64_t n, cs_prec prec, void* C_dev, void* S_dev,
                 cossin_stream_t stream);

/* As cossin, with caller-provided workspace (ws_dev, at least
 * cossin_workspace_size bytes, 256-byte aligned) so that nothing is
 * allocated, and optional forced (m, s): force_m in {4, 8, 16, 24} together
 * with force_s in [0, 64], or both -1 for the automatic choice (with a forced
 * pair the norm is still computed and reported).  force_m = 9 selects the
 * alternative k = 4 scheme that the automatic choice never takes: the 2m = 8
 * cosine with the sine T9s of eq. Algorithm5sA (5 products, exact through
 * A^9; its sine's admissible norm, not printed in the paper, is 0.17402
 * double / 1.0813 single, so the cosine's Table 1-2 value binds the pair).
 * info may be NULL. */
cs_status cossin_ex(const void* A_dev, int64_t n, cs_prec prec, void* C_dev, void* S_dev,
                    void* ws_dev, size_t ws_bytes, int32_t force_m, int32_t force_s,
                    cs_info* info, cossin_stream_t stream);

/* The Sec. 2.2 variant: C = c(t^2 A) = cos(sqrt(t^2 A)) and
 * S = s(t, A) = A^(-1/2) sin(sqrt(t^2 A)) (each a power series in t^2 A, so
 * no square root is formed), the functions that advance u'' + A u = 0 by a
 * step t.  The schemes of Sec. 2.1 run on B = (t / 2^sigma)^2 A with the
 * first product (A^2) and the sine's last product (A times ...) removed, so
 * the four families cost 2, 3, 4 and 5 products; sigma double-angle steps
 * C <- 2C^2 - I, S <- 2SC follow.  The family and sigma minimise products +
 * 2 sigma subject to ||B||_1 <= theta_cs (the paper prints no admissible
 * norms for these schemes: the library's values come from the Sec. 3 error
 * series of the scalar polynomials in B; ties go to the smaller sigma).
 *   family 0: k = 3 with P_{3,4}^s (the minus sign printed before the
 *             (6!/7!) B_4 term is read as plus), 2 products;
 *   family 1: k = 3 with P_4^s, 3 products;
 *   family 2: k = 4 (P_8^c, P_{8,12}^s on B), 4 products;
 *   family 3: k = 5 (P_12^c, P_{11,24}^s on B), 5 products.
 * Arguments as cossin_ex (same workspace size), plus the finite step t;
 * force_family in [0, 3] with force_sigma in [0, 64], or both -1.  info->m
 * holds the family, info->s sigma and info->norm1 ||t^2 A||_1.
 * CS_ENONFINITE if t^2 ||A||_1 is not finite, CS_ERANGE if sigma would
 * exceed 64, CS_EINVAL for a non-finite t or bad arguments.  ws_dev may be
 * NULL, in which case the workspace is allocated on `stream` as in cossin. */
/* The choice cossin_cs makes, on the host: the family (0..3) and sigma of
 * minimal products + 2 sigma with ||B||_1 / 4^sigma <= theta_cs (table 0:
 * double, 1: single; ties go to the smaller sigma).  CS_ENONFINITE for a
 * non-finite norm, CS_ERANGE beyond 64 steps, CS_EINVAL for a negative norm. */
cs_status cossin_cs_select(double normB, int32_t table, int32_t* family, int32_t* sigma);

cs_status cossin_cs(const void* A_dev, int64_t n, double t, cs_prec prec, void* C_dev, void* S_dev,
                    void* ws_dev, size_t ws_bytes, int32_t force_family, int32_t force_sigma,
                    cs_info* info, cossin_stream_t stream);

/* Failure-path self test (the paper has no counterpart): launches one
 * tensor-core-style bounded wait on an mbarrier that nothing arrives at, with
 * a limit of about 1 ms.  The wait gives up and raises the device error word
 * exactly as an expired wait in the tensor-core kernels would, so the next
 * call that synchronises (cossin, cossin_ex, cossin_cs, ...) returns
 * CS_ETIMEOUT and clears the word; the context stays usable.  Returns CS_OK
 * once the kernel is queued on `stream`. */
cs_status cossin_selftest_wait_timeout(cossin_stream_t stream);

/* Measured FP64 FMA throughput of the current device (the paper has no
 * counterpart): one register-only kernel, 16 independent FMA chains of
 * `rounds` steps in each of 256 threads x 4 CTAs per SM, timed with CUDA
 * events after a warm-up launch; *tflops = 2 x FMAs / time.  It is the
 * denominator of the FP64 product kernel's roofline.  Blocks until done;
 * allocates a small stream-ordered scratch. */
cs_status cossin_fp64_fma_rate(int64_t rounds, double* tflops, cossin_stream_t stream);

/* Kernels one FP64 product of an M x N result with inner dimension K
 * launches inside cossin / cossin_ex on the current device (the paper has no
 * counterpart): 2 when the tiles of its last, partial wave are split over K
 * (a second kernel adds the pieces and runs the epilogue), else 1; 0 for an
 * empty product.  For launch accounting; queues no work. */
cs_status cossin_fp64_product_launches(int64_t M, int64_t N, int64_t K, int32_t* launches);

/* Allocation-failure self test (the paper has no counterpart): the next
 * `count` device allocations the library makes for itself (the workspaces of
 * cossin, cossin_cs, cossin_unitary without ws, cossin_norm1, cossin_matmul
 * and the adjoint without ws) fail as if the device were out of memory, so
 * those calls return CS_ENOMEM before queuing any work; later calls run
 * normally.  count <= 0 clears the setting.  Host-only; touches no GPU. */
void cossin_selftest_fail_next_alloc(int32_t count);

/* One product P = X Y (n x n, row-major) on the library's product kernel for
 * `prec`, the one its Taylor chain uses: the FP64 kernel for CS_FP64, the
 * four-pass TF32 tensor-core kernel for CS_SPLIT_TF32 and CS_SPLIT_EMU (FP64
 * in and out, computed from the (hi, lo) splits of X and Y), the eight-slice
 * emulated product for CS_FP64_EMU and the four-slice BF16 product for
 * CS_SPLIT_BF16 (FP64 in and out) and CS_FP32 (FP32 in and out, the
 * operands taken to FP64 and the product rounded to FP32 once; n <= 8192
 * for these three).  These are the products the method counts (Pi_2m
 * in Tables 1-2).  P must not overlap X or Y.  Allocates and frees a
 * stream-ordered workspace for the tensor-core kinds, and for CS_FP64 when
 * the product's last wave of tiles is split over K (as inside cossin). */
cs_status cossin_matmul(const void* X_dev, const void* Y_dev, int64_t n, cs_prec prec, void* P_dev,
                        cossin_stream_t stream);

/* ------------------------------------------------------------ adjoint ---
 * Reverse mode of the computed approximant (not of the exact functions; the
 * paper has no adjoint): for each of `count` FP64 n x n matrices (contiguous
 * [count][n][n] arrays) and cotangents G_C, G_S,
 *   dA = d/dA ( <G_C, cos_r(A)> + <G_S, sin_r(A)> )
 * at the (2m, s) the forward pass uses (Table 1, or forced as in cossin_ex,
 * the same pair for every matrix).  Because the approximant is a polynomial
 * with real coefficients this equals L_cos(A^T, G_C) + L_sin(A^T, G_S).
 * The forward pass is recomputed with every product operand kept (the
 * double-angle levels included); matrices sharing (2m, s) run as one batch.
 * C, S (nullable) receive cos(A), sin(A) from that forward pass; infos_host
 * (nullable, host array of `count`) receives each matrix's norm, (2m, s) and
 * the product count 3 Pi_2m + 6 s of forward plus reverse.  Allocates its
 * workspace stream-ordered and synchronises `stream` once per (2m, s) group. */
cs_status cossin_backward(int64_t count, int64_t n, const double* A_dev, const double* G_C_dev,
                          const double* G_S_dev, double* dA_dev, double* C_dev, double* S_dev,
                          int32_t force_m, int32_t force_s, cs_info* infos_host, cossin_stream_t stream);

/* As cossin_backward, with the FP64 products of the forward and reverse
 * passes computed natively (prec = CS_FP64) or emulated on the BF16 tensor
 * cores (prec = CS_FP64_EMU, n <= 8192; see CS_FP64_EMU).  Any other prec
 * gives CS_EINVAL. */
cs_status cossin_backward_ex(int64_t count, int64_t n, const double* A_dev, const double* G_C_dev,
                             const double* G_S_dev, double* dA_dev, double* C_dev, double* S_dev, int32_t force_m,
                             int32_t force_s, cs_prec prec, cs_info* infos_host, cossin_stream_t stream);

/* Caller-workspace forms of the adjoint (the `ws, ws_bytes` contract of
 * cossin_ex): the same computation as cossin_backward_ex, with every device
 * buffer taken from ws_dev and nothing allocated.  The buffers depend on the
 * (2m, s) each matrix selects (its 1-norm, read on the device), so the size
 * is queried for the largest s the caller expects:
 *   cossin_backward_workspace_size: bytes for `count` matrices of order n in
 *     `prec` (CS_FP64 or CS_FP64_EMU) whose selected or forced s are all
 *     <= max_s, for any family.  Host-only.
 *   cossin_backward_ws: ws_dev (256-byte aligned, not overlapping the
 *     matrices) of ws_bytes; CS_EINVAL before any product is queued if the
 *     pairs the norms select need more than ws_bytes (the message gives the
 *     size).  Synchronises `stream` once for the norms and once per (2m, s)
 *     group, as cossin_backward does. */
cs_status cossin_backward_workspace_size(int64_t count, int64_t n, cs_prec prec, int32_t max_s, size_t* bytes);
cs_status cossin_backward_ws(int64_t count, int64_t n, const double* A_dev, const double* G_C_dev,
                             const double* G_S_dev, double* dA_dev, double* C_dev, double* S_dev, int32_t force_m,
                             int32_t force_s, cs_prec prec, void* ws_dev, size_t ws_bytes, cs_info* infos_host,
                             cossin_stream_t stream);

/* ------------------------------------------------------------ unitary ---
 * The propagator U = e^{-itA} = cos(tA) - i sin(tA) of a real n x n matrix
 * (Sec. 1, the Schroedinger case: unitary when A is symmetric), by the
 * cos/sin scheme at tA: ||tA||_1 = |t| ||A||_1 drives the choice of (2m, s)
 * (Tables 1-2) and t is folded into the first and last products, so no
 * scaled copy of A is made.
 *   U_dev: n x n complex, interleaved (re, im) pairs of the precision's real
 *          type (complex64 for CS_FP32, complex128 for every other prec);
 *          must not overlap A.
 *   ws_dev: at least cossin_unitary_workspace_size bytes, 256-byte aligned,
 *          or NULL to allocate on `stream`.
 * force_m / force_s and info as cossin_ex (info->norm1 = ||tA||_1).
 * CS_EINVAL for a non-finite t. */
cs_status cossin_unitary_workspace_size(int64_t n, cs_prec prec, size_t* bytes);
cs_status cossin_unitary(const void* A_dev, int64_t n, double t, cs_prec prec, void* U_dev, void* ws_dev,
                         size_t ws_bytes, int32_t force_m, int32_t force_s, cs_info* info,
                         cossin_stream_t stream);

/* Gradient of the real loss L = Re sum conj(G) .* U = <Re G, cos(tA)> +
 * <-Im G, sin(tA)> with respect to the real A (FP64; `count` matrices of
 * order n, contiguous), at the (2m, s) the forward pass uses for tA: the
 * reverse pass of cossin_backward with the cotangents (Re G, -Im G), t
 * carried by the plans' coefficients.  G_dev: interleaved complex128,
 * count x n x n.  dA_dev: real.  U_dev: optional interleaved forward output
 * (NULL to skip).  infos_host as cossin_backward.  No device-side failure
 * mode beyond those of cossin_backward. */
cs_status cossin_unitary_backward(int64_t count, int64_t n, double t, const double* A_dev, const double* G_dev,
                                  double* dA_dev, double* U_dev, int32_t force_m, int32_t force_s,
                                  cs_info* infos_host, cossin_stream_t stream);

/* ------------------------------------------------------------ batched ---
 * cos and sin of `count` FP32 matrices of orders n[i] <= 256 (host array),
 * each with its own theta, (2m, s) from Table 2, in one persistent launch:
 * every CTA takes matrices from a device work queue (largest first) and runs
 * steps 1-5 for each.  A[i], C[i], S[i] (host arrays of device pointers) are
 * row-major n[i] x n[i] FP32 matrices; C[i], S[i] must not overlap any A[j]
 * or each other.  infos_dev (device array of `count` cs_info) and status_dev
 * (device array of `count` cs_status: CS_OK, CS_ENONFINITE, CS_ERANGE; the
 * matrix's C and S are then NaN) may be NULL.  Orders > 256 go through
 * cossin() one by one.  ws_dev: cossin_batched_workspace_size bytes,
 * 256-byte aligned, owned by the caller. */
cs_status cossin_batched_workspace_size(int64_t count, const int64_t* n, size_t* bytes);

/* One-shot: uploads the batch descriptors (synchronises `stream` once) and
 * launches the persistent kernel with the tile shape the autotuner chose for
 * this batch signature earlier in the process (or the default). */
cs_status cossin_batched(int64_t count, const int64_t* n, const float* const* A, float* const* C,
                         float* const* S, void* ws_dev, size_t ws_bytes, cs_info* infos_dev,
                         int32_t* status_dev, cossin_stream_t stream);

/* Reusable plan: uploads the descriptors once, optionally autotunes (times
 * every tile shape / occupancy variant on this batch, keeps the fastest; this
 * runs the batch several times), and captures the queue reset plus the
 * persistent launch in a CUDA graph.  Each cossin_batched_plan_launch is one
 * graph launch on `stream`, recomputing every matrix from its current A.
 * The pointers and ws_dev must stay valid for the plan's lifetime. */
typedef struct cossin_batched_plan_st* cossin_batched_plan;
cs_status cossin_batched_plan_create(int64_t count, const int64_t* n, const float* const* A, float* const* C,
                                     float* const* S, void* ws_dev, size_t ws_bytes, cs_info* infos_dev,
                                     int32_t* status_dev, int32_t autotune, cossin_stream_t stream,
                                     cossin_batched_plan* plan);
cs_status cossin_batched_plan_launch(cossin_batched_plan plan, cossin_stream_t stream);
/* The variant the plan runs: CTA tile edge (64 or 128) and CTAs per SM. */
cs_status cossin_batched_plan_info(cossin_batched_plan plan, int32_t* tile, int32_t* ctas_per_sm);
cs_status cossin_batched_plan_destroy(cossin_batched_plan plan);

/* Last error message of the calling thread ("" if none). */
const char* cossin_last_error(void);

/* Synchronises `stream` and reports a device-side failure of earlier calls:
 * CS_ETIMEOUT if a kernel gave up on a bounded wait (the flag is then
 * cleared), CS_ECUDA if the stream holds a CUDA error, else CS_OK.  The same
 * check runs inside every cossin / cossin_ex call at its one synchronisation. */
cs_status cossin_device_status(cossin_stream_t stream);

/* Kernel timing hooks used by the benchmark.  While enabled, the library
 * records CUDA events around each launch of the kinds below on the launch
 * stream; cossin_prof_read synchronises those events and returns the summed
 * device time (ms), the number of launches and the algorithmic flops or
 * bytes of those launches since the last reset. */
typedef enum {
  CS_KERNEL_NORM1 = 0,      /* bytes = n^2 * element size */
  CS_KERNEL_GEMM_F64 = 1,   /* flops = 2 M N K */
  CS_KERNEL_GEMM_TF32 = 2,  /* flops = 2 M N K (algorithmic, not the 4 passes) */
  CS_KERNEL_BATCHED = 3,    /* flops = sum over matrices of 2 n^3 (Pi_2m + 2 s) */
  CS_KERNEL_ADJOINT = 4,    /* flops = 2 M N K of the reverse-pass products */
  CS_KERNEL_OTHER = 5,      /* splits and conversions; bytes moved */
  CS_KERNEL_GEMM_EMU = 6,   /* flops = 2 M N K (the emulated FP64 product, not its 36 slice products) */
  CS_KERNEL_KINDS = 7
} cs_kernel_kind;

void cossin_prof_enable(int32_t on);
void cossin_prof_reset(void);
cs_status cossin_prof_read(int32_t kind, double* ms, int64_t* launches, double* work);

#ifdef __cplusplus
}
#endif
#endif /* COSSIN_H */
